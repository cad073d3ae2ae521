"""GPU: the continuous-batching render server (cloud_server_*).

* a session's frames are the same alone and in a mix of concurrent sessions
  (bitwise: each view is the same computation in any batch);
* served frames match the FP64 oracle chain (render -> motion -> TAA);
* sessions are admitted against a device-memory budget;
* a paused server makes waits time out (host-side failure detection), and
  the queued requests complete after it resumes."""
import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_05344_gb300 import _native, api as A
    _native.build()
    return A


def _orbit(sid, f):
    return I.orbit_camera(f, seed=100 + sid)


def _run_alone(api, vol, w, h, frames, steps):
    srv = api.Server(vol, I.params(), history_fmt="fp32", max_batch_views=8)
    sid = srv.open_session(w, h)
    outs = []
    for f in range(frames):
        srv.wait(srv.submit(sid, _orbit(0, f), steps))
        outs.append(srv.output(sid))
    srv.close()
    return outs


def test_same_alone_and_in_the_mix(api):
    vol = api.Volume(I.volume_desc("full", seed=3))
    w, h, frames = 96, 64, 5
    alone = _run_alone(api, vol, w, h, frames, 8)
    srv = api.Server(vol, I.params(), history_fmt="fp32", max_batch_views=8, slots=2)
    rng = np.random.default_rng(0)
    sids = [srv.open_session(w, h)] + [srv.open_session(int(rng.integers(20, 200)),
                                                        int(rng.integers(20, 120)))
                                       for _ in range(7)]
    mixed = []
    for f in range(frames):
        tickets = {}
        order = list(rng.permutation(len(sids)))
        for k in order:  # submit in random order; other sessions compete for the batch
            tickets[k] = srv.submit(sids[k], _orbit(k, f), 16 if k % 2 else 8)
        infos = {k: srv.wait(t) for k, t in tickets.items()}
        mixed.append(srv.output(sids[0]))
    st = srv.stats()
    srv.close()
    assert st["batches"] < st["completed"]  # requests were batched together
    for a, m in zip(alone, mixed):
        assert np.array_equal(a, m)


def test_served_frames_match_oracle(api, oracle):
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    prm = I.params()
    w, h = 80, 48
    srv = api.Server(vol, prm, history_fmt="fp32")
    sid = srv.open_session(w, h)
    ohist = None
    for f in range(4):
        cam = _orbit(0, f)
        srv.wait(srv.submit(sid, cam, 8))
        ocur, _ = oracle.render(ovol, cam, prm, w, h, 8, 6, jitter_frame=f, nthreads=8)
        omot = oracle.motion(desc, prm, _orbit(0, f - 1), cam, w, h) if f else np.zeros((h, w, 2))
        ohist = oracle.taa(ohist, ocur, omot, blend=0.1)
        assert np.abs(srv.output(sid).astype(np.float64) - ohist).max() <= 1e-4
    srv.close()


def test_admission_by_memory_budget(api):
    from paper_1609_05344_gb300._native import CloudError, ERR_OUT_OF_MEMORY
    vol = api.Volume(I.volume_desc("tiny"))
    one = 640 * 360 * (16 + 2 * 8)  # current + 2 FP16 histories
    srv = api.Server(vol, I.params(), history_fmt="fp16", budget_bytes=3 * one)
    sids = [srv.open_session(640, 360) for _ in range(3)]
    with pytest.raises(CloudError) as e:
        srv.open_session(640, 360)
    assert e.value.status == ERR_OUT_OF_MEMORY
    srv.close_session(sids[0])
    sids[0] = srv.open_session(640, 360)  # freed memory admits a new session
    assert srv.stats()["open_sessions"] == 3
    srv.close()


def test_pause_times_out_then_resumes(api):
    from paper_1609_05344_gb300._native import CloudError, ERR_TIMEOUT
    vol = api.Volume(I.volume_desc("tiny"))
    srv = api.Server(vol, I.params())
    sid = srv.open_session(64, 32)
    srv.pause(True)
    t = srv.submit(sid, _orbit(0, 0), 8)
    with pytest.raises(CloudError) as e:
        srv.wait(t, timeout_ms=100)
    assert e.value.status == ERR_TIMEOUT
    assert srv.stats()["queued"] == 1
    srv.pause(False)
    info = srv.wait(t, timeout_ms=10000)
    assert info["latency_ms"] >= 100.0
    srv.close()


def test_failed_request_is_reported_not_hung(api):
    # a request whose launch fails (camera with tan_half_fovy = 0) makes the
    # server's error sticky: its wait and later submits report it, nothing hangs
    from paper_1609_05344_gb300._native import CloudError, ERR_INVALID_ARG
    vol = api.Volume(I.volume_desc("tiny"))
    srv = api.Server(vol, I.params())
    sid = srv.open_session(32, 16)
    ok = srv.wait(srv.submit(sid, _orbit(0, 0), 8))
    assert ok["latency_ms"] > 0
    bad = dict(_orbit(0, 1), tan_half_fovy=0.0)
    t = srv.submit(sid, bad, 8)
    with pytest.raises(CloudError) as e:
        srv.wait(t, timeout_ms=5000)
    assert e.value.status == ERR_INVALID_ARG
    assert srv.stats()["status"] == ERR_INVALID_ARG
    with pytest.raises(CloudError):
        srv.submit(sid, _orbit(0, 2), 8)
    srv.close()


def test_concurrent_submitters(api):
    """Four host threads drive their own sessions at once (the binding releases
    the interpreter lock inside each call): every session's frames are bitwise
    the frames of the same session served alone."""
    import threading
    vol = api.Volume(I.volume_desc("full", seed=3))
    w, h, frames = 48, 32, 4
    alone = {k: _run_alone_orbit(api, vol, w, h, frames, k) for k in range(4)}
    srv = api.Server(vol, I.params(), history_fmt="fp32", max_batch_views=16, slots=2)
    sids = {k: srv.open_session(w, h) for k in range(4)}
    got, errors = {}, []

    def drive(k):
        try:
            outs = []
            for f in range(frames):
                srv.wait(srv.submit(sids[k], _orbit(k, f), 8))
                outs.append(srv.output(sids[k]))
            got[k] = outs
        except Exception as exc:  # reported below, never swallowed
            errors.append(exc)

    threads = [threading.Thread(target=drive, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=60)
    st = srv.stats()
    srv.close()
    assert not errors and all(not t.is_alive() for t in threads)
    assert st["completed"] == 4 * frames
    for k in range(4):
        for a, m in zip(alone[k], got[k]):
            assert np.array_equal(a, m)


def _run_alone_orbit(api, vol, w, h, frames, k):
    srv = api.Server(vol, I.params(), history_fmt="fp32", max_batch_views=8)
    sid = srv.open_session(w, h)
    outs = []
    for f in range(frames):
        srv.wait(srv.submit(sid, _orbit(k, f), 8))
        outs.append(srv.output(sid))
    srv.close()
    return outs


def test_served_full_size_fp16(api, oracle):
    """The served configuration at its largest session (1920x1080, FP16 tiles
    and FP16 history) next to a small one in the same batches: three frames of
    each against the FP64 oracle chain (render -> motion -> TAA), within the
    reduced-precision tolerance 3e-3."""
    desc = I.volume_desc("full", seed=3, precision="fp16")
    vol, ovol = api.Volume(desc), oracle.Volume(dict(desc, precision="fp32"))
    prm = I.params()
    sizes = [(1920, 1080), (640, 360)]
    srv = api.Server(vol, prm, history_fmt="fp16", max_batch_views=8, slots=2)
    sids = [srv.open_session(w, h) for w, h in sizes]
    ohist = [None, None]
    worst = 0.0
    for f in range(3):
        tickets = [srv.submit(sid, _orbit(k, f), 8) for k, sid in enumerate(sids)]
        for t in tickets:
            srv.wait(t)
        for k, (w, h) in enumerate(sizes):
            cam = _orbit(k, f)
            ocur, _ = oracle.render(ovol, cam, prm, w, h, 8, 6, jitter_frame=f, nthreads=16)
            omot = (oracle.motion(desc, prm, _orbit(k, f - 1), cam, w, h) if f
                    else np.zeros((h, w, 2)))
            ohist[k] = oracle.taa(ohist[k], ocur, omot, blend=0.1)
            worst = max(worst, float(np.abs(srv.output(sids[k]).astype(np.float64) - ohist[k]).max()))
    srv.close()
    print(f"served fp16 full size: max abs err {worst:.3e}")
    assert worst <= 3e-3


def test_served_frames_equal_session_frames(api):
    """The server's batched raymarch and batched resolve compute each frame
    exactly as a session does with its single-view launches (bitwise)."""
    import torch
    vol = api.Volume(I.volume_desc("full", seed=3))
    prm = I.params()
    w, h, frames = 72, 40, 4
    sess = api.Session(vol, w, h, "fp32")
    host = torch.empty((h, w, 4), dtype=torch.float32, pin_memory=True)
    srv = api.Server(vol, prm, history_fmt="fp32", max_batch_views=8)
    sid = srv.open_session(w, h)
    other = srv.open_session(50, 30)  # a second view in the same batches
    for f in range(frames):
        sess.frame(_orbit(0, f), prm, 8, 6, host_out=host)
        t = srv.submit(sid, _orbit(0, f), 8)
        t2 = srv.submit(other, _orbit(1, f), 16)
        srv.wait(t)
        srv.wait(t2)
        assert np.array_equal(srv.output(sid), host.numpy()), f
    srv.close()
    sess.close()
