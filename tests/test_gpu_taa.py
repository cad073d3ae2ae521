"""GPU parity of motion (cloud_motion), the TAA resolve (taa_resolve) and the
session frame loop against the FP64 oracle.

The resolve is compared on identical seeded synthetic inputs (history,
current frame, motion with off-screen pixels); each side takes the same
off-screen and bilinear-weight decisions exactly, so FP32 history agrees to
rounding (1e-6) and FP16 history to its storage rounding (2e-3 for values up
to 2).  The frame loop runs each side's own chain (render -> motion -> TAA)
over an orbit and compares at the FP32 tolerance 1e-4."""
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


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("w,h", [(160, 90), (37, 23), (1920, 1080)])
def test_motion_parity(api, oracle, w, h):
    desc = I.volume_desc("full", seed=3)
    vol = api.Volume(desc)
    prm = I.params()
    for f in (1, 9):
        prev, cur = I.orbit_camera(f - 1, 3), I.orbit_camera(f, 3)
        got = api.motion(vol, prm, prev, cur, w, h).cpu().numpy()
        ref = oracle.motion(desc, prm, prev, cur, w, h)
        err = np.abs(got - ref).max()
        print(f"motion {w}x{h} frame {f}: max abs err {err:.3e} px")
        assert err <= 1e-4
    # a camera turned away: every point is behind the previous camera
    prev = I.camera((0.0, 0.0, 500.0), 180.0, 20.0, 60.0)
    cur = I.camera((0.0, 0.0, 500.0), 0.0, 20.0, 60.0)
    got = api.motion(vol, prm, prev, cur, 16, 8).cpu().numpy()
    assert np.all(got == np.float32(1e9))


@pytest.mark.parametrize("w,h", [(64, 48), (33, 17), (1, 1), (1920, 1080)])
@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_taa_parity_synthetic(api, oracle, w, h, fmt):
    rng = np.random.default_rng(w * 7 + h)
    hist = I.synthetic_frame(rng, h, w)
    cur = I.synthetic_frame(rng, h, w)
    mot = I.synthetic_motion(rng, h, w)
    hist_in = hist.astype(np.float16) if fmt == "fp16" else hist
    got = api.taa(_t(hist_in), _t(cur), _t(mot), blend=0.1, history_fmt=fmt).cpu().numpy()
    ref = oracle.taa(hist_in.astype(np.float64), cur.astype(np.float64), mot.astype(np.float64))
    tol = 1e-6 if fmt == "fp32" else 2e-3
    assert np.abs(got.astype(np.float64) - ref).max() <= tol
    first = api.taa(None, _t(cur), _t(mot), history_fmt=fmt).cpu().numpy()
    assert np.abs(first.astype(np.float64) - cur).max() <= (0 if fmt == "fp32" else 2e-3)


def test_taa_rejects_overlap(api):
    import torch
    from paper_1609_05344_gb300._native import CloudError
    buf = torch.zeros((8, 8, 4), dtype=torch.float32, device="cuda")
    mot = torch.zeros((8, 8, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(CloudError):
        api.taa(buf, buf, mot, out=buf)


# FP16 history: each resolve rounds its output by at most 2^-11 (values below
# 2) and the blend carries 0.9 of that forward, so after 8 frames the chain
# error is at most 2^-11 sum_{k<8} 0.9^k = 2^-11 * 5.7 = 2.8e-3, plus the
# render tolerance: within the reduced-precision tolerance 3e-3.
@pytest.mark.parametrize("fmt,tol", [("fp32", 1e-4), ("fp16", 3e-3)])
def test_session_matches_oracle_chain(api, oracle, fmt, tol):
    import torch
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    prm = I.params()
    w, h, frames = 120, 68, 8
    sess = api.Session(vol, w, h, history_fmt=fmt)
    host = torch.empty((h, w, 4), dtype=torch.float32 if fmt == "fp32" else torch.float16,
                       pin_memory=True)
    ohist = None
    for f in range(frames):
        cam = I.orbit_camera(f, 3)
        sess.frame(cam, prm, 8, 6, blend=0.1, host_out=host)
        ocur, _ = oracle.render(ovol, cam, prm, w, h, 8, 6, jitter_frame=f, nthreads=8)
        omot = (oracle.motion(desc, prm, I.orbit_camera(f - 1, 3), cam, w, h) if f
                else np.zeros((h, w, 2)))
        ohist = oracle.taa(ohist, ocur, omot, blend=0.1)
        err = np.abs(host.numpy().astype(np.float64) - ohist).max()
        print(f"session {fmt} frame {f}: max abs err {err:.3e}")
        assert err <= tol, (f, err)
    sess.close()


@pytest.mark.parametrize("w,h", [(37, 23), (1920, 1080), (1, 1)])
@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_fused_reprojection_equals_separate(api, w, h, fmt):
    import torch
    rng = np.random.default_rng(w + h)
    vol = api.Volume(I.volume_desc("full", seed=3))
    prm = I.params()
    dt = np.float16 if fmt == "fp16" else np.float32
    hist = _t(I.synthetic_frame(rng, h, w).astype(dt))
    cur = _t(I.synthetic_frame(rng, h, w))
    prev_cam, cur_cam = I.orbit_camera(4, 3), I.orbit_camera(5, 3)
    mot = api.motion(vol, prm, prev_cam, cur_cam, w, h)
    sep = api.taa(hist, cur, mot, blend=0.1, history_fmt=fmt).cpu().numpy()
    fused = api.taa_reproject(vol, prm, prev_cam, cur_cam, hist, cur, blend=0.1,
                              history_fmt=fmt).cpu().numpy()
    assert np.array_equal(sep, fused)
    first = api.taa_reproject(vol, prm, None, cur_cam, None, cur, history_fmt=fmt).cpu().numpy()
    assert np.array_equal(first, api.taa(None, cur, mot, history_fmt=fmt).cpu().numpy())


def test_async_session_frames_match_sync(api):
    import torch
    desc = I.volume_desc("full", seed=3)
    vol = api.Volume(desc)
    prm = I.params()
    w, h, frames = 200, 120, 7
    ref = api.Session(vol, w, h)
    host = torch.empty((h, w, 4), dtype=torch.float32, pin_memory=True)
    want = []
    for f in range(frames):
        ref.frame(I.orbit_camera(f, 3), prm, 8, 6, host_out=host)
        want.append(host.numpy().copy())
    ref.close()
    s = api.Session(vol, w, h)
    bufs = [torch.empty((h, w, 4), dtype=torch.float32, pin_memory=True) for _ in range(3)]
    idx = []
    for f in range(frames):
        idx.append(s.frame_async(I.orbit_camera(f, 3), prm, 8, 6, bufs[f % 3]))
        if f >= 2:  # the oldest in-flight read-back, then its buffer is reused
            s.wait_frame(idx[f - 2])
            assert np.array_equal(bufs[(f - 2) % 3].numpy(), want[f - 2])
    for f in (frames - 2, frames - 1):
        s.wait_frame(idx[f])
        assert np.array_equal(bufs[f % 3].numpy(), want[f])
    s.wait_frame(idx[0])  # long finished: returns at once
    s.close()


@pytest.mark.parametrize("src,dst,fmt", [((960, 540), (1920, 1080), "fp32"),
                                         ((480, 270), (1920, 1080), "fp16"),
                                         ((37, 23), (100, 61), "fp32"), ((5, 3), (5, 3), "fp32")])
def test_composite_parity(api, oracle, src, dst, fmt):
    rng = np.random.default_rng(src[0])
    cloud = I.synthetic_frame(rng, src[1], src[0])
    if fmt == "fp16":
        cloud = cloud.astype(np.float16)
    bg = rng.uniform(0, 1, (dst[1], dst[0], 4)).astype(np.float32)
    got = api.composite(_t(cloud), _t(bg)).cpu().numpy()
    ref = oracle.composite(cloud.astype(np.float64), bg.astype(np.float64))
    assert np.abs(got - ref).max() <= 1e-5


def test_session_frame_device_view_and_buffer_checks(api):
    """Without host_out a session frame is a zero-copy view of the resolved
    history; mis-sized or device-side host buffers are refused before any launch."""
    import torch
    vol = api.Volume(I.volume_desc("full", seed=3))
    prm = I.params()
    for fmt, dt in (("fp32", torch.float32), ("fp16", torch.float16)):
        sess = api.Session(vol, 64, 48, fmt)
        host = torch.empty((48, 64, 4), dtype=dt, pin_memory=True)
        sess.frame(I.orbit_camera(0, 3), prm, 8, 6, host_out=host)
        view = sess.frame(I.orbit_camera(1, 3), prm, 8, 6)
        assert view.is_cuda and view.dtype == dt and tuple(view.shape) == (48, 64, 4)
        torch.cuda.synchronize()
        got = view.cpu().numpy().copy()
        ref = api.Session(vol, 64, 48, fmt)
        ref.frame(I.orbit_camera(0, 3), prm, 8, 6, host_out=host)
        ref.frame(I.orbit_camera(1, 3), prm, 8, 6, host_out=host)
        assert np.array_equal(got, host.numpy())
        with pytest.raises(ValueError):
            sess.frame(I.orbit_camera(2, 3), prm, 8, 6, host_out=torch.empty(10, dtype=dt))
        with pytest.raises(ValueError):
            sess.frame(I.orbit_camera(2, 3), prm, 8, 6, host_out=view)
        sess.close()
        ref.close()
    with pytest.raises(ValueError):
        api.render(vol, I.orbit_camera(0, 3), prm, 64, 48, 8, 6,
                   out=torch.empty((48, 63, 4), device="cuda"))
    with pytest.raises(ValueError):
        api.taa(None, torch.empty((48, 64, 4), device="cuda"), torch.empty((48, 64, 1), device="cuda"))


@pytest.mark.parametrize("jump", ["yaw-40", "behind", "translate-2km", "above-layer"])
def test_fused_resolve_large_camera_jumps(api, oracle, jump):
    """Camera jumps that push much of the history off screen or behind the
    previous camera: the fused kernel against the oracle's motion + resolve on
    the same current frame and history."""
    rng = np.random.default_rng(11)
    desc = I.volume_desc("full", seed=3)
    vol = api.Volume(desc)
    prm = I.params()
    w, h = 97, 61
    cur_cam = I.camera((0.0, 0.0, 500.0), 30.0, 15.0, 60.0)
    prev_cam = {
        "yaw-40": I.camera((0.0, 0.0, 500.0), 70.0, 15.0, 60.0),
        "behind": I.camera((0.0, 0.0, 500.0), 210.0, 15.0, 60.0),
        "translate-2km": I.camera((1500.0, -1300.0, 500.0), 30.0, 15.0, 60.0),
        "above-layer": I.camera((0.0, 0.0, 5000.0), 30.0, -20.0, 60.0),
    }[jump]
    hist = I.synthetic_frame(rng, h, w)
    cur = I.synthetic_frame(rng, h, w)
    got = api.taa_reproject(vol, prm, prev_cam, cur_cam, _t(hist), _t(cur), blend=0.1).cpu().numpy()
    omot = oracle.motion(desc, prm, prev_cam, cur_cam, w, h)
    ref = oracle.taa(hist.astype(np.float64), cur.astype(np.float64), omot, blend=0.1)
    off = (omot[..., 0] > np.arange(w)[None, :] + 0.5) | (omot[..., 0] < np.arange(w)[None, :] + 0.5 - w) | \
          (omot[..., 1] > np.arange(h)[:, None] + 0.5) | (omot[..., 1] < np.arange(h)[:, None] + 0.5 - h)
    assert off.any()  # the jump really sends pixels off screen
    assert np.abs(got.astype(np.float64) - ref).max() <= 1e-4


def test_fast_1080p_full_orbit_chain(api, oracle):
    """The benchmarked configuration end to end: 1920x1080, 8 jittered x 6 light
    steps, FP32 tiles, render + fused reprojection + TAA over the whole 32-frame
    orbit, every resolved frame against the FP64 oracle chain at 1e-4."""
    import time
    import torch
    wl = I.workload("fast-1080p")
    desc = wl.volume
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    prm = I.params()
    W, H = wl.width, wl.height
    sess = api.Session(vol, W, H, history_fmt="fp32")
    host = torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True)
    ohist, worst, t0 = None, 0.0, time.perf_counter()
    seed = desc["seed"]
    for f in range(wl.frames):
        cam = I.orbit_camera(f, seed)
        sess.frame(cam, prm, wl.steps, wl.light_steps, blend=0.1, host_out=host)
        ocur, _ = oracle.render(ovol, cam, prm, W, H, wl.steps, wl.light_steps, jitter_frame=f,
                                nthreads=16)
        omot = (oracle.motion(desc, prm, I.orbit_camera(f - 1, seed), cam, W, H) if f
                else np.zeros((H, W, 2)))
        ohist = oracle.taa(ohist, ocur, omot, blend=0.1)
        err = float(np.abs(host.numpy().astype(np.float64) - ohist).max())
        worst = max(worst, err)
        assert err <= 1e-4, (f, err)
    sess.close()
    print(f"fast-1080p orbit chain: worst max abs err {worst:.3e} over {wl.frames} frames "
          f"({time.perf_counter() - t0:.0f} s)")


def test_fused_resolve_random_camera_pairs(api, oracle):
    """Seeded random (previous, current) camera pairs, sizes and blends: the fused
    reprojection + resolve against the oracle's motion + resolve on the same
    current frame and history, FP32 history at 1e-4."""
    rng = np.random.default_rng(77)
    desc = I.volume_desc("full", seed=3)
    vol = api.Volume(desc)
    prm = I.params()
    worst = 0.0
    for _ in range(16):
        def cam():
            return I.camera((float(rng.uniform(-3000, 3000)), float(rng.uniform(-3000, 3000)),
                             float(rng.uniform(0, 6000))), float(rng.uniform(0, 360)),
                            float(rng.uniform(-50, 70)), float(rng.uniform(30, 90)))
        cur_cam = cam()
        prev_cam = cam() if rng.uniform() < 0.5 else dict(
            cur_cam, pos=tuple(np.array(cur_cam["pos"]) + rng.normal(0, 30, 3)))
        w, h = int(rng.integers(1, 90)), int(rng.integers(1, 60))
        blend = float(rng.uniform(0.02, 0.5))
        hist = I.synthetic_frame(rng, h, w)
        cur = I.synthetic_frame(rng, h, w)
        got = api.taa_reproject(vol, prm, prev_cam, cur_cam, _t(hist), _t(cur),
                                blend=blend).cpu().numpy()
        omot = oracle.motion(desc, prm, prev_cam, cur_cam, w, h)
        ref = oracle.taa(hist.astype(np.float64), cur.astype(np.float64), omot, blend=blend)
        worst = max(worst, float(np.abs(got.astype(np.float64) - ref).max()))
    assert worst <= 1e-4


@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_session_snapshot_restore_continues_bitwise(api, fmt):
    """A session checkpointed mid-orbit and restored into a fresh session
    continues bitwise like the uninterrupted one (history, jitter index and
    previous camera all carried over); malformed or mismatched snapshots are
    refused."""
    import torch
    from paper_1609_05344_gb300 import _native as N
    vol = api.Volume(I.volume_desc("full", seed=3))
    prm = I.params()
    w, h = 96, 54
    dt = torch.float32 if fmt == "fp32" else torch.float16
    a = api.Session(vol, w, h, history_fmt=fmt)
    host = torch.empty((h, w, 4), dtype=dt, pin_memory=True)
    for f in range(4):
        a.frame(I.orbit_camera(f, 3), prm, 8, 6, host_out=host)
    snap = a.snapshot()
    cont = [a.frame(I.orbit_camera(f, 3), prm, 8, 6, host_out=torch.empty_like(host)).clone()
            for f in range(4, 7)]
    b = api.Session(vol, w, h, history_fmt=fmt)
    b.frame(I.orbit_camera(30, 3), prm, 8, 6, host_out=host)  # state that the restore replaces
    b.restore(snap)
    got = [b.frame(I.orbit_camera(f, 3), prm, 8, 6, host_out=torch.empty_like(host)).clone()
           for f in range(4, 7)]
    for x, y in zip(cont, got):
        assert torch.equal(x, y)
    bad = bytearray(snap)
    bad[0] ^= 0xFF
    with pytest.raises(N.CloudError):
        b.restore(bytes(bad))
    other = api.Session(vol, w + 1, h, history_fmt=fmt)
    with pytest.raises(N.CloudError):
        other.restore(snap)
    # a snapshot of a session without history restores to a first frame
    fresh = api.Session(vol, w, h, history_fmt=fmt)
    snap0 = fresh.snapshot()
    b.restore(snap0)
    x = b.frame(I.orbit_camera(0, 3), prm, 8, 6, host_out=torch.empty_like(host)).clone()
    y = fresh.frame(I.orbit_camera(0, 3), prm, 8, 6, host_out=torch.empty_like(host)).clone()
    assert torch.equal(x, y)
    for sess in (a, b, other, fresh):
        sess.close()


def test_resolve_wait_give_up_is_reported(api):
    """The fused resolve's bounded wait for its tile copy, made to give up at
    once (poll budget 0): every tile's outputs stay unwritten, the give-ups are
    counted, a session reports CLOUD_ERR_TIMEOUT (sticky until reset) and a
    server request fails with it.  The copy itself is a valid in-bounds load
    that the kernel's second bounded wait still sees land before it exits."""
    import torch
    from paper_1609_05344_gb300 import _native as N
    vol = api.Volume(I.volume_desc("tiny", seed=1))
    prm = I.params()
    w, h, tiles = 70, 37, 3 * 2  # FP32 history: 32x32-pixel tiles, 3 columns, 2 rows (ragged)
    cams = [I.orbit_camera(f, 1) for f in range(3)]
    torch.cuda.synchronize()
    before = api.device_wait_timeouts()
    cur0 = api.render(vol, cams[0], prm, w, h, 8, 6, jitter_frame=0)
    cur1 = api.render(vol, cams[1], prm, w, h, 8, 6, jitter_frame=1)
    hist0 = api.taa_reproject(vol, prm, None, cams[0], None, cur0)
    host = torch.empty((h, w, 4), dtype=torch.float32, pin_memory=True)
    sess, ref = api.Session(vol, w, h), api.Session(vol, w, h)
    srv = api.Server(vol, prm, history_fmt="fp32", max_sessions=2, max_batch_views=4, slots=1,
                     reserve_bytes=0)
    sid = srv.open_session(w, h)
    try:
        api.set_wait_polls(0)
        out = api.taa_reproject(vol, prm, cams[0], cams[1], hist0, cur1,
                                out=torch.full((h, w, 4), -7.0, device="cuda"))
        torch.cuda.synchronize()
        assert api.device_wait_timeouts() - before == tiles
        assert bool((out == -7.0).all())
        with pytest.raises(N.CloudError) as e:
            sess.frame(cams[0], prm, 8, 6, host_out=host)
        assert e.value.status == N.ERR_TIMEOUT
        with pytest.raises(N.CloudError) as e:  # sticky: refused without rendering
            sess.frame(cams[1], prm, 8, 6, host_out=host)
        assert e.value.status == N.ERR_TIMEOUT
        with pytest.raises(N.CloudError) as e:
            srv.wait(srv.submit(sid, cams[0], 8), 20000)
        assert e.value.status == N.ERR_TIMEOUT
    finally:
        api.set_wait_polls(-1)
    torch.cuda.synchronize()
    assert api.device_wait_timeouts() - before == 3 * tiles
    # after a reset the session continues exactly like one that never failed:
    # frame index 1 as a first frame, then frame 2 with history
    ref.frame(cams[0], prm, 8, 6, host_out=host)
    ref.reset()
    sess.reset()
    for f in (1, 2):
        a = sess.frame(cams[f], prm, 8, 6, host_out=torch.empty_like(host)).clone()
        b = ref.frame(cams[f], prm, 8, 6, host_out=torch.empty_like(host)).clone()
        assert torch.equal(a, b)
    # the server session's next frame is a first frame and succeeds
    srv.wait(srv.submit(sid, cams[1], 8), 20000)
    srv.close()
    sess.close()
    ref.close()
    if before == 0:
        api.device_wait_timeouts(reset=True)


def test_zz_no_device_wait_gave_up(api):
    """Every bounded wait of the resolve kernels in this module's other tests
    completed (the tile copies all landed)."""
    import torch
    torch.cuda.synchronize()
    assert api.device_wait_timeouts() == 0
