"""GPU: multi-view persistent launches (cloud_batch_*) and the tile-shape
autotuner.  Every view of a batch is the same computation as cloud_render of
that view, so outputs must be bitwise equal; a few views are also checked
against the FP64 oracle (1e-4)."""
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


def _single(api, vol, v):
    return api.render(vol, v["camera"], I.params(), v["width"], v["height"], v["steps"], 6,
                      jitter_frame=v["jitter_frame"]).cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "unorm16"])
def test_batch_equals_single_views(api, precision):
    vol = api.Volume(I.volume_desc("full", seed=3, precision=precision))
    views = I.random_views(12, seed=9, max_size=(300, 200), min_size=(1, 1))
    b = api.Batch(vol, I.params(), views)
    outs = [o.cpu().numpy() for o in b.render()]
    for v, o in zip(views, outs):
        assert np.array_equal(o, _single(api, vol, v))
    outs_g = [o.cpu().numpy() for o in b.render(graph=True)]
    for a, c in zip(outs, outs_g):
        assert np.array_equal(a, c)
    for o in b.outputs:
        o.zero_()
    outs_p = [o.cpu().numpy() for o in b.render_per_view()]
    for a, c in zip(outs, outs_p):
        assert np.array_equal(a, c)
    b.close()


def test_batch_set_views_and_graph_replay(api):
    vol = api.Volume(I.volume_desc("full", seed=3))
    views = I.random_views(6, seed=2, max_size=(160, 120), min_size=(8, 8))
    b = api.Batch(vol, I.params(), views)
    b.render(graph=True)
    for frame in range(3):
        moved = [dict(v, camera=I.camera(np.array(v["camera"]["pos"]) + [50.0 * frame, 0, 0],
                                         10.0 * frame, 15.0), jitter_frame=frame) for v in views]
        b.set_views(moved)
        outs = [o.cpu().numpy() for o in b.render(graph=True)]
        for v, o in zip(moved, outs):
            assert np.array_equal(o, _single(api, vol, v))
    with pytest.raises(Exception):
        b.set_views([dict(views[0], width=views[0]["width"] + 1)] + views[1:])
    b.close()


def test_batch_matches_oracle(api, oracle):
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    views = I.random_views(4, seed=5, max_size=(64, 48), min_size=(17, 9))
    b = api.Batch(vol, I.params(), views)
    outs = [o.cpu().numpy() for o in b.render()]
    for v, o in zip(views, outs):
        ref, _ = oracle.render(ovol, v["camera"], I.params(), v["width"], v["height"], v["steps"],
                               6, jitter_frame=v["jitter_frame"], nthreads=8)
        assert np.abs(o - ref).max() <= 1e-4
    b.close()


def test_autotune_shapes_equal_results(api):
    keep = api.launch_config("fp32", 6)
    try:
        _autotune_checks(api)
    finally:  # later tests run in the launch configuration the bench uses
        api.set_launch_config("fp32", 6, keep)


def _autotune_checks(api):
    vol = api.Volume(I.volume_desc("full", seed=3))
    cam = I.orbit_camera(0, 3)
    base = api.render(vol, cam, I.params(), 333, 177, 8, 6, jitter_frame=3).cpu().numpy()
    best, times = api.autotune_render(vol, cam, I.params(), 333, 177, 8, 6, jitter_frame=3,
                                      repeats=2)
    assert 0 <= best < 8 and len(times) == 8 and all(t > 0 for t in times)
    again = api.render(vol, cam, I.params(), 333, 177, 8, 6, jitter_frame=3).cpu().numpy()
    assert np.array_equal(base, again)  # the launch configuration does not change any pixel
    views = I.random_views(5, seed=11, max_size=(200, 100), min_size=(8, 8))
    b = api.Batch(vol, I.params(), views)
    ref = [o.cpu().numpy() for o in b.render()]
    best, times = b.autotune(repeats=2)
    assert 0 <= best < 8 and len(times) == 8
    for a, o in zip(ref, b.render(graph=True)):
        assert np.array_equal(a, o.cpu().numpy())
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_every_launch_config_bitwise_equal(api, precision):
    """Tile shape and view steps per warp iteration (8 or 16) change the work
    order only: every configuration gives bitwise the same pixels, for one view,
    a multi-view batch and a ray count that needs more than one 16-step chunk."""
    from paper_1609_05344_gb300 import _native as N
    vol = api.Volume(I.volume_desc("full", seed=3, precision=precision))
    cam = I.orbit_camera(2, 3)
    keep = api.launch_config(precision, 6)
    views = I.random_views(4, seed=5, max_size=(160, 90), min_size=(8, 8), steps=(8, 24, 40))
    try:
        outs, bouts = [], []
        for cfg in range(N.TUNE_CONFIGS):
            api.set_launch_config(precision, 6, cfg)
            outs.append(api.render(vol, cam, I.params(), 203, 77, 40, 6, jitter_frame=1).cpu().numpy())
            b = api.Batch(vol, I.params(), views)
            bouts.append([o.cpu().numpy() for o in b.render()])
            b.close()
        for cfg in range(1, N.TUNE_CONFIGS):
            assert np.array_equal(outs[0], outs[cfg]), N.config_parts(cfg)
            for a, o in zip(bouts[0], bouts[cfg]):
                assert np.array_equal(a, o), N.config_parts(cfg)
    finally:
        api.set_launch_config(precision, 6, keep)


@pytest.mark.parametrize("precision,tol", [
    ("fp32", 1e-4), ("fp16", 3e-3),
    pytest.param("bf16", 3e-3, marks=pytest.mark.xfail(
        strict=True, reason="BF16 differences from an exactly stored corner still round the "
                            "base tile's texel differences to ~2.4e-4; the 8-step views exceed "
                            "3e-3 (the 16- to 128-step views meet it)"))])
def test_batched_64_full_size_sampled(api, oracle, precision, tol):
    """The batched workload at its full size (64 seeded views, 256x256 .. 1920x1080,
    8 / 16 / 32 / 128 steps) in the launch the bench times (one persistent launch
    from a CUDA graph), checked on sampled pixels of every view against the FP64
    oracle: FP32 tiles at the 1e-4 bar, FP16 and BF16 tiles at 3e-3."""
    desc = I.volume_desc("full", seed=3, precision=precision)
    vol, ovol = api.Volume(desc), oracle.Volume(dict(desc, precision="fp32"))
    views = I.random_views(64, seed=4)
    b = api.Batch(vol, I.params(), views)
    outs = b.render(graph=True)
    rng = np.random.default_rng(9)
    worst = 0.0
    for v, o in zip(views, outs):
        xs = rng.integers(0, v["width"], 24)
        ys = rng.integers(0, v["height"], 24)
        got = o.cpu().numpy()[ys, xs]
        ref, _ = oracle.render_pixels(ovol, v["camera"], I.params(), v["width"], v["height"],
                                      v["steps"], 6, xs, ys, jitter_frame=v["jitter_frame"],
                                      nthreads=8)
        worst = max(worst, float(np.abs(got - ref).max()))
    b.close()
    print(f"batched-64 {precision}: max abs err {worst:.3e} on 1536 sampled pixels")
    assert worst <= tol
