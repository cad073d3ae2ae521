"""GPU parity of the raymarch (cloud_render) against the FP64 oracle.

Tolerances (max-abs RGBA): 1e-4 for FP32 volumes, 3e-3 for FP16 volumes;
the closed-form and telescoping identities to 2e-5 / 2e-6.  Small cases are
compared on every pixel (sizes with ragged tails over several 16x8 tiles);
the full-size workloads are compared on seeded pixel samples the oracle
evaluates one by one, from a full-size launch."""
import math

import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_FP16 = 3e-3


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_05344_gb300 import _native, api as A
    _native.build()
    return A


def _max_err(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).max())


def test_hash_bitwise(api, oracle):
    import torch
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1 << 32, (1 << 20, 4), dtype=np.uint64).astype(np.uint32)
    keys[:1024, :] = np.arange(4096, dtype=np.uint32).reshape(1024, 4)  # structured keys too
    got = api.hash4(torch.from_numpy(keys.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.hash4_batch(keys))


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-7), ("fp16", 7.7e-6), ("bf16", 7.7e-6),
                                           ("unorm16", 7.7e-6)])
def test_volume_generation(api, oracle, precision, tol):
    desc = I.volume_desc("full", seed=2, precision=precision, base_n=64)
    tiles = api.Volume(desc).export()
    ov = oracle.Volume(desc)
    assert _max_err(tiles["base"].cpu().numpy(), ov.base) <= tol
    assert _max_err(tiles["detail"].cpu().numpy(), ov.detail) <= tol
    assert _max_err(tiles["weather"].cpu().numpy(), ov.weather) <= tol


@pytest.mark.parametrize("w,h", [(128, 128), (37, 23), (1, 1), (200, 9)])
def test_plain_tiny_full_image(api, oracle, w, h):
    wl = I.workload("plain-tiny")
    vol, ovol = api.Volume(wl.volume), oracle.Volume(wl.volume)
    cam = I.ground_camera()
    if (w, h) == (1, 1):
        cam = I.camera((0.0, 0.0, 500.0), 0.0, 45.0, 60.0)  # the single ray hits the layer
    got = api.render(vol, cam, I.params(), w, h, wl.steps, wl.light_steps).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, I.params(), w, h, wl.steps, wl.light_steps, nthreads=8)
    assert _max_err(got, ref) <= TOL_FP32
    if w * h > 1:
        assert ref[..., 3].max() > 0.1


@pytest.mark.parametrize("frame", [0, 5, 31])
@pytest.mark.parametrize("integration", ["analytic", "basic"])
def test_full_volume_jittered_small(api, oracle, frame, integration):
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    cam = I.orbit_camera(frame, 3)
    w, h = 96, 54
    got = api.render(vol, cam, I.params(), w, h, 8, 6, jitter_frame=frame,
                     integration=integration).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, I.params(), w, h, 8, 6, jitter_frame=frame,
                           integration=1 if integration == "basic" else 0, nthreads=8)
    assert _max_err(got, ref) <= TOL_FP32


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_FP32), ("fp16", TOL_FP16)])
def test_non_dyadic_detail_period(api, oracle, precision, tol):
    """The standard tile sizes with a base tile period that is not 2^k detail
    periods (6400 m / 1000 m): the march then converts the detail coordinates
    separately (the generic kernel) and the occupancy grid bounds the detail
    term by the whole detail tile's minimum.  Every pixel against the FP64
    oracle, and the grid's skips bitwise exact."""
    desc = I.volume_desc("full", seed=5, detail_period=1000.0)
    vol = api.Volume(dict(desc, precision=precision))
    ovol = oracle.Volume(desc)
    cam = I.orbit_camera(4, 5)
    w, h = 80, 45
    got = api.render(vol, cam, I.params(), w, h, 8, 6, jitter_frame=4).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, I.params(), w, h, 8, 6, jitter_frame=4, nthreads=8)
    assert _max_err(got, ref) <= tol
    assert ref[..., 3].max() > 0.1
    api.set_occupancy(False)
    try:
        plain = api.render(vol, cam, I.params(), w, h, 8, 6, jitter_frame=4).cpu().numpy()
    finally:
        api.set_occupancy(True)
    assert np.array_equal(plain, got)


def _sampled(api, oracle, wl, cam, frame, n, seed, precision="fp32", steps=None):
    desc = dict(wl.volume, precision=precision)
    vol = api.Volume(desc)
    ovol = oracle.Volume(dict(wl.volume, precision="fp32"))
    steps = steps or wl.steps
    img = api.render(vol, cam, I.params(), wl.width, wl.height, steps, wl.light_steps,
                     jitter_frame=frame).cpu().numpy()
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, wl.width, n)
    ys = rng.integers(0, wl.height, n)
    # the last row/column and the four corners are always checked
    xs = np.concatenate([xs, [0, wl.width - 1, 0, wl.width - 1], rng.integers(0, wl.width, 16),
                         np.full(16, wl.width - 1)])
    ys = np.concatenate([ys, [0, 0, wl.height - 1, wl.height - 1], np.full(16, wl.height - 1),
                         rng.integers(0, wl.height, 16)])
    ref, _ = oracle.render_pixels(ovol, cam, I.params(), wl.width, wl.height, steps,
                                  wl.light_steps, xs, ys, jitter_frame=frame, nthreads=8)
    return _max_err(img[ys, xs], ref), img


@pytest.mark.parametrize("frame", [0, 7, 19])
def test_fast_1080p_sampled(api, oracle, frame):
    wl = I.workload("fast-1080p")
    err, img = _sampled(api, oracle, wl, I.orbit_camera(frame, 3), frame, 60000, 100 + frame)
    assert err <= TOL_FP32
    assert np.isfinite(img).all()


def test_reference_720p_fp16_volumes(api, oracle):
    wl = I.workload("reference")
    err, _ = _sampled(api, oracle, wl, I.ground_camera(), -1, 4000, 6, precision="fp16")
    assert err <= TOL_FP16


@pytest.mark.parametrize("frame", [3, 11])
def test_fast_1080p_unorm16_volumes(api, oracle, frame):
    # 16-bit fixed-point texels (error <= 2^-17) meet the reduced-precision
    # tolerance on the 8-step fast path at half the bytes of FP32
    wl = I.workload("fast-1080p")
    err, _ = _sampled(api, oracle, wl, I.orbit_camera(frame, 3), frame, 40000, 5 + frame,
                      precision="unorm16")
    print(f"fast-1080p unorm16 volumes frame {frame}: max abs err {err:.3e}")
    assert err <= TOL_FP16


@pytest.mark.parametrize("frame", [3, 11])
def test_fast_1080p_fp16_volumes(api, oracle, frame):
    # FP16 records (corner 0 as 16-bit fixed point, the other corners as half
    # differences from it) meet the reduced-precision tolerance on the 8-step
    # fast path at half the record bytes of FP32
    wl = I.workload("fast-1080p")
    err, _ = _sampled(api, oracle, wl, I.orbit_camera(frame, 3), frame, 40000, 5 + frame,
                      precision="fp16")
    print(f"fast-1080p fp16 volumes frame {frame}: max abs err {err:.3e}")
    assert err <= TOL_FP16


@pytest.mark.xfail(strict=True, reason="BF16 keeps 8 significant bits: even as differences from "
                                       "an exactly stored corner, the base tile's texel "
                                       "differences (up to ~0.13) round to ~2.4e-4, which 8 view "
                                       "steps of up to 3.5 km amplify past 3e-3")
def test_fast_1080p_bf16_volumes(api, oracle):
    wl = I.workload("fast-1080p")
    err, _ = _sampled(api, oracle, wl, I.orbit_camera(3, 3), 3, 40000, 5, precision="bf16")
    print(f"fast-1080p bf16 volumes: max abs err {err:.3e}")
    assert err <= TOL_FP16


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "unorm16"])
@pytest.mark.parametrize("frame", [3, 20])
def test_occupancy_skip_is_bitwise_exact(api, frame, precision):
    """Skipping the memory reads of lookups in macro-cells the occupancy grid
    proves empty changes no pixel: a full-size fast-1080p frame is bitwise the
    same with the grid in use and with every lookup evaluated."""
    import torch
    wl = I.workload("fast-1080p", precision=precision)
    vol = api.Volume(wl.volume)
    cam = I.orbit_camera(frame, 3)
    try:
        api.set_occupancy(False)
        full, n_full = api.render(vol, cam, I.params(), wl.width, wl.height, wl.steps,
                                  wl.light_steps, jitter_frame=frame, count=True)
        api.set_occupancy(True)
        skip, n_skip = api.render(vol, cam, I.params(), wl.width, wl.height, wl.steps,
                                  wl.light_steps, jitter_frame=frame, count=True)
    finally:
        api.set_occupancy(True)
    assert torch.equal(full, skip)
    assert int(n_full.item()) == int(n_skip.item())  # the same lookups, fewer of them read memory


def _half_lattice(t):
    """Trilinear values of a periodic texel lattice at every half-texel point:
    index 2k is texel k, 2k + 1 the midpoint of texels k and k + 1 (per axis)."""
    h = np.zeros((2 * t.shape[0],) * 3)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                acc, cnt = 0.0, 0
                for oz in range(dz + 1):
                    for oy in range(dy + 1):
                        for ox in range(dx + 1):
                            acc = acc + np.roll(t, (-oz, -oy, -ox), (0, 1, 2))
                            cnt += 1
                h[dz::2, dy::2, dx::2] = acc / cnt
    return h


def test_occupancy_grid_is_conservative(api, oracle):
    """Every cell the grid marks empty really has no density, checked on the FP64
    oracle texels, and the grid marks a substantial share of the cells empty.
    A grid cell is half a base texel on each axis: over it, trilinear B is
    largest at one of the cell's 8 corners (half-texel lattice points), and Dt
    over the same box (detail coordinate = 2 x base + 1/2 here) is smallest at
    one of the 27 points formed by its corners and the detail lattice plane
    inside; max B - w_d min Dt - c must then be negative."""
    desc = I.volume_desc("full", seed=3)
    occ = api.Volume(desc).occupancy()
    ov = oracle.Volume(desc)
    B, Dt = ov.base, ov.detail
    nb, nd = B.shape[0], Dt.shape[0]
    assert occ.shape == (2 * nb,) * 3
    assert desc["base_period"] / desc["detail_period"] * nd / nb == 2.0
    bh = np.pad(_half_lattice(B), ((0, 1),) * 3, mode="wrap")
    bmax = np.full(occ.shape, -np.inf)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                bmax = np.maximum(bmax, bh[dz:dz + 2 * nb, dy:dy + 2 * nb, dx:dx + 2 * nb])
    # cell u: detail coordinates [u + 1/2, u + 3/2) -> half-lattice points 2u+1, 2u+2, 2u+3
    dh = _half_lattice(Dt)
    dhp = np.pad(dh, ((0, 3),) * 3, mode="wrap")
    dmin = np.full(dh.shape, np.inf)
    for oz in (1, 2, 3):
        for oy in (1, 2, 3):
            for ox in (1, 2, 3):
                dmin = np.minimum(dmin, dhp[oz:oz + 2 * nd, oy:oy + 2 * nd, ox:ox + 2 * nd])
    k = np.arange(2 * nb) % nd
    dmin_cells = dmin[::2, ::2, ::2][np.ix_(k, k, k)]
    bound = bmax - desc["detail_weight"] * dmin_cells - desc["coverage"]
    empty = ~occ
    assert empty.mean() > 0.5
    assert bound[empty].max() < 0.0


def test_reference_720p_sampled(api, oracle):
    wl = I.workload("reference")
    err, _ = _sampled(api, oracle, wl, I.ground_camera(), -1, 4000, 9)
    assert err <= TOL_FP32


@pytest.mark.parametrize("integration", ["analytic", "basic"])
def test_reference_720p_full_image(api, oracle, integration):
    """The reference-quality configuration (1280x720, 128 x 6 steps, full tiles,
    no jitter) on every pixel, for both integration rules."""
    wl = I.workload("reference")
    vol, ovol = api.Volume(wl.volume), oracle.Volume(wl.volume)
    cam, prm = I.ground_camera(), I.params()
    got = api.render(vol, cam, prm, wl.width, wl.height, wl.steps, wl.light_steps,
                     integration=integration).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, prm, wl.width, wl.height, wl.steps, wl.light_steps,
                           integration=oracle.ANALYTIC if integration == "analytic" else oracle.BASIC,
                           nthreads=16)
    assert _max_err(got, ref) <= TOL_FP32


def _closed_form(oracle, desc, prm, cam, w, h, rho0, ls):
    out = np.zeros((h, w, 4))
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    for y in range(h):
        for x in range(w):
            d = oracle.pixel_ray(cam, w, h, x, y)
            hit, t0, t1 = oracle.slab_clip(desc, prm, cam["pos"], d)
            if not hit:
                continue
            ph = oracle.hg(float(np.dot(d, s)), prm["hg_g"])
            lin = (np.array(prm["sun_radiance"]) * math.exp(-rho0 * prm["absorption"] * ls *
                                                            prm["light_step"]) * ph
                   + np.array(prm["ambient"]))
            a = -math.expm1(-rho0 * prm["absorption"] * (t1 - t0))
            out[y, x, :3], out[y, x, 3] = lin * a, a
    return out


@pytest.mark.parametrize("steps", [1, 3, 8, 128])
def test_homogeneous_slab_closed_form_on_gpu(api, oracle, steps):
    rho0 = 0.004
    desc = I.volume_desc("constant", rho0=rho0)
    prm = I.params(tau_max=0.0)
    cam = I.ground_camera()
    w, h = 40, 24
    got = api.render(api.Volume(desc), cam, prm, w, h, steps, 6, jitter_frame=2).cpu().numpy()
    assert _max_err(got, _closed_form(oracle, desc, prm, cam, w, h, rho0, 6)) <= 2e-5


@pytest.mark.parametrize("steps", [1, 2, 3, 8])
def test_basic_rule_homogeneous_closed_form_on_gpu(api, oracle, steps):
    """Basic rule (Sec. 3.1) in a homogeneous slab: the transmittance advanced
    over a step weights that step's light, RGB = L_in sigma D sum_{i=1..N}
    e^{-i sigma D}, summed as a geometric series."""
    rho0 = 0.004
    desc = I.volume_desc("constant", rho0=rho0)
    prm = I.params(tau_max=0.0)
    cam = I.ground_camera()
    w, h = 40, 24
    got = api.render(api.Volume(desc), cam, prm, w, h, steps, 6, jitter_frame=2,
                     integration="basic").cpu().numpy()
    exp = np.zeros((h, w, 4))
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    sigma = rho0 * prm["absorption"]
    for y in range(h):
        for x in range(w):
            d = oracle.pixel_ray(cam, w, h, x, y)
            hit, t0, t1 = oracle.slab_clip(desc, prm, cam["pos"], d)
            if not hit:
                continue
            ph = oracle.hg(float(np.dot(d, s)), prm["hg_g"])
            lin = (np.array(prm["sun_radiance"]) * math.exp(-sigma * 6 * prm["light_step"]) * ph
                   + np.array(prm["ambient"]))
            sd = sigma * (t1 - t0) / steps
            geo = math.exp(-sd) * -math.expm1(-steps * sd) / -math.expm1(-sd)
            exp[y, x, :3], exp[y, x, 3] = lin * sd * geo, -math.expm1(-sigma * (t1 - t0))
    assert exp[..., 3].max() > 0.3
    assert _max_err(got, exp) <= 2e-5


def test_telescoping_no_sun_on_gpu(api):
    desc = I.volume_desc("full", seed=3)
    prm = I.params(sun_radiance=(0.0, 0.0, 0.0))
    got = api.render(api.Volume(desc), I.orbit_camera(0, 3), prm, 160, 90, 8, 6,
                     jitter_frame=4).cpu().numpy().astype(np.float64)
    amb = np.array(prm["ambient"])
    assert _max_err(got[..., :3], got[..., 3:4] * amb) <= 2e-6
    assert got[..., 3].max() > 0.5


@pytest.mark.parametrize("case", ["inside-layer", "looking-down", "no-light-steps", "one-step",
                                  "no-early-out", "horizontal", "above-layer", "above-looking-up",
                                  "on-bottom", "on-top-looking-down", "far-clip",
                                  "horizontal-below"])
def test_edge_cases(api, oracle, case):
    desc = I.volume_desc("full", seed=5)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    prm = I.params()
    cam = I.ground_camera()
    steps, ls = 8, 6
    if case == "inside-layer":
        cam = I.camera((100.0, 200.0, 2600.0), 40.0, 5.0, 60.0)
    elif case == "looking-down":
        cam = I.camera((0.0, 0.0, 500.0), 0.0, -60.0, 40.0)
    elif case == "no-light-steps":
        ls = 0
    elif case == "one-step":
        steps = 1
    elif case == "no-early-out":
        prm = I.params(tau_max=0.0)
    elif case == "horizontal":
        cam = I.camera((0.0, 0.0, 2000.0), 10.0, 0.0, 50.0)
    elif case == "above-layer":  # enters from the top; rays near the horizon miss
        cam = I.camera((300.0, -200.0, 6000.0), 70.0, -25.0, 70.0)
    elif case == "above-looking-up":  # every ray misses (quick test from above)
        cam = I.camera((300.0, -200.0, 6000.0), 70.0, 30.0, 40.0)
    elif case == "on-bottom":  # camera exactly on the layer bottom
        cam = I.camera((50.0, 80.0, 1500.0), 15.0, 20.0, 60.0)
    elif case == "on-top-looking-down":  # exactly on the top, looking into the layer
        cam = I.camera((50.0, 80.0, 4000.0), 200.0, -30.0, 60.0)
    elif case == "far-clip":  # shallow rays: t_max = 40 km ends most marches
        cam = I.camera((0.0, 0.0, 0.0), 30.0, 3.0, 10.0)
    elif case == "horizontal-below":  # the middle row is exactly horizontal and misses
        cam = I.camera((0.0, 0.0, 500.0), 10.0, 0.0, 50.0)
    w, h = 33, 17
    got = api.render(vol, cam, prm, w, h, steps, ls, jitter_frame=1).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, prm, w, h, steps, ls, jitter_frame=1, nthreads=8)
    assert _max_err(got, ref) <= TOL_FP32
    if case in ("looking-down", "above-looking-up"):
        assert np.all(got == 0.0)
    if case == "above-layer":
        assert ref[..., 3].max() > 0.5 and (ref[..., 3] == 0).any()
    if case == "horizontal-below":
        assert np.all(got[h // 2] == 0.0)


def test_lookup_count_matches_oracle(api, oracle):
    wl = I.workload("plain-tiny")
    vol, ovol = api.Volume(wl.volume), oracle.Volume(wl.volume)
    cam = I.ground_camera()
    _, ctr = api.render(vol, cam, I.params(), 64, 48, 16, 6, count=True)
    _, n = oracle.render(ovol, cam, I.params(), 64, 48, 16, 6)
    # the two sides may disagree on a handful of near-threshold rho > 0 / early-out decisions
    assert abs(int(ctr.item()) - n) <= 0.001 * n


def test_invalid_arguments_raise(api):
    import torch
    from paper_1609_05344_gb300._native import CloudError
    vol = api.Volume(I.volume_desc("tiny"))
    out = torch.empty((8, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(CloudError):
        api.render(vol, I.ground_camera(), I.params(), 8, 8, 0, 6, out=out)
    with pytest.raises(CloudError):
        api.render(vol, I.ground_camera(), I.params(), 8, 8, 8, 33, out=out)
    with pytest.raises(CloudError):
        api.render(vol, I.ground_camera(), I.params(sun_dir=(0.0, 1.0, -0.2)), 8, 8, 8, 6, out=out)
    with pytest.raises(CloudError):
        api.Volume(I.volume_desc("tiny", base_n=100))


def test_per_frame_jitter_mode(api, oracle):
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    prm = I.params(jitter_mode="frame")
    cam = I.orbit_camera(2, 3)
    got = api.render(vol, cam, prm, 80, 45, 8, 6, jitter_frame=9).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, prm, 80, 45, 8, 6, jitter_frame=9, nthreads=8)
    assert _max_err(got, ref) <= TOL_FP32


@pytest.mark.parametrize("ls", [1, 3, 32])
def test_generic_light_step_counts(api, oracle, ls):
    # light-step counts other than 6 use the generic (runtime-length) light loop
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    cam = I.orbit_camera(6, 3)
    prm = I.params(light_step=40.0)
    got = api.render(vol, cam, prm, 64, 36, 8, ls, jitter_frame=6).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, prm, 64, 36, 8, ls, jitter_frame=6, nthreads=8)
    assert _max_err(got, ref) <= TOL_FP32


def test_maximum_sizes(api, oracle):
    desc = I.volume_desc("full", seed=3)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    cam = I.camera((0.0, 0.0, 500.0), 0.0, 25.0, 40.0)
    # widest image (16384 x 3: a ragged row of tiles) and the most view steps
    wide = api.render(vol, cam, I.params(), 16384, 3, 8, 6, jitter_frame=1).cpu().numpy()
    xs = np.array([0, 1, 8191, 16383, 12345, 16382])
    ys = np.array([0, 2, 1, 2, 0, 1])
    ref, _ = oracle.render_pixels(ovol, cam, I.params(), 16384, 3, 8, 6, xs, ys, jitter_frame=1)
    assert _max_err(wide[ys, xs], ref) <= TOL_FP32
    deep = api.render(vol, cam, I.params(tau_max=0.0), 6, 4, 4096, 6).cpu().numpy()
    ref, _ = oracle.render(ovol, cam, I.params(tau_max=0.0), 6, 4, 4096, 6, nthreads=8)
    assert _max_err(deep, ref) <= TOL_FP32


def test_random_cameras_and_settings(api, oracle):
    """Seeded random cameras (inside, below and above the layer, any yaw, pitch
    from -70 to 80 degrees, fov 15-100), step counts, light steps, offsets and
    integration rules on small ragged images, against the oracle at 1e-4."""
    rng = np.random.default_rng(2024)
    desc = I.volume_desc("full", seed=9)
    vol, ovol = api.Volume(desc), oracle.Volume(desc)
    worst = 0.0
    for _ in range(24):
        cam = I.camera((float(rng.uniform(-5000, 5000)), float(rng.uniform(-5000, 5000)),
                        float(rng.choice([rng.uniform(0, 1400), rng.uniform(1600, 3900),
                                          rng.uniform(4100, 7000)]))),
                       float(rng.uniform(0, 360)), float(rng.uniform(-70, 80)),
                       float(rng.uniform(15, 100)))
        w, h = int(rng.integers(1, 24)), int(rng.integers(1, 16))
        steps, ls = int(rng.integers(1, 25)), int(rng.integers(0, 9))
        frame = int(rng.integers(-1, 50))
        integ = str(rng.choice(["analytic", "basic"]))
        prm = I.params(jitter_mode=str(rng.choice(["pixel", "frame"])))
        got = api.render(vol, cam, prm, w, h, steps, ls, jitter_frame=frame,
                         integration=integ).cpu().numpy()
        ref, _ = oracle.render(ovol, cam, prm, w, h, steps, ls, jitter_frame=frame,
                               integration=oracle.ANALYTIC if integ == "analytic" else oracle.BASIC,
                               nthreads=8)
        worst = max(worst, _max_err(got, ref))
    assert worst <= TOL_FP32
