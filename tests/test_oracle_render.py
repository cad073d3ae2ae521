"""Pins for the oracle's raymarch: phase function, camera rays, slab clipping
and the integration rules of Sec. 3.1.

* Henyey-Greenstein (Sec. 1): normalisation and mean cosine by quadrature.
* Homogeneous slab: with density rho0 everywhere, the analytic rule gives
  RGB = L_in (1 - e^{-rho0 alpha (t1 - t0)}) for EVERY step count and jitter
  (the step-length independence claimed in Sec. 3.1 / Fig. 2); the basic rule
  S = T L does not, and converges to it as the step shrinks.
* Basic rule, homogeneous slab: the transmittance advanced over a step weights
  that step's light, so RGB = L_in sigma D sum_{i=1..N} e^{-i sigma D} (a
  geometric series, summed in closed form).
* Telescoping: with no sun, RGB = A * alpha exactly for any density field.
* Beer-Lambert (Sec. 1): alpha = 1 - exp(-alpha D sum_i rho_i), independent
  of the lighting.
* Convergence: analytic and basic rules approach the same limit as N grows.
* By hand: one and two (jittered) view steps of a pixel written out from the
  method's formulas, sharing only the separately pinned density and hash with
  the oracle, pin the light-march placement and sum and the step chaining;
  every pixel of small images recomputed the same way pins the assembled
  image, the early out and the lookup count.
"""
import math

import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I


@pytest.mark.parametrize("g", [0.0, 0.3, 0.6, -0.5, 0.85])
def test_hg_normalised_and_mean_cosine(oracle, g):
    mu, w = np.polynomial.legendre.leggauss(400)
    p = np.array([oracle.hg(m, g) for m in mu])
    assert 2 * math.pi * np.sum(w * p) == pytest.approx(1.0, abs=1e-9)
    assert 2 * math.pi * np.sum(w * mu * p) == pytest.approx(g, abs=1e-9)


def test_hg_isotropic_and_forward_peak(oracle):
    for m in (-1.0, -0.2, 0.5, 1.0):
        assert oracle.hg(m, 0.0) == pytest.approx(1.0 / (4 * math.pi), abs=1e-15)
    assert oracle.hg(1.0, 0.6) > oracle.hg(0.0, 0.6) > oracle.hg(-1.0, 0.6)


def test_centre_pixel_is_forward_and_edge_angle(oracle):
    cam = I.camera((1.0, 2.0, 500.0), 33.0, 20.0, 60.0)
    d = oracle.pixel_ray(cam, 101, 51, 50, 25)
    assert np.allclose(d, cam["forward"], atol=1e-15)
    # top row, centre column: tan(angle to forward) = (1 - 1/H) tan(fovy/2) along up
    d = oracle.pixel_ray(cam, 101, 51, 50, 0)
    f, u = np.array(cam["forward"]), np.array(cam["up"])
    assert np.dot(d, u) / np.dot(d, f) == pytest.approx((1 - 1 / 51) * math.tan(math.radians(30)),
                                                        rel=1e-13)
    # rightmost column: aspect ratio applies
    d = oracle.pixel_ray(cam, 101, 51, 100, 25)
    r = np.array(cam["right"])
    assert np.dot(d, r) / np.dot(d, f) == pytest.approx(
        (1 - 1 / 101) * (101 / 51) * math.tan(math.radians(30)), rel=1e-13)
    assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-15)


def test_slab_clip_cases(oracle):
    desc, prm = I.volume_desc("tiny"), I.params()
    up = np.array([0.0, math.cos(math.radians(30)), math.sin(math.radians(30))])
    hit, t0, t1 = oracle.slab_clip(desc, prm, (0, 0, 500.0), up)
    assert hit and t0 == pytest.approx(2000.0) and t1 == pytest.approx(7000.0)
    hit, _, _ = oracle.slab_clip(desc, prm, (0, 0, 500.0), -up)
    assert not hit
    flat = np.array([1.0, 0.0, 0.0])
    hit, t0, t1 = oracle.slab_clip(desc, prm, (0, 0, 2000.0), flat)
    assert hit and t0 == 0.0 and t1 == prm["t_max"]
    hit, _, _ = oracle.slab_clip(desc, prm, (0, 0, 500.0), flat)
    assert not hit
    hit, t0, t1 = oracle.slab_clip(desc, prm, (0, 0, 2000.0), up)   # inside the layer
    assert hit and t0 == 0.0 and t1 == pytest.approx(4000.0)
    grazing = np.array([math.cos(0.03), 0.0, math.sin(0.03)])      # clipped by t_max
    hit, t0, t1 = oracle.slab_clip(desc, prm, (0, 0, 500.0), grazing)
    assert hit and t0 == pytest.approx(1000.0 / math.sin(0.03)) and t1 == prm["t_max"]


def _closed_form_pixel(oracle, desc, prm, cam, w, h, x, y, rho0, light_steps):
    d = oracle.pixel_ray(cam, w, h, x, y)
    hit, t0, t1 = oracle.slab_clip(desc, prm, cam["pos"], d)
    if not hit:
        return np.zeros(4)
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    tau_sun = rho0 * prm["absorption"] * light_steps * prm["light_step"]
    ph = oracle.hg(float(np.dot(d, s)), prm["hg_g"])
    l_in = np.array(prm["sun_radiance"]) * math.exp(-tau_sun) * ph + np.array(prm["ambient"])
    a = -math.expm1(-rho0 * prm["absorption"] * (t1 - t0))
    return np.concatenate([l_in * a, [a]])


@pytest.mark.parametrize("steps", [1, 2, 3, 8, 16, 128])
@pytest.mark.parametrize("jitter_frame", [-1, 0, 5])
def test_homogeneous_slab_closed_form(oracle, steps, jitter_frame):
    rho0 = 0.004
    desc = I.volume_desc("constant", rho0=rho0)
    prm = I.params(tau_max=0.0)
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    w, h = 24, 16
    img, _ = oracle.render(vol, cam, prm, w, h, steps, 6, jitter_frame=jitter_frame)
    hits = 0
    for y in range(h):
        for x in range(w):
            exp = _closed_form_pixel(oracle, desc, prm, cam, w, h, x, y, rho0, 6)
            assert np.allclose(img[y, x], exp, atol=1e-12, rtol=0), (x, y)
            hits += exp[3] > 0
    assert hits > w * h // 3


def _basic_closed_form_pixel(oracle, desc, prm, cam, w, h, x, y, rho0, light_steps, n):
    """Basic rule (Sec. 3.1: the transmittance is advanced over a step before it
    weights that step's light) in a homogeneous slab, summed in closed form: with
    q = e^{-sigma D}, RGB = L_in sigma D (q + q^2 + ... + q^N)
    = L_in sigma D q (1 - q^N) / (1 - q); alpha = 1 - q^N.  Weighting by the
    transmittance before the step instead would drop one factor q."""
    d = oracle.pixel_ray(cam, w, h, x, y)
    hit, t0, t1 = oracle.slab_clip(desc, prm, cam["pos"], d)
    if not hit:
        return np.zeros(4)
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    tau_sun = rho0 * prm["absorption"] * light_steps * prm["light_step"]
    ph = oracle.hg(float(np.dot(d, s)), prm["hg_g"])
    l_in = np.array(prm["sun_radiance"]) * math.exp(-tau_sun) * ph + np.array(prm["ambient"])
    sd = rho0 * prm["absorption"] * (t1 - t0) / n
    q = math.exp(-sd)
    geo = q * -math.expm1(-n * sd) / -math.expm1(-sd)
    return np.concatenate([l_in * sd * geo, [-math.expm1(-rho0 * prm["absorption"] * (t1 - t0))]])


@pytest.mark.parametrize("steps", [1, 2, 3, 8])
@pytest.mark.parametrize("jitter_frame", [-1, 4])
def test_basic_rule_homogeneous_closed_form(oracle, steps, jitter_frame):
    rho0 = 0.004
    desc = I.volume_desc("constant", rho0=rho0)
    prm = I.params(tau_max=0.0)
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    w, h = 24, 16
    img, _ = oracle.render(vol, cam, prm, w, h, steps, 6, jitter_frame=jitter_frame,
                           integration=oracle.BASIC)
    hits = 0
    for y in range(h):
        for x in range(w):
            exp = _basic_closed_form_pixel(oracle, desc, prm, cam, w, h, x, y, rho0, 6, steps)
            assert np.allclose(img[y, x], exp, atol=1e-12, rtol=0), (x, y)
            hits += exp[3] > 0.3
    assert hits > w * h // 4


def test_basic_rule_depends_on_step_length(oracle):
    rho0 = 0.004
    desc = I.volume_desc("constant", rho0=rho0)
    prm = I.params(tau_max=0.0)
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    ref = _closed_form_pixel(oracle, desc, prm, cam, 8, 8, 4, 1, rho0, 6)
    errs = []
    for n in (2, 8, 32, 128, 512):
        img, _ = oracle.render(vol, cam, prm, 8, 8, n, 6, integration=oracle.BASIC)
        errs.append(np.abs(img[1, 4, :3] - ref[:3]).max())
    assert errs[0] > 0.05                           # visibly darker with few steps (Fig. 2)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < errs[0] / 100                 # first-order convergence in the step length


@pytest.mark.parametrize("jitter_frame", [-1, 3])
def test_telescoping_no_sun(oracle, jitter_frame):
    desc = I.volume_desc("tiny", seed=1)
    prm = I.params(sun_radiance=(0.0, 0.0, 0.0))
    vol = oracle.Volume(desc)
    img, _ = oracle.render(vol, I.ground_camera(), prm, 32, 24, 8, 6, jitter_frame=jitter_frame)
    amb = np.array(prm["ambient"])
    assert np.allclose(img[..., :3], img[..., 3:4] * amb, atol=1e-12, rtol=0)
    assert img[..., 3].max() > 0.5


def test_alpha_is_beer_lambert_of_density_sum(oracle):
    desc = I.volume_desc("tiny", seed=1)
    prm = I.params(tau_max=0.0)
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    w, h, n = 16, 12, 8
    img, _ = oracle.render(vol, cam, prm, w, h, n, 6, jitter_frame=2)
    img2, _ = oracle.render(vol, cam, I.params(tau_max=0.0, sun_radiance=(5, 0, 1), hg_g=-0.2,
                                               ambient=(0, 1, 0)), w, h, n, 6, jitter_frame=2)
    assert np.array_equal(img[..., 3], img2[..., 3])
    for (x, y) in [(3, 2), (8, 6), (15, 11), (0, 0)]:
        d = oracle.pixel_ray(cam, w, h, x, y)
        hit, t0, t1 = oracle.slab_clip(desc, prm, cam["pos"], d)
        if not hit:
            assert img[y, x, 3] == 0.0
            continue
        D = (t1 - t0) / n
        u = oracle.jitter(desc["seed"], x, y, 2)
        rho = sum(vol.density(np.array(cam["pos"]) + (t0 + (i + u) * D) * d) for i in range(n))
        assert img[y, x, 3] == pytest.approx(-math.expm1(-prm["absorption"] * D * rho), abs=1e-13)


def test_early_out_bound(oracle):
    desc = I.volume_desc("tiny", seed=1)
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    a, n_on = oracle.render(vol, cam, I.params(), 32, 32, 64, 6)
    b, n_off = oracle.render(vol, cam, I.params(tau_max=0.0), 32, 32, 64, 6)
    assert n_on < n_off
    # after tau >= 11.5 the rest of the ray carries at most e^-11.5 of the radiance
    lmax = 2.0 * oracle.hg(1.0, 0.6) + 0.3
    assert np.abs(a - b).max() <= math.exp(-11.5) * lmax


@pytest.mark.slow
def test_convergence_in_step_count(oracle):
    desc = I.volume_desc("tiny", seed=1)
    prm = I.params(tau_max=0.0)
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    w = h = 8
    ref, _ = oracle.render(vol, cam, prm, w, h, 4096, 6, nthreads=4)
    basic, _ = oracle.render(vol, cam, prm, w, h, 4096, 6, integration=oracle.BASIC, nthreads=4)
    errs = []
    for n in (256, 512, 1024, 2048):
        img, _ = oracle.render(vol, cam, prm, w, h, n, 6, nthreads=4)
        errs.append(np.abs(img - ref).max())
    assert all(b < a for a, b in zip(errs, errs[1:]))
    # the two rules differ by O(D): at N = 4096 they agree closely
    assert np.abs(basic - ref).max() < 5e-3
    assert np.abs(basic - ref).max() < np.abs(
        oracle.render(vol, cam, prm, w, h, 256, 6, integration=oracle.BASIC, nthreads=4)[0] - ref).max()


def test_per_frame_jitter_shares_one_offset(oracle):
    # Sec. 4: one random offset shared by all rays of a frame; every pixel
    # uses the offset of pixel (0, 0); alpha = 1 - exp(-alpha D sum rho(t0 + (i+u) D))
    desc = I.volume_desc("tiny", seed=1)
    prm = I.params(tau_max=0.0, jitter_mode="frame")
    vol = oracle.Volume(desc)
    cam = I.ground_camera()
    w, h, n = 12, 9, 8
    img, _ = oracle.render(vol, cam, prm, w, h, n, 6, jitter_frame=5)
    u = oracle.jitter(desc["seed"], 0, 0, 5)
    for (x, y) in [(3, 2), (11, 8), (6, 4)]:
        d = oracle.pixel_ray(cam, w, h, x, y)
        hit, t0, t1 = oracle.slab_clip(desc, prm, cam["pos"], d)
        if not hit:
            continue
        D = (t1 - t0) / n
        rho = sum(vol.density(np.array(cam["pos"]) + (t0 + (i + u) * D) * d) for i in range(n))
        assert img[y, x, 3] == pytest.approx(-math.expm1(-prm["absorption"] * D * rho), abs=1e-13)
    pix, _ = oracle.render(vol, cam, I.params(tau_max=0.0), w, h, n, 6, jitter_frame=5)
    assert not np.allclose(pix, img)  # per-pixel jitter differs


@pytest.mark.parametrize("light_steps", [1, 6, 32])
def test_one_step_pixel_by_hand(oracle, light_steps):
    """One view step of one pixel, written out from Sec. 1 / Sec. 3.1 with the
    oracle's (separately pinned) density as the only shared piece: the view
    sample at the middle of the layer segment, light samples at
    p + (j + 1/2) dl s towards the sun (zero density above the layer), tau_sun =
    alpha dl sum rho_j, L_in = E e^{-tau_sun} p_HG(d.s) + A, and the analytic
    step C = L_in (1 - e^{-alpha rho D}).  Pins the light-march placement,
    direction and sum, which a constant-density slab cannot see."""
    desc = I.volume_desc("full", seed=7)
    vol = oracle.Volume(desc)
    prm = I.params()
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    checked = above = 0
    for yaw in range(0, 360, 5):
        for pitch in (8.0, 20.0, 45.0):
            cam = I.camera((0.0, 0.0, 500.0), float(yaw), pitch, 60.0)
            d = oracle.pixel_ray(cam, 1, 1, 0, 0)
            o = np.array(cam["pos"])
            hit, t0, t1 = oracle.slab_clip(desc, prm, o, d)
            if not hit:
                continue
            D = t1 - t0
            p = o + (t0 + 0.5 * D) * d
            rho = vol.density(p)
            if rho <= 0.0:
                continue
            qs = [p + (j + 0.5) * prm["light_step"] * s for j in range(light_steps)]
            above += sum(q[2] > desc["slab_hi"] for q in qs)
            tau_sun = prm["absorption"] * prm["light_step"] * sum(vol.density(q) for q in qs)
            lin = (np.array(prm["sun_radiance"]) * math.exp(-tau_sun) *
                   oracle.hg(float(np.dot(d, s)), prm["hg_g"]) + np.array(prm["ambient"]))
            a = -math.expm1(-prm["absorption"] * rho * D)
            want = np.concatenate([lin * a, [a]])
            got, _ = oracle.render(vol, cam, prm, 1, 1, 1, light_steps, nthreads=1)
            assert np.allclose(got[0, 0], want, rtol=1e-12, atol=1e-14), (yaw, pitch)
            checked += 1
    assert checked >= 10
    if light_steps == 32:
        assert above > 0  # some light samples left the layer (density 0 there)


def test_two_jittered_steps_by_hand(oracle):
    """Two view steps with the Sec. 3.2 offset, by hand: samples at
    t0 + (i + u) D with u the pixel's jitter value, each step's light from its
    own light march, and the second step attenuated by the first's optical
    depth (C = L_1 (1 - e^{-s_1}) + e^{-s_1} L_2 (1 - e^{-s_2}), s_i = alpha rho_i D)."""
    desc = I.volume_desc("full", seed=7)
    vol = oracle.Volume(desc)
    prm = I.params()
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    al, dl = prm["absorption"], prm["light_step"]
    checked = 0
    for yaw in range(0, 360, 7):
        cam = I.camera((0.0, 0.0, 500.0), float(yaw), 12.0, 60.0)
        w = h = 3
        x, y, frame = 2, 1, 5
        d = oracle.pixel_ray(cam, w, h, x, y)
        o = np.array(cam["pos"])
        hit, t0, t1 = oracle.slab_clip(desc, prm, o, d)
        if not hit:
            continue
        u = oracle.jitter(desc["seed"], x, y, frame)
        D = (t1 - t0) / 2
        ph = oracle.hg(float(np.dot(d, s)), prm["hg_g"])
        c, tau = np.zeros(3), 0.0
        for i in range(2):
            p = o + (t0 + (i + u) * D) * d
            rho = vol.density(p)
            if rho <= 0.0:
                continue
            tsun = al * dl * sum(vol.density(p + (j + 0.5) * dl * s) for j in range(6))
            lin = np.array(prm["sun_radiance"]) * math.exp(-tsun) * ph + np.array(prm["ambient"])
            c += math.exp(-tau) * lin * -math.expm1(-al * rho * D)
            tau += al * rho * D
        want = np.concatenate([c, [-math.expm1(-tau)]])
        got, _ = oracle.render(vol, cam, prm, w, h, 2, 6, jitter_frame=frame, nthreads=1)
        assert np.allclose(got[y, x], want, rtol=1e-12, atol=1e-14), yaw
        checked += tau > 0
    assert checked >= 5


def _pixel_by_hand(oracle, vol, desc, prm, cam, w, h, x, y, n, ls, frame, basic):
    """One pixel of Sec. 1 / Sec. 3.1 / Sec. 3.2 written out: view samples at
    t0 + (i + u) D, a light march of ls samples towards the sun where the view
    density is positive, L_in = E e^{-tau_sun} p_HG + A, the analytic (or basic)
    step, and the early out once tau reaches tau_max.  Returns RGBA and the
    number of density lookups (view samples walked plus light samples)."""
    s = np.array(prm["sun_dir"]) / np.linalg.norm(prm["sun_dir"])
    al, dl = prm["absorption"], prm["light_step"]
    d = oracle.pixel_ray(cam, w, h, x, y)
    o = np.array(cam["pos"])
    hit, t0, t1 = oracle.slab_clip(desc, prm, o, d)
    if not hit:
        return np.zeros(4), 0
    u = oracle.jitter(desc["seed"], x, y, frame) if frame >= 0 else 0.5
    D = (t1 - t0) / n
    ph = oracle.hg(float(np.dot(d, s)), prm["hg_g"])
    c, tau, looks = np.zeros(3), 0.0, 0
    for i in range(n):
        p = o + (t0 + (i + u) * D) * d
        rho = vol.density(p)
        looks += 1
        if rho > 0.0:
            tsun = al * dl * sum(vol.density(p + (j + 0.5) * dl * s) for j in range(ls))
            looks += ls
            lin = np.array(prm["sun_radiance"]) * math.exp(-tsun) * ph + np.array(prm["ambient"])
            sd = al * rho * D
            if basic:
                c += math.exp(-(tau + sd)) * sd * lin
            else:
                c += math.exp(-tau) * lin * -math.expm1(-sd)
            tau += sd
        if tau >= prm["tau_max"]:
            break
    return np.concatenate([c, [-math.expm1(-tau)]]), looks


@pytest.mark.parametrize("pos,yaw,pitch", [((0.0, 0.0, 500.0), 30.0, 14.0),
                                           ((300.0, -200.0, 2600.0), 200.0, -4.0),
                                           ((0.0, 0.0, 6000.0), 120.0, -28.0)])
@pytest.mark.parametrize("tau_max,basic", [(11.5, False), (0.7, False), (11.5, True)])
def test_small_images_by_hand(oracle, pos, yaw, pitch, tau_max, basic):
    """Every pixel of small jittered images, camera below, inside and above the
    layer, recomputed from the method's formulas with only the separately
    pinned pieces (pixel ray, layer clip, jitter hash, density, HG) shared with
    the oracle: pins the assembled image -- sample placement, light marches,
    step chaining, both integration rules, the early out (tau_max = 0.7 trips
    it) and the lookup count -- to 1e-12."""
    desc = I.volume_desc("full", seed=11)
    vol = oracle.Volume(desc)
    prm = I.params(tau_max=tau_max)
    cam = I.camera(pos, yaw, pitch, 70.0)
    w, h, n, ls, frame = 7, 5, 8, 6, 3
    integ = oracle.BASIC if basic else oracle.ANALYTIC
    got, n_got = oracle.render(vol, cam, prm, w, h, n, ls, jitter_frame=frame, integration=integ)
    n_want, lit, early = 0, 0, 0
    for y in range(h):
        for x in range(w):
            want, looks = _pixel_by_hand(oracle, vol, desc, prm, cam, w, h, x, y, n, ls, frame, basic)
            n_want += looks
            lit += want[3] > 0
            early += looks < n * (1 + ls) and want[3] >= -math.expm1(-tau_max)
            assert np.allclose(got[y, x], want, rtol=1e-12, atol=1e-14), (x, y)
    assert n_got == n_want
    assert lit >= 10  # most pixels see cloud
    if tau_max < 1.0:
        assert early >= 2  # the early out ended rays
