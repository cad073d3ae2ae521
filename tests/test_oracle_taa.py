"""Pins for the oracle's reprojection motion and TAA resolve (Sec. 3.2).

Motion: a static camera gives zero motion; a sideways translation moves a
point at depth z by f * dx / z pixels; a pure yaw moves the centre pixel by
f * tan(yaw) pixels (f = W / (2 aspect tan(fovy/2)) the focal length in pixels).
TAA: an unchanged frame is a fixed point; an integer motion is an exact texel
shift; the clamped output stays inside the current frame's 3x3 range; with the
clamp off and no motion the resolve is the exponential moving average
out_n = b sum_k (1-b)^k c_{n-k} + (1-b)^n c_0.
"""
import math

import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I


def test_static_camera_zero_motion(oracle):
    cam = I.orbit_camera(4)
    m = oracle.motion(I.volume_desc("tiny"), I.params(), cam, cam, 40, 30)
    assert np.abs(m).max() < 1e-9


def test_translation_motion_closed_form(oracle):
    w, h = 41, 31
    cur = I.camera((0.0, 0.0, 500.0), 0.0, 30.0, 60.0)
    dx = 7.0
    prev = dict(cur, pos=tuple(np.array(cur["pos"]) - dx * np.array(cur["right"])))
    m = oracle.motion(I.volume_desc("tiny"), I.params(), prev, cur, w, h)
    # centre pixel looks along forward and enters the layer at 1000 / sin 30 = 2000 m
    f_px = w / (2 * (w / h) * cur["tan_half_fovy"])
    assert m[15, 20, 0] == pytest.approx(-f_px * dx / 2000.0, rel=1e-12)
    assert m[15, 20, 1] == pytest.approx(0.0, abs=1e-9)


def test_yaw_motion_closed_form(oracle):
    w, h = 41, 31
    delta = 0.4
    prev = I.camera((10.0, 20.0, 500.0), 30.0, 0.0, 60.0)
    cur = I.camera((10.0, 20.0, 500.0), 30.0 + delta, 0.0, 60.0)
    m = oracle.motion(I.volume_desc("tiny"), I.params(), prev, cur, w, h)
    f_px = w / (2 * (w / h) * cur["tan_half_fovy"])
    assert m[15, 20, 0] == pytest.approx(f_px * math.tan(math.radians(delta)), rel=1e-12)
    assert m[15, 20, 1] == pytest.approx(0.0, abs=1e-9)


def test_point_behind_previous_camera(oracle):
    prev = I.camera((0.0, 0.0, 500.0), 180.0, 20.0, 60.0)
    cur = I.camera((0.0, 0.0, 500.0), 0.0, 20.0, 60.0)
    m = oracle.motion(I.volume_desc("tiny"), I.params(), prev, cur, 16, 8)
    assert np.all(m == 1e9)


def test_taa_identity_and_first_frame(oracle):
    rng = np.random.default_rng(1)
    c = I.synthetic_frame(rng, 20, 30).astype(np.float64)
    zero = np.zeros((20, 30, 2))
    assert np.array_equal(oracle.taa(c, c, zero), c)
    assert np.array_equal(oracle.taa(None, c, zero), c)


def test_taa_integer_shift(oracle):
    rng = np.random.default_rng(2)
    hst = I.synthetic_frame(rng, 20, 30).astype(np.float64)
    c = I.synthetic_frame(rng, 20, 30).astype(np.float64)
    mot = np.zeros((20, 30, 2))
    mot[..., 0], mot[..., 1] = 2.0, -1.0
    out = oracle.taa(hst, c, mot, blend=0.1, clamp=False)
    # pixel (x, y) reads history at (x - 2, y + 1)
    exp = 0.9 * hst[1:, :-2] + 0.1 * c[:-1, 2:]
    assert np.allclose(out[:-1, 2:], exp, atol=1e-15, rtol=0)


def test_taa_half_pixel_bilinear(oracle):
    rng = np.random.default_rng(3)
    hst = I.synthetic_frame(rng, 10, 12).astype(np.float64)
    c = I.synthetic_frame(rng, 10, 12).astype(np.float64)
    mot = np.zeros((10, 12, 2))
    mot[..., 0] = 0.5
    out = oracle.taa(hst, c, mot, blend=0.25, clamp=False)
    exp = 0.75 * 0.5 * (hst[:, :-1] + hst[:, 1:]) + 0.25 * c[:, 1:]
    assert np.allclose(out[:, 1:], exp, atol=1e-15, rtol=0)


def test_taa_clamp_bounds_and_offscreen(oracle):
    rng = np.random.default_rng(4)
    h, w = 24, 32
    hst = I.synthetic_frame(rng, h, w).astype(np.float64) * 3.0
    c = I.synthetic_frame(rng, h, w).astype(np.float64)
    mot = I.synthetic_motion(rng, h, w).astype(np.float64)
    out = oracle.taa(hst, c, mot)
    pad = np.pad(c, ((1, 1), (1, 1), (0, 0)), mode="edge")
    win = np.stack([pad[dy:dy + h, dx:dx + w] for dy in range(3) for dx in range(3)])
    mn, mx = win.min(axis=0), win.max(axis=0)
    assert np.all(out >= mn - 1e-15) and np.all(out <= mx + 1e-15)
    qx = np.arange(w)[None, :] + 0.5 - mot[..., 0]
    qy = np.arange(h)[:, None] + 0.5 - mot[..., 1]
    off = (qx < 0) | (qx > w) | (qy < 0) | (qy > h)
    assert off.sum() > 0
    assert np.array_equal(out[off], c[off])


def test_taa_ema_closed_form(oracle):
    rng = np.random.default_rng(5)
    frames = [I.synthetic_frame(rng, 8, 10).astype(np.float64) for _ in range(12)]
    zero = np.zeros((8, 10, 2))
    b = 0.1
    hist = None
    for c in frames:
        hist = oracle.taa(hist, c, zero, blend=b, clamp=False)
    n = len(frames) - 1
    exp = (1 - b) ** n * frames[0] + sum(b * (1 - b) ** k * frames[n - k] for k in range(n))
    assert np.allclose(hist, exp, atol=1e-13, rtol=0)


def test_composite_pins(oracle):
    rng = np.random.default_rng(8)
    cloud = I.synthetic_frame(rng, 10, 16).astype(np.float64)
    bg = rng.uniform(0, 1, (20, 32, 4))
    out = oracle.composite(cloud, bg)
    # exact 2x upsample: output pixel (2i+1/2.., ) centres fall at +-1/4 texel; pixel (1,1)
    # samples the cloud at (0.25, 0.25): weights 0.75/0.25 of texels 0 and 1
    c = 0.5625 * cloud[0, 0] + 0.1875 * (cloud[0, 1] + cloud[1, 0]) + 0.0625 * cloud[1, 1]
    assert np.allclose(out[1, 1], c + (1 - c[3]) * bg[1, 1], atol=1e-15)
    # transparent cloud leaves the background; same size is a plain "over"
    assert np.allclose(oracle.composite(np.zeros((4, 4, 4)), bg[:4, :4]), bg[:4, :4])
    same = oracle.composite(cloud, bg[:10, :16])
    assert np.allclose(same, cloud + (1 - cloud[..., 3:4]) * bg[:10, :16], atol=1e-15)
