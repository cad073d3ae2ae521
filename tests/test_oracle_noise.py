"""Pins for the oracle's noise volumes and density (the sampled density of Sec. 1).

Lattice exactness ties fBm values to the hash; zero second differences at odd
voxels pin plain (fade-free) trilinear interpolation and the octave cell counts;
periodicity pins the wrap; texel-centre sampling pins the half-texel offset
and the x-fastest layout; the height-profile knots pin g(h).
"""
import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I

OCT_KEY = 0x9E37


def _lattice_value(oracle, seed, salt, o, ix, iy, iz, m):
    return oracle.unit(oracle.hash4(ix % m, iy % m, iz % m, seed ^ (o * OCT_KEY) ^ salt))


@pytest.mark.parametrize("n", [16, 32, 64])
def test_fbm_lattice_exact(oracle, n):
    seed, salt = 77, oracle.SALT_BASE
    # at voxels that are multiples of 16 every octave coordinate k*M_o/N is an integer
    for k in [(0, 0, 0), (16, 0, 0), (0, 16, 16), (n - 16, 16 % n, 0)]:
        expect = 0.0
        for o in range(4):
            m = (n // 16) << o
            c = [kk * m // n for kk in k]
            expect += 0.5 ** o * _lattice_value(oracle, seed, salt, o, *c, m)
        expect /= 1.875
        assert oracle.fbm3(seed, salt, n, k) == pytest.approx(expect, abs=1e-15)


def test_fbm_piecewise_linear_no_fade(oracle):
    # knots of octave o for N=64 are at multiples of 16/2^o >= 2: at odd x the
    # second difference of a sum of trilinear (not smoothstep) cells vanishes
    n, seed, salt = 64, 5, oracle.SALT_BASE
    for ky, kz in [(3, 7), (10, 1), (33, 60)]:
        for kx in range(1, n, 2):
            f = [oracle.fbm3(seed, salt, n, (kx + d, ky, kz)) for d in (-1, 0, 1)]
            assert abs(f[0] - 2 * f[1] + f[2]) < 1e-14
        # and the second difference is not zero everywhere (the knots exist)
    f = [oracle.fbm3(seed, salt, n, (8 + d, 3, 7)) for d in (-2, 0, 2)]
    assert abs(f[0] - 2 * f[1] + f[2]) > 1e-6


def test_fbm_periodic_and_in_range(oracle):
    n = 32
    for k in [(0, 0, 0), (5, 9, 31), (31, 31, 31)]:
        v = oracle.fbm3(9, oracle.SALT_DETAIL, n, k)
        assert 0.0 <= v < 1.0
        assert oracle.fbm3(9, oracle.SALT_DETAIL, n, (k[0] + n, k[1], k[2] - n)) == v
    v2 = oracle.fbm2(9, oracle.SALT_WEATHER, 64, (3, 4))
    assert oracle.fbm2(9, oracle.SALT_WEATHER, 64, (3 + 64, 4 - 128)) == v2


def test_weather_lattice_exact(oracle):
    n, seed, salt = 64, 21, oracle.SALT_WEATHER
    expect = 0.0
    for o in range(4):
        m = (n // 16) << o
        expect += 0.5 ** o * oracle.unit(oracle.hash4(32 * m // n % m, 16 * m // n % m, 0,
                                                      seed ^ (o * OCT_KEY) ^ salt))
    assert oracle.fbm2(seed, salt, n, (32, 16)) == pytest.approx(expect / 1.875, abs=1e-15)


def test_volume_arrays_layout(oracle):
    d = I.volume_desc("tiny", seed=4, base_n=16)
    v = oracle.Volume(d)
    b = v.base
    assert b.shape == (16, 16, 16)
    for (x, y, z) in [(1, 2, 3), (15, 0, 7), (4, 11, 0)]:
        assert b[z, y, x] == oracle.fbm3(4, oracle.SALT_BASE, 16, (x, y, z))
    assert 0.0 <= b.min() and b.max() < 1.0


def test_height_gradient_knots(oracle):
    d = I.volume_desc("tiny")
    lo, hi = d["slab_lo"], d["slab_hi"]
    th = hi - lo
    cases = [(lo - 10, 0.0), (lo, 0.0), (lo + 0.05 * th, 0.5), (lo + 0.1 * th, 1.0),
             (lo + 0.6 * th, 1.0), (lo + 0.8 * th, 0.5), (hi, 0.0), (hi + 5, 0.0)]
    for z, g in cases:
        assert oracle.height_gradient(d, z) == pytest.approx(g, abs=1e-12)


def test_density_texel_centres_and_remap(oracle):
    d = I.volume_desc("tiny", seed=6, base_n=16)
    v = oracle.Volume(d)
    b = v.base
    vox = d["base_period"] / 16
    # pick voxels whose centre lies in the full-density band of the layer
    for (x, y) in [(1, 2), (7, 7), (13, 4)]:
        for z in range(16):
            zc = (z + 0.5) * vox
            g = oracle.height_gradient(d, zc)
            if g != 1.0:
                continue
            p = ((x + 0.5) * vox, (y + 0.5) * vox, zc)
            expect = max(0.0, (b[z, y, x] - 0.5) / 0.5)
            assert v.density(p) == pytest.approx(expect, abs=1e-12)
            # wrap: one tile over in x and y samples the same texel
            q = (p[0] + d["base_period"], p[1] - 3 * d["base_period"], zc)
            assert v.density(q) == pytest.approx(expect, abs=1e-12)


def test_density_trilinear_midpoint(oracle):
    d = I.volume_desc("tiny", seed=6, base_n=64)
    v = oracle.Volume(d)
    b = v.base
    vox = d["base_period"] / 64
    checked = 0
    for z in range(20, 36):
        zc = (z + 0.5) * vox
        if oracle.height_gradient(d, zc) != 1.0:
            continue
        for y in range(0, 64, 7):
            for x in range(63):
                if b[z, y, x] > 0.5 and b[z, y, x + 1] > 0.5:
                    p = ((x + 1.0) * vox, (y + 0.5) * vox, zc)
                    expect = ((b[z, y, x] + b[z, y, x + 1]) / 2 - 0.5) / 0.5
                    assert v.density(p) == pytest.approx(expect, abs=1e-12)
                    checked += 1
    assert checked > 10


def test_density_full_volume_components(oracle):
    # 16^3 base (400 m texels), 16^3 detail (50 m texels), 16^2 weather (2500 m texels)
    d = I.volume_desc("full", seed=2, base_n=16, detail_n=16, weather_n=16)
    v = oracle.Volume(d)
    b, dt, w = v.base, v.detail, v.weather
    p = (200.0, 600.0, 3000.0)            # base texel centre (0, 1, 7); g(3000 m) = 1
    assert oracle.height_gradient(d, p[2]) == 1.0
    # detail coordinates 3.5, 11.5, 59.5: half-way between texels on every axis
    dsum = 0.125 * sum(dt[(11 + dz) % 16, (11 + dy) % 16, (3 + dx) % 16]
                       for dz in (0, 1) for dy in (0, 1) for dx in (0, 1))
    # weather coordinates 200/2500*16 - 1/2 = 0.78, 600/2500*16 - 1/2 = 3.34
    sx, sy = 200.0 / 2500.0 * 16 - 0.5, 600.0 / 2500.0 * 16 - 0.5
    ix, iy = int(np.floor(sx)), int(np.floor(sy))
    fx, fy = sx - ix, sy - iy
    wv = ((1 - fy) * ((1 - fx) * w[iy % 16, ix % 16] + fx * w[iy % 16, (ix + 1) % 16])
          + fy * ((1 - fx) * w[(iy + 1) % 16, ix % 16] + fx * w[(iy + 1) % 16, (ix + 1) % 16]))
    expect = wv * max(0.0, (b[7, 1, 0] - 0.3 * dsum - 0.5) / 0.5)
    assert v.density(p) == pytest.approx(expect, abs=1e-12)


def test_density_constant_mode(oracle):
    v = oracle.Volume(I.volume_desc("constant", rho0=0.37))
    for p in [(0, 0, 0), (1e4, -3e3, 2500.0), (5, 5, 1e5)]:
        assert v.density(p) == 0.37
