"""Randomised invariants of the oracle (property-based; skipped where the
hypothesis package is absent).  Each draws cameras, seeds, step counts,
offsets and lighting and checks identities that hold for every input:

* telescoping (no sun): RGB = A * alpha, since the per-step weights
  e^{-tau_{i-1}} (1 - e^{-s_i}) sum to 1 - e^{-tau_N} (Sec. 3.1 analytic rule);
* alpha is lighting-independent: two renders that differ only in the sun and
  ambient colours have the same alpha;
* colour is linear in the lights: the render with sun E and ambient A equals
  the sum of the renders with (E, 0) and (0, A);
* the TAA output lies in the current frame's 3x3 range or equals the current
  value (off screen / first frame)."""
import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

_cams = st.tuples(st.floats(-3000, 3000), st.floats(-3000, 3000), st.floats(0, 5500),
                  st.floats(0, 360), st.floats(-60, 75), st.floats(20, 90))


def _cam(c):
    x, y, z, yaw, pitch, fov = c
    return I.camera((x, y, z), yaw, pitch, fov)


_VOLS = {}


def _vol(oracle, seed):
    """One full-tile volume per seed (building the FP64 tiles is the slow part)."""
    if seed not in _VOLS:
        _VOLS[seed] = oracle.Volume(I.volume_desc("full", seed=seed))
    return _VOLS[seed]


@settings(max_examples=25, deadline=None)
@given(c=_cams, seed=st.integers(1, 3), steps=st.integers(1, 24), frame=st.integers(-1, 40))
def test_telescoping_random(oracle, c, seed, steps, frame):
    prm = I.params(sun_radiance=(0.0, 0.0, 0.0))
    img, _ = oracle.render(_vol(oracle, seed), _cam(c), prm, 5, 4, steps, 6, jitter_frame=frame)
    assert np.allclose(img[..., :3], img[..., 3:4] * np.array(prm["ambient"]), atol=1e-12, rtol=0)


@settings(max_examples=20, deadline=None)
@given(c=_cams, seed=st.integers(1, 3), steps=st.integers(1, 16),
       sun=st.tuples(st.floats(0, 5), st.floats(0, 5), st.floats(0, 5)),
       amb=st.tuples(st.floats(0, 1), st.floats(0, 1), st.floats(0, 1)))
def test_alpha_independent_and_colour_linear_in_lights(oracle, c, seed, steps, sun, amb):
    vol, cam = _vol(oracle, seed), _cam(c)

    def render(e, a):
        img, _ = oracle.render(vol, cam, I.params(sun_radiance=e, ambient=a), 4, 3, steps, 6,
                               jitter_frame=2)
        return img
    both, sun_only, amb_only = render(sun, amb), render(sun, (0, 0, 0)), render((0, 0, 0), amb)
    assert np.array_equal(both[..., 3], sun_only[..., 3])
    assert np.array_equal(both[..., 3], amb_only[..., 3])
    assert np.allclose(both[..., :3], sun_only[..., :3] + amb_only[..., :3], atol=1e-12, rtol=1e-12)


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 10000), h=st.integers(1, 12), w=st.integers(1, 12),
       blend=st.floats(0, 1), first=st.booleans())
def test_taa_output_in_range_or_current(oracle, seed, h, w, blend, first):
    rng = np.random.default_rng(seed)
    hist = None if first else rng.uniform(0, 3, (h, w, 4))
    cur = rng.uniform(0, 1, (h, w, 4))
    mot = rng.uniform(-4, 4, (h, w, 2))
    out = oracle.taa(hist, cur, mot, blend=blend)
    pad = np.pad(cur, ((1, 1), (1, 1), (0, 0)), mode="edge")
    win = np.stack([pad[dy:dy + h, dx:dx + w] for dy in range(3) for dx in range(3)])
    inside = np.all((out >= win.min(0) - 1e-12) & (out <= win.max(0) + 1e-12), axis=-1)
    assert np.all(inside | np.all(out == cur, axis=-1))
