"""Seeded synthetic inputs for the cloud raymarch and TAA resolve.

This module only builds input descriptions (volume descriptors, cameras,
lighting constants, synthetic frames and motion fields) from seeds.  It holds
none of the method's arithmetic and imports nothing else from this package,
so both the CUDA path and the independent FP64 checker can be fed from it.

The paper (Toft, Bowles, Zimmermann, arXiv 1609.05344) publishes no scene, so
the workloads below are stand-ins with the shapes the paper describes: a
1920x1080 display (Sec. 4 table), about 128 view steps x 6 light steps for
full quality and 8 jittered steps for the fast path (Sec. 1, Sec. 3.2), a
cloud layer seen from the ground, and a moving camera for TAA.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

# Lighting and march constants shared by every workload.
SUN_DIR = (0.3, 0.2, 0.5)           # towards the sun; normalised by consumers
SUN_RADIANCE = (2.0, 1.9, 1.8)      # colour x intensity of the sun
AMBIENT = (0.20, 0.24, 0.30)        # constant ambient radiance
HG_G = 0.6                          # Henyey-Greenstein asymmetry
ABSORPTION = 0.04                   # alpha, 1/m at density 1
LIGHT_STEP_M = 100.0                # light-march step length
TAU_MAX = 11.5                      # early-out optical depth (alpha >= 1 - 1e-5)
T_MAX_M = 40000.0                   # far clip of a view ray
SLAB_LO_M, SLAB_HI_M = 1500.0, 4000.0


def params(**over) -> dict:
    """Lighting / march constants as a plain dictionary."""
    p = dict(sun_dir=SUN_DIR, sun_radiance=SUN_RADIANCE, ambient=AMBIENT, hg_g=HG_G,
             absorption=ABSORPTION, light_step=LIGHT_STEP_M, tau_max=TAU_MAX, t_max=T_MAX_M,
             jitter_mode="pixel")
    p.update(over)
    return p


def volume_desc(kind: str = "tiny", seed: int = 1, precision: str = "fp32", **over) -> dict:
    """Volume descriptors.

    tiny   : 64^3 base fBm only (coverage 0.5, 6.4 km tile).
    full   : 128^3 base, 32^3 detail subtracted at weight 0.3 (0.8 km tile),
             512^2 weather map tiled over 40 km.
    constant: homogeneous density everywhere (closed-form checks).
    """
    d = dict(seed=seed, base_n=64, detail_n=0, weather_n=0, detail_weight=0.0,
             base_period=6400.0, detail_period=800.0, weather_period=40000.0, coverage=0.5,
             slab_lo=SLAB_LO_M, slab_hi=SLAB_HI_M, density_mode="noise", constant_density=0.0,
             precision=precision)
    if kind == "full":
        d.update(base_n=128, detail_n=32, weather_n=512, detail_weight=0.3)
    elif kind == "constant":
        d.update(density_mode="constant", constant_density=over.pop("rho0", 0.05))
    elif kind != "tiny":
        raise ValueError(kind)
    d.update(over)
    return d


def camera(pos, yaw_deg: float, pitch_deg: float, fovy_deg: float = 60.0) -> dict:
    """Pinhole camera, z up, right-handed; yaw about +z from +x, pitch up."""
    cy, sy = math.cos(math.radians(yaw_deg)), math.sin(math.radians(yaw_deg))
    cp, sp = math.cos(math.radians(pitch_deg)), math.sin(math.radians(pitch_deg))
    fwd = (cp * cy, cp * sy, sp)
    right = (sy, -cy, 0.0)
    up = (right[1] * fwd[2] - right[2] * fwd[1], right[2] * fwd[0] - right[0] * fwd[2],
          right[0] * fwd[1] - right[1] * fwd[0])
    return dict(pos=tuple(float(v) for v in pos), forward=fwd, right=right, up=up,
                tan_half_fovy=math.tan(math.radians(fovy_deg) * 0.5))


def ground_camera() -> dict:
    """Still view from 500 m, pitched 20 degrees up, 60 degree vertical FOV."""
    return camera((0.0, 0.0, 500.0), 0.0, 20.0, 60.0)


@functools.lru_cache(maxsize=None)
def _orbit_start(seed: int) -> float:
    return float(np.random.default_rng(seed).uniform(0.0, 360.0))


def orbit_camera(frame: int, seed: int = 3) -> dict:
    """Seeded orbit: radius 3 km at 500 m height, facing the centre, pitched
    12 degrees up; the orbit angle advances 0.25 degrees per frame."""
    start = _orbit_start(seed)
    phi = start + 0.25 * frame
    pos = (3000.0 * math.cos(math.radians(phi)), 3000.0 * math.sin(math.radians(phi)), 500.0)
    return camera(pos, phi + 180.0, 12.0, 60.0)


@dataclass
class Workload:
    name: str
    width: int
    height: int
    steps: int
    light_steps: int
    jitter: bool
    taa: bool
    frames: int
    volume: dict = field(default_factory=dict)
    integration: str = "analytic"


def workload(name: str, precision: str = "fp32") -> Workload:
    """The three single-view workloads.

    plain-tiny : 128x128, 64^3 fBm, 16 x 6 steps, no jitter, one frame.
    reference  : 1280x720, full volumes, 128 x 6 steps, no jitter.
    fast-1080p : 1920x1080, full volumes, 8 x 6 jittered steps, TAA blend 0.1
                 over a 32-frame seeded orbit.
    """
    if name == "plain-tiny":
        return Workload(name, 128, 128, 16, 6, False, False, 1, volume_desc("tiny", 1, precision))
    if name == "reference":
        return Workload(name, 1280, 720, 128, 6, False, False, 1,
                        volume_desc("full", 2, precision))
    if name == "fast-1080p":
        return Workload(name, 1920, 1080, 8, 6, True, True, 32, volume_desc("full", 3, precision))
    raise ValueError(name)


def synthetic_frame(rng: np.random.Generator, height: int, width: int) -> np.ndarray:
    """Cloud-buffer-like premultiplied RGBA: smooth blobs plus per-pixel noise
    (what 8 jittered steps look like), RGB in [0, 2], alpha in [0, 1]."""
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    a = np.zeros((height, width))
    for _ in range(6):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        r = rng.uniform(0.1, 0.4) * max(width, height)
        a += np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (r * r))
    a = np.clip(a * 0.7 + rng.normal(0.0, 0.15, a.shape), 0.0, 1.0)
    rgb = a[..., None] * rng.uniform(0.4, 2.0, (1, 1, 3)) * (1.0 + rng.normal(0, 0.2, a.shape))[
        ..., None]
    out = np.concatenate([np.clip(rgb, 0.0, 2.0), a[..., None]], axis=-1)
    return out.astype(np.float32)


def synthetic_motion(rng: np.random.Generator, height: int, width: int,
                     max_px: float = 6.0, offscreen_frac: float = 0.02) -> np.ndarray:
    """Smooth random motion field in pixels, with a few off-screen pixels."""
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    m = np.zeros((height, width, 2))
    for k in range(2):
        c = rng.uniform(-1, 1, 4)
        m[..., k] = max_px * (c[0] + c[1] * xx / width + c[2] * yy / height
                              + 0.3 * np.sin(c[3] * 6.0 + xx / 37.0 + yy / 23.0))
    m += rng.normal(0.0, 0.05, m.shape)
    off = rng.uniform(0, 1, (height, width)) < offscreen_frac
    m[off] = 1e9
    return m.astype(np.float32)


def random_views(n: int, seed: int = 4, max_size=(1920, 1080), min_size=(256, 256),
                 steps=(8, 16, 32, 128)) -> list:
    """Uneven multi-view workload: n views with seeded sizes in
    [min_size, max_size], step counts drawn from `steps`, cameras on seeded
    positions below the cloud layer looking up at seeded yaw/pitch."""
    rng = np.random.default_rng(seed)
    views = []
    for i in range(n):
        w = int(rng.integers(min_size[0], max_size[0] + 1))
        h = int(rng.integers(min_size[1], max_size[1] + 1))
        pos = (float(rng.uniform(-20000, 20000)), float(rng.uniform(-20000, 20000)),
               float(rng.uniform(0.0, 1200.0)))
        cam = camera(pos, float(rng.uniform(0, 360)), float(rng.uniform(2.0, 40.0)),
                     float(rng.uniform(40.0, 75.0)))
        views.append(dict(camera=cam, width=w, height=h, steps=int(rng.choice(steps)),
                          jitter_frame=int(rng.integers(0, 1000))))
    return views
