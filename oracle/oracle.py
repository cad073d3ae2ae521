"""Python face of the FP64 CPU oracle (``cloud_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, double-precision
restatement of the cloud raymarch and TAA resolve of Toft, Bowles and
Zimmermann, "Optimisations for Real-Time Volumetric Cloudscapes" (Sec. 1,
Sec. 3.1, Sec. 3.2).  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library: inputs arrive as plain dictionaries of numbers, and the C source is
compiled here with gcc into ``oracle/_build``.

Parity status of each function (what pins it, tests/test_oracle_*.py):
  hash / jitter      PCG permutation inverted exactly; uniformity; avalanche
  noise volumes      lattice exactness, periodicity, range, interpolation
  density            height-profile knots, remap threshold, texel centres
  HG phase           normalisation, g=0 isotropy, mean cosine = g (quadrature)
  pixel ray / slab   centre pixel = forward, closed-form slab crossing
  render (analytic)  homogeneous-slab closed form for every N and jitter;
                     telescoping identity RGB = A * alpha with E_sun = 0;
                     alpha = 1 - exp(-alpha D sum rho); convergence in N
  render (basic)     convergence to the analytic limit; step dependence
  motion             static camera = 0; closed-form translation and yaw
  TAA                identity, integer shift, clamp bounds, EMA closed form
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cloud_oracle.c")
_HDR = os.path.join(_HERE, "cloud_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libcloud_oracle.so")

ANALYTIC = 0
BASIC = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB_PATH) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
               "-shared", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _VolDesc(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("base_n", ctypes.c_int), ("detail_n", ctypes.c_int),
                ("weather_n", ctypes.c_int), ("detail_weight", ctypes.c_double),
                ("base_period", ctypes.c_double), ("detail_period", ctypes.c_double),
                ("weather_period", ctypes.c_double), ("coverage", ctypes.c_double),
                ("slab_lo", ctypes.c_double), ("slab_hi", ctypes.c_double),
                ("density_mode", ctypes.c_int), ("constant_density", ctypes.c_double)]


class _Vol(ctypes.Structure):
    _fields_ = [("d", _VolDesc), ("base", ctypes.POINTER(ctypes.c_double)),
                ("detail", ctypes.POINTER(ctypes.c_double)),
                ("weather", ctypes.POINTER(ctypes.c_double))]


_D3 = ctypes.c_double * 3


class _Cam(ctypes.Structure):
    _fields_ = [("pos", _D3), ("forward", _D3), ("right", _D3), ("up", _D3),
                ("tan_half_fovy", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("sun_dir", _D3), ("sun_radiance", _D3), ("ambient", _D3),
                ("hg_g", ctypes.c_double), ("absorption", ctypes.c_double),
                ("light_step", ctypes.c_double), ("tau_max", ctypes.c_double),
                ("t_max", ctypes.c_double), ("jitter_mode", ctypes.c_int)]


_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_ip = _P(ctypes.c_int)
_up = _P(ctypes.c_uint32)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_pcg.argtypes = [ctypes.c_uint32]
        lib.orc_pcg.restype = ctypes.c_uint32
        lib.orc_hash4.argtypes = [ctypes.c_uint32] * 4
        lib.orc_hash4.restype = ctypes.c_uint32
        lib.orc_hash4_batch.argtypes = [_up, ctypes.c_long, _up]
        lib.orc_hash4_batch.restype = None
        lib.orc_unit.argtypes = [ctypes.c_uint32]
        lib.orc_unit.restype = ctypes.c_double
        lib.orc_volume_build.argtypes = [_P(_VolDesc), _P(_Vol)]
        lib.orc_volume_build.restype = ctypes.c_int
        lib.orc_volume_free.argtypes = [_P(_Vol)]
        lib.orc_volume_free.restype = None
        lib.orc_fbm3.argtypes = [ctypes.c_uint32, ctypes.c_uint32] + [ctypes.c_int] * 4
        lib.orc_fbm3.restype = ctypes.c_double
        lib.orc_fbm2.argtypes = [ctypes.c_uint32, ctypes.c_uint32] + [ctypes.c_int] * 3
        lib.orc_fbm2.restype = ctypes.c_double
        lib.orc_height_gradient.argtypes = [_P(_VolDesc), ctypes.c_double]
        lib.orc_height_gradient.restype = ctypes.c_double
        lib.orc_density.argtypes = [_P(_Vol), _dp]
        lib.orc_density.restype = ctypes.c_double
        lib.orc_hg.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_hg.restype = ctypes.c_double
        lib.orc_pixel_ray.argtypes = [_P(_Cam), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _dp]
        lib.orc_pixel_ray.restype = None
        lib.orc_slab_clip.argtypes = [_P(_VolDesc), _P(_Params), _dp, _dp, _dp, _dp]
        lib.orc_slab_clip.restype = ctypes.c_int
        lib.orc_jitter.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_jitter.restype = ctypes.c_double
        lib.orc_render_pixel.argtypes = [_P(_Vol), _P(_Cam), _P(_Params)] + [ctypes.c_int] * 8 + [
            _dp, _P(ctypes.c_longlong)]
        lib.orc_render_pixel.restype = None
        lib.orc_render.argtypes = [_P(_Vol), _P(_Cam), _P(_Params)] + [ctypes.c_int] * 7 + [_dp]
        lib.orc_render.restype = ctypes.c_longlong
        lib.orc_render_pixels.argtypes = [_P(_Vol), _P(_Cam), _P(_Params)] + [ctypes.c_int] * 6 + [
            _ip, _ip, ctypes.c_int, ctypes.c_int, _dp]
        lib.orc_render_pixels.restype = ctypes.c_longlong
        lib.orc_motion_pixel.argtypes = [_P(_VolDesc), _P(_Params), _P(_Cam), _P(_Cam)] + [
            ctypes.c_int] * 4 + [_dp]
        lib.orc_motion_pixel.restype = None
        lib.orc_motion.argtypes = [_P(_VolDesc), _P(_Params), _P(_Cam), _P(_Cam), ctypes.c_int,
                                   ctypes.c_int, _dp]
        lib.orc_motion.restype = None
        lib.orc_taa.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, _dp]
        lib.orc_taa.restype = None
        lib.orc_taa_pixel.argtypes = [_dp, _dp, _dp] + [ctypes.c_int] * 4 + [
            ctypes.c_double, ctypes.c_int, _dp]
        lib.orc_taa_pixel.restype = None
        lib.orc_composite.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                      ctypes.c_int, _dp]
        lib.orc_composite.restype = None
        _lib = lib
        return lib


def _vec3(v):
    return _D3(*[float(a) for a in v])


def _desc(d: dict) -> _VolDesc:
    mode = d.get("density_mode", "noise")
    return _VolDesc(int(d.get("seed", 0)) & 0xFFFFFFFF, int(d.get("base_n", 0)),
                    int(d.get("detail_n", 0)), int(d.get("weather_n", 0)),
                    float(d.get("detail_weight", 0.0)), float(d.get("base_period", 6400.0)),
                    float(d.get("detail_period", 800.0)), float(d.get("weather_period", 40000.0)),
                    float(d.get("coverage", 0.5)), float(d.get("slab_lo", 1500.0)),
                    float(d.get("slab_hi", 4000.0)), 1 if mode == "constant" else 0,
                    float(d.get("constant_density", 0.0)))


def _cam(c: dict) -> _Cam:
    return _Cam(_vec3(c["pos"]), _vec3(c["forward"]), _vec3(c["right"]), _vec3(c["up"]),
                float(c["tan_half_fovy"]))


def _params(p: dict) -> _Params:
    return _Params(_vec3(p["sun_dir"]), _vec3(p["sun_radiance"]), _vec3(p["ambient"]),
                   float(p["hg_g"]), float(p["absorption"]), float(p["light_step"]),
                   float(p["tau_max"]), float(p["t_max"]),
                   1 if p.get("jitter_mode", "pixel") == "frame" else 0)


def _ptr(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def pcg(v: int) -> int:
    return int(_load().orc_pcg(v & 0xFFFFFFFF))


def hash4(a: int, b: int, c: int, d: int) -> int:
    return int(_load().orc_hash4(a & 0xFFFFFFFF, b & 0xFFFFFFFF, c & 0xFFFFFFFF, d & 0xFFFFFFFF))


def hash4_batch(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1, 4)
    out = np.empty(keys.shape[0], dtype=np.uint32)
    _load().orc_hash4_batch(_ptr(keys, ctypes.c_uint32), keys.shape[0], _ptr(out, ctypes.c_uint32))
    return out


def unit(h: int) -> float:
    return float(_load().orc_unit(h & 0xFFFFFFFF))


def fbm3(seed: int, salt: int, n: int, k) -> float:
    return float(_load().orc_fbm3(seed & 0xFFFFFFFF, salt, n, int(k[0]), int(k[1]), int(k[2])))


def fbm2(seed: int, salt: int, n: int, k) -> float:
    return float(_load().orc_fbm2(seed & 0xFFFFFFFF, salt, n, int(k[0]), int(k[1])))


SALT_BASE, SALT_DETAIL, SALT_WEATHER = 0xB45E, 0xDE7A, 0x3EA7


def hg(mu: float, g: float) -> float:
    return float(_load().orc_hg(mu, g))


def jitter(seed: int, x: int, y: int, frame: int) -> float:
    return float(_load().orc_jitter(seed & 0xFFFFFFFF, x, y, frame))


def height_gradient(desc: dict, z: float) -> float:
    d = _desc(desc)
    return float(_load().orc_height_gradient(ctypes.byref(d), z))


def pixel_ray(cam: dict, width: int, height: int, x: int, y: int) -> np.ndarray:
    out = np.zeros(3)
    c = _cam(cam)
    _load().orc_pixel_ray(ctypes.byref(c), width, height, x, y, _ptr(out))
    return out


def slab_clip(desc: dict, params: dict, o, d):
    t0 = ctypes.c_double()
    t1 = ctypes.c_double()
    od = np.asarray(o, dtype=np.float64)
    dd = np.asarray(d, dtype=np.float64)
    vd, pp = _desc(desc), _params(params)
    hit = _load().orc_slab_clip(ctypes.byref(vd), ctypes.byref(pp), _ptr(od), _ptr(dd),
                                ctypes.byref(t0), ctypes.byref(t1))
    return bool(hit), t0.value, t1.value


class Volume:
    """FP64 noise volumes built from a descriptor dictionary."""

    def __init__(self, desc: dict):
        lib = _load()
        self.desc = dict(desc)
        self._d = _desc(desc)
        self._v = _Vol()
        rc = lib.orc_volume_build(ctypes.byref(self._d), ctypes.byref(self._v))
        if rc != 0:
            raise ValueError(f"oracle volume build failed ({rc}) for {desc}")

    def close(self):
        if self._v is not None:
            _load().orc_volume_free(ctypes.byref(self._v))
            self._v = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, ptr, n, dims):
        if not ptr:
            return None
        return np.ctypeslib.as_array(ptr, shape=(n ** dims,)).reshape((n,) * dims).copy()

    @property
    def base(self):
        return self._arr(self._v.base, self._d.base_n, 3)

    @property
    def detail(self):
        return self._arr(self._v.detail, self._d.detail_n, 3)

    @property
    def weather(self):
        return self._arr(self._v.weather, self._d.weather_n, 2)

    def density(self, p) -> float:
        pd = np.asarray(p, dtype=np.float64)
        return float(_load().orc_density(ctypes.byref(self._v), _ptr(pd)))


def render(vol: Volume, cam: dict, params: dict, width: int, height: int, steps: int,
           light_steps: int, jitter_frame: int = -1, integration: int = ANALYTIC,
           nthreads: int = 1):
    """Whole image, (H, W, 4) premultiplied RGBA in float64, plus lookup count."""
    out = np.zeros((height, width, 4), dtype=np.float64)
    c, p = _cam(cam), _params(params)
    n = _load().orc_render(ctypes.byref(vol._v), ctypes.byref(c), ctypes.byref(p), width, height,
                           steps, light_steps, jitter_frame, integration, nthreads, _ptr(out))
    return out, int(n)


def render_pixels(vol: Volume, cam: dict, params: dict, width: int, height: int, steps: int,
                  light_steps: int, xs, ys, jitter_frame: int = -1,
                  integration: int = ANALYTIC, nthreads: int = 1):
    """Selected pixels, (n, 4) float64, plus lookup count."""
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    out = np.zeros((xs.size, 4), dtype=np.float64)
    c, p = _cam(cam), _params(params)
    n = _load().orc_render_pixels(ctypes.byref(vol._v), ctypes.byref(c), ctypes.byref(p), width,
                                  height, steps, light_steps, jitter_frame, integration,
                                  _ptr(xs, ctypes.c_int), _ptr(ys, ctypes.c_int), xs.size,
                                  nthreads, _ptr(out))
    return out, int(n)


def motion(desc: dict, params: dict, prev: dict, cur: dict, width: int, height: int):
    out = np.zeros((height, width, 2), dtype=np.float64)
    d, p, a, b = _desc(desc), _params(params), _cam(prev), _cam(cur)
    _load().orc_motion(ctypes.byref(d), ctypes.byref(p), ctypes.byref(a), ctypes.byref(b), width,
                       height, _ptr(out))
    return out


def taa(history, current, motion_px, blend: float = 0.1, clamp: bool = True):
    """TAA resolve of a whole frame; history None means the first frame."""
    cur = np.ascontiguousarray(current, dtype=np.float64)
    h, w = cur.shape[:2]
    mot = np.ascontiguousarray(motion_px, dtype=np.float64)
    out = np.zeros_like(cur)
    hist_p = None
    if history is not None:
        hist = np.ascontiguousarray(history, dtype=np.float64)
        hist_p = _ptr(hist)
    _load().orc_taa(hist_p, _ptr(cur), _ptr(mot), w, h, blend, 1 if clamp else 0, _ptr(out))
    return out


def composite(cloud, background):
    """Bilinear upsample of the premultiplied cloud buffer to the background's
    size, laid over it (Sec. 3.2 composite)."""
    c = np.ascontiguousarray(cloud, dtype=np.float64)
    b = np.ascontiguousarray(background, dtype=np.float64)
    out = np.zeros_like(b)
    _load().orc_composite(_ptr(c), c.shape[1], c.shape[0], _ptr(b), b.shape[1], b.shape[0],
                          _ptr(out))
    return out
