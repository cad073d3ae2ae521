"""Build and load libcloudvol.so, and mirror its C ABI (include/cloudvol.h)
with ctypes.  Argument marshalling only: every computation runs in the CUDA
kernels of the library.  There is no fallback: if the library is missing or
fails to load, the calls raise.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
CSRC = os.path.join(_HERE, "csrc")
BUILD_DIR = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_HERE, "libcloudvol.so")
# the checked build (kernels verify their index ranges into a status word; for
# tests), loaded instead of the normal library when CLOUDVOL_CHECKED=1
CHECKED_BUILD_DIR = os.path.join(_HERE, "_build_checked")
CHECKED_LIB_PATH = os.path.join(_HERE, "libcloudvol_checked.so")
HEADER = os.path.join(_ROOT, "include", "cloudvol.h")
SOURCES = ["volume.cu", "render.cu", "batch.cu", "march8_view.cu", "march16_view.cu",
           "march8_batch.cu", "march16_batch.cu", "taa.cu", "session.cu", "server.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", ARCH, "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr"]

# status codes and enumerations (include/cloudvol.h)
OK = 0
ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5
PRECISION = {"fp32": 0, "fp16": 1, "bf16": 2, "unorm16": 3}
DENSITY = {"noise": 0, "constant": 1}
INTEGRATION = {"analytic": 0, "basic": 1}
HISTORY = {"fp32": 0, "fp16": 1}
JITTER = {"pixel": 0, "frame": 1}
MAX_LIGHT_STEPS, MAX_STEPS, MAX_DIM, MAX_VIEWS, STATIC_MAX_VIEWS = 32, 4096, 16384, 4096, 256
TUNE_CONFIGS = 8  # launch configurations: tile shape + 4 * (view steps per iteration: 8, 16)


def config_parts(config: int):
    """(tile shape, view steps per warp iteration) of a launch configuration."""
    return config % 4, (8, 16)[config // 4]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (in parallel) and link the library
    (with checked=True the checked build, into its own directory and file)."""
    build_dir = CHECKED_BUILD_DIR if checked else BUILD_DIR
    lib_path = CHECKED_LIB_PATH if checked else LIB_PATH
    flags = NVCC_FLAGS + (["-DCLOUDVOL_CHECKED=1"] if checked else [])
    os.makedirs(build_dir, exist_ok=True)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [
        os.path.join(CSRC, h) for h in ("common.cuh", "march.cuh", "march_kernels.cuh")] + [HEADER]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest:
        return lib_path
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose:
                print(log)
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


class VolumeDesc(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("base_n", ctypes.c_int32), ("detail_n", ctypes.c_int32),
                ("weather_n", ctypes.c_int32), ("detail_weight", ctypes.c_double),
                ("base_period_m", ctypes.c_double), ("detail_period_m", ctypes.c_double),
                ("weather_period_m", ctypes.c_double), ("coverage", ctypes.c_double),
                ("slab_lo_m", ctypes.c_double), ("slab_hi_m", ctypes.c_double),
                ("density_mode", ctypes.c_int32), ("constant_density", ctypes.c_double),
                ("precision", ctypes.c_int32)]


_D3 = ctypes.c_double * 3


class Camera(ctypes.Structure):
    _fields_ = [("pos", _D3), ("forward", _D3), ("right", _D3), ("up", _D3),
                ("tan_half_fovy", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("sun_dir", _D3), ("sun_radiance", _D3), ("ambient", _D3), ("hg_g", ctypes.c_double),
                ("absorption_per_m", ctypes.c_double), ("light_step_m", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("t_max_m", ctypes.c_double),
                ("jitter_mode", ctypes.c_int32)]


class View(ctypes.Structure):
    _fields_ = [("camera", Camera), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("steps", ctypes.c_int32), ("jitter_frame", ctypes.c_int32),
                ("out_rgba", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch_views", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("max_sessions", ctypes.c_int32), ("history_fmt", ctypes.c_int32),
                ("blend", ctypes.c_float), ("reserve_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("session", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class ServerCounters(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("batched_views", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("open_sessions", ctypes.c_int32), ("session_bytes", ctypes.c_uint64)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_P = ctypes.POINTER
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)

# (name, restype, argtypes) for every entry point declared in include/cloudvol.h
SIGNATURES = [
    ("cloud_status_string", ctypes.c_char_p, [_i]),
    ("cloud_last_error_message", ctypes.c_char_p, []),
    ("cloud_volume_create", _i, [_P(VolumeDesc), _vp, _P(_vp)]),
    ("cloud_volume_destroy", _i, [_vp]),
    ("cloud_volume_export", _i, [_vp, _vp, _vp, _vp, _vp]),
    ("cloud_render", _i, [_vp, _P(Camera), _P(Params), _i, _i, _i, _i, _i, _i, _vp, _vp]),
    ("cloud_render_count", _i, [_vp, _P(Camera), _P(Params), _i, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    ("cloud_motion", _i, [_vp, _P(Params), _P(Camera), _P(Camera), _i, _i, _vp, _vp]),
    ("taa_resolve", _i, [_vp, _vp, _vp, _vp, _i, _i, _i, ctypes.c_float, _vp]),
    ("cloud_taa_reproject", _i, [_vp, _P(Params), _P(Camera), _P(Camera), _vp, _vp, _vp, _i, _i, _i,
                                 ctypes.c_float, _vp]),
    ("cloud_device_wait_timeouts", _i, [_P(ctypes.c_uint), _i]),
    ("cloud_composite", _i, [_vp, _i, _i, _i, _vp, _vp, _i, _i, _vp]),
    ("cloud_session_create", _i, [_vp, _i, _i, _i, _P(_vp)]),
    ("cloud_session_destroy", _i, [_vp]),
    ("cloud_session_frame", _i, [_vp, _P(Camera), _P(Params), _i, _i, _i, ctypes.c_float, _vp,
                                 _P(_vp), _vp]),
    ("cloud_session_reset", _i, [_vp]),
    ("cloud_session_frame_async", _i, [_vp, _P(Camera), _P(Params), _i, _i, _i, ctypes.c_float,
                                       _vp, _ip, _vp]),
    ("cloud_session_wait_frame", _i, [_vp, _i, _i]),
    ("cloud_session_snapshot_bytes", _i, [_vp, _P(ctypes.c_size_t)]),
    ("cloud_session_snapshot", _i, [_vp, _vp, ctypes.c_size_t, _vp]),
    ("cloud_session_restore", _i, [_vp, _vp, ctypes.c_size_t, _vp]),
    ("cloud_hash4_batch", _i, [_vp, ctypes.c_int64, _vp, _vp]),
    ("cloud_debug_set_wait_polls", _i, [_i]),
    ("cloud_debug_set_occupancy", _i, [_i]),
    ("cloud_debug_check_status", _i, [_P(ctypes.c_uint), _i]),
    ("cloud_volume_occupancy", _i, [_vp, _vp, ctypes.c_int64, _ip, _vp]),
    ("cloud_get_launch_config", _i, [_i, _i, _P(_i)]),
    ("cloud_set_launch_config", _i, [_i, _i, _i]),
    ("cloud_autotune_render", _i, [_vp, _P(Camera), _P(Params), _i, _i, _i, _i, _i, _i, _vp, _i,
                                   _fp, _ip, _vp]),
    ("cloud_batch_create", _i, [_vp, _P(Params), _i, _i, _P(View), _i, _P(_vp)]),
    ("cloud_batch_destroy", _i, [_vp]),
    ("cloud_batch_set_views", _i, [_vp, _P(View), _i, _vp]),
    ("cloud_batch_render", _i, [_vp, _vp]),
    ("cloud_batch_render_graph", _i, [_vp, _vp]),
    ("cloud_batch_render_per_view", _i, [_vp, _vp]),
    ("cloud_batch_autotune", _i, [_vp, _i, _fp, _ip, _vp]),
    ("cloud_batch_render_static", _i, [_vp, _P(Params), _i, _i, _P(View), _i, _vp]),
    ("cloud_server_create", _i, [_vp, _P(Params), _i, _P(ServerConfig), _P(_vp)]),
    ("cloud_server_destroy", _i, [_vp]),
    ("cloud_server_open_session", _i, [_vp, _i, _i, _ip]),
    ("cloud_server_close_session", _i, [_vp, _i]),
    ("cloud_server_submit", _i, [_vp, _i, _P(Camera), _i, _P(ctypes.c_uint64)]),
    ("cloud_server_wait", _i, [_vp, ctypes.c_uint64, _i, _P(RequestInfo)]),
    ("cloud_server_session_output", _i, [_vp, _i, _P(_vp)]),
    ("cloud_server_copy_output", _i, [_vp, _i, _vp, ctypes.c_size_t]),
    ("cloud_server_pause", _i, [_vp, _i]),
    ("cloud_server_stats", _i, [_vp, _P(ServerCounters)]),
]

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = CHECKED_LIB_PATH if os.environ.get("CLOUDVOL_CHECKED") == "1" else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        h = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
        return h


class CloudError(RuntimeError):
    def __init__(self, status: int, where: str):
        l = lib()
        msg = l.cloud_last_error_message().decode() or l.cloud_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def check(status: int, where: str):
    if status != OK:
        raise CloudError(status, where)


def volume_desc(d: dict) -> VolumeDesc:
    return VolumeDesc(int(d.get("seed", 0)) & 0xFFFFFFFF, int(d.get("base_n", 0)),
                      int(d.get("detail_n", 0)), int(d.get("weather_n", 0)),
                      float(d.get("detail_weight", 0.0)), float(d.get("base_period", 6400.0)),
                      float(d.get("detail_period", 800.0)), float(d.get("weather_period", 40000.0)),
                      float(d.get("coverage", 0.5)), float(d.get("slab_lo", 1500.0)),
                      float(d.get("slab_hi", 4000.0)), DENSITY[d.get("density_mode", "noise")],
                      float(d.get("constant_density", 0.0)), PRECISION[d.get("precision", "fp32")])


def camera(c: dict) -> Camera:
    return Camera(_D3(*c["pos"]), _D3(*c["forward"]), _D3(*c["right"]), _D3(*c["up"]),
                  float(c["tan_half_fovy"]))


def params(p: dict) -> Params:
    return Params(_D3(*p["sun_dir"]), _D3(*p["sun_radiance"]), _D3(*p["ambient"]), float(p["hg_g"]),
                  float(p["absorption"]), float(p["light_step"]), float(p["tau_max"]),
                  float(p["t_max"]), JITTER[p.get("jitter_mode", "pixel")])
