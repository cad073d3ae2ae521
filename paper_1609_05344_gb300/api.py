"""Python binding of libcloudvol.so (include/cloudvol.h).

PyTorch supplies device memory and streams; every computation runs in the
library's CUDA kernels.  Inputs are the plain dictionaries produced by
``inputs.py`` (volume descriptors, cameras, lighting constants).
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _require_cuda(t: torch.Tensor, name: str, dtype=None, shape=None):
    """A kernel reads or writes exactly the elements its sizes imply, on the
    current device: anything else is refused here, before a launch."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise ValueError(f"{name} must be {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")


class _DeviceArray:
    """A library-owned device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 2, "strides": None}


def _device_view(ptr: int, shape, typestr: str) -> torch.Tensor:
    """Zero-copy tensor view of a library-owned device buffer (valid as long as
    the library keeps that buffer)."""
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


def _require_host(t, name: str, nbytes: int):
    """A host buffer the library copies exactly nbytes into."""
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CPU tensor (pinned for asynchronous copies)")
    if t.numel() * t.element_size() != nbytes:
        raise ValueError(f"{name} must hold exactly {nbytes} bytes")


class Volume:
    """A cloud density volume generated on the device (cloud_volume_create)."""

    def __init__(self, desc: dict, stream=None):
        self.desc = dict(desc)
        self._h = ctypes.c_void_p()
        d = N.volume_desc(desc)
        N.check(N.lib().cloud_volume_create(ctypes.byref(d), _stream(stream), ctypes.byref(self._h)),
                "cloud_volume_create")

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise RuntimeError("volume destroyed")
        return self._h

    def close(self):
        if self._h:
            torch.cuda.synchronize()
            N.check(N.lib().cloud_volume_destroy(self._h), "cloud_volume_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def occupancy(self, stream=None):
        """The occupancy grid as a (C, C, C) bool numpy array indexed [z, y, x]
        (cloud_volume_occupancy), or None for a constant-density volume."""
        import numpy as np
        lc = ctypes.c_int()
        N.check(N.lib().cloud_volume_occupancy(self.handle, None, 0, ctypes.byref(lc),
                                               _stream(stream)), "cloud_volume_occupancy")
        if lc.value < 0:
            return None
        cells = 1 << (3 * lc.value)
        words = torch.empty((cells + 31) // 32, dtype=torch.int32, device="cuda")
        N.check(N.lib().cloud_volume_occupancy(self.handle, _ptr(words), words.numel(),
                                               ctypes.byref(lc), _stream(stream)),
                "cloud_volume_occupancy")
        w = words.cpu().numpy().view(np.uint32)
        bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:cells]
        c = 1 << lc.value
        return bits.astype(bool).reshape(c, c, c)

    def export(self, stream=None) -> dict:
        """Noise tiles as float32 CUDA tensors in [0, 1), indexed [z, y, x] / [y, x]."""
        d = self.desc
        out = {}
        if d.get("density_mode", "noise") == "noise":
            n = d["base_n"]
            out["base"] = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
            if d.get("detail_n"):
                m = d["detail_n"]
                out["detail"] = torch.empty((m, m, m), dtype=torch.float32, device="cuda")
            if d.get("weather_n"):
                m = d["weather_n"]
                out["weather"] = torch.empty((m, m), dtype=torch.float32, device="cuda")
        N.check(N.lib().cloud_volume_export(self.handle, _ptr(out.get("base")),
                                            _ptr(out.get("detail")), _ptr(out.get("weather")),
                                            _stream(stream)), "cloud_volume_export")
        return out


def render(vol: Volume, cam: dict, prm: dict, width: int, height: int, steps: int,
           light_steps: int, jitter_frame: int = -1, integration: str = "analytic", out=None,
           count: bool = False, stream=None):
    """Raymarch one image (cloud_render).  Returns an (H, W, 4) float32 CUDA
    tensor of premultiplied RGBA; with count=True also the number of density
    lookups the launch executed (a 1-element int64 CUDA tensor)."""
    if out is None:
        out = torch.empty((height, width, 4), dtype=torch.float32, device="cuda")
    _require_cuda(out, "out", torch.float32, (height, width, 4))
    c, p = N.camera(cam), N.params(prm)
    if count:
        ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
        N.check(N.lib().cloud_render_count(vol.handle, ctypes.byref(c), ctypes.byref(p), width,
                                           height, steps, light_steps, jitter_frame,
                                           N.INTEGRATION[integration], _ptr(out), _ptr(ctr),
                                           _stream(stream)), "cloud_render_count")
        return out, ctr
    N.check(N.lib().cloud_render(vol.handle, ctypes.byref(c), ctypes.byref(p), width, height, steps,
                                 light_steps, jitter_frame, N.INTEGRATION[integration], _ptr(out),
                                 _stream(stream)), "cloud_render")
    return out


def motion(vol: Volume, prm: dict, prev: dict, cur: dict, width: int, height: int, out=None,
           stream=None):
    """Per-pixel reprojection motion (cloud_motion): (H, W, 2) float32."""
    if out is None:
        out = torch.empty((height, width, 2), dtype=torch.float32, device="cuda")
    _require_cuda(out, "out", torch.float32, (height, width, 2))
    a, b, p = N.camera(prev), N.camera(cur), N.params(prm)
    N.check(N.lib().cloud_motion(vol.handle, ctypes.byref(p), ctypes.byref(a), ctypes.byref(b),
                                 width, height, _ptr(out), _stream(stream)), "cloud_motion")
    return out


def taa(history, current: torch.Tensor, motion_px: torch.Tensor, blend: float = 0.1, out=None,
        history_fmt: str = "fp32", stream=None):
    """TAA resolve (taa_resolve).  history None means the first frame.
    history/out are float32 (H, W, 4) or float16 (H, W, 4) per history_fmt."""
    _require_cuda(current, "current", torch.float32)
    if current.dim() != 3 or current.shape[2] != 4:
        raise ValueError("current must have shape (H, W, 4)")
    h, w = current.shape[:2]
    dt = torch.float32 if history_fmt == "fp32" else torch.float16
    if out is None:
        out = torch.empty((h, w, 4), dtype=dt, device="cuda")
    _require_cuda(motion_px, "motion", torch.float32, (h, w, 2))
    _require_cuda(out, "out", dt, (h, w, 4))
    if history is not None:
        _require_cuda(history, "history", dt, (h, w, 4))
    N.check(N.lib().taa_resolve(_ptr(history), _ptr(current), _ptr(motion_px), _ptr(out), w, h,
                                N.HISTORY[history_fmt], float(blend), _stream(stream)),
            "taa_resolve")
    return out


def taa_reproject(vol: Volume, prm: dict, prev, cur: dict, history, current: torch.Tensor,
                  blend: float = 0.1, out=None, history_fmt: str = "fp32", stream=None):
    """Motion (prev -> cur) and TAA resolve fused (cloud_taa_reproject); history
    None is a first frame."""
    _require_cuda(current, "current", torch.float32)
    if current.dim() != 3 or current.shape[2] != 4:
        raise ValueError("current must have shape (H, W, 4)")
    h, w = current.shape[:2]
    dt = torch.float32 if history_fmt == "fp32" else torch.float16
    if out is None:
        out = torch.empty((h, w, 4), dtype=dt, device="cuda")
    _require_cuda(out, "out", dt, (h, w, 4))
    if history is not None:
        _require_cuda(history, "history", dt, (h, w, 4))
    pc = N.camera(prev) if prev is not None else None
    c, p = N.camera(cur), N.params(prm)
    N.check(N.lib().cloud_taa_reproject(vol.handle, ctypes.byref(p),
                                        ctypes.byref(pc) if pc is not None else None,
                                        ctypes.byref(c), _ptr(history), _ptr(current), _ptr(out),
                                        w, h, N.HISTORY[history_fmt], float(blend), _stream(stream)),
            "cloud_taa_reproject")
    return out


def composite(cloud: torch.Tensor, background: torch.Tensor, out=None, stream=None):
    """Upsample the premultiplied cloud buffer (float32 or float16 (h, w, 4)) to
    the background's size and lay it over the background (cloud_composite)."""
    _require_cuda(cloud, "cloud", (torch.float32, torch.float16))
    _require_cuda(background, "background", torch.float32)
    if cloud.dim() != 3 or cloud.shape[2] != 4 or background.dim() != 3 or background.shape[2] != 4:
        raise ValueError("cloud and background must have shape (H, W, 4)")
    fmt = "fp32" if cloud.dtype == torch.float32 else "fp16"
    h, w = background.shape[:2]
    if out is None:
        out = torch.empty_like(background)
    _require_cuda(out, "out", torch.float32, (h, w, 4))
    N.check(N.lib().cloud_composite(_ptr(cloud), N.HISTORY[fmt], cloud.shape[1], cloud.shape[0],
                                    _ptr(background), _ptr(out), w, h, _stream(stream)),
            "cloud_composite")
    return out


class Session:
    """One camera's stream of jittered frames resolved by TAA (cloud_session_*)."""

    def __init__(self, vol: Volume, width: int, height: int, history_fmt: str = "fp32"):
        self.vol, self.width, self.height, self.history_fmt = vol, width, height, history_fmt
        self._h = ctypes.c_void_p()
        N.check(N.lib().cloud_session_create(vol.handle, width, height, N.HISTORY[history_fmt],
                                             ctypes.byref(self._h)), "cloud_session_create")

    def close(self):
        if self._h:
            torch.cuda.synchronize()
            N.check(N.lib().cloud_session_destroy(self._h), "cloud_session_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        N.check(N.lib().cloud_session_reset(self._h), "cloud_session_reset")

    def snapshot(self, stream=None) -> bytes:
        """Checkpoint of the session's state (cloud_session_snapshot) as bytes."""
        n = ctypes.c_size_t()
        N.check(N.lib().cloud_session_snapshot_bytes(self._h, ctypes.byref(n)),
                "cloud_session_snapshot_bytes")
        buf = ctypes.create_string_buffer(n.value)
        N.check(N.lib().cloud_session_snapshot(self._h, buf, n.value, _stream(stream)),
                "cloud_session_snapshot")
        return buf.raw

    def restore(self, snap: bytes, stream=None):
        """Load a checkpoint taken by snapshot() (cloud_session_restore)."""
        buf = ctypes.create_string_buffer(bytes(snap), len(snap))
        N.check(N.lib().cloud_session_restore(self._h, buf, len(snap), _stream(stream)),
                "cloud_session_restore")

    def _frame_bytes(self) -> int:
        return self.width * self.height * (16 if self.history_fmt == "fp32" else 8)

    def frame_async(self, cam: dict, prm: dict, steps: int, light_steps: int, host_out,
                    blend: float = 0.1, integration: str = "analytic", stream=None) -> int:
        """Render + resolve one frame and start copying it into host_out on the
        session's copy stream; returns the frame index to pass to wait_frame."""
        _require_host(host_out, "host_out", self._frame_bytes())
        c, p = N.camera(cam), N.params(prm)
        idx = ctypes.c_int()
        N.check(N.lib().cloud_session_frame_async(self._h, ctypes.byref(c), ctypes.byref(p), steps,
                                                  light_steps, N.INTEGRATION[integration],
                                                  float(blend), ctypes.c_void_p(host_out.data_ptr()),
                                                  ctypes.byref(idx), _stream(stream)),
                "cloud_session_frame_async")
        return idx.value

    def wait_frame(self, index: int, timeout_ms: int = 10000):
        N.check(N.lib().cloud_session_wait_frame(self._h, index, timeout_ms),
                "cloud_session_wait_frame")

    def frame(self, cam: dict, prm: dict, steps: int, light_steps: int, blend: float = 0.1,
              integration: str = "analytic", host_out=None, stream=None):
        """Render + motion + resolve one frame.  With host_out (a pinned CPU
        tensor of H*W*4 elements) the resolved frame is copied there and the
        call waits; otherwise returns a CUDA tensor view of the resolved frame
        (valid until the next frame)."""
        if host_out is not None:
            _require_host(host_out, "host_out", self._frame_bytes())
        c, p = N.camera(cam), N.params(prm)
        dev = ctypes.c_void_p()
        hp = ctypes.c_void_p(host_out.data_ptr()) if host_out is not None else ctypes.c_void_p()
        N.check(N.lib().cloud_session_frame(self._h, ctypes.byref(c), ctypes.byref(p), steps,
                                            light_steps, N.INTEGRATION[integration], float(blend),
                                            hp, ctypes.byref(dev), _stream(stream)),
                "cloud_session_frame")
        if host_out is not None:
            return host_out
        return _device_view(dev.value, (self.height, self.width, 4),
                            "<f4" if self.history_fmt == "fp32" else "<f2")


def hash4(keys: torch.Tensor, stream=None) -> torch.Tensor:
    """Device hash of (n, 4) int32/uint32 keys (cloud_hash4_batch) -> (n,) int32 bits."""
    _require_cuda(keys, "keys")
    if keys.element_size() != 4 or keys.shape[-1] != 4:
        raise ValueError("keys must be (n, 4) 32-bit")
    n = keys.numel() // 4
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    N.check(N.lib().cloud_hash4_batch(_ptr(keys), n, _ptr(out), _stream(stream)),
            "cloud_hash4_batch")
    return out


def device_wait_timeouts(reset: bool = False) -> int:
    """Bounded device waits that gave up (cloud_device_wait_timeouts); 0 normally."""
    n = ctypes.c_uint()
    N.check(N.lib().cloud_device_wait_timeouts(ctypes.byref(n), int(reset)),
            "cloud_device_wait_timeouts")
    return n.value


def check_status(reset: bool = False) -> int:
    """Site bits of failed index checks of the checked build
    (cloud_debug_check_status); raises CloudError (unsupported) in a normal build."""
    n = ctypes.c_uint()
    N.check(N.lib().cloud_debug_check_status(ctypes.byref(n), int(reset)), "cloud_debug_check_status")
    return n.value


def set_occupancy(enabled: bool = True):
    """Use of the occupancy grid by the raymarch (cloud_debug_set_occupancy)."""
    N.check(N.lib().cloud_debug_set_occupancy(1 if enabled else 0), "cloud_debug_set_occupancy")


def set_wait_polls(first_polls: int = -1):
    """Poll budget of the fused resolve's first bounded wait for its tile copy
    (cloud_debug_set_wait_polls; -1 restores the default).  For tests of the
    failure reporting."""
    N.check(N.lib().cloud_debug_set_wait_polls(int(first_polls)), "cloud_debug_set_wait_polls")


def launch_config(precision: str, light_steps: int) -> int:
    """The launch configuration renders of this precision and light-step count
    use (cloud_get_launch_config)."""
    c = ctypes.c_int()
    N.check(N.lib().cloud_get_launch_config(N.PRECISION[precision], light_steps, ctypes.byref(c)),
            "cloud_get_launch_config")
    return c.value


def set_launch_config(precision: str, light_steps: int, config: int):
    """Pin the launch configuration (cloud_set_launch_config)."""
    N.check(N.lib().cloud_set_launch_config(N.PRECISION[precision], light_steps, config),
            "cloud_set_launch_config")


def autotune_render(vol: Volume, cam: dict, prm: dict, width: int, height: int, steps: int,
                    light_steps: int, jitter_frame: int = -1, integration: str = "analytic",
                    repeats: int = 5, stream=None):
    """Time every launch configuration (tile shape x view steps per warp
    iteration, see _native.config_parts) on this workload and make the fastest
    the default for the volume's precision (cloud_autotune_render).  Returns
    (best_config, [ms per configuration])."""
    out = torch.empty((height, width, 4), dtype=torch.float32, device="cuda")
    c, p = N.camera(cam), N.params(prm)
    times = (ctypes.c_float * N.TUNE_CONFIGS)()
    best = ctypes.c_int()
    N.check(N.lib().cloud_autotune_render(vol.handle, ctypes.byref(c), ctypes.byref(p), width,
                                          height, steps, light_steps, jitter_frame,
                                          N.INTEGRATION[integration], _ptr(out), repeats, times,
                                          ctypes.byref(best), _stream(stream)),
            "cloud_autotune_render")
    return best.value, list(times)


class Batch:
    """Many views rendered in one persistent launch (cloud_batch_*).

    views: list of dicts {camera, width, height, steps, jitter_frame}; the
    batch allocates one (H, W, 4) float32 output per view (``outputs``)."""

    def __init__(self, vol: Volume, prm: dict, views: list, light_steps: int = 6,
                 integration: str = "analytic"):
        self.vol = vol
        self.outputs = [torch.empty((v["height"], v["width"], 4), dtype=torch.float32,
                                    device="cuda") for v in views]
        self._views = views
        arr = self._array(views)
        self._h = ctypes.c_void_p()
        p = N.params(prm)
        N.check(N.lib().cloud_batch_create(vol.handle, ctypes.byref(p), light_steps,
                                           N.INTEGRATION[integration], arr, len(views),
                                           ctypes.byref(self._h)), "cloud_batch_create")

    def _array(self, views):
        arr = (N.View * len(views))()
        for i, v in enumerate(views):
            arr[i] = N.View(N.camera(v["camera"]), v["width"], v["height"], v["steps"],
                            v.get("jitter_frame", -1), self.outputs[i].data_ptr())
        return arr

    def set_views(self, views: list, stream=None):
        arr = self._array(views)
        N.check(N.lib().cloud_batch_set_views(self._h, arr, len(views), _stream(stream)),
                "cloud_batch_set_views")
        self._views = views

    def render(self, graph: bool = False, stream=None):
        fn = N.lib().cloud_batch_render_graph if graph else N.lib().cloud_batch_render
        N.check(fn(self._h, _stream(stream)), "cloud_batch_render")
        return self.outputs

    def render_per_view(self, stream=None):
        N.check(N.lib().cloud_batch_render_per_view(self._h, _stream(stream)),
                "cloud_batch_render_per_view")
        return self.outputs

    def autotune(self, repeats: int = 3, stream=None):
        """Time every launch configuration on this batch and keep the fastest;
        returns (best_config, [ms per configuration])."""
        times = (ctypes.c_float * N.TUNE_CONFIGS)()
        best = ctypes.c_int()
        N.check(N.lib().cloud_batch_autotune(self._h, repeats, times, ctypes.byref(best),
                                             _stream(stream)), "cloud_batch_autotune")
        return best.value, list(times)

    def close(self):
        if self._h:
            torch.cuda.synchronize()
            N.check(N.lib().cloud_batch_destroy(self._h), "cloud_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching render server (cloud_server_*): many TAA sessions of
    one volume, frames batched into persistent launches as they arrive."""

    def __init__(self, vol: Volume, prm: dict, light_steps: int = 6, max_batch_views: int = 64,
                 slots: int = 2, max_sessions: int = 512, history_fmt: str = "fp16",
                 blend: float = 0.1, reserve_bytes: int = 1 << 30, budget_bytes: int = 0):
        self.vol, self.history_fmt = vol, history_fmt
        cfg = N.ServerConfig(max_batch_views, slots, max_sessions, N.HISTORY[history_fmt],
                             float(blend), reserve_bytes, budget_bytes)
        p = N.params(prm)
        self._h = ctypes.c_void_p()
        N.check(N.lib().cloud_server_create(vol.handle, ctypes.byref(p), light_steps,
                                            ctypes.byref(cfg), ctypes.byref(self._h)),
                "cloud_server_create")
        self.sizes = {}

    def open_session(self, width: int, height: int) -> int:
        sid = ctypes.c_int()
        N.check(N.lib().cloud_server_open_session(self._h, width, height, ctypes.byref(sid)),
                "cloud_server_open_session")
        self.sizes[sid.value] = (width, height)
        return sid.value

    def close_session(self, sid: int):
        N.check(N.lib().cloud_server_close_session(self._h, sid), "cloud_server_close_session")
        self.sizes.pop(sid, None)

    def submit(self, sid: int, cam: dict, steps: int) -> int:
        t = ctypes.c_uint64()
        c = N.camera(cam)
        N.check(N.lib().cloud_server_submit(self._h, sid, ctypes.byref(c), steps, ctypes.byref(t)),
                "cloud_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 10000) -> dict:
        info = N.RequestInfo()
        N.check(N.lib().cloud_server_wait(self._h, ticket, timeout_ms, ctypes.byref(info)),
                "cloud_server_wait")
        return dict(session=info.session, steps=info.steps, batch_size=info.batch_size,
                    queue_ms=info.queue_ms, latency_ms=info.latency_ms)

    def output(self, sid: int):
        """The session's latest resolved frame (history format) as a numpy array."""
        w, h = self.sizes[sid]
        dt = torch.float32 if self.history_fmt == "fp32" else torch.float16
        host = torch.empty((h, w, 4), dtype=dt)
        N.check(N.lib().cloud_server_copy_output(self._h, sid, ctypes.c_void_p(host.data_ptr()),
                                                 host.numel() * host.element_size()),
                "cloud_server_copy_output")
        return host.numpy()

    def pause(self, paused: bool = True):
        N.check(N.lib().cloud_server_pause(self._h, 1 if paused else 0), "cloud_server_pause")

    def stats(self) -> dict:
        st = N.ServerCounters()
        rc = N.lib().cloud_server_stats(self._h, ctypes.byref(st))
        return dict(completed=st.completed, batches=st.batches, batched_views=st.batched_views,
                    queued=st.queued, open_sessions=st.open_sessions,
                    session_bytes=st.session_bytes, status=rc)

    def close(self):
        if self._h:
            N.check(N.lib().cloud_server_destroy(self._h), "cloud_server_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
