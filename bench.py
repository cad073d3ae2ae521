"""Benchmark of the cloud raymarch + TAA frame loop on GB300.

Workload (fast path of the paper, Sec. 3.2 / Sec. 4): 1920x1080, 8 jittered
view steps x 6 light steps per ray, analytic integration, TAA resolve with
blend 0.1 over a seeded 32-frame camera orbit; 128^3 base + 32^3 detail noise
and a 512^2 weather map (FP32 by default, --precision fp16 for half volumes).

One step = one frame: raymarch (jitter frame f) -> reprojection motion ->
TAA resolve.  Metric: nominal Gsamples/s = W*H*steps*(1+light_steps) / frame
time, plus ms/frame.  L2 is flushed (256 MiB write) between timed frames,
outside the timed events.

    python bench.py [--gpus N --steps K --warmup W --precision fp32|fp16]
    python bench.py --impl reference      # the FP64 CPU oracle on host cores

Multi-GPU (torchrun): every rank renders its own replica of the frame loop
(independent views; no collective on the data path); value = sum over ranks
of the samples / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsamples/s & ms/frame 1080p 8-step+TAA; served p50/p99 latency; err vs FP64"
UNIT = "Gsamples/s"
L1TEX_BYTES_PER_CLK_PER_SM = 128
FLUSH_BYTES = 256 << 20


class L2Flush:
    """Evicts L2 between timed steps, outside the timed events: writes a
    256 MiB buffer (larger than the 126 MB L2), then reads another 256 MiB
    buffer so the dirty lines of the write are written back before the next
    step starts instead of during it."""

    def __init__(self):
        import torch
        self.w = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        self.r = torch.zeros(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        self(0)  # the first reduction may be compiled on the fly: keep that out of any timing
        torch.cuda.synchronize()

    def __call__(self, k: int):
        self.w.fill_(k & 0xFF)
        self.r.max()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=d.get("hbm_gbs", 6800.0), sm_max_mhz=d.get("sm_max_mhz", 2070.0),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc and self.proc.poll() is not None:
            return
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _code_sha1(files):
    """SHA-1 (12 hex digits) of sources with comments and blank lines removed:
    it changes when the code does, not when a comment does."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1609_05344_gb300", "csrc")
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(csrc, f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            line = line.split("//")[0].rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:12]


def march_code_sha1():
    """Comment-insensitive SHA-1 of the march sources."""
    return _code_sha1(("march.cuh", "march_kernels.cuh", "render.cu", "common.cuh"))


def taa_code_sha1():
    """Comment-insensitive SHA-1 (12 hex digits) of the resolve's source."""
    return _code_sha1(("taa.cu", "common.cuh"))


def _profile_data(name, code_hash):
    """Counters from the data file committed beside an ncu summary
    (profiles/<name>.json), or {} when the kernel code has changed since they
    were taken."""
    path = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        d = json.load(f)
    return d if d.get("code_sha1") == code_hash else {}


def taa_profile():
    """DRAM bytes per launch of the fused resolve from the committed ncu capture."""
    d = _profile_data("taa_motion_kernels_fast-1080p", taa_code_sha1())
    return {"traffic": d["traffic_bytes_per_launch"]} if d else {}


def march_profile():
    """Counters of the march from the committed ncu capture (DRAM bytes per
    launch, ncu's L1TEX throughput in % of peak)."""
    d = _profile_data("march_kernel_fast-1080p", march_code_sha1())
    return ({"traffic": d["traffic_bytes_per_launch"], "l1tex_pct": d["l1tex_throughput_pct"]}
            if d else {})


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(
        os.environ.get("LOCAL_RANK", 0))


def make_reduce_max(world: int, device):
    """Max over ranks of a per-rank number (NCCL on the GPU path, gloo on CPU)."""
    def reduce_max(v: float) -> float:
        if world == 1:
            return v
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return reduce_max


def aggregate(step_ms: float, samples: float, world: int, reduce_max=None):
    """Whole-job throughput: all ranks' samples over the slowest rank's time."""
    worst = reduce_max(step_ms) if reduce_max else step_ms
    return samples * world / (worst * 1e-3) / 1e9, worst


def cpu_baseline(wl, prm, budget_s=12.0, gpu_frame=None):
    """The FP64 oracle (test infrastructure) timed on the host cores over whole
    frames of the workload (render + motion + TAA), as many as fit budget_s."""
    import numpy as np
    from oracle import oracle as O
    from paper_1609_05344_gb300 import inputs as I
    cores = os.cpu_count() or 1
    ovol = O.Volume(dict(wl.volume, precision="fp32"))
    frames, t0 = 0, time.perf_counter()
    hist, first_img = None, None
    while True:
        cam = I.orbit_camera(frames, wl.volume["seed"])
        img, _ = O.render(ovol, cam, prm, wl.width, wl.height, wl.steps, wl.light_steps,
                          jitter_frame=frames, nthreads=cores)
        if first_img is None:
            first_img = img
        mot = (O.motion(wl.volume, prm, I.orbit_camera(frames - 1, wl.volume["seed"]), cam,
                        wl.width, wl.height) if frames else np.zeros((wl.height, wl.width, 2)))
        hist = O.taa(hist, img, mot, blend=0.1)
        frames += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    samples = wl.width * wl.height * wl.steps * (1 + wl.light_steps) * frames
    # one thread: the raymarch of one frame (the bulk of the oracle's work)
    t1 = time.perf_counter()
    O.render(ovol, I.orbit_camera(0, wl.volume["seed"]), prm, wl.width, wl.height, wl.steps,
             wl.light_steps, jitter_frame=0, nthreads=1)
    dt1 = time.perf_counter() - t1
    err = None
    if gpu_frame is not None:
        err = float(np.abs(gpu_frame.astype(np.float64) - first_img).max())
    return {"value": samples / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{frames} whole frame(s) of the workload (render+motion+TAA), FP64, "
                      f"{cores} threads, {dt:.1f} s",
            "single_thread": {"value": wl.width * wl.height * wl.steps * (1 + wl.light_steps) / dt1 / 1e9,
                              "unit": UNIT, "sample": f"the raymarch of one frame, 1 thread, {dt1:.1f} s"}}, err


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (there is no
    published implementation of the paper to run), timed over whole frames of
    the workload: each step renders one 1920x1080 frame (row-parallel over the
    host cores), computes its motion from the previous camera and resolves it
    into the history, exactly the work of one GPU step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    from paper_1609_05344_gb300 import inputs as I
    wl = I.workload("fast-1080p")
    prm = I.params()
    cores = os.cpu_count() or 1
    ovol = O.Volume(wl.volume)
    seed = wl.volume["seed"]
    hist, times = None, []
    t_run = time.perf_counter()
    for f in range(args.warmup + args.steps):
        cam = I.orbit_camera(f % wl.frames, seed)
        t0 = time.perf_counter()
        img, _ = O.render(ovol, cam, prm, wl.width, wl.height, wl.steps, wl.light_steps,
                          jitter_frame=f, nthreads=cores)
        mot = (O.motion(wl.volume, prm, I.orbit_camera((f - 1) % wl.frames, seed), cam, wl.width,
                        wl.height) if hist is not None else np.zeros((wl.height, wl.width, 2)))
        hist = O.taa(hist, img, mot, blend=0.1)
        dt = time.perf_counter() - t0
        if f >= args.warmup:
            times.append(dt)
    t_run = time.perf_counter() - t_run
    frame_s = statistics.mean(times)
    value = wl.width * wl.height * wl.steps * (1 + wl.light_steps) / frame_s / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": frame_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "fast-1080p", "width": wl.width, "height": wl.height,
                       "steps": wl.steps, "light_steps": wl.light_steps, "jitter": "pixel",
                       "taa": True, "blend": 0.1, "volume_precision": "fp64 (the oracle's own)",
                       "volumes": "128^3 base + 32^3 detail + 512^2 weather",
                       "frames": "32-frame seeded orbit"},
            "frame_ms_p10_p50_p90": [float(np.percentile(times, q)) * 1e3 for q in (10, 50, 90)],
            "wall_s": t_run,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} whole frames (render + motion + TAA), FP64, "
                                       f"render on {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1609_05344_gb300 import _native, api, inputs as I

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    _native.build()

    wl = I.workload("fast-1080p", precision=args.precision)
    prm = I.params(jitter_mode="frame" if args.jitter == "frame" else "pixel")
    W, H, S, LS = wl.width, wl.height, wl.steps, wl.light_steps
    jit = (lambda f: -1) if args.jitter == "none" else (lambda f: f)
    seed = wl.volume["seed"] + 1000 * rank  # each replica its own orbit start
    vol = api.Volume(wl.volume)
    stream = torch.cuda.current_stream()
    cur = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    hist = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    flush = L2Flush()

    def cam(f):
        return I.orbit_camera(f % wl.frames, seed)

    state = {"latest": None, "n": 0}

    def frame(f, ev=None):
        """One frame: raymarch (jitter frame f), then reprojection motion and TAA
        resolve fused in one kernel.  Returns the number of launches."""
        if ev:
            ev[0].record(stream)
        api.render(vol, cam(f), prm, W, H, S, LS, jitter_frame=jit(f), out=cur)
        if ev:
            ev[1].record(stream)
            ev[2].record(stream)
        src = hist[state["latest"]] if state["latest"] is not None else None
        nxt = 1 if state["latest"] == 0 else 0
        api.taa_reproject(vol, prm, cam(f - 1) if src is not None else None, cam(f), src, cur,
                          blend=0.1, out=hist[nxt])
        if ev:
            ev[3].record(stream)
        state["latest"] = nxt
        return 2

    # untimed: the autotuner picks the launch configuration (tile shape, view
    # steps per warp iteration) the frame loop then uses, unless one is given
    # (profiling runs pin it: under a profiler the tuner's timings are not the
    # kernels' own)
    if args.launch_config >= 0:
        api.set_launch_config(args.precision, LS, args.launch_config)
        tuned, tune_ms = args.launch_config, None
    else:
        tuned, tune_ms = api.autotune_render(vol, cam(0), prm, W, H, S, LS, jitter_frame=jit(0),
                                             repeats=3)
    # clocks are sampled (every 200 ms) from the start of the warm-up through the
    # timed frames; warm-up continues, untimed, until the sampler is running
    clk = ClockSampler(local).__enter__()
    fi = 0
    t_warm = time.perf_counter()
    while fi < args.warmup or (len(clk.rows) < 3 and time.perf_counter() - t_warm < 5.0):
        frame(fi)
        fi += 1
        if fi >= args.warmup:
            torch.cuda.synchronize()
    # effective lookups per frame (untimed counting launches over the timed cameras)
    counted = []
    for k in range(min(args.steps, 8)):
        _, ctr = api.render(vol, cam(fi + k), prm, W, H, S, LS, jitter_frame=jit(fi + k), out=cur,
                            count=True)
        counted.append(int(ctr.item()))
    eff_lookups = statistics.mean(counted)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush(k)  # evict L2 (outside the timed events)
        launches += frame(fi + k, evs[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk.__exit__()
    if world > 1:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    march_ms = [e[0].elapsed_time(e[1]) for e in evs]
    taa_ms = [e[2].elapsed_time(e[3]) for e in evs]
    ms = statistics.mean(step_ms)

    # the 32-frame orbit as one CUDA graph (render + fused resolve per frame), replayed
    # back to back without L2 flushes: the steady state of a renderer whose tiles stay
    # L2-resident between frames (reported beside, not as, the flushed number)
    graph_ms = None
    try:
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gs):
            frame(fi + args.steps)  # first use of this stream, outside the capture
        torch.cuda.current_stream().wait_stream(gs)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            for k in range(wl.frames):
                frame(fi + args.steps + 1 + k)
        g.replay()
        torch.cuda.synchronize()
        ge = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ge[0].record()
        for _ in range(3):
            g.replay()
        ge[1].record()
        torch.cuda.synchronize()
        graph_ms = ge[0].elapsed_time(ge[1]) / (3 * wl.frames)
        del g
    except RuntimeError as exc:  # capture is reported, never worked around
        graph_ms = f"capture failed: {exc}"

    reduce_max = make_reduce_max(world, "cuda")

    samples = W * H * S * (1 + LS)
    value, worst = aggregate(ms, samples, world, reduce_max)

    # end to end through the session API: every step renders, resolves and reads its
    # resolved frame back into pinned host memory (33 MB); the read-back of frame k runs on
    # the session's copy stream while frame k+1 renders (three host buffers in rotation)
    # (at least 64 frames, so that filling and draining the two-frame pipeline is a
    # small share; the host-side camera descriptions are prepared before the clock)
    hosts = [torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True) for _ in range(3)]
    sess = api.Session(vol, W, H, "fp32")
    for f in range(args.warmup):
        sess.wait_frame(sess.frame_async(cam(f), prm, S, LS, hosts[f % 3]))
    n_e2e = max(args.steps, 64)
    cams_e2e = [cam(fi + k) for k in range(n_e2e)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pending = []
    for k in range(n_e2e):
        pending.append(sess.frame_async(cams_e2e[k], prm, S, LS, hosts[k % 3]))
        if len(pending) > 2:
            sess.wait_frame(pending.pop(0))
    for idx in pending:
        sess.wait_frame(idx)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_value, _ = aggregate(e2e_s * 1e3, samples, world, reduce_max)
    sess.close()

    pk = _peaks()
    mprof = march_profile()
    sm_mhz = pk["sm_max_mhz"]
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    l1_peak_gbs = sms * L1TEX_BYTES_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e9
    # scattered 32-byte records: at most one L1 data-pipe wavefront (sector) per clock per SM
    sector_peak_gbs = sms * 32 * sm_mhz * 1e6 / 1e9
    texel_b = 4 if args.precision == "fp32" else 2  # bytes per stored texel
    bytes_per_lookup = 20 * texel_b  # 8 base + 8 detail + 4 weather texels
    march_avg = statistics.mean(march_ms)
    achieved = eff_lookups * bytes_per_lookup / (march_avg * 1e-3) / 1e9
    taa_avg = statistics.mean(taa_ms)
    taa_bytes_px = 48  # current 16 + history 16 + resolved 16 (motion fused, never stored)
    taa_gbs = W * H * taa_bytes_px / (taa_avg * 1e-3) / 1e9

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": worst, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "fast-1080p", "width": W, "height": H, "steps": S,
                   "light_steps": LS, "jitter": args.jitter, "taa": True, "blend": 0.1,
                   "volume_precision": args.precision,
                   "volumes": "128^3 base + 32^3 detail + 512^2 weather",
                   "frames": "32-frame seeded orbit", "l2": "flushed between steps (256 MiB write + 256 MiB read, untimed)",
                   "parallelism": f"replicas x{world}", "launch_config": tuned,
                   "tile_shape_and_steps_per_iteration": list(_native.config_parts(tuned)),
                   "config_ms": tune_ms},
        "ms_per_frame": worst, "march_ms": march_avg, "taa_reproject_ms": taa_avg,
        "frame_ms_p10_p50_p90": [float(np.percentile(step_ms, q)) for q in (10, 50, 90)],
        "graph_32_frames": {"ms_per_frame": graph_ms,
                            "l2": "warm: 32 frames replayed back to back from one CUDA graph, "
                                  "no flush between frames"},
        "motion": "fused into the TAA resolve", "wall_ms_per_step_incl_flush": t_wall / args.steps * 1e3,
        "effective_lookups_per_frame": eff_lookups,
        "effective_gsamples_s": eff_lookups / (ms * 1e-3) / 1e9,
        "roofline": {"bound": "l1tex", "achieved": achieved, "peak": l1_peak_gbs, "unit": "GB/s",
                     "frac": achieved / l1_peak_gbs, "traffic": mprof.get("traffic"),
                     "ncu_l1tex_throughput_pct_of_peak": mprof.get("l1tex_pct"),
                     "kernel": "march_kernel",
                     "peak_source": f"L1TEX data path {sms} SMs x 128 B/clk x {sm_mhz:.0f} MHz "
                                    f"({pk['source']} clock)",
                     "algorithmic_bytes_per_lookup": bytes_per_lookup,
                     "sector_rate_peak": sector_peak_gbs,
                     "frac_of_sector_rate": achieved / sector_peak_gbs,
                     "note": "achieved counts every lookup of the method with its 80 algorithmic "
                             "bytes, including the view lookups the occupancy grid proves empty "
                             "(they return 0 without reading a record), so it can exceed the "
                             "scattered-sector rate; traffic is what the kernel actually reads"},
        "taa_roofline": {"bound": "hbm", "achieved": taa_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": taa_gbs / pk["hbm_gbs"], "bytes_per_pixel": taa_bytes_px,
                         "traffic": taa_profile().get("traffic"),
                         "kernel": "taa_reproject_kernel",
                         "peak_source": pk["source"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_s * 1e3, "frames": n_e2e,
                "h2d_bytes_per_step": 216, "d2h_bytes_per_step": W * H * 16,
                "api": "cloud_session_frame_async + cloud_session_wait_frame (read-back "
                       "overlapped with the next frame)",
                "l2": "not flushed: frames back to back through the session API, as an "
                      "application runs them (wall clock over all frames incl. pipeline "
                      "fill and drain)"},
        "gpu_launches": launches,
        "device_wait_timeouts": api.device_wait_timeouts(),
        "clocks": dict(clk.summary(), window="warm-up and timed frames"),
    }
    if not args.no_extra_workloads:
        # the other two configurations' headline comparisons, measured in the
        # same run (BF16 tiles for the 64-view batch, FP16 tiles and history for
        # serving, as the configurations state), each with its error vs FP64
        bvol = api.Volume(I.volume_desc("full", seed=3, precision="bf16"))
        line["batched_64"] = dict(
            batched_measure(bvol, I.random_views(64, seed=4 + 1000 * rank), I.params(), 3, 3,
                            local, oracle_pixels=8 if rank == 0 else 0),
            volume_precision="bf16", views=64, steps="{8,16,32,128}",
            sizes="256x256..1920x1080 seeded", timed_steps=3)
        bvol.close()
        # the same batch with FP16 tiles, the 16-bit format that meets 3e-3
        hvol = api.Volume(I.volume_desc("full", seed=3, precision="fp16"))
        line["batched_64_fp16"] = dict(
            batched_measure(hvol, I.random_views(64, seed=4 + 1000 * rank), I.params(), 3, 3,
                            local, oracle_pixels=8 if rank == 0 else 0),
            volume_precision="fp16", timed_steps=3)
        hvol.close()
        svol = api.Volume(I.volume_desc("full", seed=3, precision="fp16"))
        line["served"] = dict(served_measure(svol, I.params(), 500, 75, rank,
                                             oracle_frames=3 if rank == 0 else 0),
                              volume_precision="fp16", history="fp16")
        svol.close()
    if world == 1 and not args.no_cpu_baseline:
        gpu0 = api.render(vol, I.orbit_camera(0, wl.volume["seed"]), prm, W, H, S, LS,
                          jitter_frame=0).cpu().numpy()
        base, err = cpu_baseline(wl, prm, gpu_frame=gpu0)
        line["cpu_baseline"] = base
        line["max_abs_err_vs_fp64"] = err
    print(json.dumps(line))
    vol.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def batched_measure(vol, views, prm, steps, warmup, local, oracle_pixels=0):
    """Config 4 (64 uneven views): one persistent launch replayed from a CUDA
    graph, the same launch without the graph, and one launch per view, each
    timed over `steps` steps with the L2 flushed between them; optionally the
    max-abs error of the graph launch against the FP64 oracle on
    `oracle_pixels` sampled pixels per view."""
    import numpy as np
    import torch

    from paper_1609_05344_gb300 import _native, api
    batch = api.Batch(vol, prm, views)
    best, times = batch.autotune(repeats=2)
    flush = L2Flush()
    stream = torch.cuda.current_stream()

    def launch(mode):
        if mode == "graph":
            batch.render(graph=True)
        elif mode == "persistent":
            batch.render()
        else:
            batch.render_per_view()

    res = {}
    for mode in ("graph", "persistent", "per_view"):
        for k in range(warmup):
            batch.set_views([dict(v, jitter_frame=k) for v in views])
            launch(mode)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for k in range(steps):
            flush(k)
            batch.set_views([dict(v, jitter_frame=warmup + k) for v in views])
            evs[k][0].record(stream)
            launch(mode)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        res[mode] = statistics.mean(a.elapsed_time(b) for a, b in evs)
    samples = sum(v["width"] * v["height"] * v["steps"] * 7 for v in views)
    out = {"ms_graph": res["graph"], "ms_persistent_no_graph": res["persistent"],
           "ms_one_launch_per_view": res["per_view"],
           "speedup_vs_per_view": res["per_view"] / res["graph"],
           "gsamples_s": samples / (res["graph"] * 1e-3) / 1e9, "launch_config": best,
           "tile_shape_and_steps_per_iteration": list(_native.config_parts(best)),
           "config_ms": times}
    if oracle_pixels:
        from oracle import oracle as O
        batch.set_views(views)
        outs = batch.render(graph=True)
        ovol = O.Volume(dict(vol.desc, precision="fp32"))
        rng = np.random.default_rng(9)
        worst = 0.0
        for v, o in zip(views, outs):
            xs = rng.integers(0, v["width"], oracle_pixels)
            ys = rng.integers(0, v["height"], oracle_pixels)
            ref, _ = O.render_pixels(ovol, v["camera"], prm, v["width"], v["height"], v["steps"], 6,
                                     xs, ys, jitter_frame=v["jitter_frame"],
                                     nthreads=os.cpu_count() or 1)
            worst = max(worst, float(np.abs(o.cpu().numpy()[ys, xs] - ref).max()))
        ovol.close()
        out["max_abs_err_vs_fp64"] = worst
        out["err_sample"] = f"{oracle_pixels} seeded pixels of each view"
    batch.close()
    return out


def run_batched(args):
    """Multi-view workload: 64 views of uneven size (256x256 .. 1920x1080, seeded),
    step counts from {8, 16, 32, 128}, seeded cameras, one volume set; all
    views in one persistent launch replayed from a CUDA graph, against one
    launch per view.  One step = every view rendered once (new jitter frame)."""
    import torch

    from paper_1609_05344_gb300 import _native, api, inputs as I
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _native.build()
    prec = args.precision if args.precision != "fp32" or args.precision_set else "bf16"
    vol = api.Volume(I.volume_desc("full", seed=3, precision=prec))
    prm = I.params()
    views = I.random_views(64, seed=4 + 1000 * rank)
    pixels = sum(v["width"] * v["height"] for v in views)
    clk = ClockSampler(local).__enter__()
    r = batched_measure(vol, views, prm, args.steps, args.warmup, local)
    clk.__exit__()
    ms = r["ms_graph"]
    line = {"metric": "Gsamples/s, 64 uneven views in one persistent launch (CUDA graph)",
            "value": r["gsamples_s"] * world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched-64", "views": 64, "pixels": pixels,
                       "sizes": "256x256..1920x1080 seeded", "steps": "{8,16,32,128}",
                       "light_steps": 6, "volume_precision": prec,
                       "l2": "flushed between steps (256 MiB write + 256 MiB read, untimed)",
                       "launch_config": r["launch_config"],
                       "tile_shape_and_steps_per_iteration": r["tile_shape_and_steps_per_iteration"],
                       "config_ms": r["config_ms"]},
            "ms_persistent_no_graph": r["ms_persistent_no_graph"],
            "ms_one_launch_per_view": r["ms_one_launch_per_view"],
            "speedup_vs_per_view": r["speedup_vs_per_view"],
            "gpu_launches": args.steps, "clocks": dict(clk.summary(), window="all modes")}
    if rank == 0:
        print(json.dumps(line))
    return 0


def served_measure(vol, prm, n_req, n_warm, rank=0, oracle_frames=0):
    """Config 5: Poisson arrivals at 2000 requests/s over 256 sessions
    (640x360..1920x1080, 8 or 16 steps, FP16 history), the same trace served by
    continuous batching (<= 64 requests per persistent launch, two batches in
    flight) and by the plain per-frame form (one request per launch set, one in
    flight), paced and saturated (all requests queued at once).  Latency is
    submit -> device work complete.  Optionally the max-abs error of a served
    640x360 session over `oracle_frames` frames against the FP64 oracle chain
    (render -> motion -> TAA)."""
    import numpy as np

    from paper_1609_05344_gb300 import api, inputs as I
    rng = np.random.default_rng(55 + rank)
    n_sess = 256
    sizes = [(int(rng.integers(640, 1921)), int(rng.integers(360, 1081))) for _ in range(n_sess)]

    def trace(seed, n):
        r = np.random.default_rng(seed)
        t = np.cumsum(r.exponential(1.0 / 2000.0, n))
        return t, r.integers(0, n_sess, n), r.choice([8, 16], n)

    def run(mode, t_arr, sess, steps, paced):
        cfg = dict(max_batch_views=64, slots=2) if mode == "continuous" else dict(
            max_batch_views=1, slots=1)
        srv = api.Server(vol, prm, history_fmt="fp16", max_sessions=n_sess, **cfg)
        sids = [srv.open_session(w, h) for (w, h) in sizes]
        wt = [srv.submit(sids[k % n_sess], I.orbit_camera(0, 100 + k % n_sess), 8)
              for k in range(n_warm)]
        for t in wt:
            srv.wait(t, 60000)
        frame = [1 if k < n_warm else 0 for k in range(n_sess)]
        tickets = []
        t0 = time.perf_counter()
        for k in range(len(t_arr)):
            if paced:
                while time.perf_counter() - t0 < t_arr[k]:
                    pass
            sk = int(sess[k])
            tickets.append(srv.submit(sids[sk], I.orbit_camera(frame[sk], 100 + sk), int(steps[k])))
            frame[sk] += 1
        infos = [srv.wait(t, 120000) for t in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array([i["latency_ms"] for i in infos])
        bs = np.array([i["batch_size"] for i in infos])
        return dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                    mean_ms=float(lat.mean()), frames_per_s=len(infos) / wall,
                    mean_batch=float(bs.mean()), batches=int(st["batches"]))

    t_arr, sess, steps = trace(7 + rank, n_req)
    res = {}
    for mode in ("continuous", "per_frame"):
        res[mode] = run(mode, t_arr, sess, steps, paced=True)
        res[mode + "_saturated"] = run(mode, t_arr, sess, steps, paced=False)
    out = {"requests": n_req, "sessions": n_sess, "arrivals": "Poisson 2000/s",
           "mean_pixels_per_request": float(np.mean([sizes[int(k)][0] * sizes[int(k)][1]
                                                     for k in sess])),
           "p50_ms": res["continuous"]["p50_ms"], "p99_ms": res["continuous"]["p99_ms"],
           "frames_per_s_saturated": res["continuous_saturated"]["frames_per_s"],
           "per_frame_p50_ms": res["per_frame"]["p50_ms"],
           "per_frame_p99_ms": res["per_frame"]["p99_ms"],
           "per_frame_frames_per_s_saturated": res["per_frame_saturated"]["frames_per_s"],
           "speedup_saturated": (res["continuous_saturated"]["frames_per_s"]
                                 / res["per_frame_saturated"]["frames_per_s"]),
           "runs": res}
    if oracle_frames:
        from oracle import oracle as O
        w, h = 640, 360
        srv = api.Server(vol, prm, history_fmt="fp16", max_batch_views=8, slots=2)
        sid, other = srv.open_session(w, h), srv.open_session(1920, 1080)
        ovol = O.Volume(dict(vol.desc, precision="fp32"))
        ohist, worst = None, 0.0
        for f in range(oracle_frames):
            cam = I.orbit_camera(f, 100)
            t1 = srv.submit(sid, cam, 8)
            t2 = srv.submit(other, I.orbit_camera(f, 101), 16)  # batched beside a large view
            srv.wait(t1)
            srv.wait(t2)
            ocur, _ = O.render(ovol, cam, prm, w, h, 8, 6, jitter_frame=f,
                               nthreads=os.cpu_count() or 1)
            omot = (O.motion(vol.desc, prm, I.orbit_camera(f - 1, 100), cam, w, h) if f
                    else np.zeros((h, w, 2)))
            ohist = O.taa(ohist, ocur, omot, blend=0.1)
            worst = max(worst, float(np.abs(srv.output(sid).astype(np.float64) - ohist).max()))
        srv.close()
        ovol.close()
        out["max_abs_err_vs_fp64"] = worst
        out["err_sample"] = (f"every pixel of a served 640x360 session (batched with a 1920x1080 "
                             f"one) over {oracle_frames} frames, against the oracle chain")
    return out


def run_served(args):
    """Serving workload (config 5): see served_measure."""
    import torch

    from paper_1609_05344_gb300 import _native, api, inputs as I
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _native.build()
    prec = args.precision if args.precision_set else "fp16"
    vol = api.Volume(I.volume_desc("full", seed=3, precision=prec))
    prm = I.params()
    clk = ClockSampler(local).__enter__()
    r = served_measure(vol, prm, max(1, args.steps) * 125, max(3, args.warmup) * 25, rank)
    clk.__exit__()
    line = {"metric": "served frames/s (saturated) and p50/p99 latency at 2000 req/s, 256 sessions",
            "value": r["frames_per_s_saturated"] * world, "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / r["frames_per_s_saturated"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "served", "sessions": r["sessions"], "requests": r["requests"],
                       "arrivals": "Poisson 2000/s", "sizes": "640x360..1920x1080 seeded",
                       "steps": "{8,16}", "light_steps": 6, "history": "fp16",
                       "volume_precision": prec,
                       "mean_pixels_per_request": r["mean_pixels_per_request"],
                       "continuous": "<=64 requests per persistent launch, 2 in flight",
                       "per_frame": "1 request per launch set, 1 in flight"},
            "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
            "served": r["runs"], "clocks": dict(clk.summary(), window="all runs")}
    if rank == 0:
        print(json.dumps(line))
    return 0


# The paper's draw times (GTX 1080, Unity/RenderDoc, median of five; Sec. 4 table).
PAPER_MS = {("full", 128, "none"): 297.7, ("half", 128, "none"): 128.0, ("half", 8, "none"): 2.3,
            ("half", 8, "pixel"): 7.5, ("half", 8, "pixel+taa"): 7.5,
            ("quarter", 8, "pixel+taa"): 2.4}


def run_paper_table(args):
    """The paper's Sec. 4 table re-measured on GB300 (1920x1080 display; half
    and quarter read per axis), plus the per-frame-constant offset of Sec. 4,
    the composite of the low-resolution buffer over a 1920x1080 background,
    and Fig. 1 / Fig. 2 as numbers: the error of each 8-step variant against
    the 128-step image of the same static view (TAA accumulated 32 frames)."""
    import numpy as np
    import torch

    from paper_1609_05344_gb300 import _native, api, inputs as I
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    _native.build()
    vol = api.Volume(I.volume_desc("full", seed=3))
    cam = I.orbit_camera(0, 3)
    res = {"full": (1920, 1080), "half": (960, 540), "quarter": (480, 270)}
    flush = L2Flush()
    stream = torch.cuda.current_stream()

    def frame_fn(size, steps, mode):
        w, h = res[size]
        prm = I.params(jitter_mode="frame" if "frame" in mode else "pixel")
        cur = torch.empty((h, w, 4), device="cuda")
        hist = [torch.empty((h, w, 4), device="cuda") for _ in range(2)]
        bg = torch.rand((1080, 1920, 4), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        disp = torch.empty_like(bg)
        st = {"k": 0}

        def run(f):
            jf = f if mode != "none" else -1
            api.render(vol, cam, prm, w, h, steps, 6, jitter_frame=jf, out=cur)
            if "taa" in mode:
                src = hist[st["k"] % 2] if f > 0 else None
                api.taa_reproject(vol, prm, cam if src is not None else None, cam, src, cur,
                                  out=hist[(st["k"] + 1) % 2])
                st["k"] += 1
                if "composite" in mode:
                    api.composite(hist[st["k"] % 2], bg, out=disp)
        return run

    rows = []
    for size, steps, mode in [("full", 128, "none"), ("half", 128, "none"), ("half", 8, "none"),
                              ("half", 8, "pixel"), ("half", 8, "pixel+taa"),
                              ("quarter", 8, "pixel+taa"), ("half", 8, "frame"),
                              ("half", 8, "frame+taa"), ("full", 8, "pixel+taa"),
                              ("half", 8, "pixel+taa+composite"),
                              ("quarter", 8, "pixel+taa+composite")]:
        run = frame_fn(size, steps, mode)
        for f in range(args.warmup):
            run(f)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush(k)
            evs[k][0].record(stream)
            run(args.warmup + k)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in evs)
        rows.append({"resolution": size, "steps": steps, "jitter_taa": mode, "ms": ms,
                     "paper_gtx1080_ms": PAPER_MS.get((size, steps, mode))})

    # quality (half resolution, static view): error against the 128-step image
    w, h = res["half"]
    prm = I.params()
    ref = api.render(vol, cam, prm, w, h, 128, 6).cpu().numpy().astype(np.float64)

    def err(img):
        d = img.astype(np.float64) - ref
        return {"rmse_rgb": float(np.sqrt((d[..., :3] ** 2).mean())),
                "mean_rgb": float(d[..., :3].mean()), "rmse_alpha": float(np.sqrt((d[..., 3] ** 2).mean()))}

    q = {"8 steps": err(api.render(vol, cam, prm, w, h, 8, 6).cpu().numpy()),
         "8 steps, basic S = T L": err(api.render(vol, cam, prm, w, h, 8, 6,
                                                  integration="basic").cpu().numpy()),
         "128 steps, basic S = T L": err(api.render(vol, cam, prm, w, h, 128, 6,
                                                    integration="basic").cpu().numpy()),
         "8 steps, jitter, 1 frame": err(api.render(vol, cam, prm, w, h, 8, 6,
                                                    jitter_frame=0).cpu().numpy())}
    for label, pm in (("8 steps, jitter, TAA 32 frames", prm),
                      ("8 steps, per-frame jitter, TAA 32 frames", I.params(jitter_mode="frame"))):
        cur = torch.empty((h, w, 4), device="cuda")
        hist = None
        for f in range(32):
            api.render(vol, cam, pm, w, h, 8, 6, jitter_frame=f, out=cur)
            hist = api.taa_reproject(vol, pm, cam if hist is not None else None, cam, hist, cur)
        q[label] = err(hist.cpu().numpy())
    half = next(r for r in rows if (r["resolution"], r["steps"], r["jitter_taa"]) ==
                ("half", 8, "pixel+taa"))
    line = {"metric": "ms/frame of the paper's Sec. 4 rows on GB300", "value": half["ms"],
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": half["ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper-table", "display": "1920x1080",
                       "half": "960x540", "quarter": "480x270", "volumes": "full, FP32",
                       "l2": "flushed between steps (256 MiB write + 256 MiB read, untimed)"},
            "rows": rows, "quality_vs_128_steps_half_res": q}
    print(json.dumps(line))
    return 0


def run_config_table(args):
    """The three single-view configurations (plain tiny, 720p reference quality,
    1080p fast path with FP32 and FP16 tiles) on GB300 beside the FP64 oracle
    timed on one host thread and on all host cores (the oracle on 16 evenly
    spaced rows, scaled to a frame), with the max-abs RGBA error of the GPU
    render against the oracle on those rows."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1609_05344_gb300 import _native, api, inputs as I
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    _native.build()
    cores = os.cpu_count() or 1
    flush = L2Flush()
    stream = torch.cuda.current_stream()
    prm = I.params()
    rows = []
    cases = [("plain-tiny", "fp32"), ("reference", "fp32"), ("fast-1080p", "fp32"),
             ("fast-1080p", "fp16")]
    for name, prec in cases:
        wl = I.workload(name, precision=prec)
        W, H, S, LS = wl.width, wl.height, wl.steps, wl.light_steps
        vol = api.Volume(wl.volume)
        cam = (lambda f: I.orbit_camera(f, wl.volume["seed"])) if wl.taa else (
            lambda f: I.ground_camera())
        jit = (lambda f: f) if wl.jitter else (lambda f: -1)
        cur = torch.empty((H, W, 4), device="cuda")
        hist = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]

        def frame(f):
            api.render(vol, cam(f), prm, W, H, S, LS, jitter_frame=jit(f), out=cur)
            if wl.taa:
                api.taa_reproject(vol, prm, cam(f - 1) if f else None, cam(f),
                                  hist[(f + 1) % 2] if f else None, cur, out=hist[f % 2])
        for f in range(args.warmup):
            frame(f)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush(k)
            evs[k][0].record(stream)
            frame(args.warmup + k)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        gpu_ms = statistics.median(a.elapsed_time(b) for a, b in evs)
        # oracle rows (FP64 tiles regardless of the GPU's storage precision)
        ys = np.unique(np.linspace(0, H - 1, min(16, H)).astype(np.int32))
        xs_all = np.tile(np.arange(W, dtype=np.int32), ys.size)
        ys_all = np.repeat(ys, W)
        ovol = O.Volume(dict(wl.volume, precision="fp32"))
        f0 = 0
        t = {}
        for nt in (1, cores):
            t0 = time.perf_counter()
            ref, _ = O.render_pixels(ovol, cam(f0), prm, W, H, S, LS, xs_all, ys_all,
                                     jitter_frame=jit(f0), nthreads=nt)
            t[nt] = (time.perf_counter() - t0) * H / ys.size
        gpu = api.render(vol, cam(f0), prm, W, H, S, LS, jitter_frame=jit(f0)).cpu().numpy()
        err = float(np.abs(gpu[ys_all, xs_all].astype(np.float64) - ref).max())
        ovol.close()
        vol.close()
        samples = W * H * S * (1 + LS)
        rows.append({"config": name, "volume_precision": prec, "size": f"{W}x{H}",
                     "steps": S, "light_steps": LS, "jitter": wl.jitter, "taa": wl.taa,
                     "gpu_ms_per_frame": gpu_ms,
                     "gpu_nominal_gsamples_s": samples / (gpu_ms * 1e-3) / 1e9,
                     "oracle_1_thread_ms_per_frame": t[1] * 1e3,
                     "oracle_all_cores_ms_per_frame": t[cores] * 1e3, "cores": cores,
                     "oracle_sample": f"render of {ys.size} evenly spaced rows, scaled to a frame",
                     "max_abs_err_vs_fp64_on_those_rows": err})
    fast = next(r for r in rows if r["config"] == "fast-1080p" and r["volume_precision"] == "fp32")
    line = {"metric": "ms/frame per configuration on GB300 beside the FP64 oracle",
            "value": fast["gpu_ms_per_frame"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fast["gpu_ms_per_frame"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "config-table",
                       "l2": "flushed between frames (256 MiB write + 256 MiB read, untimed)"},
            "rows": rows}
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "unorm16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch-config", type=int, default=-1,
                    help="fast-1080p: pin the march launch configuration (0..7) instead of "
                         "autotuning it")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="fast-1080p only: skip the 64-view batch and serving summaries")
    ap.add_argument("--jitter", default="pixel", choices=["pixel", "frame", "none"],
                    help="fast-1080p start offsets: per pixel (Sec. 3.2), one per frame "
                         "(Sec. 4), or none (midpoint samples)")
    ap.add_argument("--workload", default="fast-1080p",
                    choices=["fast-1080p", "batched-64", "served", "paper-table", "config-table"])
    args = ap.parse_args(argv)
    args.precision_set = any(a.startswith("--precision") for a in (argv or sys.argv[1:]))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched-64":
        return run_batched(args)
    if args.workload == "config-table":
        return run_config_table(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "paper-table":
        return run_paper_table(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
