"""Driver of tests/test_gpu_checked.py, run in a process of its own with
CLOUDVOL_CHECKED=1 so that the binding loads the checked build of the library
(kernels that verify their index arithmetic stays in range, skip an access
that fails and record its site in a device status word).

Every kernel of the render path runs on tiny configurations and on edge
cases -- 1x1, 8x8 and ragged images, 16^3 tiles, the standard tile sizes,
cameras inside, below and above the layer, 0 to 32 light steps, both
integration rules, per-pixel and per-frame offsets, FP32 and 16-bit tiles, a
multi-view batch, session frames with FP32 and FP16 history and a camera
jump, the separate motion and resolve passes, the composite and the render
server -- and FP32 results are compared with the FP64 oracle on every pixel.
Prints "CHECKED OK" when every check held and every comparison passed."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1609_05344_gb300 import api, inputs as I  # noqa: E402

TOL = 1e-4


def main():
    assert os.environ.get("CLOUDVOL_CHECKED") == "1"
    torch.cuda.set_device(0)
    api.check_status(reset=True)
    worst = 0.0
    cams = {
        "ground": I.ground_camera(),
        "orbit": I.orbit_camera(2, 3),
        "inside": I.camera((100.0, -50.0, 2600.0), 30.0, 5.0, 60.0),
        "above-down": I.camera((0.0, 0.0, 5200.0), 45.0, -35.0, 50.0),
        "horizontal": I.camera((0.0, 0.0, 2000.0), 10.0, 0.0, 60.0),
    }
    descs = {
        "tiny": I.volume_desc("tiny", seed=1),
        "small": I.volume_desc("full", seed=2, base_n=16, detail_n=16, weather_n=16),
        "full": I.volume_desc("full", seed=3),
    }
    sizes = [(8, 8), (1, 1), (37, 23)]
    for dname, desc in descs.items():
        ovol = O.Volume(desc)
        for prec in ("fp32", "fp16", "bf16", "unorm16"):
            vol = api.Volume(dict(desc, precision=prec))
            for cname, cam in cams.items():
                for (w, h) in sizes:
                    for steps, ls, jf, integ, jm in ((8, 6, 3, "analytic", "pixel"),
                                                     (16, 1, -1, "basic", "pixel"),
                                                     (3, 0, 5, "analytic", "frame"),
                                                     (20, 32, 1, "analytic", "pixel")):
                        prm = I.params(jitter_mode=jm)
                        got = api.render(vol, cam, prm, w, h, steps, ls, jitter_frame=jf,
                                         integration=integ).cpu().numpy()
                        assert np.isfinite(got).all(), (dname, prec, cname, w, h)
                        if prec == "fp32":
                            ref, _ = O.render(ovol, cam, prm, w, h, steps, ls, jitter_frame=jf,
                                              integration=O.ANALYTIC if integ == "analytic"
                                              else O.BASIC, nthreads=8)
                            err = float(np.abs(got - ref).max())
                            worst = max(worst, err)
                            assert err <= TOL, (dname, cname, w, h, steps, ls, err)
            # one multi-view launch against single renders (bitwise)
            views = [dict(camera=cams["orbit"], width=37, height=23, steps=8, jitter_frame=1),
                     dict(camera=cams["ground"], width=1, height=1, steps=16, jitter_frame=-1),
                     dict(camera=cams["inside"], width=8, height=8, steps=5, jitter_frame=2)]
            b = api.Batch(vol, I.params(), views)
            for v, o in zip(views, b.render(graph=True)):
                one = api.render(vol, v["camera"], I.params(), v["width"], v["height"], v["steps"],
                                 6, jitter_frame=v["jitter_frame"])
                assert torch.equal(o, one)
            b.close()
            vol.close()
        ovol.close()
    # session frames (fused motion + resolve, TMA tile with clamped borders), a camera jump
    desc = descs["full"]
    vol, ovol = api.Volume(desc), O.Volume(desc)
    prm = I.params()
    w, h = 37, 23
    frames = [I.orbit_camera(0, 3), I.orbit_camera(1, 3), I.camera((400.0, 300.0, 700.0), 80.0, 15.0)]
    for fmt in ("fp32", "fp16"):
        sess = api.Session(vol, w, h, history_fmt=fmt)
        host = torch.empty((h, w, 4), dtype=torch.float32 if fmt == "fp32" else torch.float16,
                           pin_memory=True)
        ohist = None
        for f, cam in enumerate(frames):
            sess.frame(cam, prm, 8, 6, host_out=host)
            ocur, _ = O.render(ovol, cam, prm, w, h, 8, 6, jitter_frame=f, nthreads=8)
            omot = O.motion(desc, prm, frames[f - 1], cam, w, h) if f else np.zeros((h, w, 2))
            ohist = O.taa(ohist, ocur, omot, blend=0.1)
            if fmt == "fp32":
                err = float(np.abs(host.numpy() - ohist).max())
                worst = max(worst, err)
                assert err <= TOL, ("session", f, err)
        sess.close()
    # the separate motion and resolve passes, and the composite
    cur = api.render(vol, frames[1], prm, w, h, 8, 6, jitter_frame=1)
    hist = api.render(vol, frames[0], prm, w, h, 8, 6, jitter_frame=0)
    mot = api.motion(vol, prm, frames[0], frames[1], w, h)
    out = api.taa(hist, cur, mot)
    ref = O.taa(hist.cpu().numpy().astype(np.float64), cur.cpu().numpy().astype(np.float64),
                mot.cpu().numpy().astype(np.float64))
    worst = max(worst, float(np.abs(out.cpu().numpy() - ref).max()))
    bg = torch.rand((61, 90, 4), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    comp = api.composite(out, bg)
    oref = O.composite(out.cpu().numpy().astype(np.float64), bg.cpu().numpy().astype(np.float64))
    worst = max(worst, float(np.abs(comp.cpu().numpy() - oref).max()))
    assert worst <= TOL, worst
    # the render server: two sessions of different sizes batched together
    srv = api.Server(vol, prm, history_fmt="fp32", max_sessions=4, max_batch_views=4, slots=2,
                     reserve_bytes=0)
    sids = [srv.open_session(8, 8), srv.open_session(37, 23)]
    for f in range(2):
        ts = [srv.submit(s, I.orbit_camera(f, 10 + k), 8) for k, s in enumerate(sids)]
        for t in ts:
            srv.wait(t, 20000)
    srv.close()
    torch.cuda.synchronize()
    bits = api.check_status()
    assert bits == 0, f"index checks failed at sites {bits:#x}"
    print(f"CHECKED OK (max abs error of the FP32 comparisons {worst:.2e})")


if __name__ == "__main__":
    main()
