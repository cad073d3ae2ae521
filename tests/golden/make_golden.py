"""Writes tests/golden/oracle_regression.json by calling only the FP64 oracle.

The paper prints no worked example, so these values are a regression record
of the oracle itself (pinned separately by closed forms and identities in
tests/test_oracle_*.py): a change to the oracle's arithmetic shows up here.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1609_05344_gb300 import inputs as I  # noqa: E402

CASES = [
    # name, workload, frame, jitter
    ("plain-tiny", "plain-tiny", 0, False),
    ("reference-small", "reference", 0, False),
    ("fast-1080p-f7", "fast-1080p", 7, True),
]


def main():
    out = {"note": "FP64 oracle regression values; premultiplied RGBA per pixel", "cases": []}
    rng = np.random.default_rng(1234)
    for name, wl_name, frame, jit in CASES:
        wl = I.workload(wl_name)
        vol = O.Volume(wl.volume)
        cam = I.orbit_camera(frame, wl.volume["seed"]) if wl.taa else I.ground_camera()
        xs = rng.integers(0, wl.width, 24)
        ys = rng.integers(0, wl.height, 24)
        steps = wl.steps if wl_name != "reference" else 32
        rgba, n = O.render_pixels(vol, cam, I.params(), wl.width, wl.height, steps, wl.light_steps,
                                  xs, ys, jitter_frame=frame if jit else -1)
        out["cases"].append(dict(name=name, workload=wl_name, frame=frame, jitter=jit, steps=steps,
                                 xs=xs.tolist(), ys=ys.tolist(), rgba=rgba.tolist(), lookups=n))
    with open(os.path.join(os.path.dirname(__file__), "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
