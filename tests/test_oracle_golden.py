"""Regression record of the oracle (tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np

from paper_1609_05344_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")


def test_oracle_matches_regression_record(oracle):
    with open(GOLDEN) as f:
        data = json.load(f)
    for case in data["cases"]:
        wl = I.workload(case["workload"])
        vol = oracle.Volume(wl.volume)
        cam = I.orbit_camera(case["frame"], wl.volume["seed"]) if wl.taa else I.ground_camera()
        rgba, n = oracle.render_pixels(vol, cam, I.params(), wl.width, wl.height, case["steps"],
                                       wl.light_steps, case["xs"], case["ys"],
                                       jitter_frame=case["frame"] if case["jitter"] else -1)
        assert n == case["lookups"]
        assert np.allclose(rgba, np.array(case["rgba"]), atol=1e-12, rtol=0), case["name"]
