"""The checked build of the library: every kernel verifies that its index
arithmetic (tile records, occupancy words, work lists, pixels, history texels,
shared tiles, views) stays in range and records any failure in a device status
word instead of reading or writing out of bounds.  The build runs on tiny and
edge-case configurations (tests/_checked_run.py, in a process of its own that
loads the checked library) with every FP32 result compared against the FP64
oracle; the test passes when no check failed.  Normal builds report the status
query as unsupported."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_05344_gb300 import _native as N
    N.build()
    return N


def test_normal_build_has_no_checks(native):
    from paper_1609_05344_gb300 import api
    with pytest.raises(native.CloudError) as e:
        api.check_status()
    assert e.value.status == native.ERR_UNSUPPORTED


def test_checked_build_tiny_and_edge_configurations(native):
    native.build(checked=True)
    env = dict(os.environ, CLOUDVOL_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    print(r.stdout[-2000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "CHECKED OK" in r.stdout
