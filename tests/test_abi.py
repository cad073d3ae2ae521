"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every entry point include/cloudvol.h declares, and rejects bad arguments on
the host before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1609_05344_gb300 import _native as N

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "cloudvol.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\([^;]*\)\s*;", text, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    N.build()
    return N.lib()


def test_header_declares_expected_calls():
    names = set(_declared_functions())
    for required in ("cloud_volume_create", "cloud_render", "taa_resolve", "cloud_motion",
                     "cloud_volume_destroy", "cloud_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(n for n, _, _ in N.SIGNATURES) == sorted(names)


def test_status_strings(lib):
    assert lib.cloud_status_string(0) == b"ok"
    assert lib.cloud_status_string(-1) == b"invalid argument"
    assert lib.cloud_status_string(-5) == b"unsupported"
    assert lib.cloud_status_string(7) == b"unknown status"


def test_host_side_validation_without_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.cloud_volume_create(None, None, ctypes.byref(out)) == N.ERR_INVALID_ARG
    assert b"null" in lib.cloud_last_error_message()
    d = N.volume_desc(dict(base_n=48))  # not a power of two
    assert lib.cloud_volume_create(ctypes.byref(d), None, ctypes.byref(out)) == N.ERR_INVALID_ARG
    assert b"base_n" in lib.cloud_last_error_message()
    d = N.volume_desc(dict(base_n=64, slab_lo=4000.0, slab_hi=1500.0))
    assert lib.cloud_volume_create(ctypes.byref(d), None, ctypes.byref(out)) == N.ERR_INVALID_ARG
    assert lib.cloud_render(None, None, None, 8, 8, 8, 6, -1, 0, None, None) == N.ERR_INVALID_ARG
    assert lib.taa_resolve(None, None, None, None, 8, 8, 0, ctypes.c_float(0.1), None) == \
        N.ERR_INVALID_ARG
    assert lib.cloud_hash4_batch(None, -1, None, None) == N.ERR_INVALID_ARG
    assert lib.cloud_session_create(None, 8, 8, 0, ctypes.byref(out)) == N.ERR_INVALID_ARG
    assert lib.cloud_volume_destroy(None) == N.ERR_INVALID_ARG
    assert not out.value  # never set on failure


def test_struct_layouts_match_header():
    # field order and sizes of the descriptors mirror include/cloudvol.h
    assert ctypes.sizeof(N.Camera) == 13 * 8
    assert ctypes.sizeof(N.Params) == 15 * 8  # 14 doubles + jitter_mode (padded)
    assert N.VolumeDesc.seed.offset == 0 and N.VolumeDesc.detail_weight.offset == 16
    assert N.VolumeDesc.precision.offset == 88
