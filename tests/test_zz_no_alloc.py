"""GPU: the allocation-free multi-view entry point (cloud_batch_render_static).

Some callers cannot allocate device memory while rendering (a real-time
render thread, an engine with a fixed device-memory budget), because
cudaMalloc/cudaFree may block, synchronize the device or fail there.  This
entry point takes its scratch from a static device array inside the library.
The test calls it through the C ABI twice in a row (different cameras and
jitter frames, so the second call reuses the scratch the first one left
behind) and checks both results against the allocating batch entry point,
with the FP32 tolerance the other render tests use.  This file sorts last so
that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_1609_05344_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_05344_gb300 import _native, api as A
    _native.build()
    return A


def _view_array(N, views, outs):
    arr = (N.View * len(views))()
    for i, v in enumerate(views):
        arr[i] = N.View(N.camera(v["camera"]), v["width"], v["height"], v["steps"],
                        v["jitter_frame"], outs[i].data_ptr())
    return arr


def test_static_scratch_entry_matches_batch(api):
    import torch
    from paper_1609_05344_gb300 import _native as N
    vol = api.Volume(I.volume_desc("full", seed=3))
    prm = I.params()
    views = I.random_views(9, seed=21, max_size=(180, 120), min_size=(5, 3))
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = N.params(prm)
    for call in range(2):
        if call == 1:  # new cameras and jitter frames, same scratch
            views = [dict(v, camera=I.camera(np.array(v["camera"]["pos"]) + [120.0, -40.0, 0.0],
                                             33.0 * (i + 1), 14.0), jitter_frame=v["jitter_frame"] + 7)
                     for i, v in enumerate(views)]
        arr = _view_array(N, views, outs)
        rc = N.lib().cloud_batch_render_static(vol.handle, ctypes.byref(p), 6, 0, arr, len(views),
                                               stream)
        assert rc == 0, N.lib().cloud_last_error_message()
        got = [o.cpu().numpy() for o in outs]
        ref_batch = api.Batch(vol, prm, views)
        ref = [o.cpu().numpy() for o in ref_batch.render()]
        ref_batch.close()
        for g, r in zip(got, ref):
            assert np.abs(g - r).max() <= TOL_FP32


def test_static_scratch_rejects_too_many_views(api):
    import torch
    from paper_1609_05344_gb300 import _native as N
    vol = api.Volume(I.volume_desc("tiny"))
    out = torch.empty((4, 4, 4), device="cuda")
    v = dict(camera=I.ground_camera(), width=4, height=4, steps=4, jitter_frame=0)
    arr = _view_array(N, [v] * (N.STATIC_MAX_VIEWS + 1), [out] * (N.STATIC_MAX_VIEWS + 1))
    p = N.params(I.params())
    rc = N.lib().cloud_batch_render_static(vol.handle, ctypes.byref(p), 6, 0, arr,
                                           N.STATIC_MAX_VIEWS + 1, None)
    assert rc == N.ERR_INVALID_ARG
    assert b"256" in N.lib().cloud_last_error_message()
