"""pt_render_noalloc: rendering for callers that may not allocate device memory.

A host program under a fixed device-memory budget, or embedded in an application that
owns all device allocations, cannot let the library call cudaMalloc.  pt_render_noalloc
runs the same wavefront kernels as pt_render with its work queues in a fixed array
compiled into the library, so its accumulators must match pt_render's call for call.
This file is collected last so that a failure here does not hide the other GPU tests.
"""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call_noalloc(scene, cam, spp, depth, seed, acc):
    from paper_2407_19977_gb300 import api
    from paper_2407_19977_gb300 import native as N
    opts = N.pt_render_opts()
    opts.sort_by_material = -1
    code = N.load().pt_render_noalloc(scene.h, C.byref(api.make_camera(cam)), spp, depth, C.c_uint64(seed),
                                      C.byref(acc.c), C.byref(opts), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code


def test_noalloc_matches_pt_render_on_two_calls():
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    sc = scenes.cornell_box(width=128, height=96, spp=1, max_depth=6)
    g = api.Scene(sc)
    ref = api.Accum(128, 96)
    out = api.Accum(128, 96)
    for spp, seed in ((3, 11), (2, 11)):   # two calls in a row: the second continues the first
        g.render(spp, max_depth=6, seed=seed, accum=ref, mode=N.PT_MODE_WAVEFRONT)
        assert _call_noalloc(g, sc.camera, spp, 6, seed, out) == N.PT_OK
        torch.cuda.synchronize()
        assert out.spp_done == ref.spp_done
        a = out.sum.cpu().numpy().astype(np.float64)
        b = ref.sum.cpu().numpy().astype(np.float64)
        rmse = math.sqrt(((a - b) ** 2).mean())
        assert rmse <= 1e-3 * b.mean() / max(ref.spp_done, 1) * ref.spp_done
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7)
    assert g.stats()["error_flags"] == 0


def test_noalloc_rejects_windows_beyond_its_array():
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    sc = scenes.cornell_box(width=256, height=256, spp=1, max_depth=2)
    g = api.Scene(sc)
    acc = api.Accum(256, 256)   # 65,536 pixels > 16,384
    assert _call_noalloc(g, sc.camera, 1, 2, 0, acc) == 1
    assert b"16384" in N.load().pt_last_error()
    assert acc.spp_done == 0
