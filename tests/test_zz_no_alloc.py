"""pt_render_noalloc: rendering for callers that may not allocate device memory.

A host program under a fixed device-memory budget, or embedded in an application that
owns all device allocations, cannot let the library call cudaMalloc.  pt_render_noalloc
runs the per-bounce wavefront kernels of pt_render with its work queues in a fixed array
compiled into the library, so its accumulators must equal pt_render's bit for bit, call for
call.  This file is collected last so that a failure here does not hide the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_PIXELS = 16384


def _call_noalloc(scene, cam, spp, depth, seed, acc, crop=(0, 0), flags=0):
    from paper_2407_19977_gb300 import api
    from paper_2407_19977_gb300 import native as N
    opts = N.pt_render_opts()
    opts.sort_by_material = -1
    opts.crop_x0, opts.crop_y0 = crop
    opts.flags = flags
    return N.load().pt_render_noalloc(scene.h, C.byref(api.make_camera(cam)), spp, depth, C.c_uint64(seed),
                                      C.byref(acc.c), C.byref(opts), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _same(out, ref):
    torch.cuda.synchronize()
    assert out.spp_done == ref.spp_done
    assert torch.equal(out.sum, ref.sum) and torch.equal(out.comp, ref.comp)


@pytest.mark.parametrize("width,height,calls", [
    (128, 96, ((3, 11), (2, 11))),      # 12,288 pixels: one sample per wave
    (64, 64, ((5, 7), (3, 7))),         # 4,096 pixels: four samples per wave, a ragged last wave
    (128, 128, ((2, 3), (1, 3))),       # exactly the array's 16,384 pixels
])
def test_noalloc_matches_pt_render_on_two_calls(width, height, calls):
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    sc = scenes.cornell_box(width=width, height=height, spp=1, max_depth=6)
    g = api.Scene(sc)
    ref = api.Accum(width, height)
    out = api.Accum(width, height)
    for spp, seed in calls:   # two calls in a row: the second continues the first
        g.render(spp, max_depth=6, seed=seed, accum=ref, mode=N.PT_MODE_WAVEFRONT)
        assert _call_noalloc(g, sc.camera, spp, 6, seed, out) == N.PT_OK
        _same(out, ref)
    assert g.stats()["error_flags"] == 0


def test_noalloc_tiles_equal_pt_render_crops_and_allocate_nothing():
    """A 256 x 128 frame (twice the array) rendered as four 128 x 64 tiles, each against
    pt_render's crop of the same window; the second pass over the tiles leaves the device's
    free memory unchanged."""
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    sc = scenes.pushbutton(width=256, height=128)
    g = api.Scene(sc)
    tiles = [(x0, y0) for y0 in (0, 64) for x0 in (0, 128)]
    refs = {t: api.Accum(128, 64) for t in tiles}
    outs = {t: api.Accum(128, 64) for t in tiles}
    free = []
    for p in range(2):
        for t in tiles:
            g.render(1, seed=5, accum=refs[t], crop=(t[0], t[1], 128, 64), mode=N.PT_MODE_WAVEFRONT)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        for t in tiles:
            assert _call_noalloc(g, sc.camera, 1, sc.max_depth, 5, outs[t], crop=t) == N.PT_OK
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        for t in tiles:
            _same(outs[t], refs[t])
    assert free[3] == free[2], (free, "the second pass changed the device's free memory")
    assert g.stats()["error_flags"] == 0


def test_noalloc_rejects_what_it_cannot_do():
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    sc = scenes.cornell_box(width=256, height=256, spp=1, max_depth=2)
    g = api.Scene(sc)
    acc = api.Accum(256, 256)   # 65,536 pixels > 16,384
    assert _call_noalloc(g, sc.camera, 1, 2, 0, acc) == N.PT_ERR_INVALID_ARG
    assert str(MAX_PIXELS).encode() in N.load().pt_last_error()
    assert acc.spp_done == 0
    small = api.Accum(128, 128)
    assert _call_noalloc(g, sc.camera, 1, 2, 0, small, flags=N.PT_FLAG_COUNT) == N.PT_ERR_INVALID_ARG
    assert small.spp_done == 0 and not bool(small.sum.any())
    assert _call_noalloc(g, sc.camera, 1, 2, 0, small, crop=(200, 0)) == N.PT_ERR_INVALID_ARG
