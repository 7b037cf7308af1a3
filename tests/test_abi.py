"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol that
include/pt.h declares; argument validation that needs no device is checked too."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_t")))


def test_library_exports_every_declared_symbol():
    from paper_2407_19977_gb300 import native
    lib = native.load()
    declared = _declared_functions()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps each of them with the same name
    assert set(declared) <= set(native.SIGNATURES)


def test_status_strings_and_struct_sizes():
    from paper_2407_19977_gb300 import native as N
    lib = N.load()
    for code, name in enumerate(N.STATUS):
        assert lib.pt_status_string(code).decode() == name
    assert C.sizeof(N.pt_openpbr) == 34 * 4
    assert C.sizeof(N.pt_quad_light) == 13 * 4
    assert C.sizeof(N.pt_camera) == 14 * 4
    assert C.sizeof(N.pt_accum) == 32
    assert C.sizeof(N.pt_bvh_opts) == 24   # leaf_size, builder, collapse, tri_cost, box_cost, max_width
    assert C.sizeof(N.pt_stats) == 26 * 8   # 21 counters, error_flags + bvh_width, 4 box-test counters
    assert (N.PT_BVH_LBVH, N.PT_BVH_PLOC, N.PT_COLLAPSE_OPTIMAL, N.PT_COLLAPSE_GREEDY) == (1, 2, 1, 2)


def test_host_side_validation_needs_no_gpu():
    import numpy as np
    from paper_2407_19977_gb300 import native as N
    lib = N.load()
    h = C.c_void_p()
    # no triangles and no lights
    assert lib.pt_scene_create(None, 0, None, 0, None, None, 0, None, 0, None, 0, 0, 0, None, C.byref(h)) == 1
    # a material out of range is rejected before any device work
    v = np.zeros((3, 3), np.float32)
    idx = np.array([[0, 1, 2]], np.uint32)
    mid = np.zeros(1, np.uint32)
    m = (N.pt_openpbr * 1)()
    m[0].v[:] = [1, .8, .8, .8, 0, 0, 1, 1, 1, 1, .3, 0.9, 0, 1, 1, 1, 0, 1, 1, 1, 0, 1.6, 0, 1, 1, 1, 0, 0, 0,
                 0, 1, 1, 1, .5]  # ior 0.9
    code = lib.pt_scene_create(v.ctypes.data_as(C.c_void_p), 3, idx.ctypes.data_as(C.c_void_p), 1,
                               mid.ctypes.data_as(C.c_void_p), m, 1, None, 0, None, 0, 0, 0, None, C.byref(h))
    assert code == 1 and b"specular_ior" in lib.pt_last_error()
    idx_bad = np.array([[0, 1, 7]], np.uint32)
    m[0].v[11] = 1.5
    code = lib.pt_scene_create(v.ctypes.data_as(C.c_void_p), 3, idx_bad.ctypes.data_as(C.c_void_p), 1,
                               mid.ctypes.data_as(C.c_void_p), m, 1, None, 0, None, 0, 0, 0, None, C.byref(h))
    assert code == 1 and b"index" in lib.pt_last_error()
    m[0].v[26] = 0.5                      # geometry_thin_walled is 0 or 1
    code = lib.pt_scene_create(v.ctypes.data_as(C.c_void_p), 3, idx.ctypes.data_as(C.c_void_p), 1,
                               mid.ctypes.data_as(C.c_void_p), m, 1, None, 0, None, 0, 0, 0, None, C.byref(h))
    assert code == 1 and b"thin_walled" in lib.pt_last_error()
    m[0].v[26] = 0.0
    # anisotropy, rotation and the fuzz parameters in [0, 1]
    for i, bad in ((27, 1.5), (28, -0.25), (29, 1.25), (31, -0.5), (33, 2.0)):
        m[0].v[i] = bad
        code = lib.pt_scene_create(v.ctypes.data_as(C.c_void_p), 3, idx.ctypes.data_as(C.c_void_p), 1,
                                   mid.ctypes.data_as(C.c_void_p), m, 1, None, 0, None, 0, 0, 0, None, C.byref(h))
        assert code == 1 and f"parameter {i} ".encode() in lib.pt_last_error()
        m[0].v[i] = 0.5
    assert lib.pt_render(None, None, 1, 1, 0, None, None, None) == 1


def test_restir_and_denoiser_arguments_are_checked_on_the_host():
    """The ReSTIR options and the denoiser entry points reject bad arguments before any CUDA
    call (no GPU needed); pt_restir_opts and pt_render_opts have the declared layout."""
    from paper_2407_19977_gb300 import native as N
    lib = N.load()
    assert C.sizeof(N.pt_restir_opts) == 16
    assert N.pt_render_opts.restir.offset % 8 == 0
    # traversal and tail_bounce close the struct: 96 bytes on a 64-bit host
    assert (N.pt_render_opts.traversal.offset, N.pt_render_opts.tail_bounce.offset) == (88, 92)
    assert C.sizeof(N.pt_render_opts) == 96
    buf = (C.c_float * 48)()
    # NULL pointers, block outside 4..32, offset not below the block
    assert lib.pt_denoise_bmfr(None, None, 4, 4, 16, 0, 0, None, None) == 1
    for block, ox, oy in ((3, 0, 0), (33, 0, 0), (16, 16, 0), (16, 0, 17)):
        assert lib.pt_denoise_bmfr(buf, buf, 2, 2, block, ox, oy, buf, None) == 1, (block, ox, oy)
    assert lib.pt_render_features(None, None, 0, 0, 1, 1, 0, 1, C.c_uint64(0), None, None) == 1
    # an empty image is a no-op
    aligned = (C.c_float * 64)()
    addr = C.addressof(aligned)
    p = C.c_void_p(addr + (-addr) % 16)
    assert lib.pt_denoise_bmfr(p, p, 0, 5, 16, 0, 0, p, None) == 0
