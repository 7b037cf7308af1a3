"""Thin ctypes binding of include/pt.h: same names, argument marshalling only.

Every computation happens in libpt_gb300.so (CUDA, sm_103a).  PyTorch is used for device
memory and streams: tensors are passed by data_ptr(), streams by cuda_stream handle.
Loading fails loudly if the library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

u32 = C.c_uint32
u64 = C.c_uint64
f32 = C.c_float
vp = C.c_void_p


class pt_openpbr(C.Structure):
    _fields_ = [("v", f32 * 34)]


class pt_quad_light(C.Structure):
    _fields_ = [("p0", f32 * 3), ("e1", f32 * 3), ("e2", f32 * 3), ("radiance", f32 * 3),
                ("two_sided", C.c_int32)]


class pt_camera(C.Structure):
    _fields_ = [("origin", f32 * 3), ("target", f32 * 3), ("up", f32 * 3), ("vfov_deg", f32),
                ("width", u32), ("height", u32), ("lens_radius", f32), ("focus_distance", f32)]


class pt_accum(C.Structure):
    _fields_ = [("sum", vp), ("comp", vp), ("spp_done", u64), ("width", u32), ("height", u32)]


class pt_restir_opts(C.Structure):
    _fields_ = [("candidates", u32), ("spatial_neighbors", u32), ("spatial_radius", u32), ("later_candidates", u32)]


class pt_render_opts(C.Structure):
    _fields_ = [("crop_x0", u32), ("crop_y0", u32), ("flags", u32), ("mode", u32), ("wave_paths", u32),
                ("sort_by_material", C.c_int32), ("block_size", u32), ("sample_out", vp), ("nrc", vp),
                ("nrc_train", u32), ("kernel_ms", C.POINTER(f32)), ("kernel_launches", C.POINTER(u32)),
                ("tail_paths", C.c_int32), ("use_graph", u32), ("restir", C.POINTER(pt_restir_opts)),
                ("traversal", u32), ("tail_bounce", u32)]


class pt_bvh_opts(C.Structure):
    _fields_ = [("leaf_size", u32), ("builder", u32), ("collapse", u32), ("tri_cost", C.c_float),
                ("box_cost", C.c_float), ("max_width", u32)]


class pt_stats(C.Structure):
    _fields_ = [("ext_rays", u64), ("shadow_rays", u64), ("paths", u64), ("nan_dropped", u64),
                ("rr_terminated", u64), ("nrc_queries", u64), ("kernel_launches", u64), ("bvh_nodes", u64),
                ("bvh_depth", u64), ("n_triangles", u64), ("trace_nodes", u64), ("trace_tris", u64),
                ("shadow_nodes", u64), ("shadow_tris", u64), ("tail_ext_rays", u64), ("tail_shadow_rays", u64),
                ("tail_trace_nodes", u64), ("tail_trace_tris", u64), ("tail_shadow_nodes", u64),
                ("tail_shadow_tris", u64), ("graph_replays", u64), ("error_flags", u32), ("bvh_width", u32),
                ("trace_boxes", u64), ("shadow_boxes", u64), ("tail_trace_boxes", u64), ("tail_shadow_boxes", u64)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class pt_job(C.Structure):
    _fields_ = [("scene", vp), ("camera", pt_camera), ("spp", u32), ("max_depth", u32), ("seed", u64),
                ("accum", C.POINTER(pt_accum))]


class pt_batch_opts(C.Structure):
    _fields_ = [("mode", u32), ("streams", u32), ("tile_pixels", u32), ("blocks_per_sm", u32), ("use_graph", u32),
                ("merged", u32), ("wave_paths", u32)]


class pt_nrc_opts(C.Structure):
    _fields_ = [("n_levels", u32), ("log2_table", u32), ("base_resolution", u32), ("per_level_scale", f32),
                ("n_hidden", u32), ("learning_rate", f32), ("batch", u32), ("seed", u64),
                ("scene_min", f32 * 3), ("scene_max", f32 * 3), ("frame_samples", u32), ("tcgen05", u32),
                ("train_kernels", u32)]


PT_OK = 0
PT_ERR_INVALID_ARG = 1
STATUS = ["PT_OK", "PT_ERR_INVALID_ARG", "PT_ERR_OOM", "PT_ERR_CUDA", "PT_ERR_NOT_BUILT", "PT_ERR_TIMEOUT",
          "PT_ERR_QUEUE_OVERFLOW", "PT_ERR_UNSUPPORTED"]
PT_FLAG_NO_NEE = 1
PT_FLAG_NO_RR = 2
PT_FLAG_COUNT = 4
PT_TRAVERSAL_AUTO, PT_TRAVERSAL_PER_LANE, PT_TRAVERSAL_COOP = 0, 1, 2
PT_BVH_DEFAULT, PT_BVH_LBVH, PT_BVH_PLOC = 0, 1, 2
PT_COLLAPSE_DEFAULT, PT_COLLAPSE_OPTIMAL, PT_COLLAPSE_GREEDY = 0, 1, 2
PT_TUNE_BVH = 1
PT_TONEMAP_SRGB = 1
KERNEL_KINDS = ("raygen", "trace", "sort", "shade", "shadow", "accum", "tail", "restir")
PT_MODE_AUTO, PT_MODE_WAVEFRONT, PT_MODE_MEGAKERNEL = 0, 1, 2

# symbol -> (restype, argtypes); every symbol declared in include/pt.h
SIGNATURES = {
    "pt_scene_create": (C.c_int, [vp, u32, vp, u32, vp, C.POINTER(pt_openpbr), u32, C.POINTER(pt_quad_light), u32,
                                  vp, u32, u32, C.c_int, vp, C.POINTER(vp)]),
    "pt_bvh_build": (C.c_int, [vp, C.POINTER(pt_bvh_opts), vp]),
    "pt_render": (C.c_int, [vp, C.POINTER(pt_camera), u32, u32, u64, C.POINTER(pt_accum),
                            C.POINTER(pt_render_opts), vp]),
    "pt_render_noalloc": (C.c_int, [vp, C.POINTER(pt_camera), u32, u32, u64, C.POINTER(pt_accum),
                                    C.POINTER(pt_render_opts), vp]),
    "pt_render_batch": (C.c_int, [C.POINTER(pt_job), u32, C.POINTER(pt_batch_opts), vp]),
    "pt_tonemap": (C.c_int, [C.POINTER(pt_accum), f32, u32, vp, vp]),
    "pt_render_features": (C.c_int, [vp, C.POINTER(pt_camera), u32, u32, u32, u32, u32, u32, C.c_uint64, vp, vp]),
    "pt_denoise_bmfr": (C.c_int, [vp, vp, u32, u32, u32, u32, u32, vp, vp]),
    "pt_autotune": (C.c_int, [vp, C.POINTER(pt_camera), u32, u32, u32, u32, C.POINTER(pt_render_opts),
                              C.POINTER(f32), vp]),
    "pt_autotune_batch": (C.c_int, [C.POINTER(pt_job), u32, u32, u32, C.POINTER(pt_batch_opts), C.POINTER(f32),
                                     vp]),
    "pt_trace": (C.c_int, [vp, vp, u32, C.c_int, vp, vp, vp, vp]),
    "pt_bsdf_eval": (C.c_int, [vp, vp, vp, vp, u32, vp, vp, vp]),
    "pt_bsdf_sample": (C.c_int, [vp, vp, vp, vp, u32, vp, vp, vp, vp, vp]),
    "pt_camera_rays": (C.c_int, [C.POINTER(pt_camera), u64, vp, u32, vp, vp]),
    "pt_uniforms": (C.c_int, [u64, vp, u32, vp, vp]),
    "pt_env_sample": (C.c_int, [vp, vp, u32, vp, vp, vp]),
    "pt_env_pdf": (C.c_int, [vp, vp, u32, vp, vp]),
    "pt_bvh_export": (C.c_int, [vp, vp, vp, C.POINTER(u32), C.POINTER(u32), vp]),
    "pt_get_stats": (C.c_int, [vp, C.POINTER(pt_stats)]),
    "pt_scene_sync": (C.c_int, [vp]),
    "pt_scene_destroy": (None, [vp]),
    "pt_launch_count": (u64, []),
    "pt_nrc_create": (C.c_int, [C.POINTER(pt_nrc_opts), vp, C.POINTER(vp)]),
    "pt_nrc_train": (C.c_int, [vp, vp, u32, vp]),
    "pt_nrc_infer": (C.c_int, [vp, vp, u32, vp, vp]),
    "pt_nrc_gradients": (C.c_int, [vp, vp, u32, vp, vp, vp]),
    "pt_nrc_params": (C.c_int, [vp, C.c_int, C.POINTER(vp), C.POINTER(u64)]),
    "pt_nrc_commit": (C.c_int, [vp, vp]),
    "pt_nrc_last_loss": (C.c_int, [vp, C.POINTER(f32)]),
    "pt_nrc_destroy": (None, [vp]),
    "pt_status_string": (C.c_char_p, [C.c_int]),
    "pt_last_error": (C.c_char_p, []),
}


class PtError(RuntimeError):
    def __init__(self, fn, code, detail):
        self.code = code
        name = STATUS[code] if 0 <= code < len(STATUS) else str(code)
        super().__init__(f"{fn} -> {name}: {detail}")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpt_gb300.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2407_19977_gb300.build.build() (needs nvcc)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(fn_name: str, code: int):
    if code != PT_OK:
        detail = load().pt_last_error().decode(errors="replace")
        raise PtError(fn_name, code, detail)


def call(fn_name: str, *args):
    """Call a status-returning entry point and raise PtError on failure."""
    code = getattr(load(), fn_name)(*args)
    check(fn_name, code)
    return code
