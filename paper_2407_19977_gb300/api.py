"""Convenience layer over the C-ABI binding (native.py): scenes, accumulators, rendering.

Torch tensors hold the device buffers; every computation is a call into libpt_gb300.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native as N


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def make_camera(cam) -> N.pt_camera:
    c = N.pt_camera()
    c.origin[:] = [float(x) for x in cam.origin]
    c.target[:] = [float(x) for x in cam.target]
    c.up[:] = [float(x) for x in cam.up]
    c.vfov_deg = float(cam.vfov_deg)
    c.width = int(cam.width)
    c.height = int(cam.height)
    c.lens_radius = float(getattr(cam, "lens_radius", 0.0))
    c.focus_distance = float(getattr(cam, "focus_distance", 1.0))
    return c


class Accum:
    """Caller-owned progressive accumulator (Kahan sum + compensation, float32 RGB)."""

    def __init__(self, width: int, height: int, device="cuda"):
        self.sum = torch.zeros((height, width, 3), dtype=torch.float32, device=device)
        self.comp = torch.zeros((height, width, 3), dtype=torch.float32, device=device)
        self.c = N.pt_accum(C.c_void_p(self.sum.data_ptr()), C.c_void_p(self.comp.data_ptr()), 0, width, height)

    @property
    def spp_done(self) -> int:
        return int(self.c.spp_done)

    def reset(self):
        self.sum.zero_()
        self.comp.zero_()
        self.c.spp_done = 0

    def image(self) -> torch.Tensor:
        return self.sum / max(self.spp_done, 1)

    def tonemap(self, exposure=1.0, srgb=True, out=None, stream=None) -> torch.Tensor:
        """Display resolve through pt_tonemap: (height, width, 4) uint8 RGBA on the device."""
        h, w = self.sum.shape[0], self.sum.shape[1]
        if out is None:
            out = torch.empty((h, w, 4), dtype=torch.uint8, device=self.sum.device)
        N.call("pt_tonemap", C.byref(self.c), float(exposure), N.PT_TONEMAP_SRGB if srgb else 0, _ptr(out),
               _stream_handle(stream))
        return out


class Scene:
    """A scene uploaded through pt_scene_create and (by default) built with pt_bvh_build."""

    def __init__(self, sc, stream=None, build=True, leaf_size=4, on_device=False, builder=0):
        lib = N.load()
        self.desc = sc
        self._stream = stream
        v = np.ascontiguousarray(sc.vertices, dtype=np.float32)
        idx = np.ascontiguousarray(sc.indices, dtype=np.uint32)
        mid = np.ascontiguousarray(sc.material_ids, dtype=np.uint32)
        mats = (N.pt_openpbr * len(sc.materials))()
        for i, row in enumerate(np.asarray(sc.materials, dtype=np.float32)):
            mats[i].v[:] = [float(x) for x in row]
        nq = len(sc.lights)
        quads = (N.pt_quad_light * max(nq, 1))()
        for i, q in enumerate(np.asarray(sc.lights, dtype=np.float32)):
            quads[i].p0[:] = [float(x) for x in q[0:3]]
            quads[i].e1[:] = [float(x) for x in q[3:6]]
            quads[i].e2[:] = [float(x) for x in q[6:9]]
            quads[i].radiance[:] = [float(x) for x in q[9:12]]
            quads[i].two_sided = int(q[12] != 0)
        env = None if sc.env is None else np.ascontiguousarray(sc.env, dtype=np.float32)
        keep = []
        if on_device:
            tv = torch.from_numpy(v).cuda()
            ti = torch.from_numpy(idx.view(np.int32)).cuda()
            tm = torch.from_numpy(mid.view(np.int32)).cuda()
            te = None if env is None else torch.from_numpy(env).cuda()
            keep += [tv, ti, tm, te]
            pv, pi, pm = _ptr(tv), _ptr(ti), _ptr(tm)
            pe = _ptr(te) if te is not None else None
        else:
            pv = v.ctypes.data_as(C.c_void_p)
            pi = idx.ctypes.data_as(C.c_void_p)
            pm = mid.ctypes.data_as(C.c_void_p)
            pe = env.ctypes.data_as(C.c_void_p) if env is not None else None
        h = C.c_void_p()
        ew, eh = (0, 0) if env is None else (env.shape[1], env.shape[0])
        N.call("pt_scene_create", pv, v.shape[0], pi, idx.shape[0], pm, mats, len(sc.materials),
               quads if nq else None, nq, pe, ew, eh, 1 if on_device else 0, _stream_handle(stream), C.byref(h))
        torch.cuda.synchronize()
        self.h = h
        self.n_tris = idx.shape[0] + 2 * nq
        if build:
            self.build(leaf_size, builder=builder)

    def build(self, leaf_size=4, stream=None, builder=0, collapse=0, tri_cost=0.0, box_cost=0.0, max_width=0):
        """pt_bvh_build; builder N.PT_BVH_LBVH or N.PT_BVH_PLOC (0: the default, PLOC); collapse
        N.PT_COLLAPSE_OPTIMAL or N.PT_COLLAPSE_GREEDY (0: optimal) with tri_cost and box_cost
        (0: defaults); max_width the most children of a node, 2..8 (0: 8)."""
        o = N.pt_bvh_opts(leaf_size, builder, collapse, float(tri_cost), float(box_cost), int(max_width))
        N.call("pt_bvh_build", self.h, C.byref(o), _stream_handle(stream))

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                N.load().pt_scene_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def render(self, spp, max_depth=None, seed=0, accum=None, camera=None, crop=None, flags=0,
               mode=N.PT_MODE_AUTO, wave_paths=0, sort=-1, sample_out=None, block_size=0, stream=None,
               kernel_ms=None, kernel_launches=None, nrc=None, nrc_train=False, tail_paths=0, use_graph=False,
               restir=None, traversal=N.PT_TRAVERSAL_AUTO, tail_bounce=0):
        cam = camera or self.desc.camera
        max_depth = self.desc.max_depth if max_depth is None else max_depth
        if crop is None:
            crop = (0, 0, cam.width, cam.height)
        x0, y0, cw, ch = crop
        if accum is None:
            accum = Accum(cw, ch)
        o = N.pt_render_opts()
        o.crop_x0, o.crop_y0, o.flags, o.mode = x0, y0, flags, mode
        o.wave_paths, o.sort_by_material, o.block_size = wave_paths, sort, block_size
        o.tail_paths = int(tail_paths)
        o.use_graph = 1 if use_graph else 0
        o.traversal = int(traversal)
        o.tail_bounce = int(tail_bounce)
        if restir is not None:
            # (M candidates, K neighbours, radius R[, L later candidates]): ReSTIR DI at the
            # primary vertex, resampled next-event estimation at later vertices if L > 0
            r4 = (tuple(restir) + (0,))[:4]
            ro = N.pt_restir_opts(int(r4[0]), int(r4[1]), int(r4[2]), int(r4[3]))
            o.restir = C.pointer(ro)
        o.sample_out = _ptr(sample_out) if sample_out is not None else None
        if nrc is not None:
            o.nrc = nrc.h
            o.nrc_train = 1 if nrc_train else 0
        if kernel_ms is not None:
            o.kernel_ms = C.cast(kernel_ms, C.POINTER(N.f32))
        if kernel_launches is not None:
            o.kernel_launches = C.cast(kernel_launches, C.POINTER(N.u32))
        N.call("pt_render", self.h, C.byref(make_camera(cam)), int(spp), int(max_depth), C.c_uint64(int(seed)),
               C.byref(accum.c), C.byref(o), _stream_handle(stream))
        return accum

    def features(self, spp, s0=0, seed=0, crop=None, camera=None, stream=None) -> torch.Tensor:
        """pt_render_features: (h, w, 12) primary-hit features (normal, scattering fraction,
        position, albedo) averaged over the samples s0 .. s0+spp-1 of pt_render's rays."""
        cam = camera or self.desc.camera
        x0, y0, cw, ch = crop if crop is not None else (0, 0, cam.width, cam.height)
        out = torch.empty((ch, cw, 12), dtype=torch.float32, device="cuda")
        N.call("pt_render_features", self.h, C.byref(make_camera(cam)), x0, y0, cw, ch, int(s0), int(spp),
               C.c_uint64(int(seed)), _ptr(out), _stream_handle(stream))
        return out

    def autotune(self, spp=1, max_depth=None, frames=2, bvh=False, camera=None, stream=None):
        """pt_autotune: the fastest schedule for frames like this one (stored in the scene for
        PT_MODE_AUTO).  Returns (options dict, ms per frame)."""
        cam = camera or self.desc.camera
        max_depth = self.desc.max_depth if max_depth is None else max_depth
        best = N.pt_render_opts()
        ms = N.f32()
        N.call("pt_autotune", self.h, C.byref(make_camera(cam)), int(spp), int(max_depth), int(frames),
               N.PT_TUNE_BVH if bvh else 0, C.byref(best), C.byref(ms), _stream_handle(stream))
        keys = ("mode", "wave_paths", "sort_by_material", "block_size", "tail_paths", "use_graph", "traversal",
                "tail_bounce")
        return {k: int(getattr(best, k)) for k in keys}, float(ms.value)

    def trace(self, origins: torch.Tensor, dirs: torch.Tensor, tmax=None, any_hit=False, count=False,
              coop=False, stream=None):
        n = origins.shape[0]
        rays = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
        rays[:, 0:3] = origins
        rays[:, 3:6] = dirs
        rays[:, 6] = float("inf") if tmax is None else tmax
        tri = torch.empty(n, dtype=torch.int32, device="cuda")
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        uv = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        flags = (1 if any_hit else 0) | (2 if count else 0) | (4 if coop else 0)
        N.call("pt_trace", self.h, _ptr(rays), n, flags, _ptr(tri), _ptr(t), _ptr(uv), _stream_handle(stream))
        return tri, t, uv

    def env_sample(self, u: torch.Tensor, stream=None):
        n = u.shape[0]
        d = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        p = torch.empty(n, dtype=torch.float32, device="cuda")
        N.call("pt_env_sample", self.h, _ptr(u.contiguous()), n, _ptr(d), _ptr(p), _stream_handle(stream))
        return d, p

    def env_pdf(self, dirs: torch.Tensor, stream=None):
        n = dirs.shape[0]
        p = torch.empty(n, dtype=torch.float32, device="cuda")
        N.call("pt_env_pdf", self.h, _ptr(dirs.contiguous()), n, _ptr(p), _stream_handle(stream))
        return p

    def export_bvh(self):
        """Host copies of the wide BVH nodes (n, 20) uint32 and leaf-ordered triangles (m, 12)."""
        nn, nt = N.u32(), N.u32()
        N.call("pt_bvh_export", self.h, None, None, C.byref(nn), C.byref(nt), _stream_handle())
        nodes = np.zeros((nn.value, 20), dtype=np.uint32)
        tris = np.zeros((nt.value, 12), dtype=np.float32)
        N.call("pt_bvh_export", self.h, nodes.ctypes.data_as(C.c_void_p), tris.ctypes.data_as(C.c_void_p),
               C.byref(nn), C.byref(nt), _stream_handle())
        return nodes, tris

    def stats(self) -> dict:
        s = N.pt_stats()
        N.call("pt_get_stats", self.h, C.byref(s))
        return s.as_dict()


def bsdf_eval(mats: torch.Tensor, front: torch.Tensor, wo: torch.Tensor, wi: torch.Tensor, stream=None):
    n = wo.shape[0]
    f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pdf = torch.empty(n, dtype=torch.float32, device="cuda")
    N.call("pt_bsdf_eval", _ptr(mats), _ptr(front), _ptr(wo), _ptr(wi), n, _ptr(f), _ptr(pdf), _stream_handle(stream))
    return f, pdf


def bsdf_sample(mats, front, wo, u, stream=None):
    n = wo.shape[0]
    wi = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    w = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    pdf = torch.empty(n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.int32, device="cuda")
    N.call("pt_bsdf_sample", _ptr(mats), _ptr(front), _ptr(wo), _ptr(u), n, _ptr(wi), _ptr(w), _ptr(pdf), _ptr(fl),
           _stream_handle(stream))
    return wi, w, pdf, fl


def camera_rays(camera, seed, pixels: torch.Tensor, stream=None):
    n = pixels.shape[0]
    out = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    N.call("pt_camera_rays", C.byref(make_camera(camera)), C.c_uint64(int(seed)), _ptr(pixels), n, _ptr(out),
           _stream_handle(stream))
    return out


def uniforms(seed, keys: torch.Tensor, stream=None):
    n = keys.shape[0]
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    N.call("pt_uniforms", C.c_uint64(int(seed)), _ptr(keys), n, _ptr(out), _stream_handle(stream))
    return out


def bmfr(color: torch.Tensor, features: torch.Tensor, block=32, offset=(0, 0), out=None, stream=None) -> torch.Tensor:
    """pt_denoise_bmfr: blockwise feature regression of a mean-radiance image (h, w, 3) on the
    primary-hit features (h, w, 12) of Scene.features; returns the denoised (h, w, 3)."""
    h, w = color.shape[0], color.shape[1]
    color = color.contiguous()
    features = features.contiguous()
    if out is None:
        out = torch.empty_like(color)
    N.call("pt_denoise_bmfr", _ptr(color), _ptr(features), w, h, int(block), int(offset[0]), int(offset[1]),
           _ptr(out), _stream_handle(stream))
    return out


def render_batch(jobs, tile_pixels=0, blocks_per_sm=0, use_graph=False, mode=0, streams=0, merged=False,
                 wave_paths=0, stream=None):
    """jobs: list of (Scene, camera, spp, max_depth, seed, Accum).  merged (wavefront mode):
    one wavefront whose waves hold the paths of every job."""
    arr = _job_array(jobs)
    o = N.pt_batch_opts(mode, streams, tile_pixels, blocks_per_sm, 1 if use_graph else 0, 1 if merged else 0,
                        int(wave_paths))
    N.call("pt_render_batch", arr, len(jobs), C.byref(o), _stream_handle(stream))


def _job_array(jobs):
    arr = (N.pt_job * len(jobs))()
    for i, (scene, cam, spp, depth, seed, acc) in enumerate(jobs):
        arr[i].scene = scene.h
        arr[i].camera = make_camera(cam)
        arr[i].spp = spp
        arr[i].max_depth = depth
        arr[i].seed = seed
        arr[i].accum = C.pointer(acc.c)
    return arr


def autotune_batch(jobs, frames=2, stream=None, bvh=False):
    """pt_autotune_batch over (Scene, camera, spp, max_depth, seed, Accum) jobs; the jobs'
    accumulators are not touched.  With bvh the jobs' scenes are rebuilt at the fastest BVH
    width first (N.PT_TUNE_BVH).  Returns (the chosen pt_batch_opts fields, ms per batch)."""
    arr = _job_array(jobs)
    best = N.pt_batch_opts()
    ms = N.f32()
    N.call("pt_autotune_batch", arr, len(jobs), int(frames), N.PT_TUNE_BVH if bvh else 0, C.byref(best),
           C.byref(ms), _stream_handle(stream))
    return {"mode": int(best.mode), "streams": int(best.streams), "tile_pixels": int(best.tile_pixels),
            "blocks_per_sm": int(best.blocks_per_sm), "use_graph": int(best.use_graph),
            "merged": int(best.merged), "wave_paths": int(best.wave_paths)}, float(ms.value)


def launch_count() -> int:
    return int(N.load().pt_launch_count())


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory (no copy)."""

    def __init__(self, ptr, n, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Nrc:
    """Neural radiance cache (hash grid + 64-wide MLP) owned by the library."""

    def __init__(self, n_levels=16, log2_table=19, base_resolution=16, per_level_scale=0.0, learning_rate=1e-2,
                 batch=8192, seed=0, box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), frame_samples=32768, tcgen05=False,
                 train_kernels=0, stream=None):
        o = N.pt_nrc_opts()
        o.n_levels, o.log2_table, o.base_resolution = n_levels, log2_table, base_resolution
        o.per_level_scale, o.n_hidden, o.learning_rate, o.batch, o.seed = per_level_scale, 4, learning_rate, batch, seed
        o.scene_min[:] = [float(x) for x in box[0]]
        o.scene_max[:] = [float(x) for x in box[1]]
        o.frame_samples = int(frame_samples)
        o.tcgen05 = 1 if tcgen05 else 0
        o.train_kernels = int(train_kernels)
        self.opts = o
        h = C.c_void_p()
        N.call("pt_nrc_create", C.byref(o), _stream_handle(stream), C.byref(h))
        self.h = h
        self.n_levels, self.log2_table = n_levels, log2_table

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                N.load().pt_nrc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def params(self, which: int) -> torch.Tensor:
        """Live FP32 view of the MLP weights (0) or the grid table (1); call commit() after writing."""
        p, n = C.c_void_p(), N.u64()
        N.call("pt_nrc_params", self.h, which, C.byref(p), C.byref(n))
        return torch.as_tensor(_DevArray(p.value, n.value), device="cuda")

    def commit(self, stream=None):
        N.call("pt_nrc_commit", self.h, _stream_handle(stream))

    def infer(self, queries: torch.Tensor, stream=None) -> torch.Tensor:
        n = queries.shape[0]
        out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        N.call("pt_nrc_infer", self.h, _ptr(queries.contiguous()), n, _ptr(out), _stream_handle(stream))
        return out[:, :3]

    def train(self, samples: torch.Tensor, stream=None):
        N.call("pt_nrc_train", self.h, _ptr(samples.contiguous()), samples.shape[0], _stream_handle(stream))

    def gradients(self, samples: torch.Tensor, stream=None):
        nw = self.params(0).numel()
        ng = self.params(1).numel()
        dw = torch.empty(nw, dtype=torch.float32, device="cuda")
        dg = torch.empty(ng, dtype=torch.float32, device="cuda")
        N.call("pt_nrc_gradients", self.h, _ptr(samples.contiguous()), samples.shape[0], _ptr(dw), _ptr(dg),
               _stream_handle(stream))
        return dw, dg

    def last_loss(self) -> float:
        v = N.f32()
        N.call("pt_nrc_last_loss", self.h, C.byref(v))
        return float(v.value)
