"""CPU oracle for the path tracer -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
import this package.  The product path (paper_2407_19977_gb300) never imports it and
shares no code with it.

`pt_oracle.c` is a plain double-precision recursive path tracer written from the paper
("Physically-based Path Tracer using WebGPU and OpenPBR": Sec. 1.1 rendering equation,
Sec. 5.1.1 BVH, Sec. 5.1.2 ray generator, Sec. 5.1.3 path tracer, Sec. 5.1.4 progressive
averaging) plus the readings fixed where the paper is silent.  `nrc.py` is the NRC oracle
(hash-grid encoding + MLP, forward and backward) in numpy float64.

Parity status: every function here is pinned by tests under tests/test_oracle_*.py
(closed forms, Monte Carlo identities, brute force, a library Philox); none is unpinned
except the end-to-end NRC estimate, which is stochastic and biased by design.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int)
_i64p = C.POINTER(C.c_longlong)


def build(force: bool = False) -> str:
    """Compile pt_oracle.c with gcc into oracle/_build/liboracle.so (host code only)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.oracle_uniform.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64]
        lib.oracle_uniform.restype = C.c_double
        lib.oracle_fresnel_dielectric.argtypes = [C.c_double, C.c_double]
        lib.oracle_fresnel_dielectric.restype = C.c_double
        lib.oracle_fresnel_f82.argtypes = [_dp, _dp, C.c_double, _dp]
        lib.oracle_ggx_D.argtypes = [_dp, C.c_double, C.c_double]
        lib.oracle_ggx_D.restype = C.c_double
        lib.oracle_ggx_G1.argtypes = [_dp, C.c_double, C.c_double]
        lib.oracle_ggx_G1.restype = C.c_double
        lib.oracle_ggx_vndf_sample.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        lib.oracle_tangent_frame.argtypes = [_dp, _dp, C.c_double, _dp, _dp]
        lib.oracle_bsdf_eval.argtypes = [_dp, C.c_int, _dp, _dp, _dp, _dp]
        lib.oracle_bsdf_sample.argtypes = [_dp, C.c_int, _dp, _dp, _dp, _dp, _dp, _i32p]
        lib.oracle_bsdf_sample.restype = C.c_int
        lib.oracle_lobe_probs.argtypes = [_dp, C.c_int, C.c_double, _dp]
        lib.oracle_sheen_D.argtypes = [C.c_double, C.c_double]
        lib.oracle_sheen_D.restype = C.c_double
        lib.oracle_sheen_area.argtypes = [C.c_double, C.c_double]
        lib.oracle_sheen_area.restype = C.c_double
        lib.oracle_sheen_albedo.argtypes = [C.c_double, C.c_double]
        lib.oracle_sheen_albedo.restype = C.c_double
        lib.oracle_sheen_f.argtypes = [_dp, _dp, C.c_double]
        lib.oracle_sheen_f.restype = C.c_double
        lib.oracle_sah_reference.argtypes = [_dp, C.c_int, C.c_int, _dp]
        lib.oracle_scene_create.argtypes = [_dp, C.c_int, _u32p, C.c_int, _u32p, _dp, C.c_int,
                                            _dp, C.c_int, _dp, C.c_int, C.c_int, C.c_int]
        lib.oracle_scene_create.restype = C.c_void_p
        lib.oracle_scene_destroy.argtypes = [C.c_void_p]
        lib.oracle_scene_eps.argtypes = [C.c_void_p]
        lib.oracle_scene_eps.restype = C.c_double
        lib.oracle_intersect.argtypes = [C.c_void_p, _dp, C.c_int, C.c_int, _i32p, _dp, _dp]
        lib.oracle_env_sample.argtypes = [C.c_void_p, C.c_double, C.c_double, _dp, _dp, _dp]
        lib.oracle_env_sample.restype = C.c_int
        lib.oracle_env_pdf.argtypes = [C.c_void_p, _dp]
        lib.oracle_env_pdf.restype = C.c_double
        lib.oracle_render.argtypes = [C.c_void_p, _dp, C.c_double, C.c_int, C.c_int, C.c_int,
                                      C.c_int, C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_int,
                                      C.c_uint64, C.c_int, C.c_int, C.c_int, _dp, _dp, _i64p, _i32p]
        lib.oracle_features.argtypes = [C.c_void_p, _dp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_uint64, _dp]
        lib.oracle_camera_ray.argtypes = [_dp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_uint32, C.c_uint64, _dp, _dp]
        lib.oracle_bsdf_eval_batch.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        lib.oracle_bsdf_sample_batch.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp,
                                                 _i32p, _i32p]
        lib.oracle_uniform_batch.argtypes = [C.c_int, _u32p, _u32p, _u32p, _u32p, C.c_uint64, _dp]
        _lib = lib
        return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


# ----------------------------------------------------------------------------------------
# RNG
# ----------------------------------------------------------------------------------------

def philox4x32_10(counter, key):
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in counter])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(pixel, sample, bounce, dim, seed):
    return _load().oracle_uniform(pixel, sample, bounce, dim, seed)


# ----------------------------------------------------------------------------------------
# BSDF pieces (local frame: shading normal = +z)
# ----------------------------------------------------------------------------------------

def fresnel_dielectric(cos_i, eta):
    return _load().oracle_fresnel_dielectric(float(cos_i), float(eta))


def fresnel_f82(f0, tint, mu):
    f0, pf = _d(f0)
    t, pt = _d(tint)
    o = np.zeros(3)
    _load().oracle_fresnel_f82(pf, pt, float(mu), o.ctypes.data_as(_dp))
    return o


def ggx_D(h, alpha, alpha_y=None):
    """GGX D in the local frame; alpha along the tangent (x), alpha_y (default alpha) along y."""
    h, ph = _d(h)
    return _load().oracle_ggx_D(ph, float(alpha), float(alpha if alpha_y is None else alpha_y))


def ggx_G1(w, alpha, alpha_y=None):
    w, pw = _d(w)
    return _load().oracle_ggx_G1(pw, float(alpha), float(alpha if alpha_y is None else alpha_y))


def ggx_vndf_sample(wo, alpha, u1, u2, alpha_y=None):
    wo, p = _d(wo)
    o = np.zeros(3)
    _load().oracle_ggx_vndf_sample(p, float(alpha), float(alpha if alpha_y is None else alpha_y), float(u1),
                                   float(u2), o.ctypes.data_as(_dp))
    return o


def tangent_frame(n, e1, rot):
    """(t, b) of an anisotropic surface with normal n, first triangle edge e1, rotation rot turns."""
    n, pn = _d(n)
    e1, pe = _d(e1)
    t, b = np.zeros(3), np.zeros(3)
    _load().oracle_tangent_frame(pn, pe, float(rot), t.ctypes.data_as(_dp), b.ctypes.data_as(_dp))
    return t, b


def sheen_D(cos_m, alpha):
    """Charlie microfacet distribution of the fuzz lobe (width alpha)."""
    return _load().oracle_sheen_D(float(cos_m), float(alpha))


def sheen_area(mu, alpha):
    """Projected area A(mu) = int <w, m>+ D(m) dm of the fuzz distribution (G1 = mu / A)."""
    return _load().oracle_sheen_area(float(mu), float(alpha))


def sheen_albedo(mu, alpha):
    """Directional albedo E(mu) of the uncoloured fuzz lobe."""
    return _load().oracle_sheen_albedo(float(mu), float(alpha))


def sheen_f(wo, wi, alpha):
    """The uncoloured fuzz lobe f_s(wo, wi) (0 unless both are above the surface)."""
    wo, po = _d(wo)
    wi, pi = _d(wi)
    return _load().oracle_sheen_f(po, pi, float(alpha))


def sah_reference(verts, leaf_max=4):
    """Surface-area cost of a binned-SAH binary BVH over the triangles (n, 3, 3): expected box
    tests and triangle tests of a ray through the root box, and the tree's node count."""
    v, pv = _d(np.asarray(verts, dtype=np.float64).reshape(-1, 9))
    out = np.zeros(3)
    _load().oracle_sah_reference(pv, int(v.shape[0]), int(leaf_max), out.ctypes.data_as(_dp))
    return {"box_tests": float(out[0]), "tri_tests": float(out[1]), "nodes": int(out[2])}


def bsdf_eval(mat, front, wo, wi):
    """Non-delta part of f(wo, wi) (RGB) and the mixture sampling pdf of wi."""
    m, pm = _d(mat)
    wo, po = _d(wo)
    wi, pi = _d(wi)
    f = np.zeros(3)
    pdf = C.c_double()
    _load().oracle_bsdf_eval(pm, int(front), po, pi, f.ctypes.data_as(_dp), C.byref(pdf))
    return f, pdf.value


def bsdf_sample(mat, front, wo, u):
    """-> (ok, wi, weight, pdf, is_delta); u = (u_lobe, u1, u2, u_refract)."""
    m, pm = _d(mat)
    wo, po = _d(wo)
    u, pu = _d(u)
    wi = np.zeros(3)
    w = np.zeros(3)
    pdf = C.c_double()
    dl = C.c_int()
    ok = _load().oracle_bsdf_sample(pm, int(front), po, pu, wi.ctypes.data_as(_dp),
                                    w.ctypes.data_as(_dp), C.byref(pdf), C.byref(dl))
    return bool(ok), wi, w, pdf.value, bool(dl.value)


def bsdf_eval_batch(mat, front, wo, wi):
    """Vectorised bsdf_eval over rows of wo, wi (n, 3) -> f (n, 3), pdf (n,)."""
    m, pm = _d(mat)
    wo, po = _d(wo)
    wi, pi = _d(wi)
    n = wo.shape[0]
    f = np.zeros((n, 3))
    pdf = np.zeros(n)
    _load().oracle_bsdf_eval_batch(pm, int(front), n, po, pi, f.ctypes.data_as(_dp),
                                   pdf.ctypes.data_as(_dp))
    return f, pdf


def bsdf_sample_batch(mat, front, wo, u):
    """Vectorised bsdf_sample: wo (n, 3), u (n, 4) -> ok, wi, weight, pdf, is_delta."""
    m, pm = _d(mat)
    wo, po = _d(wo)
    u, pu = _d(u)
    n = wo.shape[0]
    wi = np.zeros((n, 3))
    w = np.zeros((n, 3))
    pdf = np.zeros(n)
    dl = np.zeros(n, dtype=np.int32)
    ok = np.zeros(n, dtype=np.int32)
    _load().oracle_bsdf_sample_batch(pm, int(front), n, po, pu, wi.ctypes.data_as(_dp),
                                     w.ctypes.data_as(_dp), pdf.ctypes.data_as(_dp),
                                     dl.ctypes.data_as(_i32p), ok.ctypes.data_as(_i32p))
    return ok.astype(bool), wi, w, pdf, dl.astype(bool)


def uniform_batch(pixel, sample, bounce, dim, seed):
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.uint32),
                                                 np.broadcast_shapes(*[np.shape(x) for x in
                                                                       (pixel, sample, bounce, dim)])))
            for a in (pixel, sample, bounce, dim)]
    n = arrs[0].size
    out = np.zeros(n)
    _load().oracle_uniform_batch(n, *[a.ravel().ctypes.data_as(_u32p) for a in arrs], int(seed),
                                 out.ctypes.data_as(_dp))
    return out.reshape(arrs[0].shape)


def lobe_probs(mat, front, mu_o):
    """Selection probabilities of the lobes (coat, metal, dielectric, diffuse, fuzz) at mu_o."""
    m, pm = _d(mat)
    o = np.zeros(5)
    _load().oracle_lobe_probs(pm, int(front), float(mu_o), o.ctypes.data_as(_dp))
    return o


# ----------------------------------------------------------------------------------------
# Scenes, intersection, environment, rendering
# ----------------------------------------------------------------------------------------

class OracleScene:
    """The oracle's own copy of a scene (double precision, optional median-split BVH)."""

    def __init__(self, scene, use_bvh=True):
        lib = _load()
        self._keep = []
        v, pv = _d(scene.vertices)
        idx = np.ascontiguousarray(scene.indices, dtype=np.uint32)
        mid = np.ascontiguousarray(scene.material_ids, dtype=np.uint32)
        mats, pm = _d(scene.materials)
        quads, pq = _d(scene.lights if len(scene.lights) else np.zeros((0, 13)))
        if scene.env is not None:
            env, pe = _d(scene.env)
            ew, eh = scene.env.shape[1], scene.env.shape[0]
        else:
            env, pe, ew, eh = None, None, 0, 0
        self._keep += [v, idx, mid, mats, quads, env]
        self.h = lib.oracle_scene_create(pv, v.shape[0], idx.ctypes.data_as(_u32p), idx.shape[0],
                                         mid.ctypes.data_as(_u32p), pm, mats.shape[0], pq,
                                         quads.shape[0], pe, ew, eh, 1 if use_bvh else 0)
        self.scene = scene
        self.n_tris = idx.shape[0] + 2 * quads.shape[0]

    def __del__(self):
        try:
            if getattr(self, "h", None):
                _load().oracle_scene_destroy(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def eps(self):
        return _load().oracle_scene_eps(self.h)

    def intersect(self, origins, dirs, tmax=None, brute=False):
        """Closest hit per ray -> (tri id or -1, t, (u, v)); ties go to the lower id."""
        n = origins.shape[0]
        rays = np.zeros((n, 8))
        rays[:, 0:3] = origins
        rays[:, 3:6] = dirs
        rays[:, 6] = np.inf if tmax is None else tmax
        tri = np.zeros(n, dtype=np.int32)
        t = np.zeros(n)
        uv = np.zeros((n, 2))
        _load().oracle_intersect(self.h, rays.ctypes.data_as(_dp), n, 1 if brute else 0,
                                 tri.ctypes.data_as(_i32p), t.ctypes.data_as(_dp),
                                 uv.ctypes.data_as(_dp))
        return tri, t, uv

    def env_sample(self, u3, u4):
        d = np.zeros(3)
        L = np.zeros(3)
        pdf = C.c_double()
        ok = _load().oracle_env_sample(self.h, float(u3), float(u4), d.ctypes.data_as(_dp),
                                       C.byref(pdf), L.ctypes.data_as(_dp))
        return bool(ok), d, pdf.value, L

    def env_pdf(self, d):
        d, p = _d(d)
        return _load().oracle_env_pdf(self.h, p)

    def render(self, camera=None, spp=None, max_depth=None, seed=0, s0=0, crop=None,
               threads=None, row_step=1, keep_samples=False, no_nee=False, no_rr=False, restir=None):
        """Sum of sample radiance over the crop (ch, cw, 3), optional per-sample values and
        stats dict.  crop = (x0, y0, w, h) in full-frame pixels.  restir = (M candidates,
        K neighbours, radius R[, L later candidates]) renders with ReSTIR DI at the primary
        vertex over the crop (and resampled NEE with L candidates at later vertices)."""
        sc = self.scene
        cam = camera or sc.camera
        spp = sc.spp if spp is None else spp
        max_depth = sc.max_depth if max_depth is None else max_depth
        x0, y0, cw, ch = crop if crop is not None else (0, 0, cam.width, cam.height)
        cam9 = np.array([*cam.origin, *cam.target, *cam.up, getattr(cam, "lens_radius", 0.0),
                         getattr(cam, "focus_distance", 1.0)], dtype=np.float64)
        out = np.zeros((ch, cw, 3))
        samples = np.zeros((ch, cw, spp, 3)) if keep_samples else None
        stats = np.zeros(5, dtype=np.int64)
        threads = threads or (os.cpu_count() or 1)
        rp = None if restir is None else np.array([int(v) for v in (tuple(restir) + (0,))[:4]], dtype=np.int32)
        if rp is not None:
            assert rp[0] >= 1 and 0 <= rp[1] <= 64 and rp[2] >= 1 and rp[3] >= 0
        _load().oracle_render(self.h, cam9.ctypes.data_as(_dp), float(cam.vfov_deg), cam.width,
                              cam.height, x0, y0, cw, ch, int(s0), int(spp), int(max_depth),
                              int(seed), (1 if no_nee else 0) | (2 if no_rr else 0), int(threads),
                              int(row_step), out.ctypes.data_as(_dp),
                              samples.ctypes.data_as(_dp) if keep_samples else None,
                              stats.ctypes.data_as(_i64p), rp.ctypes.data_as(_i32p) if rp is not None else None)
        st = dict(zip(("ext_rays", "shadow_rays", "nan_dropped", "rr_terminated", "paths"),
                      map(int, stats)))
        return out, samples, st


def _cam9(cam):
    return np.array([*cam.origin, *cam.target, *cam.up, getattr(cam, "lens_radius", 0.0),
                     getattr(cam, "focus_distance", 1.0)], dtype=np.float64)


def features(oscene, spp, seed=0, s0=0, crop=None, camera=None):
    """Primary-hit features (ch, cw, 12): normal[3], scattering fraction, position[3], 0,
    albedo[3], 0 -- the means over the render's samples s0 .. s0+spp-1."""
    cam = camera or oscene.scene.camera
    x0, y0, cw, ch = crop if crop is not None else (0, 0, cam.width, cam.height)
    out = np.zeros((ch, cw, 12))
    _load().oracle_features(oscene.h, _cam9(cam).ctypes.data_as(_dp), float(cam.vfov_deg), cam.width, cam.height,
                            x0, y0, cw, ch, int(s0), int(spp), int(seed), out.ctypes.data_as(_dp))
    return out


def camera_ray(camera, px, py, sample, seed):
    cam9 = np.array([*camera.origin, *camera.target, *camera.up, getattr(camera, "lens_radius", 0.0),
                     getattr(camera, "focus_distance", 1.0)], dtype=np.float64)
    o = np.zeros(3)
    d = np.zeros(3)
    _load().oracle_camera_ray(cam9.ctypes.data_as(_dp), float(camera.vfov_deg), camera.width,
                              camera.height, int(px), int(py), int(sample), int(seed),
                              o.ctypes.data_as(_dp), d.ctypes.data_as(_dp))
    return o, d
