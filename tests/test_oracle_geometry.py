"""Pins of the oracle's geometry: intersection (BVH vs brute force vs an independent
Moller-Trumbore in numpy), watertightness, tie rule, camera and environment mapping."""
import math

import numpy as np
import pytest
from scipy.stats import chi2 as chi2d

import oracle
from paper_2407_19977_gb300 import scenes

RNG = np.random.default_rng(7)


def _soup(n_tris, seed):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1, 1, (n_tris, 1, 3))
    v = (centers + rng.normal(0, 0.15, (n_tris, 3, 3))).reshape(-1, 3)
    idx = np.arange(3 * n_tris, dtype=np.uint32).reshape(-1, 3)
    mats = scenes.diffuse((0.5, 0.5, 0.5))[None]
    cam = scenes.Camera((0, 0, -3), (0, 0, 0), (0, 1, 0), 40.0, 8, 8)
    return scenes.Scene("soup", v.astype(np.float32), idx, np.zeros(n_tris, np.uint32), mats,
                        np.zeros((0, 13), np.float32), None, cam, 1, 1)


def _random_rays(n, rng=RNG):
    o = rng.uniform(-2, 2, (n, 3))
    tgt = rng.uniform(-0.8, 0.8, (n, 3))
    d = tgt - o
    return o, d / np.linalg.norm(d, axis=1, keepdims=True)


def _moller_trumbore(o, d, v0, v1, v2):
    """Closest hit by the Moller-Trumbore test (a different algorithm), numpy double."""
    e1, e2 = v1 - v0, v2 - v0
    best_t = np.full(o.shape[0], np.inf)
    best = np.full(o.shape[0], -1)
    for i in range(v0.shape[0]):
        p = np.cross(d, e2[i])
        det = p @ e1[i]
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            s = o - v0[i]
            u = np.einsum("ij,ij->i", s, p) * inv
            q = np.cross(s, e1[i])
            v = np.einsum("ij,ij->i", d, q) * inv
            t = q @ e2[i] * inv
        ok = (np.abs(det) > 1e-14) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0) & (t < best_t)
        best_t = np.where(ok, t, best_t)
        best = np.where(ok, i, best)
    return best, best_t


def test_bvh_matches_brute_force_and_moller_trumbore():
    sc = _soup(300, 3)
    osc = oracle.OracleScene(sc, use_bvh=True)
    o, d = _random_rays(3000)
    tri_b, t_b, uv_b = osc.intersect(o, d, brute=True)
    tri_v, t_v, uv_v = osc.intersect(o, d, brute=False)
    assert np.array_equal(tri_b, tri_v)
    assert np.array_equal(t_b, t_v)
    assert (tri_b >= 0).sum() > 1000
    v = sc.vertices.astype(np.float64)[sc.indices.astype(np.int64)]
    tri_m, t_m = _moller_trumbore(o, d, v[:, 0], v[:, 1], v[:, 2])
    agree = tri_m == tri_b
    assert agree.mean() > 0.999
    hit = agree & (tri_b >= 0)
    assert np.allclose(t_b[hit], t_m[hit], rtol=1e-9)
    # barycentrics reconstruct the hit point
    p = o[hit] + t_b[hit, None] * d[hit]
    w1, w2 = uv_b[hit, 0:1], uv_b[hit, 1:2]
    vv = v[tri_b[hit]]
    q = (1 - w1 - w2) * vv[:, 0] + w1 * vv[:, 1] + w2 * vv[:, 2]
    assert np.allclose(p, q, atol=1e-9)


def test_bvh_matches_brute_force_on_cornell():
    sc = scenes.cornell_box()
    osc = oracle.OracleScene(sc, use_bvh=True)
    o = RNG.uniform(0.02, 0.98, (5000, 3))
    d = RNG.normal(size=(5000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tri_b, t_b, _ = osc.intersect(o, d, brute=True)
    tri_v, t_v, _ = osc.intersect(o, d)
    assert np.array_equal(tri_b, tri_v) and np.array_equal(t_b, t_v)
    # from inside the box only rays heading out through the open front (z = 0) can miss
    assert (tri_b >= 0).mean() > 0.5
    assert np.all(d[tri_b < 0, 2] < 0)
    assert osc.n_tris == 36


def test_watertight_closed_mesh():
    v, f = scenes.icosphere(3)
    sc = scenes.Scene("ico", v.astype(np.float32), f.astype(np.uint32),
                      np.zeros(f.shape[0], np.uint32), scenes.diffuse((1, 1, 1))[None],
                      np.zeros((0, 13), np.float32), None, scenes.Camera((0, 0, -3), (0, 0, 0),
                                                                         (0, 1, 0), 40, 4, 4), 1, 1)
    osc = oracle.OracleScene(sc)
    vf = v.astype(np.float32).astype(np.float64)
    targets = [vf]                                                    # every vertex
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    targets.append(0.5 * (vf[e[:, 0]] + vf[e[:, 1]]))                 # every edge midpoint
    targets = np.concatenate(targets)
    for origin in (np.zeros(3), np.array([0.11, -0.07, 0.05]), np.array([-0.3, 0.2, 0.1])):
        d = targets - origin
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        tri, t, _ = osc.intersect(np.tile(origin, (d.shape[0], 1)), d)
        assert (tri >= 0).all(), "ray leaked through a shared edge or vertex"


def test_equal_t_goes_to_lower_id():
    v = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0]], np.float32)
    v = np.concatenate([v, v])
    idx = np.array([[3, 4, 5], [0, 1, 2]], np.uint32)   # identical triangles, ids 0 and 1
    sc = scenes.Scene("dup", v, idx, np.zeros(2, np.uint32), scenes.diffuse((1, 1, 1))[None],
                      np.zeros((0, 13), np.float32), None,
                      scenes.Camera((0, 0, -3), (0, 0, 0), (0, 1, 0), 40, 4, 4), 1, 1)
    osc = oracle.OracleScene(sc)
    tri, t, _ = osc.intersect(np.array([[0.1, 0.0, -2.0]]), np.array([[0.0, 0.0, 1.0]]))
    assert tri[0] == 0 and t[0] == pytest.approx(2.0)


def test_tmax_is_exclusive():
    sc = _soup(1, 0)
    osc = oracle.OracleScene(sc)
    v = sc.vertices.astype(np.float64)
    c = v.mean(0)
    o = c + np.array([0.0, 0.0, -1.0])
    d = (c - o) / np.linalg.norm(c - o)
    tri, t, _ = osc.intersect(o[None], d[None])
    assert tri[0] == 0
    tri2, _, _ = osc.intersect(o[None], d[None], tmax=t[0])
    assert tri2[0] == -1


def test_thin_lens_camera():
    """Thin-lens depth of field: radius 0 is the pinhole ray; otherwise every ray starts on the
    lens disk (in the plane through the camera origin perpendicular to the view direction),
    passes through the point where the pinhole ray of the same pixel jitter meets the plane of
    focus, and the lens points are uniform over the disk (concentric map)."""
    base = dict(origin=(0.3, 0.2, -1.0), target=(0.5, 0.4, 1.0), up=(0, 1, 0), vfov_deg=45.0, width=40,
                height=30)
    pin = scenes.Camera(**base)
    zero = scenes.Camera(**base, lens_radius=0.0, focus_distance=2.0)
    lens = scenes.Camera(**base, lens_radius=0.05, focus_distance=1.7)
    o0 = np.array(base["origin"], float)
    fwd = np.subtract(base["target"], base["origin"])
    fwd = fwd / np.linalg.norm(fwd)
    radii = []
    for s in range(400):
        px, py = s % 40, (7 * s) % 30
        op, dp = oracle.camera_ray(pin, px, py, s, 11)
        oz, dz = oracle.camera_ray(zero, px, py, s, 11)
        assert np.array_equal(op, oz) and np.array_equal(dp, dz)
        ol, dl = oracle.camera_ray(lens, px, py, s, 11)
        off = ol - o0
        assert abs(off @ fwd) < 1e-12                       # on the lens plane
        radii.append(np.linalg.norm(off))
        focus = op + dp * (1.7 / (dp @ fwd))                 # pinhole ray on the plane of focus
        t = (focus - ol) @ dl
        assert np.linalg.norm(ol + t * dl - focus) < 1e-10   # the lens ray passes through it
        assert abs(np.linalg.norm(dl) - 1.0) < 1e-12
    radii = np.array(radii) / 0.05
    assert radii.max() <= 1.0 + 1e-12
    # uniform on the disk: P(r < 1/2) = 1/4, P(r < 1/sqrt 2) = 1/2 (binomial, 400 samples)
    assert abs((radii < 0.5).mean() - 0.25) < 0.07
    assert abs((radii < 2 ** -0.5).mean() - 0.5) < 0.08


def test_camera_frustum_geometry():
    cam = scenes.Camera((0, 0, 0), (0, 0, 1), (0, 1, 0), 60.0, 64, 32)
    # every ray of the top row points up by less than 30 deg, of row 0..: by ~30 deg at the edge
    ups = []
    for s in range(32):
        o, d = oracle.camera_ray(cam, 32, 0, s, 5)
        assert np.allclose(o, 0)
        ups.append(math.degrees(math.atan2(d[1], d[2])))
    ups = np.array(ups)
    # pixel row 0 spans vertical angles atan(tan30 * (1 - 2*[0, 1/32]))
    assert ups.max() <= 30.0 + 1e-9
    assert ups.min() >= math.degrees(math.atan(math.tan(math.radians(30)) * (1 - 2 / 32))) - 1e-9
    # aspect 2: horizontal half-angle atan(2 tan 30); +x of the world is the image's left
    o, d = oracle.camera_ray(cam, 0, 16, 0, 5)
    assert d[0] > 0
    half_h = math.degrees(math.atan(2 * math.tan(math.radians(30))))
    assert math.degrees(math.atan2(d[0], d[2])) <= half_h + 1e-9
    assert math.degrees(math.atan2(d[0], d[2])) >= math.degrees(
        math.atan(2 * math.tan(math.radians(30)) * (1 - 2 / 64))) - 1e-9


# ------------------------------------------------------------------ environment map

def _index_env(w=16, h=8):
    env = np.zeros((h, w, 3), np.float64)
    env[..., :] = (1.0 + np.arange(w * h).reshape(h, w))[..., None]
    return env


def _env_scene(env):
    sc = _soup(1, 0)
    sc.env = env
    return oracle.OracleScene(sc)


def test_env_direction_mapping():
    env = _index_env()
    h, w = env.shape[:2]
    osc = _env_scene(env)
    st = np.sin(math.pi * (np.arange(h) + 0.5) / h)
    total = (env[..., 0] * st[:, None]).sum()

    def texel_of(d):
        d = np.asarray(d, float) / np.linalg.norm(d)
        p = osc.env_pdf(d)
        s = math.sqrt(max(0.0, 1 - d[1] ** 2))
        lum_st = p * 2 * math.pi ** 2 * s * total / (w * h)
        cand = np.argwhere(np.isclose(env[..., 0] * st[:, None], lum_st, rtol=1e-9))
        assert len(cand) == 1
        return tuple(cand[0])

    eps = 1e-3
    assert texel_of([0, -1, 0.0 + eps])[0] == h - 1
    assert texel_of([0, 1, -eps])[0] == 0
    # azimuth: -z is the centre column, +x three quarters, -x one quarter
    assert texel_of([0, 0.1, -1]) == (h // 2 - 1, w // 2)
    assert texel_of([1, 0.1, -eps])[1] == 3 * w // 4 - 1
    assert texel_of([-1, 0.1, -eps])[1] == w // 4


def test_env_sampling_distribution_and_pdf():
    env = scenes.analytic_sky(32, 16, seed=3).astype(np.float64)
    h, w = env.shape[:2]
    # a tiny per-texel offset makes every texel's radiance unique (identifies the texel)
    env += 1e-6 * (1.0 + np.arange(w * h).reshape(h, w))[..., None]
    osc = _env_scene(env)
    lumi = env @ np.array([0.2126, 0.7152, 0.0722])
    wts = lumi * np.sin(math.pi * (np.arange(h) + 0.5) / h)[:, None]
    n_side = 300
    us = (np.arange(n_side) + 0.5) / n_side
    counts = np.zeros((h, w))
    mism = 0
    for u3 in us:
        for u4 in us:
            ok, d, pdf, L = osc.env_sample(u3, u4)
            assert ok
            # texel from the radiance returned (unique per texel with overwhelming probability)
            idx = np.argwhere(np.all(np.isclose(env, L, rtol=0, atol=0), axis=-1))[0]
            counts[idx[0], idx[1]] += 1
            p2 = osc.env_pdf(d)
            if not math.isclose(pdf, p2, rel_tol=1e-9):
                mism += 1
    assert mism <= 0.002 * n_side * n_side  # only at texel boundaries
    n = n_side * n_side
    exp = wts / wts.sum() * n
    keep = exp >= 5
    stat = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    # stratified u makes the counts much tighter than multinomial; chi-square is an upper bound
    assert chi2d.sf(stat, keep.sum() - 1) > 1e-3
    # the pdf integrates to one over the sphere
    nt, nph = 8 * h, 8 * w
    t = (np.arange(nt) + 0.5) / nt * math.pi
    ph = ((np.arange(nph) + 0.5) / nph - 0.5) * 2 * math.pi
    acc = 0.0
    for ti in t:
        for pj in ph[::1]:
            d = [math.sin(ti) * math.sin(pj), math.cos(ti), -math.sin(ti) * math.cos(pj)]
            acc += osc.env_pdf(d) * math.sin(ti)
    acc *= (math.pi / nt) * (2 * math.pi / nph)
    assert acc == pytest.approx(1.0, rel=1e-9)
