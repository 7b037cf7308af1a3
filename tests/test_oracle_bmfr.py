"""Pins of the regression denoiser oracle (oracle/bmfr.py) and of the oracle's primary-hit
features: least-squares facts that hold whatever the implementation, and the features'
closed forms on simple geometry."""
import math

import numpy as np
import pytest

import oracle
from oracle import bmfr as ob
from paper_2407_19977_gb300 import scenes

RNG = np.random.default_rng(17)


def _smooth_features(h, w, frac=1.0):
    """Features of a curved, bumpy surface patch: positions on a paraboloid, normals of a
    bump pattern that is not an affine function of position within any block, albedo."""
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    u, v = xs / w, ys / h
    p = np.stack([u, 0.3 * u * u + 0.2 * v * v, v + 2.0], -1)
    n = np.stack([np.sin(31.0 * u + 3.0 * v), np.ones_like(u), np.cos(23.0 * v - 2.0 * u)], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    alb = np.stack([0.2 + 0.5 * u, 0.6 * np.ones_like(u), 0.3 + 0.4 * v], -1)
    f = np.zeros((h, w, 12))
    f[..., 0:3], f[..., 3], f[..., 4:7], f[..., 8:11] = n, frac, p, alb
    return f


def test_colour_in_the_feature_span_comes_back_unchanged():
    h, w = 70, 90                                   # several blocks and ragged edges
    f = _smooth_features(h, w)
    n, p, a = f[..., 0:3], f[..., 4:7], f[..., 8:11]
    coef = RNG.normal(size=(10, 3))
    # (1) a quadratic in x and z plus a linear term in the paraboloid's height: in the span
    # of every block's kept columns whatever the block's shape (a column left out as
    # dependent here is exactly dependent, e.g. q^2 over two distinct values)
    base = coef[0] + p @ coef[4:7] + (p[..., 0:1] ** 2) * coef[7] + (p[..., 2:3] ** 2) * coef[9]
    c = (a + ob.ALBEDO_EPS) * base
    for block, off in ((32, (0, 0)), (16, (5, 11)), (8, (3, 0))):
        out = ob.bmfr(c, f, block=block, offset=off)
        assert np.allclose(out, c, rtol=1e-9, atol=1e-12), (block, off, np.abs(out - c).max())
    # (2) every feature: on the 32-pixel grid each block keeps all its columns but one (the
    # paraboloid ties q_y to q_x^2 and q_z^2, so the last of the three, q_z^2, is left out)
    for y0, y1, x0, x1 in ob._blocks(h, w, 32, (0, 0)):
        full = ob.design_matrix(f[y0:y1, x0:x1].reshape(-1, 12))
        assert ob.kept_columns(full).shape[1] == full.shape[1] - 1
    base = coef[0] + n @ coef[1:4] + p @ coef[4:7] + (p * p) @ coef[7:10]
    c = (a + ob.ALBEDO_EPS) * base
    out = ob.bmfr(c, f, block=32)
    assert np.allclose(out, c, rtol=1e-9, atol=1e-12), np.abs(out - c).max()


def test_fit_is_idempotent_and_residual_is_orthogonal():
    h, w = 40, 48
    f = _smooth_features(h, w)
    c = RNG.gamma(2.0, 0.5, (h, w, 3))
    y = ob.bmfr(c, f, block=16)
    assert np.allclose(ob.bmfr(y, f, block=16), y, rtol=1e-9, atol=1e-12)
    # one block: the demodulated residual is orthogonal to every kept column
    fb = f[16:32, 16:32].reshape(-1, 12)
    A = ob.kept_columns(ob.design_matrix(fb))
    a = fb[:, 8:11] + ob.ALBEDO_EPS
    r = (c[16:32, 16:32].reshape(-1, 3) - y[16:32, 16:32].reshape(-1, 3)) / a
    g = A.T @ r
    assert np.abs(g).max() < 1e-9 * np.abs(A).sum(0).max() * np.abs(r).max()
    # and the fit is the orthogonal projection (normal equations through the pseudo-inverse)
    b = c[16:32, 16:32].reshape(-1, 3) / a
    assert np.allclose(A @ (np.linalg.pinv(A) @ b), y[16:32, 16:32].reshape(-1, 3) / a, rtol=1e-8, atol=1e-12)


def test_non_scattering_pixels_pass_through_and_blocks_are_independent():
    h, w = 48, 64
    f = _smooth_features(h, w)
    f[5:9, 40:50, 3] = 0.5                          # partly sky / light
    c = RNG.gamma(2.0, 0.5, (h, w, 3))
    y = ob.bmfr(c, f, block=16, offset=(4, 4))
    assert np.array_equal(y[5:9, 40:50], c[5:9, 40:50])
    c2 = c.copy()
    c2[20:28, 30:40] += 5.0                         # inside the block x in [28, 44), y in [12, 28)
    y2 = ob.bmfr(c2, f, block=16, offset=(4, 4))
    changed = np.any(y2 != y, axis=-1)
    ys, xs = np.nonzero(changed)
    assert ys.min() >= 12 and ys.max() < 28 and xs.min() >= 28 and xs.max() < 44


def test_near_constant_and_dependent_features_are_left_out():
    """A flat wall (constant normal, one position axis constant up to rounding) keeps only the
    columns that vary; a normal that is an affine copy of a position axis adds nothing."""
    h, w = 32, 32
    f = _smooth_features(h, w)
    f[..., 0:3] = [0.0, 0.0, -1.0]
    f[..., 6] = 1.0 + 1e-8 * RNG.standard_normal((h, w))   # z: rounding-level variation
    A = ob.kept_columns(ob.design_matrix(f.reshape(-1, 12)))
    assert A.shape[1] == 5                          # 1, q_x, q_y, q_x^2, q_y^2
    g = _smooth_features(h, w)
    g[..., 0] = 0.3 * g[..., 4] - 0.1               # n_x affine in p_x: the same direction
    full = ob.design_matrix(g.reshape(-1, 12))
    kept = ob.kept_columns(full)
    # q_x repeats n_x, and the paraboloid's q_z^2 is in the span of 1, q_y, q_x^2
    assert kept.shape[1] == full.shape[1] - 2
    c = RNG.gamma(2.0, 0.5, (h, w, 3))
    y = ob.bmfr(c, g, block=32)
    a = g.reshape(-1, 12)[:, 8:11] + ob.ALBEDO_EPS
    b = c.reshape(-1, 3) / a
    ref = full @ (np.linalg.pinv(full, rcond=1e-10) @ b)
    assert np.allclose(y.reshape(-1, 3) / a, ref, rtol=1e-8, atol=1e-10)


def test_features_closed_forms():
    """On a plane y = 0 under a camera looking straight down, every pixel's first hit has
    normal +y, height 0, the plane's albedo, and the mean position of its jittered hits."""
    sc = scenes.plane_with_quad(albedo=0.8, radiance=5.0, width=10, height=10, spp=4)
    osc = oracle.OracleScene(sc)
    f = oracle.features(osc, 4, seed=3)
    hit = f[..., 3] == 1.0
    assert hit.mean() > 0.9
    assert np.allclose(f[hit][:, 0:3], [0, 1, 0], atol=1e-12)
    assert np.allclose(f[hit][:, 5], 0.0, atol=1e-12)
    assert np.allclose(f[hit][:, 8:11], 0.8, atol=1e-12)
    cam = sc.camera
    for py, px in ((2, 3), (7, 8)):
        if not hit[py, px]:
            continue
        pts = []
        for s in range(4):
            o, d = oracle.camera_ray(cam, px, py, s, 3)
            pts.append(o + (-o[1] / d[1]) * d)
        assert np.allclose(f[py, px, 4:7], np.mean(pts, 0), atol=1e-12)


def test_denoising_lowers_the_error_of_a_noisy_render():
    """The Cornell box at 4 spp: the regression output is closer to a 512-spp reference than
    the noisy mean (a property of the method on smooth diffuse scenes)."""
    sc = scenes.cornell_box(width=64, height=64, spp=4, max_depth=4)
    osc = oracle.OracleScene(sc)
    noisy, _, _ = osc.render(spp=4, seed=1)
    noisy /= 4
    ref, _, _ = osc.render(spp=512, seed=2, s0=1000)
    ref /= 512
    f = oracle.features(osc, 4, seed=1)
    den = ob.bmfr(noisy, f, block=16)

    def relmse(x):
        return float(((x - ref) ** 2 / (ref * ref + 1e-2)).mean())

    assert relmse(den) < 0.6 * relmse(noisy), (relmse(den), relmse(noisy))
    assert math.isfinite(relmse(den))
