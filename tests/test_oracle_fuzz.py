"""Pins of the oracle's fuzz lobe (OpenPBR's fuzz layer): the Charlie distribution with its
exact Smith masking, the lobe's directional albedo, and the layer's composition with the
material under it.  Facts fixed by the mathematics: the normalisation of D, the projected area
at grazing (a Wallis integral), the albedo at grazing (every direction reflected off a
horizontal wo stays above the surface, so E(0) = A(0) / A(0) = 1), the albedo as an integral
of the lobe computed by another integrator, reciprocity and energy."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2407_19977_gb300 import scenes

ALPHAS = [0.04, 0.09, 0.25, 0.49, 1.0]   # fuzz_roughness 0.2, 0.3, 0.5, 0.7, 1


def _wallis(n):
    """int_0^{pi/2} sin^n(t) dt."""
    return 0.5 * math.sqrt(math.pi) * math.exp(special.gammaln((n + 1) / 2) - special.gammaln(n / 2 + 1))


@pytest.mark.parametrize("alpha", ALPHAS)
def test_distribution_normalisation_and_grazing_area(alpha):
    # A(1) = int D cos(theta_m) dm = 1 is the normalisation of D
    assert oracle.sheen_area(1.0, alpha) == pytest.approx(1.0, abs=1e-12)
    # seen edge-on, <w, m>+ integrates over the azimuth to 2 sin(theta_m): with
    # D = (k + 2) sin^k / (2 pi), A(0) = (k + 2) / pi * int sin^(k+2)
    k = 1.0 / alpha
    assert oracle.sheen_area(0.0, alpha) == pytest.approx((k + 2) / math.pi * _wallis(k + 2), rel=1e-10)
    # Smith's G1 = mu / A is at most 1: A(mu) >= mu (the mean normal is the surface normal)
    for mu in np.linspace(0.0, 1.0, 21):
        assert oracle.sheen_area(mu, alpha) >= mu - 1e-12


@pytest.mark.parametrize("alpha", [0.04, 0.25, 1.0])
def test_projected_area_against_a_two_dimensional_rule(alpha):
    """A(mu) with the azimuth integrated numerically (midpoint rule) instead of in closed form
    and no split at the kink: checks the closed-form inner integral and the split."""
    nt, nphi = 4000, 720
    th = (np.arange(nt) + 0.5) * (0.5 * math.pi / nt)
    d = np.array([oracle.sheen_D(math.cos(t), alpha) for t in th])
    ph = (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
    for mu in (0.05, 0.3, 0.7, 0.95):
        s = math.sqrt(1 - mu * mu)
        dot = s * np.sin(th)[:, None] * np.cos(ph)[None, :] + mu * np.cos(th)[:, None]
        inner = np.maximum(dot, 0.0).sum(1) * (2 * math.pi / nphi)
        a = float((d * np.sin(th) * inner).sum() * (0.5 * math.pi / nt))
        assert oracle.sheen_area(mu, alpha) == pytest.approx(a, rel=2e-5), (mu, alpha)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_albedo_at_grazing_is_one_and_bounded(alpha):
    """With wo horizontal, the reflected direction 2 (wo.h) h - wo has z = 2 (wo.h) h_z >= 0 for
    every visible microfacet, so no light is lost: E(0) = A(0) / A(0) = 1.  Single scattering
    with Smith masking keeps E <= 1 everywhere."""
    assert oracle.sheen_albedo(0.0, alpha) == pytest.approx(1.0, abs=1e-8)
    es = [oracle.sheen_albedo(mu, alpha) for mu in np.linspace(0.0, 1.0, 11)]
    assert all(0.0 <= e <= 1.0 + 1e-8 for e in es)


def _albedo_adaptive(mu_o, alpha):
    """E(mu_o) by scipy's adaptive quadrature of the oracle's own lobe over the hemisphere."""
    wo = np.array([math.sqrt(1 - mu_o * mu_o), 0.0, mu_o])

    def g(phi, mu_i):
        s = math.sqrt(max(0.0, 1 - mu_i * mu_i))
        return oracle.sheen_f(wo, np.array([s * math.cos(phi), s * math.sin(phi), mu_i]), alpha) * mu_i

    pts = [p for p in (0.5 * mu_o, mu_o, 2 * mu_o, 8 * mu_o) if 0 < p < 1]
    val, _ = integrate.quad(lambda m: integrate.quad(g, 0.0, math.pi, args=(m,), epsabs=1e-11, epsrel=1e-10,
                                                     limit=100)[0],
                            0.0, 1.0, epsabs=1e-10, epsrel=1e-9, limit=200, points=pts or None)
    return 2.0 * val


@pytest.mark.parametrize("alpha,mu", [(0.04, 1e-5), (0.25, 1e-4), (1.0, 1e-3), (0.04, 0.05), (0.04, 0.5),
                                      (1.0, 0.3), (1.0, 0.9), (1.0, 0.999), (1.0, 1.0), (0.09, 1e-5)])
def test_albedo_is_the_integral_of_the_lobe(alpha, mu):
    """The oracle's E (polar pieces cut at mu_o, 4 mu_o, 16 mu_o, ...; Gauss-Legendre in the
    polar angle and the azimuth) against another integrator applied to the oracle's f_s, to
    1e-7 from grazing (mu 1e-5, where the integrand turns over within mu_i ~ mu of the horizon)
    to normal incidence (alpha 1: the lobe has a cone-shaped kink at the mirror direction):
    catches a wrong symmetry factor, a wrong range, a lost piece or a lobe that does not match
    its albedo."""
    assert oracle.sheen_albedo(mu, alpha) == pytest.approx(_albedo_adaptive(mu, alpha), abs=1e-7)


def test_lobe_reciprocity_and_zero_below():
    rng = np.random.default_rng(5)
    for alpha in (0.04, 0.25, 1.0):
        for _ in range(20):
            a = rng.normal(size=3)
            b = rng.normal(size=3)
            a[2], b[2] = abs(a[2]) + 1e-3, abs(b[2]) + 1e-3
            a /= np.linalg.norm(a)
            b /= np.linalg.norm(b)
            assert oracle.sheen_f(a, b, alpha) == pytest.approx(oracle.sheen_f(b, a, alpha), rel=1e-12)
            assert oracle.sheen_f(a, b * [1, 1, -1], alpha) == 0.0


def _hemisphere_albedo(mat, mu_o, n=48):
    """int f(wo, wi) |mu_i| dwi over the upper hemisphere by a product Gauss rule."""
    x, w = np.polynomial.legendre.leggauss(n)
    mus, wm = 0.5 * (x + 1), 0.5 * w
    phs, wp = 0.5 * math.pi * (x + 1), 0.5 * math.pi * w          # [0, pi], doubled below
    M, P = np.meshgrid(mus, phs, indexing="ij")
    s = np.sqrt(1 - M * M)
    wi = np.stack([s * np.cos(P), s * np.sin(P), M], -1).reshape(-1, 3)
    wo = np.tile([math.sqrt(1 - mu_o * mu_o), 0.0, mu_o], (wi.shape[0], 1))
    f, _ = oracle.bsdf_eval_batch(mat, 1, wo, wi)
    return 2.0 * (f * wi[:, 2:3] * np.outer(wm, wp).reshape(-1, 1)).sum(0)


def test_fuzz_over_white_lambert_conserves_energy():
    """White fuzz (weight 1) over a white Lambertian base: the albedo is the fuzz's E(mu_o)
    plus what the base returns through the layer, (1 - E(mu_o)) 2 int (1 - E(mu)) mu dmu, and
    never exceeds 1."""
    alpha_r = 0.5
    mat = scenes.openpbr(base_color=(1, 1, 1), specular_weight=0.0, fuzz_weight=1.0, fuzz_roughness=alpha_r)
    alpha = alpha_r * alpha_r
    x, w = np.polynomial.legendre.leggauss(48)
    mus, wm = 0.5 * (x + 1), 0.5 * w
    through = 2.0 * sum(wk * (1 - oracle.sheen_albedo(m, alpha)) * m for m, wk in zip(mus, wm))
    for mu_o in (0.15, 0.5, 0.9):
        e_o = oracle.sheen_albedo(mu_o, alpha)
        alb = _hemisphere_albedo(mat, mu_o)
        assert np.allclose(alb, e_o + (1 - e_o) * through, rtol=2e-5), (mu_o, alb)
        assert np.all(alb <= 1.0)


def test_zero_fuzz_weight_changes_nothing():
    rng = np.random.default_rng(9)
    base = scenes.openpbr(base_color=(0.6, 0.4, 0.3), specular_roughness=0.4, coat_weight=0.5, coat_roughness=0.2)
    off = base.copy()
    off[30:34] = [0.2, 0.9, 0.4, 0.35]                 # colour and roughness without weight
    wo = rng.normal(size=(64, 3))
    wi = rng.normal(size=(64, 3))
    wo[:, 2] = np.abs(wo[:, 2])
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    fa, pa = oracle.bsdf_eval_batch(base, 1, wo, wi)
    fb, pb = oracle.bsdf_eval_batch(off, 1, wo, wi)
    assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
    assert oracle.lobe_probs(off, 1, 0.4)[4] == 0.0


def test_fuzz_lobe_weight_and_layer_scaling():
    """Lobe probabilities: the fuzz lobe gets fw lum(fc) E(mu_o) and the others are scaled by
    1 - fw E(mu_o), so their ratios are those of the material without fuzz, and the ratio of
    the fuzz lobe to the rest, r = fw lum(fc) E / ((1 - fw E) S) with S the base's own sum,
    fixes E through two fuzz weights: r(a) / r(b) = [a / (1 - a E)] / [b / (1 - b E)]."""
    def mat(fw, fc=(0.9, 0.3, 0.5)):
        return scenes.openpbr(base_color=(0.5, 0.5, 0.5), specular_roughness=0.3, fuzz_weight=fw,
                              fuzz_color=fc, fuzz_roughness=0.6)
    base = scenes.openpbr(base_color=(0.5, 0.5, 0.5), specular_roughness=0.3)
    for mu in (0.1, 0.35, 0.8):
        pb = oracle.lobe_probs(base, 1, mu)
        r = float(np.float32(0.6))           # the parameter table is float32
        e = oracle.sheen_albedo(mu, r * r)
        ratios = {}
        for fw in (0.3, 0.9):
            pf = oracle.lobe_probs(mat(fw), 1, mu)
            assert abs(pf.sum() - 1.0) < 1e-12
            assert np.allclose(pf[:4] / pf[:4].sum(), pb[:4], rtol=1e-12)
            ratios[fw] = pf[4] / pf[:4].sum()
        a3, a9 = float(np.float32(0.3)), float(np.float32(0.9))
        expect = (a3 / (1 - a3 * e)) / (a9 / (1 - a9 * e))
        assert ratios[0.3] / ratios[0.9] == pytest.approx(expect, rel=1e-10)
        # the fuzz lobe's share is linear in the luminance of its colour
        half = oracle.lobe_probs(mat(0.9, (0.45, 0.15, 0.25)), 1, mu)
        assert half[4] / half[:4].sum() == pytest.approx(0.5 * ratios[0.9], rel=1e-12)
