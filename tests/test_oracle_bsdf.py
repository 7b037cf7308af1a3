"""Pins of the oracle's OpenPBR subset: closed forms, Monte Carlo identities, reciprocity,
sample/eval consistency and a chi-square fit of the sampler against its own pdf.

Each check would fail on a plausible mistake in the lobe code: a dropped Fresnel or
shadowing factor breaks the energy bound or reciprocity, a wrong Jacobian breaks the pdf
normalisation or the chi-square fit, a wrong VNDF breaks the projected-area identity.
"""
import math

import numpy as np
import pytest
from scipy.stats import chi2 as chi2d

import oracle
from paper_2407_19977_gb300 import scenes

RNG = np.random.default_rng(20240728)


def _sphere_dirs(n, rng=RNG):
    z = 1.0 - 2.0 * rng.random(n)
    phi = 2.0 * math.pi * rng.random(n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _hemi_dir(mu, phi=0.3):
    s = math.sqrt(max(0.0, 1.0 - mu * mu))
    return np.array([s * math.cos(phi), s * math.sin(phi), mu])


def test_rough_diffuse_properties():
    """Rough diffuse base (qualitative Oren-Nayar): roughness 0 is Lambert exactly; f depends
    only on the azimuth difference; near grazing it scatters more back towards the viewer
    than forward (the backscatter that distinguishes rough from Lambertian diffuse); it does
    not gain energy (albedo <= rho at every angle)."""
    rho = 0.7
    rough = scenes.openpbr(base_color=(rho,) * 3, base_diffuse_roughness=0.9, specular_weight=0.0)
    rng = np.random.default_rng(3)
    wo = _sphere_dirs(300)
    wo[:, 2] = np.abs(wo[:, 2]) + 1e-3
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    wi = _sphere_dirs(300)
    wi[:, 2] = np.abs(wi[:, 2]) + 1e-3
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    f0, _ = oracle.bsdf_eval_batch(scenes.openpbr(base_color=(rho,) * 3, base_diffuse_roughness=0.0,
                                                  specular_weight=0.0), 1, wo, wi)
    assert np.allclose(f0, rho / math.pi, rtol=1e-14)
    # rotating both directions about the normal leaves f unchanged
    f1, _ = oracle.bsdf_eval_batch(rough, 1, wo, wi)
    ang = rng.uniform(0, 2 * math.pi)
    R = np.array([[math.cos(ang), -math.sin(ang), 0], [math.sin(ang), math.cos(ang), 0], [0, 0, 1]])
    f2, _ = oracle.bsdf_eval_batch(rough, 1, wo @ R.T, wi @ R.T)
    assert np.allclose(f1, f2, rtol=1e-12)
    # backscatter: at 75 deg, the mirror-azimuth (retro) direction beats the forward one
    th = math.radians(75)
    o = np.array([[math.sin(th), 0, math.cos(th)]])
    retro, _ = oracle.bsdf_eval_batch(rough, 1, o, o)
    fwd, _ = oracle.bsdf_eval_batch(rough, 1, o, o * np.array([-1, -1, 1]))
    assert retro[0, 0] > 1.5 * fwd[0, 0]
    # directional albedo by quadrature over the cosine-weighted hemisphere
    n = 200000
    u1, u2 = rng.random(n), rng.random(n)
    r, phi = np.sqrt(u1), 2 * math.pi * u2
    wis = np.stack([r * np.cos(phi), r * np.sin(phi), np.sqrt(1 - u1)], 1)
    for mu in (0.05, 0.3, 0.7, 1.0):
        o = np.repeat(np.array([[math.sqrt(1 - mu * mu), 0, mu]]), n, 0)
        f, _ = oracle.bsdf_eval_batch(rough, 1, o, wis)
        E = float((f[:, 0] * math.pi).mean())           # f cos / (cos/pi)
        assert E <= rho * (1 + 1e-2), (mu, E)


@pytest.mark.parametrize("sigma", [0.3, 0.7, 1.0])
def test_rough_diffuse_normalisation_fixes_the_grazing_albedo(sigma):
    """Fujii's normalisation of the qualitative Oren-Nayar term, 1 / (1 + (1/2 - 2/(3 pi)) sigma),
    is the value its s/t term integrates to at a grazing view: with wo on the horizon, t = mu_i
    where s > 0 and
      (1/pi) int (s/t) mu_i dwi = (1/pi) [int sin(th_i) cos(phi)+ dwi - int mu_i sin(th_i) cos(phi)- dwi]
                                = (1/pi) (pi/2 - 2/3),
    so the directional albedo there is exactly rho for every roughness.  A wrong constant (or a
    wrong s, t or sign) moves this albedo by about sigma times its error.  Quadrature: Gauss in
    mu_i and, split where s changes sign (phi = pi/2), in the azimuth."""
    rho = 0.8
    mat = scenes.openpbr(base_color=(rho,) * 3, base_diffuse_roughness=sigma, specular_weight=0.0)
    x, w = np.polynomial.legendre.leggauss(96)
    mus, wm = 0.5 * (x + 1), 0.5 * w
    phs = np.concatenate([0.25 * math.pi * (x + 1), 0.5 * math.pi + 0.25 * math.pi * (x + 1)])
    wp = np.concatenate([0.25 * math.pi * w, 0.25 * math.pi * w])       # [0, pi]; doubled below
    M, P = np.meshgrid(mus, phs, indexing="ij")
    sn = np.sqrt(1 - M * M)
    wi = np.stack([sn * np.cos(P), sn * np.sin(P), M], -1).reshape(-1, 3)
    mu_o = 1e-7
    wo = np.tile([math.sqrt(1 - mu_o * mu_o), 0.0, mu_o], (wi.shape[0], 1))
    f, _ = oracle.bsdf_eval_batch(mat, 1, wo, wi)
    E = 2.0 * float((f[:, 0] * wi[:, 2] * np.outer(wm, wp).reshape(-1)).sum())
    assert E == pytest.approx(rho, rel=1e-5), E
    # away from grazing the same term loses energy (no multiple-scattering compensation)
    wo1 = np.tile([0.0, 0.0, 1.0], (wi.shape[0], 1))
    f1, _ = oracle.bsdf_eval_batch(mat, 1, wo1, wi)
    E1 = 2.0 * float((f1[:, 0] * wi[:, 2] * np.outer(wm, wp).reshape(-1)).sum())
    assert E1 == pytest.approx(rho / (1 + (0.5 - 2 / (3 * math.pi)) * sigma), rel=1e-6)


def test_thin_walled_sheet():
    """A smooth white thin-walled sheet passes light straight through (wi = -wo) with
    weight 1 - F and reflects F into the mirror direction, so reflectance plus transmittance
    is exactly 1; a rough one is the same from both sides."""
    sheet = scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.0, transmission_weight=1.0,
                           geometry_thin_walled=1.0)
    rng = np.random.default_rng(9)
    for mu in (0.95, 0.6, 0.2):
        wo = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
        n = 4000
        ok, wi, w, p, dl = oracle.bsdf_sample_batch(sheet, 1, np.tile(wo, (n, 1)), rng.random((n, 4)))
        assert ok.all() and dl.all()
        trans = wi[:, 2] < 0
        assert np.allclose(wi[trans], -wo, atol=1e-12)
        assert np.allclose(wi[~trans], wo * np.array([-1, -1, 1]), atol=1e-12)
        # one-sample estimator of R + T: mean weight = 1 for a lossless sheet
        assert w[:, 0].mean() == pytest.approx(1.0, abs=0.03)
        F = float(oracle.fresnel_dielectric(mu, 1.5))
        assert np.allclose(w[trans, 0] * trans.mean(), 1 - F, rtol=0.1)
    rough = scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.5, transmission_weight=1.0,
                           geometry_thin_walled=1.0)
    a = _sphere_dirs(200)
    a[:, 2] = np.abs(a[:, 2]) + 1e-3
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = _sphere_dirs(200)
    f_front, p_front = oracle.bsdf_eval_batch(rough, 1, a, b)
    f_back, p_back = oracle.bsdf_eval_batch(rough, 0, a, b)
    assert np.array_equal(f_front, f_back) and np.array_equal(p_front, p_back)


# materials with every lobe rough enough for quadrature- and MC-based checks
MATS = {
    "diffuse_white": scenes.openpbr(base_color=(1, 1, 1), specular_weight=0.0),
    "plastic": scenes.openpbr(base_color=(0.6, 0.5, 0.4), specular_roughness=0.4),
    "metal": scenes.openpbr(base_color=(0.9, 0.7, 0.5), base_metalness=1.0, specular_roughness=0.45,
                            specular_color=(0.8, 0.9, 1.0)),
    "coated": scenes.openpbr(base_color=(0.8, 0.05, 0.05), specular_roughness=0.5, coat_weight=1.0,
                             coat_roughness=0.35, coat_ior=1.5),
    "rough_glass": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.45,
                                  transmission_weight=1.0),
    "mixed": scenes.openpbr(base_color=(0.7, 0.6, 0.9), base_metalness=0.3, specular_roughness=0.5,
                            transmission_weight=0.4, transmission_color=(0.9, 0.8, 0.7),
                            coat_weight=0.5, coat_roughness=0.4, coat_color=(0.9, 0.9, 0.6)),
    "rough_diffuse": scenes.openpbr(base_color=(1, 1, 1), base_diffuse_roughness=1.0, specular_weight=0.0),
    "rough_plastic": scenes.openpbr(base_color=(0.5, 0.6, 0.7), base_diffuse_roughness=0.6, specular_roughness=0.4),
    "thin_glass": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.4, transmission_weight=1.0,
                                 geometry_thin_walled=1.0),
    "thin_tinted": scenes.openpbr(base_color=(0.6, 0.6, 0.6), specular_roughness=0.3, transmission_weight=0.7,
                                  transmission_color=(0.9, 0.6, 0.5), coat_weight=0.4, coat_roughness=0.3,
                                  geometry_thin_walled=1.0),
    "aniso_metal": scenes.openpbr(base_color=(0.9, 0.8, 0.6), base_metalness=1.0, specular_roughness=0.5,
                                  specular_roughness_anisotropy=0.8),
    "aniso_glass": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.5, transmission_weight=1.0,
                                  specular_roughness_anisotropy=0.6),
    "aniso_coated": scenes.openpbr(base_color=(0.2, 0.4, 0.8), specular_roughness=0.45, coat_weight=1.0,
                                   coat_roughness=0.3, specular_roughness_anisotropy=0.5),
    "fuzz_velvet": scenes.openpbr(base_color=(0.5, 0.1, 0.2), specular_roughness=0.5, fuzz_weight=1.0,
                                  fuzz_color=(0.9, 0.6, 0.7), fuzz_roughness=0.4),
    "fuzz_coated_glass": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.45, transmission_weight=0.8,
                                        coat_weight=0.6, coat_roughness=0.3, fuzz_weight=0.5,
                                        fuzz_color=(0.7, 0.8, 0.9), fuzz_roughness=0.8),
}
# fuzz materials integrate their albedo in the oracle at every evaluation: fewer samples
FUZZ_SCALE = 10
WHITE = {
    "white_plastic": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.3),
    "white_metal": scenes.openpbr(base_color=(1, 1, 1), base_metalness=1.0, specular_roughness=0.3),
    "white_coated": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.6, coat_weight=1.0,
                                   coat_roughness=0.2),
    "white_glass": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.3, transmission_weight=1.0),
    "white_mixed": scenes.openpbr(base_color=(1, 1, 1), base_metalness=0.5, specular_roughness=0.35,
                                  transmission_weight=0.5, coat_weight=0.5, coat_roughness=0.3),
    "white_aniso_metal": scenes.openpbr(base_color=(1, 1, 1), base_metalness=1.0, specular_roughness=0.35,
                                        specular_roughness_anisotropy=0.9),
    "white_aniso_glass": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.4, transmission_weight=1.0,
                                        specular_roughness_anisotropy=0.7),
    "white_fuzz": scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.3, fuzz_weight=1.0,
                                 fuzz_roughness=0.3),
}


# ------------------------------------------------------------------ closed forms

def test_fresnel_closed_forms():
    assert oracle.fresnel_dielectric(1.0, 1.5) == pytest.approx(0.04, abs=1e-15)
    assert oracle.fresnel_dielectric(0.7, 1.0) == pytest.approx(0.0, abs=1e-15)
    assert oracle.fresnel_dielectric(0.0, 1.5) == pytest.approx(1.0, abs=1e-15)
    # textbook sin/tan form of Fresnel's equations (Hecht), a different formula
    for eta in (1.33, 1.5, 2.2, 1 / 1.5):
        for ci in np.linspace(0.05, 0.99, 17):
            ti = math.acos(ci)
            st = math.sin(ti) / eta
            if st >= 1.0:
                assert oracle.fresnel_dielectric(ci, eta) == 1.0  # total internal reflection
                continue
            tt = math.asin(st)
            rs = (math.sin(ti - tt) / math.sin(ti + tt)) ** 2
            rp = (math.tan(ti - tt) / math.tan(ti + tt)) ** 2
            assert oracle.fresnel_dielectric(ci, eta) == pytest.approx(0.5 * (rs + rp), rel=1e-10)
    # critical angle for eta = 1/1.5: sin(theta_c) = 1/1.5
    cc = math.cos(math.asin(1 / 1.5))
    assert oracle.fresnel_dielectric(cc - 1e-6, 1 / 1.5) == 1.0
    assert oracle.fresnel_dielectric(cc + 1e-3, 1 / 1.5) < 1.0


def test_f82_tint_closed_forms():
    f0 = np.array([0.9, 0.6, 0.3])
    tint = np.array([0.5, 0.8, 1.0])
    assert np.allclose(oracle.fresnel_f82(f0, tint, 1.0), f0, atol=1e-15)
    assert np.allclose(oracle.fresnel_f82(f0, tint, 0.0), 1.0, atol=1e-15)
    mu = 1.0 / 7.0
    schlick = f0 + (1 - f0) * (1 - mu) ** 5
    assert np.allclose(oracle.fresnel_f82(f0, tint, mu), tint * schlick, atol=1e-13)
    # unit tint reduces to Schlick's approximation
    for m in np.linspace(0, 1, 11):
        assert np.allclose(oracle.fresnel_f82(f0, np.ones(3), m), f0 + (1 - f0) * (1 - m) ** 5,
                           atol=1e-13)


@pytest.mark.parametrize("alpha", [0.02, 0.09, 0.3, 0.8])
def test_ggx_normalisation_and_projected_area(alpha):
    # integrate over theta with a substitution that resolves the peak: tan(theta) = alpha * tan(x)
    n = 4000
    x = (np.arange(n) + 0.5) / n * (math.pi / 2)
    th = np.arctan(alpha * np.tan(x))
    dth = alpha / np.cos(x) ** 2 / (1 + (alpha * np.tan(x)) ** 2) * (math.pi / 2 / n)
    D = np.array([oracle.ggx_D([math.sin(t), 0.0, math.cos(t)], alpha) for t in th])
    total = (D * np.cos(th) * np.sin(th) * dth).sum() * 2 * math.pi
    assert total == pytest.approx(1.0, abs=2e-4)
    # projected area: int G1(wo) max(0, wo.h) D(h) dh = cos(theta_o)
    for mu_o in (0.95, 0.6, 0.2):
        wo = _hemi_dir(mu_o, 0.0)
        g1 = oracle.ggx_G1(wo, alpha)
        nphi = 256
        phis = (np.arange(nphi) + 0.5) / nphi * 2 * math.pi
        acc = 0.0
        for t, dt, d in zip(th, dth, D):
            h = np.stack([math.sin(t) * np.cos(phis), math.sin(t) * np.sin(phis),
                          np.full(nphi, math.cos(t))], 1)
            oh = np.maximum(h @ wo, 0.0)
            acc += (oh * d).sum() * math.sin(t) * dt * (2 * math.pi / nphi)
        assert g1 * acc == pytest.approx(mu_o, rel=2e-3)


def _aniso_quadrature(ax, ay, nx=1500, nphi=720):
    """Hemisphere quadrature nodes for an anisotropic GGX lobe: per azimuth phi the polar angle
    is substituted by tan(theta) = a(phi) tan(x), a(phi) = (cos^2/ax^2 + sin^2/ay^2)^(-1/2) the
    lobe's width along phi, which resolves the peak.  Returns directions h and weights of dw."""
    phis = (np.arange(nphi) + 0.5) / nphi * 2 * math.pi
    x = (np.arange(nx) + 0.5) / nx * (math.pi / 2)
    P, X = np.meshgrid(phis, x, indexing="ij")
    a = 1.0 / np.sqrt(np.cos(P) ** 2 / ax ** 2 + np.sin(P) ** 2 / ay ** 2)
    T = np.arctan(a * np.tan(X))
    dT = a / np.cos(X) ** 2 / (1 + (a * np.tan(X)) ** 2) * (math.pi / 2 / nx)
    h = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    w = (np.sin(T) * dT).ravel() * (2 * math.pi / nphi)
    return h, w


def _ggx_D_vec(h, ax, ay):
    return np.array([oracle.ggx_D(v, ax, ay) for v in h])


@pytest.mark.parametrize("ax,ay", [(0.3, 0.08), (0.12, 0.5)])
def test_anisotropic_ggx_normalisation_and_projected_area(ax, ay):
    """The anisotropic lobe (widths ax along the tangent, ay along the bitangent): projected
    normals integrate to 1, the projected-area identity holds for views off both axes, and the
    lobe is elongated along the wider axis (a swapped axis or width fails one of these)."""
    h, w = _aniso_quadrature(ax, ay)
    D = _ggx_D_vec(h, ax, ay)
    assert (D * h[:, 2] * w).sum() == pytest.approx(1.0, abs=5e-4)
    for mu_o, phi in ((0.9, 0.4), (0.5, 1.2), (0.2, 2.6)):
        wo = _hemi_dir(mu_o, phi)
        acc = (np.maximum(h @ wo, 0.0) * D * w).sum()
        assert oracle.ggx_G1(wo, ax, ay) * acc == pytest.approx(mu_o, rel=2e-3), (mu_o, phi)
    # D at the normal is 1/(pi ax ay); a tilt along x falls off with ax, along y with ay
    assert oracle.ggx_D([0, 0, 1], ax, ay) == pytest.approx(1 / (math.pi * ax * ay), rel=1e-14)
    s = 0.2
    dx = oracle.ggx_D([math.sin(s), 0, math.cos(s)], ax, ay)
    dy = oracle.ggx_D([0, math.sin(s), math.cos(s)], ax, ay)
    assert (dx > dy) == (ax > ay)
    # isotropic widths give the isotropic lobe
    for v in ([0.3, 0.2, 0.93], [0.0, 0.6, 0.8]):
        v = np.array(v) / np.linalg.norm(v)
        assert oracle.ggx_D(v, 0.3, 0.3) == pytest.approx(oracle.ggx_D(v, 0.3), rel=1e-14)


def test_anisotropic_vndf_sampler():
    """Visible normals sampled for an anisotropic lobe have the moments E[hx^2], E[hy^2],
    E[hz^2] of the density G1(wo) max(0, wo.h) D(h) / wo.z (quadrature)."""
    ax, ay = 0.45, 0.1
    wo = _hemi_dir(0.5, 0.8)
    n = 60000
    u = RNG.random((n, 2))
    hs = np.array([oracle.ggx_vndf_sample(wo, ax, a, b, alpha_y=ay) for a, b in u])
    assert np.all(hs[:, 2] >= 0) and np.allclose(np.linalg.norm(hs, axis=1), 1.0)
    h, w = _aniso_quadrature(ax, ay, nx=600, nphi=360)
    dens = oracle.ggx_G1(wo, ax, ay) * np.maximum(h @ wo, 0) * _ggx_D_vec(h, ax, ay) / wo[2]
    assert (dens * w).sum() == pytest.approx(1.0, abs=3e-3)
    for c in range(3):
        est, err = (hs[:, c] ** 2).mean(), (hs[:, c] ** 2).std() / math.sqrt(n)
        ref = (dens * h[:, c] ** 2 * w).sum()
        assert abs(est - ref) < 4 * err + 2e-3, (c, est, ref)


def test_anisotropy_mapping():
    """OpenPBR's mapping of (roughness r, anisotropy a) to the two widths keeps
    ax^2 + ay^2 = 2 r^4 with ay = (1 - a) ax: checked through the lobe itself, D at the
    normal = 1/(pi ax ay), and a = 0 is the isotropic material exactly."""
    r = 0.5
    wo = _hemi_dir(0.7, 0.3)
    for a in (0.0, 0.3, 0.8):
        mat = scenes.openpbr(base_color=(1, 1, 1), base_metalness=1.0, specular_roughness=r,
                             specular_roughness_anisotropy=a)
        a = float(mat[27])                               # the float32 value the row holds
        ax = r * r * math.sqrt(2 / (1 + (1 - a) ** 2))
        ay = (1 - a) * ax
        assert ax * ax + ay * ay == pytest.approx(2 * r ** 4)
        wi = np.array([-wo[0], -wo[1], wo[2]])          # mirror direction: h = n
        f, _ = oracle.bsdf_eval(mat, 1, wo, wi)
        g2 = 1.0 / (1.0 + 2 * _lambda(wo, ax, ay))
        assert f[0] == pytest.approx(1 / (math.pi * ax * ay) * g2 / (4 * wo[2] * wo[2]), rel=1e-12)
    iso = scenes.openpbr(base_color=(0.8, 0.6, 0.4), base_metalness=1.0, specular_roughness=r)
    zero = scenes.openpbr(base_color=(0.8, 0.6, 0.4), base_metalness=1.0, specular_roughness=r,
                          specular_roughness_anisotropy=0.0, specular_rotation=0.37)
    dirs = _sphere_dirs(50)
    for wi in dirs:
        assert np.array_equal(oracle.bsdf_eval(iso, 1, wo, wi)[0], oracle.bsdf_eval(zero, 1, wo, wi)[0])


def _lambda(w, ax, ay):
    x = (ax * ax * w[0] ** 2 + ay * ay * w[1] ** 2) / w[2] ** 2
    return (-1 + math.sqrt(1 + x)) / 2


def test_tangent_frame():
    """The frame of an anisotropic surface: orthonormal and right-handed with the normal,
    the tangent along the in-plane part of the first edge at rotation 0, along n x e1 at a
    quarter turn, reversed at half a turn."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        e1 = rng.normal(size=3)
        e1 -= n * (n @ e1) * rng.uniform(0, 1)          # not necessarily in the plane
        rot = rng.uniform(0, 1)
        t, b = oracle.tangent_frame(n, e1, rot)
        M = np.stack([t, b, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(t, b), n, atol=1e-12)
        p = e1 - n * (n @ e1)
        p /= np.linalg.norm(p)
        t0, _ = oracle.tangent_frame(n, e1, 0.0)
        assert np.allclose(t0, p, atol=1e-12)
        tq, _ = oracle.tangent_frame(n, e1, 0.25)
        assert np.allclose(tq, np.cross(n, p), atol=1e-12)
        th, _ = oracle.tangent_frame(n, e1, 0.5)
        assert np.allclose(th, -p, atol=1e-12)
        assert t @ p == pytest.approx(math.cos(2 * math.pi * rot), abs=1e-12)


def test_vndf_sampler_matches_visible_normal_density():
    # E_h[h_z^2] under VNDF sampling equals the quadrature of h_z^2 G1 (wo.h) D / wo_z
    for alpha, mu_o in ((0.3, 0.8), (0.6, 0.3)):
        wo = _hemi_dir(mu_o, 0.4)
        n = 60000
        u = RNG.random((n, 2))
        hs = np.array([oracle.ggx_vndf_sample(wo, alpha, a, b) for a, b in u])
        assert np.all(hs[:, 2] >= 0) and np.allclose(np.linalg.norm(hs, axis=1), 1.0)
        assert np.all(hs @ wo >= -1e-12)
        est = (hs[:, 2] ** 2).mean()
        err = (hs[:, 2] ** 2).std() / math.sqrt(n)
        # quadrature
        nt, nphi = 600, 256
        t = (np.arange(nt) + 0.5) / nt * (math.pi / 2)
        phis = (np.arange(nphi) + 0.5) / nphi * 2 * math.pi
        T, P = np.meshgrid(t, phis, indexing="ij")
        h = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
        D = np.array([oracle.ggx_D(x, alpha) for x in h[:: 1]])
        dens = oracle.ggx_G1(wo, alpha) * np.maximum(h @ wo, 0) * D / wo[2]
        w = (np.sin(T).ravel()) * (math.pi / 2 / nt) * (2 * math.pi / nphi)
        assert (dens * w).sum() == pytest.approx(1.0, abs=3e-3)
        ref = (dens * h[:, 2] ** 2 * w).sum()
        assert abs(est - ref) < 4 * err + 2e-3


def test_lambert_closed_form():
    rho = np.array([0.3, 0.6, 0.9])
    mat = scenes.openpbr(base_color=tuple(rho), specular_weight=0.0)
    wo = _sphere_dirs(500)
    wo[:, 2] = np.abs(wo[:, 2]) + 1e-3
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    wi = _sphere_dirs(500)
    wi[:, 2] = np.abs(wi[:, 2]) + 1e-3
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    f, pdf = oracle.bsdf_eval_batch(mat, 1, wo, wi)
    assert np.allclose(f, rho / math.pi, rtol=1e-14)
    assert np.allclose(pdf, wi[:, 2] / math.pi, rtol=1e-14)
    # a below-horizon direction gets nothing
    f, pdf = oracle.bsdf_eval_batch(mat, 1, wo, wi * np.array([1, 1, -1]))
    assert np.all(f == 0) and np.all(pdf == 0)


def test_delta_lobes_weights():
    glass = scenes.openpbr(base_color=(1, 1, 1), specular_roughness=0.0, transmission_weight=1.0)
    for mu in (0.9, 0.5, 0.15):
        wo = _hemi_dir(mu)
        F = oracle.fresnel_dielectric(mu, 1.5)
        ok, wi, w, pdf, dl = oracle.bsdf_sample(glass, 1, wo, [0.5, 0.3, 0.3, F * 0.5])
        assert ok and dl and np.allclose(wi, [-wo[0], -wo[1], wo[2]])
        assert np.allclose(w, 1.0)  # F / P(reflect) with P(reflect) = F
        ok, wi, w, pdf, dl = oracle.bsdf_sample(glass, 1, wo, [0.5, 0.3, 0.3, 0.5 * (1 + F)])
        assert ok and dl and wi[2] < 0
        assert np.allclose(w, 1.0 / 1.5 ** 2)  # radiance scaling 1/eta^2
        # Snell's law on the refracted direction
        s_t = math.sqrt(wi[0] ** 2 + wi[1] ** 2)
        assert s_t == pytest.approx(math.sqrt(1 - mu * mu) / 1.5, rel=1e-12)
    # a perfect mirror conductor (F0 = 1) has reflectance 1 at every angle
    mirror = scenes.openpbr(base_color=(1, 1, 1), base_metalness=1.0, specular_roughness=0.0)
    for mu in (0.95, 0.3, 0.02):
        ok, wi, w, pdf, dl = oracle.bsdf_sample(mirror, 1, _hemi_dir(mu), [0.2, 0.5, 0.5, 0.5])
        assert ok and dl and np.allclose(w, 1.0)
    # total internal reflection from inside the glass
    cc = math.cos(math.asin(1 / 1.5))
    wo = _hemi_dir(cc * 0.5)
    for u8 in (0.1, 0.9):
        ok, wi, w, pdf, dl = oracle.bsdf_sample(glass, 0, wo, [0.5, 0.3, 0.3, u8])
        assert ok and wi[2] > 0 and np.allclose(w, 1.0)


# ------------------------------------------------------------------ Monte Carlo identities

@pytest.mark.parametrize("name", sorted(MATS))
def test_sample_eval_consistency(name):
    mat = MATS[name]
    for front in (1, 0):
        for mu in (0.9, 0.4, 0.08):
            n = 3000 // (FUZZ_SCALE if "fuzz" in name else 1)
            wo = np.tile(_hemi_dir(mu, 1.1), (n, 1))
            u = RNG.random((n, 4))
            ok, wi, w, pdf, dl = oracle.bsdf_sample_batch(mat, front, wo, u)
            sel = ok & ~dl
            assert sel.sum() > 0
            f, pdf2 = oracle.bsdf_eval_batch(mat, front, wo[sel], wi[sel])
            assert np.allclose(pdf[sel], pdf2, rtol=1e-10)
            assert np.allclose(w[sel], f * np.abs(wi[sel, 2:3]) / pdf2[:, None], rtol=1e-9)
            assert np.allclose(np.linalg.norm(wi[sel], axis=1), 1.0, atol=1e-12)


@pytest.mark.parametrize("name", sorted(MATS))
def test_pdf_integrates_to_valid_sample_fraction(name):
    mat = MATS[name]
    for front in (1, 0):
        for mu in (0.85, 0.3):
            wo = _hemi_dir(mu, 0.7)
            n = 200_000 // (FUZZ_SCALE if "fuzz" in name else 1)
            dirs = _sphere_dirs(n)
            _, pdf = oracle.bsdf_eval_batch(mat, front, np.tile(wo, (n, 1)), dirs)
            vals = pdf * 4 * math.pi
            integral, err_i = vals.mean(), vals.std() / math.sqrt(n)
            m = 100_000 // (FUZZ_SCALE if "fuzz" in name else 1)
            ok, wi, w, p, dl = oracle.bsdf_sample_batch(mat, front, np.tile(wo, (m, 1)),
                                                        RNG.random((m, 4)))
            frac = (ok & ~dl).mean()
            err_f = math.sqrt(frac * (1 - frac) / m)
            assert integral <= 1.0 + 4 * err_i
            assert abs(integral - frac) < 4.5 * math.hypot(err_i, err_f) + 1e-3, (integral, frac)


@pytest.mark.parametrize("name", sorted(WHITE))
def test_albedo_at_most_one(name):
    mat = WHITE[name]
    for front in (1, 0):
        for mu in (0.98, 0.7, 0.4, 0.15, 0.03):
            n = 40_000 // (4 * FUZZ_SCALE if "fuzz" in name else 1)
            ok, wi, w, p, dl = oracle.bsdf_sample_batch(mat, front, np.tile(_hemi_dir(mu), (n, 1)),
                                                        RNG.random((n, 4)))
            if front == 0 and "glass" in name or "mixed" in name and front == 0:
                # transmissive interfaces seen from inside: radiance scaling by eta^2 < 1 side
                w = w * np.where(wi[:, 2:3] < 0, 1.0 / 1.5 ** 2, 1.0)
            alb = w.mean(0)
            err = w.std(0) / math.sqrt(n)
            assert np.all(alb <= 1.0 + 4 * err + 1e-3), (mu, front, alb)
            assert np.all(alb > 0.0)


def test_white_lambert_albedo_exactly_one():
    mat = scenes.openpbr(base_color=(1, 1, 1), specular_weight=0.0)
    n = 2000
    ok, wi, w, p, dl = oracle.bsdf_sample_batch(mat, 1, np.tile(_hemi_dir(0.4), (n, 1)),
                                                RNG.random((n, 4)))
    assert ok.all() and np.allclose(w, 1.0, rtol=1e-12)


@pytest.mark.parametrize("name", sorted(MATS))
def test_reciprocity(name):
    mat = MATS[name]
    n = 400
    a = _sphere_dirs(n)
    b = _sphere_dirs(n)
    a[:, 2] = np.abs(a[:, 2]) + 1e-3
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    # reflection: f(a, b) = f(b, a) with both directions above the surface
    b_up = b.copy()
    b_up[:, 2] = np.abs(b_up[:, 2]) + 1e-3
    b_up /= np.linalg.norm(b_up, axis=1, keepdims=True)
    for front in (1, 0):
        f1, _ = oracle.bsdf_eval_batch(mat, front, a, b_up)
        f2, _ = oracle.bsdf_eval_batch(mat, front, b_up, a)
        assert np.allclose(f1, f2, rtol=1e-12, atol=1e-300)
    # transmission: f(a -> b)/eta_a^2 = f(b -> a)/eta_b^2, evaluated from the other side; a
    # thin-walled sheet has the same medium on both sides (eta 1 across it)
    b_dn = b_up * np.array([1, 1, -1])
    flip = np.array([1, 1, -1])
    f_fwd, _ = oracle.bsdf_eval_batch(mat, 1, a, b_dn)
    f_rev, _ = oracle.bsdf_eval_batch(mat, 0, b_dn * flip, a * flip)
    if mat[12] > 0:
        assert np.any(f_fwd > 0)
    eta2 = 1.0 if mat[26] > 0 else 1.5 ** 2
    # Grazing on the outside (wo.h -> 0) is the critical angle on the inside, where the
    # transmitted cosine is the square root of a difference that cancels: the two sides then
    # agree to about 1e-16 / (wo.h)^2 relative, not to 1e-10.
    h = a + (1.0 if mat[26] > 0 else 1.5) * (b_dn * (flip if mat[26] > 0 else 1))
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    oh = np.abs((a * h).sum(1))
    rtol = 1e-10 + 1e-15 / np.maximum(oh, 1e-300) ** 2
    assert np.all(np.abs(f_fwd - f_rev / eta2) <= rtol[:, None] * np.abs(f_rev / eta2) + 1e-300)


@pytest.mark.parametrize("name", ["plastic", "metal", "coated", "rough_glass", "mixed", "thin_glass", "rough_diffuse",
                                  "aniso_metal", "aniso_glass"])
def test_sampler_chi_square(name):
    mat = MATS[name]
    mu = 0.55
    wo = _hemi_dir(mu, 0.9)
    nz, nphi = 20, 24
    n = 150_000
    ok, wi, w, p, dl = oracle.bsdf_sample_batch(mat, 1, np.tile(wo, (n, 1)), RNG.random((n, 4)))
    assert not dl.any()
    z = wi[ok, 2]
    phi = np.mod(np.arctan2(wi[ok, 1], wi[ok, 0]), 2 * math.pi)
    obs, _, _ = np.histogram2d(z, phi, bins=[nz, nphi], range=[[-1, 1], [0, 2 * math.pi]])
    # expected mass per bin: midpoint quadrature of the pdf in (z, phi), 8 x 8 per bin
    sub = 8
    zs = -1 + (np.arange(nz * sub) + 0.5) * (2.0 / (nz * sub))
    ps = (np.arange(nphi * sub) + 0.5) * (2 * math.pi / (nphi * sub))
    Z, P = np.meshgrid(zs, ps, indexing="ij")
    R = np.sqrt(1 - Z * Z)
    dirs = np.stack([R * np.cos(P), R * np.sin(P), Z], -1).reshape(-1, 3)
    _, pdf = oracle.bsdf_eval_batch(mat, 1, np.tile(wo, (dirs.shape[0], 1)), dirs)
    cell = (2.0 / (nz * sub)) * (2 * math.pi / (nphi * sub))
    exp = (pdf.reshape(nz * sub, nphi * sub) * cell).reshape(nz, sub, nphi, sub).sum((1, 3)) * n
    invalid_obs = n - ok.sum()
    invalid_exp = n - exp.sum()
    o = np.append(obs.ravel(), invalid_obs)
    e = np.append(exp.ravel(), max(invalid_exp, 1e-9))
    keep = e >= 5
    o_m = np.append(o[keep], o[~keep].sum())
    e_m = np.append(e[keep], e[~keep].sum())
    if e_m[-1] < 5:
        o_m, e_m = o_m[:-1], e_m[:-1]
    stat = ((o_m - e_m) ** 2 / e_m).sum()
    dof = len(o_m) - 1
    assert chi2d.sf(stat, dof) > 1e-5, (stat, dof)


def test_lobe_probabilities_form_a_distribution():
    for name, mat in {**MATS, **WHITE}.items():
        for front in (1, 0):
            for mu in (0.9, 0.3, 0.01):
                p = oracle.lobe_probs(mat, front, mu)
                assert np.all(p >= 0) and p.sum() == pytest.approx(1.0, abs=1e-12), name
