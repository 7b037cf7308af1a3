"""Image-level pins of the oracle: white furnace (convex and concave), a diffuse plane under
a uniform sky, direct lighting from a quad against Lambert's polygon formula, and the
determinism properties the progressive/crop parity relies on."""
import math

import numpy as np
import pytest

import oracle
from paper_2407_19977_gb300 import scenes


def _zscores(samples):
    """Per-pixel z-score of the sample mean against its own standard error."""
    mean = samples.mean(2)
    se = samples.std(2, ddof=1) / math.sqrt(samples.shape[2])
    return mean, se


def test_white_furnace_convex():
    sc = scenes.furnace_sphere(level=2, width=24, height=24, spp=32, max_depth=4)
    osc = oracle.OracleScene(sc)
    # BSDF sampling only: every sample of an albedo-1 convex object under L = 1 is exactly 1
    s, smp, st = osc.render(no_nee=True, keep_samples=True)
    assert np.allclose(smp, 1.0, atol=1e-12)
    # with NEE + MIS the estimator is still unbiased
    s, smp, st = osc.render(keep_samples=True, spp=64)
    mean, se = _zscores(smp)
    z = (mean - 1.0) / np.maximum(se, 1e-12)
    assert np.abs(z).max() < 5.5
    assert abs(mean.mean() - 1.0) < 4 * math.sqrt((se ** 2).sum()) / mean.size + 1e-12
    assert st["shadow_rays"] > 0 and st["nan_dropped"] == 0


def test_white_furnace_concave():
    sc = scenes.furnace_sphere(level=3, displace=0.45, width=20, height=20, spp=32, max_depth=64)
    osc = oracle.OracleScene(sc)
    s, smp, st = osc.render(no_nee=True, no_rr=True, keep_samples=True)
    # BSDF sampling only: each path is 1 once it escapes; paths can only be lost by the
    # 64-bounce cap, which an open-enough concavity practically never reaches
    assert np.mean(np.isclose(smp, 1.0, atol=1e-12)) > 0.999
    assert st["ext_rays"] > 1.3 * st["paths"]   # there were interreflections
    s, smp, st = osc.render(no_rr=True, keep_samples=True, spp=64)
    mean, se = _zscores(smp)
    tot = mean.mean()
    tot_se = math.sqrt((se ** 2).sum()) / mean.size
    assert abs(tot - 1.0) < 4.5 * tot_se
    # roulette keeps it unbiased
    s, smp, st = osc.render(keep_samples=True, spp=64)
    mean, se = _zscores(smp)
    assert abs(mean.mean() - 1.0) < 4.5 * math.sqrt((se ** 2).sum()) / mean.size
    assert st["rr_terminated"] > 0


@pytest.mark.parametrize("no_nee", [False, True])
def test_diffuse_plane_under_uniform_sky(no_nee):
    rho = 0.5
    sc = scenes.plane_under_sky(albedo=rho, spp=128)
    osc = oracle.OracleScene(sc)
    s, smp, st = osc.render(keep_samples=True, no_nee=no_nee)
    mean, se = _zscores(smp)
    # E = pi L on the upper hemisphere, L_o = rho E / pi = rho
    tot_se = math.sqrt((se ** 2).sum()) / mean.size
    assert abs(mean.mean() - rho) < 4.5 * tot_se
    assert np.abs((mean - rho) / np.maximum(se, 1e-12)).max() < 5.5


def _polygon_irradiance(x, n, verts, L):
    """Lambert's polygon formula: E = L/2 * sum_i gamma_i (n . unit(u_i x u_{i+1}))."""
    u = verts - x
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    acc = 0.0
    for i in range(len(u)):
        a, b = u[i], u[(i + 1) % len(u)]
        c = np.cross(a, b)
        gamma = math.acos(max(-1.0, min(1.0, float(a @ b))))
        acc += gamma * float(n @ (c / np.linalg.norm(c)))
    return 0.5 * L * abs(acc)


@pytest.mark.parametrize("no_nee", [False, True])
def test_quad_light_direct_lighting_closed_form(no_nee):
    rho, Lq = 0.8, 5.0
    spp = 256 if not no_nee else 1024
    sc = scenes.plane_with_quad(albedo=rho, radiance=Lq, width=12, height=12, spp=spp)
    osc = oracle.OracleScene(sc)
    s, smp, st = osc.render(keep_samples=True, no_nee=no_nee)
    mean, se = _zscores(smp)
    q = sc.lights[0].astype(np.float64)
    p0, e1, e2 = q[0:3], q[3:6], q[6:9]
    verts = np.array([p0, p0 + e1, p0 + e1 + e2, p0 + e2])
    cam = sc.camera
    zs = []
    for py in range(cam.height):
        for px in range(cam.width):
            # the estimator's expectation given its own camera rays, sample by sample
            ref = []
            for s_i in range(0, spp, 16):
                o, d = oracle.camera_ray(cam, px, py, s_i, 0)
                t = -o[1] / d[1]
                xh = o + t * d
                ref.append(rho / math.pi * _polygon_irradiance(xh, np.array([0, 1.0, 0]), verts, Lq))
            ref = np.mean(ref)
            zs.append((mean[py, px, 0] - ref) / max(se[py, px, 0], 1e-12))
            assert abs(mean[py, px, 0] - ref) < 5.5 * se[py, px, 0] + 2e-3 * ref
    zs = np.array(zs)
    assert abs(zs.mean()) < 4.5 / math.sqrt(len(zs)) + 0.15


def test_progressive_and_crop_consistency():
    sc = scenes.cornell_box(width=32, height=32, spp=8)
    osc = oracle.OracleScene(sc)
    full, _, _ = osc.render(spp=8)
    again, _, _ = osc.render(spp=8, threads=3)
    assert np.array_equal(full, again)
    a, _, _ = osc.render(spp=3, s0=0)
    b, _, _ = osc.render(spp=5, s0=3)
    assert np.allclose(a + b, full, rtol=1e-12, atol=1e-15)
    crop, _, _ = osc.render(spp=8, crop=(5, 7, 11, 9))
    assert np.allclose(crop, full[7:16, 5:16], rtol=1e-13, atol=0)
    rows, _, _ = osc.render(spp=8, row_step=4)
    assert np.allclose(rows[::4], full[::4]) and np.all(rows[1::4] == 0)


def test_mse_decreases_as_one_over_spp():
    sc = scenes.cornell_box(width=16, height=16)
    osc = oracle.OracleScene(sc)
    ref, _, _ = osc.render(spp=1024, s0=100000)
    ref /= 1024
    spps = [4, 16, 64]
    mse = []
    for k, n in enumerate(spps):
        errs = []
        for rep in range(4):
            img, _, _ = osc.render(spp=n, s0=1000 * (rep + 1) + 200000 * k)
            errs.append(((img / n - ref) ** 2).mean())
        mse.append(np.mean(errs))
    slope = np.polyfit(np.log(spps), np.log(mse), 1)[0]
    assert -1.25 < slope < -0.75, (slope, mse)


@pytest.mark.parametrize("no_rr", [False, True])
def test_emissive_enclosure_closed_form(no_rr):
    rho, le = 0.6, 0.4
    sc = scenes.emissive_sphere_interior(albedo=rho, emission=le, spp=64,
                                         max_depth=60 if no_rr else 200)
    osc = oracle.OracleScene(sc)
    s, smp, st = osc.render(keep_samples=True, no_rr=no_rr)
    mean, se = _zscores(smp)
    rho, le = float(sc.materials[0, 1]), float(sc.materials[0, 22])  # float32-rounded inputs
    expect = le / (1.0 - rho) * (1.0 - rho ** 61 if no_rr else 1.0)
    tot_se = math.sqrt((se ** 2).sum()) / mean.size
    assert abs(mean.mean() - expect) < 4.5 * tot_se + 1e-12, (mean.mean(), expect, tot_se)
    if no_rr:
        # without roulette every sample is the same geometric series
        assert np.allclose(smp, le * (1 - rho ** 61) / (1 - rho), rtol=1e-12)
    else:
        assert st["rr_terminated"] == st["paths"]
