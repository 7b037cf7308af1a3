"""Pins of the display-resolve oracle (oracle/tonemap.py): facts the Khronos PBR Neutral
mapping and the sRGB transfer function fix, independent of how the oracle writes them."""
import numpy as np
import pytest

from oracle import tonemap as tm

RNG = np.random.default_rng(7)


def test_identity_region_subtracts_f90():
    """Below the knee and above the toe the mapping is c - 0.04 exactly."""
    c = RNG.uniform(0.08, 0.79, (2000, 3)).astype(np.float32)
    c = c[(c - 0.04).max(-1) < 0.76 - 1e-6]
    out = tm.pbr_neutral(c)
    assert np.array_equal(out, (c - np.float32(0.04)).astype(np.float32))


def test_toe_is_smooth_at_its_join():
    """The offset x - x^2/(4 F90) meets the constant F90 with equal value and slope at 0.08."""
    def offset(x):
        c = np.array([[x, 0.5, 0.5]], np.float32)
        return 0.5 - float(tm.pbr_neutral(c)[0, 1])      # channel 1 sees only the offset
    h = 1e-3
    assert abs(offset(0.08 - 1e-7) - 0.04) < 1e-6
    assert abs(offset(0.08 + 1e-7) - 0.04) < 1e-6
    slope_left = (offset(0.08) - offset(0.08 - h)) / h
    assert abs(slope_left) < 2e-3 * 10                    # slope 1 - 12.5 x -> 0 at the join
    assert abs(offset(0.0)) < 1e-9                        # black stays black


def test_compression_continuous_and_bounded():
    """At the knee p = K_s the compressed peak equals p; beyond it the peak approaches 1."""
    below = tm.pbr_neutral(np.array([[0.7599, 0.5, 0.5]], np.float32) + np.float32(0.04))
    above = tm.pbr_neutral(np.array([[0.7601, 0.5, 0.5]], np.float32) + np.float32(0.04))
    assert abs(float(below.max()) - float(above.max())) < 1e-3
    big = tm.pbr_neutral(np.array([[1e6, 1e6, 1e6]], np.float32))
    assert 0.999 < float(big.max()) < 1.0
    peaks = tm.pbr_neutral(np.stack([np.linspace(0.9, 50, 200, dtype=np.float32)] * 3, -1)).max(-1)
    assert np.all(np.diff(peaks) > 0)


def test_outputs_in_unit_range_and_greys_stay_grey():
    c = (RNG.random((20000, 3)) ** 3 * 200).astype(np.float32)
    out = tm.pbr_neutral(c)
    assert np.all(out >= -1e-7) and np.all(out < 1.0)
    grey = np.repeat(RNG.uniform(0, 40, (500, 1)).astype(np.float32), 3, 1)
    g = tm.pbr_neutral(grey)
    assert np.all(g[:, 0] == g[:, 1]) and np.all(g[:, 1] == g[:, 2])


def test_desaturation_moves_highlights_towards_white():
    """A saturated highlight loses chroma: its channel spread relative to the peak shrinks."""
    c = np.array([[6.0, 0.6, 0.3]], np.float32)
    out = tm.pbr_neutral(c)[0]
    x = float(c.min()) ; f = 0.04 if x >= 0.08 else x - x * x / 0.16
    shifted = c[0] - f
    assert (out.max() - out.min()) / out.max() < (shifted.max() - shifted.min()) / shifted.max()
    assert out.min() > shifted.min() * out.max() / shifted.max()


def test_desaturation_constant_half_way_to_white():
    """The desaturation step mixes the compressed colour towards white by
    g = 1 - 1 / (K_d (p - p') + 1), p - p' the amount the highlight was compressed and K_d = 0.15
    the published desaturation speed: a highlight compressed by exactly 1 / K_d = 20/3 is moved
    half-way to white.  A pure-red highlight c = (p, 0, 0) has no toe offset (the offset
    x - x^2 / (4 F90) vanishes at its minimum x = 0) and becomes (p', g p', g p'), so green
    over red reads g directly.  p solves p - p'(p) = 20/3 with p' = 1 - d^2 / (p + d - K_s),
    d = 1 - K_s (bisection in float64).  With K_d = 0.10 or 0.30 the ratio is 0.40 or 0.67."""
    ks, d = 0.76, 0.24
    lo, hi = 1.0, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid - (1 - d * d / (mid + d - ks)) < 20.0 / 3.0:
            lo = mid
        else:
            hi = mid
    p = 0.5 * (lo + hi)
    out = tm.pbr_neutral(np.array([[p, 0.0, 0.0]], np.float32))[0].astype(np.float64)
    assert out[1] == out[2]
    assert out[1] / out[0] == pytest.approx(0.5, abs=2e-6)
    assert out[0] == pytest.approx(1 - d * d / (p + d - ks), abs=2e-6)
    # at the knee (p = K_s) nothing has been compressed, so nothing is desaturated
    knee = tm.pbr_neutral(np.array([[0.76 + 1e-4, 0.0, 0.0]], np.float32))[0].astype(np.float64)
    assert knee[1] / knee[0] < 1e-5


def test_srgb_closed_forms():
    assert abs(float(tm.srgb_encode(np.float32(1.0))) - 1.0) <= 1.2e-7   # 1.055 - 0.055 in float32
    assert float(tm.srgb_encode(np.float32(0.0))) == 0.0
    half = 1.055 * 0.5 ** (1 / 2.4) - 0.055
    assert abs(float(tm.srgb_encode(np.float32(0.5))) - half) < 1e-6
    k = np.float32(0.0031308)
    assert abs(float(tm.srgb_encode(k)) - float(tm.srgb_encode(np.nextafter(k, np.float32(1))))) < 1e-5


def test_resolve_quantises_and_sets_alpha():
    s = np.zeros((2, 3, 3), np.float32)
    s[0, 0] = 1e6
    out = tm.resolve(s, 4)
    assert out.dtype == np.uint8 and out.shape == (2, 3, 4)
    assert np.all(out[..., 3] == 255)
    assert tuple(out[0, 0, :3]) == (255, 255, 255) and tuple(out[1, 2, :3]) == (0, 0, 0)
