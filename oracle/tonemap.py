"""Display resolve oracle -- TEST INFRASTRUCTURE ONLY.

The paper shows the accumulated image through a full-screen pass that applies the Khronos
PBR Neutral tone mapper (Sec. 5.1.4).  That mapper, as Khronos publishes it, has three
constants and four steps on a linear RGB colour c:

  F90 = 0.04          K_s = 0.8 - F90 (start of highlight compression)     K_d = 0.15

  1. x = min(c); the offset f = x - x^2 / (4 F90) if x < 2 F90, else F90; c <- c - f
     (a smooth toe: f and its slope are continuous at x = 2 F90)
  2. p = max(c); if p < K_s the colour is returned as it is
  3. d = 1 - K_s; p' = 1 - d^2 / (p + d - K_s); c <- c * p' / p   (p' -> 1 as p -> inf)
  4. g = 1 - 1 / (K_d (p - p') + 1); c <- (1 - g) c + g p' (1, 1, 1)   (desaturation)

The displayed image is the progressive mean (sum / spp) times an exposure (NaN read as 0,
clamped to [0, 1e30]: a guard of this library, radiance being finite and >= 0), tone mapped,
then (reading of this library) encoded with the sRGB transfer function of IEC 61966-2-1 and
quantised to 8 bits as floor(255 v + 0.5), alpha 255.

The quantisation is an integer decided by floating point, so the oracle takes it in float32
(the precision of the paper's WGSL and of the CUDA kernel), step by step in the order above.

Pins (tests/test_oracle_tonemap.py): the exact identity region (c - F90 below the knee),
continuity of the toe and of the compression at their joins, outputs in [0, 1) for any
non-negative input, greys stay grey, the sRGB closed forms and its continuity.
"""
from __future__ import annotations

import numpy as np

F90 = np.float32(0.04)
K_S = np.float32(0.8) - F90
K_D = np.float32(0.15)


def pbr_neutral(c):
    """Khronos PBR Neutral on linear RGB, float32, c (..., 3) -> (..., 3)."""
    c = np.asarray(c, dtype=np.float32)
    x = c.min(-1, keepdims=True)
    f = np.where(x < np.float32(2) * F90, x - x * x / (np.float32(4) * F90), F90).astype(np.float32)
    c = (c - f).astype(np.float32)
    p = c.max(-1, keepdims=True)
    d = np.float32(1) - K_S
    with np.errstate(divide="ignore", invalid="ignore"):
        pn = (np.float32(1) - d * d / (p + d - K_S)).astype(np.float32)
        scaled = (c * (pn / p)).astype(np.float32)
        g = (np.float32(1) - np.float32(1) / (K_D * (p - pn) + np.float32(1))).astype(np.float32)
        mixed = ((np.float32(1) - g) * scaled + g * pn).astype(np.float32)
    return np.where(p < K_S, c, mixed).astype(np.float32)


def srgb_encode(v):
    """IEC 61966-2-1 transfer function on [0, 1] (clamped), float32."""
    v = np.clip(np.asarray(v, dtype=np.float32), np.float32(0), np.float32(1))
    lo = (np.float32(12.92) * v).astype(np.float32)
    hi = (np.float32(1.055) * np.power(v, np.float32(1.0 / 2.4)) - np.float32(0.055)).astype(np.float32)
    return np.where(v <= np.float32(0.0031308), lo, hi).astype(np.float32)


def resolve_float(sum_rgb, spp, exposure=1.0, srgb=True):
    """The pre-quantisation display values (H, W, 3) float32."""
    mean = (np.asarray(sum_rgb, dtype=np.float32) * np.float32(1.0 / spp)).astype(np.float32)
    mean = (mean * np.float32(exposure)).astype(np.float32)
    # guard of this library: NaN -> 0, the mean clamped to [0, 1e30]
    mean = np.where(np.isnan(mean), np.float32(0), np.clip(mean, np.float32(0), np.float32(1e30)))
    v = pbr_neutral(mean.astype(np.float32))
    v = np.clip(v, np.float32(0), np.float32(1))
    return srgb_encode(v) if srgb else v


def resolve(sum_rgb, spp, exposure=1.0, srgb=True):
    """(H, W, 4) uint8 display image."""
    v = resolve_float(sum_rgb, spp, exposure, srgb)
    q = np.floor(v * np.float32(255) + np.float32(0.5)).astype(np.int64)
    out = np.empty(v.shape[:-1] + (4,), np.uint8)
    out[..., :3] = np.clip(q, 0, 255)
    out[..., 3] = 255
    return out
