"""Regression denoiser oracle (BMFR) -- TEST INFRASTRUCTURE ONLY.

The paper lists denoising as future work (Sec. 6.3).  This is the blockwise multi-order
feature regression of Koskela et al. 2019 (BMFR) as a plain definition, in float64, for the
GPU's `pt_denoise_bmfr` to be checked against:

  input   mean radiance c (H, W, 3) and the primary-hit features (H, W, 12) of
          `oracle.features` / `pt_render_features`: normal n[3], scattering fraction,
          position p[3], -, albedo a[3], -
  pixels  a pixel takes part iff all its samples hit a scattering surface (fraction 1);
          the others are returned unchanged
  blocks  square blocks of `block` pixels; with offset (ox, oy) block (i, j) covers
          x in [i B - ox, (i+1) B - ox), y in [j B - oy, (j+1) B - oy), clipped to the image
  columns in this order: 1, n_x, n_y, n_z, q_x, q_y, q_z, q_x^2, q_y^2, q_z^2 with
          q = 2 (p - lo) / (hi - lo) - 1 (per block and axis: lo, hi = min, max over the
          block's taking-part pixels), and n scaled the same way; a feature whose block range
          hi - lo is at most 1e-4 max(|lo|, |hi|, 1e-2) is left out (with its square)
  drop    then, in that order, a column whose part orthogonal to the span of the earlier
          kept columns has norm at most 1e-3 of its own norm is left out (reading: the
          least-squares problem is solved on the columns that add a direction)
  fit     per channel, least squares of the demodulated colour c / (a + 0.01) on the kept
          columns; the output is the fitted value times (a + 0.01)

The scaling and the left-out columns change no span (a constant column lies in the span of
the column of ones, a left-out column in the span of the kept ones), so up to those two
tolerance rules the output is the orthogonal projection of the demodulated colour onto
span{1, n, p, p^2} over each block.  numpy's least-squares routine is the solver.

Pins (tests/test_oracle_bmfr.py): colours that are (demodulated) quadratics of position and
linear in the normal come back unchanged; the fit is idempotent; residuals are orthogonal to
the kept columns; non-taking-part pixels pass through; blocks are independent; a duplicated
feature changes nothing.
"""
from __future__ import annotations

import numpy as np

ALBEDO_EPS = 1e-2
RANGE_TOL = 1e-4
DEPENDENCE_TOL = 1e-3


def _scaled(f):
    """Feature column scaled to [-1, 1] over the block, or None if near-constant."""
    lo, hi = float(f.min()), float(f.max())
    if hi - lo <= RANGE_TOL * max(abs(lo), abs(hi), 1e-2):
        return None
    return 2.0 * (f - lo) / (hi - lo) - 1.0


def design_matrix(feats):
    """Columns of one block (rows = its taking-part pixels), before the dependence rule."""
    n, p = feats[:, 0:3], feats[:, 4:7]
    cols = [np.ones(len(feats))]
    for k in range(3):
        c = _scaled(n[:, k])
        if c is not None:
            cols.append(c)
    lin, sq = [], []
    for k in range(3):
        q = _scaled(p[:, k])
        if q is not None:
            lin.append(q)
            sq.append(q * q)
    return np.stack(cols + lin + sq, 1)


def kept_columns(A):
    """Columns that add a direction, in order: the part of column k orthogonal to the span
    of the kept earlier ones has norm > DEPENDENCE_TOL * |column k|."""
    keep = []
    for k in range(A.shape[1]):
        col = A[:, k]
        if keep:
            B = A[:, keep]
            coef, *_ = np.linalg.lstsq(B, col, rcond=None)
            res = col - B @ coef
        else:
            res = col
        if np.linalg.norm(res) > DEPENDENCE_TOL * np.linalg.norm(col):
            keep.append(k)
    return A[:, keep]


def _blocks(h, w, block, offset):
    ox, oy = offset
    for by in range(-(oy % block) if oy % block else 0, h, block):
        for bx in range(-(ox % block) if ox % block else 0, w, block):
            yield max(by, 0), min(by + block, h), max(bx, 0), min(bx + block, w)


def bmfr(color, feats, block=32, offset=(0, 0)):
    """Denoised (H, W, 3) float64 image."""
    color = np.asarray(color, np.float64)
    feats = np.asarray(feats, np.float64)
    h, w = color.shape[:2]
    out = color.copy()
    for y0, y1, x0, x1 in _blocks(h, w, block, offset):
        f = feats[y0:y1, x0:x1].reshape(-1, 12)
        c = color[y0:y1, x0:x1].reshape(-1, 3)
        take = f[:, 3] >= 1.0
        if not take.any():
            continue
        A = kept_columns(design_matrix(f[take]))
        a = f[take, 8:11] + ALBEDO_EPS
        b = c[take] / a
        x, *_ = np.linalg.lstsq(A, b, rcond=None)
        fitted = (A @ x) * a
        blk = out[y0:y1, x0:x1].reshape(-1, 3)
        blk[take] = fitted
        out[y0:y1, x0:x1] = blk.reshape(y1 - y0, x1 - x0, 3)
    return out
