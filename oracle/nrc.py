"""Neural radiance cache oracle in numpy float64 -- TEST INFRASTRUCTURE ONLY.

The paper names neural radiance caching as future work to cut the samples per pixel
(Sec. 6.1).  This is the cache the GPU library implements, written plainly:

  input  x = [ hash-grid features of the position (L levels x F features),
               direction (3), normal (3), roughness (1), 1, zero padding ]   (64 wide)
  MLP    h_1 = relu(W_0 x), ..., h_4 = relu(W_3 h_3), y = W_4 h_4          (no biases)
  loss   relative L2: mean over samples and channels of (y - t)^2 / (sg(y)^2 + 0.01)
  update Adam (beta1 0.9, beta2 0.99, eps 1e-15) on the MLP weights; lazy Adam on the grid
         table: an entry whose gradient is exactly zero in a step keeps its value and its
         moments (the sparse/lazy Adam variant; a hash table receives sparse gradients)

Hash grid (multiresolution, as in Mueller et al. 2022): level l has resolution
N_l = floor(N_min * b^l); the 8 corners of the cell around p * N_l are looked up densely
when (N_l + 1)^3 <= T, else by the spatial hash (x * 1) ^ (y * 2654435761) ^ (z * 805459861)
mod T, and interpolated trilinearly.

Pins (tests/test_oracle_nrc.py): trilinear interpolation reproduces linear functions
exactly on dense levels, the backward pass matches central finite differences and torch
autograd on the CPU, and the Adam step matches torch.optim.Adam.
"""
from __future__ import annotations

import math

import numpy as np

WIDTH = 64
N_OUT = 3
PRIMES = (1, 2654435761, 805459861)


def level_resolutions(n_levels=16, base_resolution=16, per_level_scale=0.0, finest=2048):
    if per_level_scale <= 0.0:
        per_level_scale = math.exp((math.log(finest) - math.log(base_resolution)) / max(n_levels - 1, 1))
    return [int(math.floor(base_resolution * per_level_scale ** l)) for l in range(n_levels)]


def corner_indices(cell, res, table_size):
    """cell: (N, 3) int64 integer corners; returns table indices (N,)."""
    n1 = res + 1
    if n1 ** 3 <= table_size:
        return cell[:, 0] + n1 * (cell[:, 1] + n1 * cell[:, 2])
    h = (cell[:, 0].astype(np.uint64) * np.uint64(PRIMES[0])) ^ \
        (cell[:, 1].astype(np.uint64) * np.uint64(PRIMES[1])) ^ \
        (cell[:, 2].astype(np.uint64) * np.uint64(PRIMES[2]))
    h = h & np.uint64(0xFFFFFFFF)  # 32-bit arithmetic
    return (h % np.uint64(table_size)).astype(np.int64)


def encode(pos01, table, resolutions):
    """Hash-grid features.  pos01 (N, 3) in [0, 1]; table (L, T, F).
    Returns feats (N, L*F) and the (indices, weights) of every level's 8 corners."""
    n = pos01.shape[0]
    L, T, F = table.shape
    feats = np.zeros((n, L * F))
    lookups = []
    for l, res in enumerate(resolutions):
        xs = pos01 * res
        cell0 = np.floor(xs).astype(np.int64)
        cell0 = np.clip(cell0, 0, res - 1)
        fr = xs - cell0
        idx_l, w_l = [], []
        for c in range(8):
            off = np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1])
            corner = cell0 + off
            w = np.prod(np.where(off == 1, fr, 1.0 - fr), axis=1)
            idx = corner_indices(corner, res, T)
            feats[:, l * F:(l + 1) * F] += w[:, None] * table[l, idx]
            idx_l.append(idx)
            w_l.append(w)
        lookups.append((np.stack(idx_l, 1), np.stack(w_l, 1)))
    return feats, lookups


def build_input(grid_feats, dirs, normals, rough):
    """Concatenate the encoded position with direction, normal, roughness, a constant 1 and
    zero padding to 64 columns."""
    n = grid_feats.shape[0]
    x = np.zeros((n, WIDTH))
    g = grid_feats.shape[1]
    x[:, :g] = grid_feats
    x[:, g:g + 3] = dirs
    x[:, g + 3:g + 6] = normals
    x[:, g + 6] = rough
    x[:, g + 7] = 1.0
    return x


def mlp_forward(x, weights):
    """weights: [W_0 .. W_4] with W_i (out, in); returns y and the list of layer inputs."""
    acts = [x]
    h = x
    for W in weights[:-1]:
        h = np.maximum(h @ W.T, 0.0)
        acts.append(h)
    y = h @ weights[-1].T
    return y, acts


def relative_l2(y, target, eps=0.01):
    """Loss and its gradient w.r.t. y; the denominator is treated as a constant."""
    denom = y * y + eps
    n = y.size
    loss = float(((y - target) ** 2 / denom).sum() / n)
    dy = 2.0 * (y - target) / denom / n
    return loss, dy


def mlp_backward(acts, weights, dy, operand=None):
    """Gradients of the weights and of the input given dL/dy.  operand: optional function
    applied to each layer's output gradient where it enters the products (a tensor-core
    implementation holds it as an FP16 operand); None = exact."""
    grads = [None] * len(weights)
    g = dy
    for i in range(len(weights) - 1, -1, -1):
        if operand is not None:
            g = operand(g)
        a = acts[i]
        grads[i] = g.T @ a
        g = g @ weights[i]
        if i > 0:
            g = g * (acts[i] > 0.0)
    return grads, g


def grid_backward(lookups, dfeat, table_shape):
    """Scatter dL/dfeatures back onto the table entries (dense gradient array)."""
    L, T, F = table_shape
    dtable = np.zeros(table_shape)
    for l, (idx, w) in enumerate(lookups):
        g = dfeat[:, l * F:(l + 1) * F]
        for c in range(8):
            np.add.at(dtable[l], idx[:, c], w[:, c:c + 1] * g)
    return dtable


def adam(param, grad, m, v, t, lr, beta1=0.9, beta2=0.99, eps=1e-15, lazy=False):
    """One Adam step (Kingma & Ba); t counts from 1 and is shared by every entry.  Returns new
    (param, m, v).  lazy=True: entries with grad == 0 are left as they are (value and moments)."""
    m_new = beta1 * m + (1.0 - beta1) * grad
    v_new = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m_new / (1.0 - beta1 ** t)
    vhat = v_new / (1.0 - beta2 ** t)
    p_new = param - lr * mhat / (np.sqrt(vhat) + eps)
    if lazy:
        keep = grad == 0.0
        p_new = np.where(keep, param, p_new)
        m_new = np.where(keep, m, m_new)
        v_new = np.where(keep, v, v_new)
    return p_new, m_new, v_new


def effective_roughness(metalness, spec_rough, transmission):
    """'Diffuse-ish' measure of a vertex: diffuse lobes count as roughness 1."""
    return metalness * spec_rough + (1.0 - metalness) * ((1.0 - transmission) + transmission * spec_rough)


def forward_all(pos01, dirs, normals, rough, table, weights, resolutions):
    feats, lookups = encode(pos01, table, resolutions)
    x = build_input(feats, dirs, normals, rough)
    y, acts = mlp_forward(x, weights)
    return y, acts, lookups


def train_step(pos01, dirs, normals, rough, target, table, weights, resolutions):
    """Loss and gradients of one batch (no update)."""
    y, acts, lookups = forward_all(pos01, dirs, normals, rough, table, weights, resolutions)
    loss, dy = relative_l2(y, target)
    gw, dx = mlp_backward(acts, weights, dy)
    L, T, F = table.shape
    dtable = grid_backward(lookups, dx[:, :L * F], table.shape)
    return loss, gw, dtable, y
