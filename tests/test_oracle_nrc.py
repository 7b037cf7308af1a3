"""Pins of the NRC oracle (oracle/nrc.py): encoding, backward pass, loss and optimiser."""
import math

import numpy as np
import pytest

from oracle import nrc

RNG = np.random.default_rng(31)


def _small(n_levels=4, log2_t=10, base=4, finest=64):
    res = nrc.level_resolutions(n_levels, base, 0.0, finest)
    table = RNG.normal(0, 0.1, (n_levels, 2 ** log2_t, 2))
    weights = [RNG.normal(0, 1 / math.sqrt(64), (64, 64)) for _ in range(4)] + [RNG.normal(0, 0.1, (3, 64))]
    return res, table, weights


def test_resolutions_geometric():
    res = nrc.level_resolutions(16, 16, 0.0, 2048)
    assert res[0] == 16 and res[-1] in (2047, 2048)
    assert all(b >= a for a, b in zip(res, res[1:]))


def test_trilinear_reproduces_linear_functions_on_dense_levels():
    res = [3, 5, 7]
    T = 2 ** 10
    table = np.zeros((3, T, 2))
    a = np.array([0.3, -1.2, 2.0])
    b = 0.25
    for l, r in enumerate(res):
        assert (r + 1) ** 3 <= T
        g = np.stack(np.meshgrid(*[np.arange(r + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
        idx = nrc.corner_indices(g, r, T)
        assert len(set(idx.tolist())) == len(idx)  # dense indexing is a bijection
        table[l, idx, 0] = (g / r) @ a + b
        table[l, idx, 1] = -(g / r) @ a
    p = RNG.random((500, 3))
    p[0] = [1.0, 1.0, 1.0]
    p[1] = [0.0, 0.0, 0.0]
    feats, _ = nrc.encode(p, table, res)
    for l in range(3):
        assert np.allclose(feats[:, 2 * l], p @ a + b, atol=1e-12)
        assert np.allclose(feats[:, 2 * l + 1], -(p @ a), atol=1e-12)


def test_hashed_levels_stay_in_range_and_interpolate():
    res = [200]
    T = 2 ** 12
    cells = RNG.integers(0, 201, (10000, 3))
    idx = nrc.corner_indices(cells, 200, T)
    assert idx.min() >= 0 and idx.max() < T
    table = RNG.normal(size=(1, T, 2))
    p = RNG.random((1000, 3))
    feats, lookups = nrc.encode(p, table, res)
    idx, w = lookups[0]
    assert np.allclose(w.sum(1), 1.0)
    assert np.all(w >= 0)
    # a corner of the cell reproduces its table entry exactly
    q = np.array([[17, 3, 150]]) / 200.0
    f, lk = nrc.encode(q, table, res)
    i0 = nrc.corner_indices(np.array([[17, 3, 150]]), 200, T)[0]
    assert np.allclose(f[0], table[0, i0])


def _loss(pos, dirs, normals, rough, target, table, weights, res):
    y, _, _ = nrc.forward_all(pos, dirs, normals, rough, table, weights, res)
    # the relative L2 denominator is a constant (stop-gradient): freeze it at the current y
    return y


def test_backward_matches_finite_differences():
    res, table, weights = _small()
    n = 64
    pos, dirs, normals = RNG.random((n, 3)), RNG.normal(size=(n, 3)), RNG.normal(size=(n, 3))
    rough = RNG.random(n)
    target = RNG.random((n, 3))
    loss, gw, dtable, y0 = nrc.train_step(pos, dirs, normals, rough, target, table, weights, res)
    denom = y0 * y0 + 0.01

    def frozen_loss(tab, ws):
        y, _, _ = nrc.forward_all(pos, dirs, normals, rough, tab, ws, res)
        return float(((y - target) ** 2 / denom).sum() / y.size)

    h = 1e-6
    for layer in range(5):
        for _ in range(4):
            i, j = RNG.integers(0, weights[layer].shape[0]), RNG.integers(0, weights[layer].shape[1])
            wp = [w.copy() for w in weights]
            wm = [w.copy() for w in weights]
            wp[layer][i, j] += h
            wm[layer][i, j] -= h
            fd = (frozen_loss(table, wp) - frozen_loss(table, wm)) / (2 * h)
            assert fd == pytest.approx(gw[layer][i, j], rel=1e-5, abs=1e-10)
    used = np.argwhere(np.abs(dtable) > 1e-5)
    ht = 1e-4   # table gradients are small against the loss: a larger step avoids cancellation
    for k in RNG.choice(len(used), 8, replace=False):
        l, t, f = used[k]
        tp, tm = table.copy(), table.copy()
        tp[l, t, f] += ht
        tm[l, t, f] -= ht
        fd = (frozen_loss(tp, weights) - frozen_loss(tm, weights)) / (2 * ht)
        assert fd == pytest.approx(dtable[l, t, f], rel=1e-5, abs=1e-10)


def test_mlp_backward_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    _, _, weights = _small()
    x = RNG.normal(size=(37, 64))
    target = RNG.random((37, 3))
    y, acts = nrc.mlp_forward(x, weights)
    loss, dy = nrc.relative_l2(y, target)
    gw, dx = nrc.mlp_backward(acts, weights, dy)
    tx = torch.tensor(x, requires_grad=True)
    tw = [torch.tensor(w, requires_grad=True) for w in weights]
    h = tx
    for w in tw[:-1]:
        h = torch.relu(torch.nn.functional.linear(h, w))
    ty = torch.nn.functional.linear(h, tw[-1])
    denom = (ty.detach() ** 2 + 0.01)
    tl = ((ty - torch.tensor(target)) ** 2 / denom).mean()
    tl.backward()
    assert float(tl) == pytest.approx(loss, rel=1e-12)
    for a, b in zip(gw, tw):
        assert np.allclose(a, b.grad.numpy(), rtol=1e-10, atol=1e-14)
    assert np.allclose(dx, tx.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    p = RNG.normal(size=50)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.99), eps=1e-15)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 6):
        g = RNG.normal(size=50)
        p, m, v = nrc.adam(p, g, m, v, t, 1e-2)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_lazy_adam_matches_torch_sparse_adam():
    """The grid's lazy Adam against torch.optim.SparseAdam, which updates only the entries a
    sparse gradient names (torch adds eps to sqrt(v) before the bias correction; with eps
    1e-15 that is far below the tolerance)."""
    torch = pytest.importorskip("torch")
    n = 200
    p = RNG.normal(size=n)
    tp = torch.nn.Parameter(torch.tensor(p.copy()))
    opt = torch.optim.SparseAdam([tp], lr=1e-2, betas=(0.9, 0.99), eps=1e-15)
    m = np.zeros(n)
    v = np.zeros(n)
    moved_by_dense = False
    for t in range(1, 7):
        idx = np.sort(RNG.choice(n, 40, replace=False))
        g = np.zeros(n)
        g[idx] = RNG.normal(size=40)
        p_dense, _, _ = nrc.adam(p, g, m, v, t, 1e-2)
        p_new, m, v = nrc.adam(p, g, m, v, t, 1e-2, lazy=True)
        untouched = g == 0
        assert np.array_equal(p_new[untouched], p[untouched])
        moved_by_dense |= bool(np.any(p_dense[untouched] != p[untouched]))
        p = p_new
        opt.zero_grad()
        tp.grad = torch.sparse_coo_tensor(torch.tensor(idx)[None], torch.tensor(g[idx]), (n,))
        opt.step()
        assert np.allclose(p, tp.detach().numpy(), rtol=1e-9, atol=1e-12)
    # after the first step the dense rule moves untouched entries by momentum; lazy does not
    assert moved_by_dense


def test_effective_roughness():
    assert nrc.effective_roughness(0.0, 0.3, 0.0) == 1.0           # diffuse base
    assert nrc.effective_roughness(1.0, 0.2, 0.0) == pytest.approx(0.2)
    assert nrc.effective_roughness(0.0, 0.0, 1.0) == 0.0           # smooth glass
