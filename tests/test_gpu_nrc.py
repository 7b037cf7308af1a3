"""Radiance cache on the GPU vs the NRC oracle (oracle/nrc.py), through the C-ABI.

Tolerances: forward rel L2 <= 2e-3 with the same FP16-rounded weights, table and inputs;
gradients rel L2 <= 1e-2 (FP16 operands, FP32 accumulation); Adam tight (FP32 vs FP64).
"""
import math

import numpy as np
import pytest

from oracle import nrc as onrc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L, LOG2T = 8, 12

# (levels, log2 entries per level, coarsest resolution, growth per level; 0 = up to 2048):
# a small grid whose levels are mostly dense, and the cache the renderer uses (16 levels of
# 2^19 entries, resolutions 16 ... 2048, hashed from the fifth level on)
GRIDS = {"small": (8, 12, 4, 1.6), "production": (16, 19, 16, 0.0)}


def _make(seed=0, lr=1e-2, batch=4096, tcgen05=False, grid="small", train_kernels=0):
    from paper_2407_19977_gb300 import api
    nl, lt, base, scale = GRIDS[grid]
    return api.Nrc(n_levels=nl, log2_table=lt, base_resolution=base, per_level_scale=scale, learning_rate=lr,
                   batch=batch, seed=seed, tcgen05=tcgen05, train_kernels=train_kernels)


def _records(rng, n, with_target=True):
    rec = np.zeros((n, 16), np.float32)
    rec[:, 0:3] = rng.random((n, 3))
    d = rng.normal(size=(n, 3))
    rec[:, 3:6] = d / np.linalg.norm(d, axis=1, keepdims=True)
    nn = rng.normal(size=(n, 3))
    rec[:, 6:9] = nn / np.linalg.norm(nn, axis=1, keepdims=True)
    rec[:, 9] = rng.random(n)
    if with_target:
        p = rec[:, 0:3].astype(np.float64)
        rec[:, 10] = 0.5 + 0.4 * np.sin(6 * p[:, 0]) * np.cos(4 * p[:, 1])
        rec[:, 11] = 0.3 + 0.2 * p[:, 2]
        rec[:, 12] = 0.2 + 0.1 * np.cos(5 * p[:, 1] + rec[:, 3])
    return rec


def _set_random_params(net, rng):
    w = net.params(0)
    g = net.params(1)
    wn = np.zeros(w.numel(), np.float32)
    nh = 4 * 64 * 64
    wn[:nh] = rng.normal(0, 1 / math.sqrt(64), nh)
    out = np.zeros((16, 64), np.float32)
    out[:3] = rng.normal(0, 0.2, (3, 64))
    wn[nh:] = out.ravel()
    gn = rng.normal(0, 0.3, g.numel()).astype(np.float32)
    w.copy_(torch.from_numpy(wn))
    g.copy_(torch.from_numpy(gn))
    net.commit()
    torch.cuda.synchronize()
    return wn, gn


def _oracle_params(wn, gn, grid="small"):
    """FP16-rounded copies, as the kernels read them."""
    h = lambda a: a.astype(np.float16).astype(np.float64)  # noqa: E731
    nh = 4 * 64 * 64
    nl, lt, _, _ = GRIDS[grid]
    ws = [h(wn[i * 4096:(i + 1) * 4096]).reshape(64, 64) for i in range(4)] + [h(wn[nh:]).reshape(16, 64)[:3]]
    table = h(gn).reshape(nl, 2 ** lt, 2)
    return ws, table


def _resolutions(grid):
    nl, _, base, scale = GRIDS[grid]
    return onrc.level_resolutions(nl, base, scale)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("grid", ["small", "production"])
@pytest.mark.parametrize("tcgen05", [False, True])
def test_nrc_forward_matches_oracle(tcgen05, grid):
    """Inference (fused encoding + MLP) on mma.sync or on tcgen05 with tensor-memory
    accumulators, over ragged sizes around the 16- and 128-row tiles, on a small grid and on
    the production cache (16 levels x 2^19 entries, resolutions 16 ... 2048)."""
    rng = np.random.default_rng(0)
    net = _make(tcgen05=tcgen05, grid=grid)
    wn, gn = _set_random_params(net, rng)
    ws, table = _oracle_params(wn, gn, grid)
    res = _resolutions(grid)
    for n in (5000, 1, 127, 128, 129):
        rec = _records(rng, n, with_target=False)
        y = net.infer(torch.from_numpy(rec).cuda()).cpu().numpy().astype(np.float64)
        # the kernels round the 64-wide input to FP16 as well
        feats, _ = onrc.encode(rec[:, 0:3].astype(np.float64), table, res)
        x = onrc.build_input(feats, rec[:, 3:6], rec[:, 6:9], rec[:, 9]).astype(np.float16).astype(np.float64)
        yo, _ = onrc.mlp_forward(x, ws)
        assert _rel_l2(y, yo) <= 2e-3, (n, _rel_l2(y, yo))
    assert net.last_loss() == 0.0   # no device wait ran out (it would raise PT_ERR_TIMEOUT)


def _reference_forward(rec, ws, table, res):
    """The oracle's forward fed the FP16 values the kernels store (the 64-wide input and each
    layer's activations), and per sample the conditioning of its ReLU decisions: the smallest
    |z| / sum_k |h_k w_k| over the hidden units.  Below 2e-5 (five times the FP32 accumulation
    bound of a 64-term product, which also covers one input whose FP16 rounding the two
    precisions take differently) the kernel's FP32 sum and the oracle's FP64 sum may put the
    pre-activation on different sides of zero, and the sample's whole gradient then takes
    another path through the network."""
    h16 = lambda a: a.astype(np.float16).astype(np.float64)  # noqa: E731
    feats, lookups = onrc.encode(rec[:, 0:3].astype(np.float64), table, res)
    x = h16(onrc.build_input(feats, rec[:, 3:6], rec[:, 6:9], rec[:, 9]))
    acts = [x]
    hcur = x
    margin = np.full(len(rec), np.inf)
    for Wl in ws[:-1]:
        z = hcur @ Wl.T
        mag = np.abs(hcur) @ np.abs(Wl).T
        margin = np.minimum(margin, (np.abs(z) / np.maximum(mag, 1e-300)).min(1))
        hcur = h16(np.maximum(z, 0.0))
        acts.append(hcur)
    return acts, lookups, margin


@pytest.mark.parametrize("grid", ["small", "production"])
@pytest.mark.parametrize("train_kernels", [0, 1])
def test_nrc_gradients_match_oracle(grid, train_kernels):
    """Loss gradients of the weights and of the grid table, from the fused tcgen05 training
    kernel (0) and from the separate mma.sync kernels (1), against the oracle's backward, on
    the samples whose ReLU decisions are well conditioned (the others, at most 2 %, counted:
    a decision FP32 and FP64 may take differently, like a path's reflect/refract choice)."""
    rng = np.random.default_rng(1)
    net = _make(grid=grid, train_kernels=train_kernels)
    wn, gn = _set_random_params(net, rng)
    rec_all = _records(rng, 3000)
    nl, lt, _, _ = GRIDS[grid]
    ws, table = _oracle_params(wn, gn, grid)
    res = _resolutions(grid)
    _, _, margin = _reference_forward(rec_all, ws, table, res)
    ill = margin < 2e-5
    assert ill.mean() <= 2e-2, ill.mean()
    rec = np.ascontiguousarray(rec_all[~ill])
    print(f"{grid}: {int(ill.sum())} of {len(rec_all)} samples with an ill-conditioned ReLU decision left out")
    dw, dg = net.gradients(torch.from_numpy(rec).cuda())
    dw = dw.cpu().numpy().astype(np.float64)
    dg = dg.cpu().numpy().astype(np.float64).reshape(nl, 2 ** lt, 2)
    h16 = lambda a: a.astype(np.float16).astype(np.float64)  # noqa: E731
    acts, lookups, _ = _reference_forward(rec, ws, table, res)
    y = acts[-1] @ ws[-1].T
    loss, dy = onrc.relative_l2(y, rec[:, 10:13].astype(np.float64))
    # the kernels hold each layer's output gradient as an FP16 tensor-core operand, in units of
    # the loss sum (times 3n; the 1/(3n) of the mean is applied in FP32 at the end)
    n_el = float(dy.size)
    gw, dx = onrc.mlp_backward(acts, ws, dy, operand=lambda g: h16(g * n_el) / n_el)
    dtable = onrc.grid_backward(lookups, dx[:, :2 * nl], table.shape)
    for i in range(4):
        assert _rel_l2(dw[i * 4096:(i + 1) * 4096].reshape(64, 64), gw[i]) <= 2e-3, i
    out = dw[4 * 4096:].reshape(16, 64)
    assert _rel_l2(out[:3], gw[4]) <= 2e-3
    assert np.all(out[3:] == 0)
    assert _rel_l2(dg, dtable) <= 2e-3
    # against the exact backward (FP16 forward activations only): the FP16 output gradients
    # cost about 1e-3 per layer, amplified by the cancellation in each 64-term product
    gw_x, dx_x = onrc.mlp_backward(acts, ws, dy)
    dtable_x = onrc.grid_backward(lookups, dx_x[:, :2 * nl], table.shape)
    for i in range(4):
        assert _rel_l2(dw[i * 4096:(i + 1) * 4096].reshape(64, 64), gw_x[i]) <= 1e-2, i
    assert _rel_l2(dg, dtable_x) <= 1e-2


@pytest.mark.parametrize("train_kernels", [0, 1])
def test_nrc_adam_step(train_kernels):
    rng = np.random.default_rng(2)
    net = _make(lr=5e-3, train_kernels=train_kernels)
    wn, gn = _set_random_params(net, rng)
    rec = _records(rng, 2048)
    t = torch.from_numpy(rec).cuda()
    dw, dg = net.gradients(t)
    net.train(t)   # one Adam step on the same batch
    w_new = net.params(0).cpu().numpy().astype(np.float64)
    g_new = net.params(1).cpu().numpy().astype(np.float64)
    dw = dw.cpu().numpy().astype(np.float64)
    dg = dg.cpu().numpy().astype(np.float64)
    for p0, g, p1 in ((wn, dw, w_new), (gn, dg, g_new)):
        exp, _, _ = onrc.adam(p0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 5e-3)
        # grid gradients are FP32 atomic sums: entries that cancel to ~0 may change sign
        # between the two evaluations, so compare where the gradient is clearly non-zero
        sel = np.abs(g) > 1e-4 * np.abs(g).max()
        assert sel.mean() > 0.01
        assert np.allclose(p1[sel], exp[sel], rtol=1e-5, atol=1e-7)
        assert np.allclose(p1[g == 0], p0[g == 0])
    # second step on samples from another part of the box: grid entries with a zero gradient
    # keep their value although their moments are non-zero (lazy Adam), the touched ones move
    rec2 = _records(rng, 512)
    rec2[:, 0] = 0.5 * rec2[:, 0] + 0.5
    t2 = torch.from_numpy(rec2).cuda()
    _, dg2 = net.gradients(t2)
    dg2 = dg2.cpu().numpy()
    net.train(t2)
    g_2 = net.params(1).cpu().numpy().astype(np.float64)
    moved1 = (g_new != gn) & (dg2 == 0)
    assert moved1.sum() > 100
    assert np.array_equal(g_2[dg2 == 0], g_new[dg2 == 0])
    assert np.mean(g_2[dg2 != 0] != g_new[dg2 != 0]) > 0.99


def test_nrc_training_reduces_loss():
    rng = np.random.default_rng(3)
    net = _make(lr=1e-2, batch=4096)
    rec = torch.from_numpy(_records(rng, 4096)).cuda()
    net.train(rec)
    first = net.last_loss()
    for _ in range(200):
        net.train(torch.from_numpy(_records(rng, 4096)).cuda())
    last = net.last_loss()
    assert last < 0.2 * first, (first, last)
    # the trained cache predicts held-out points of the smooth target
    test = _records(rng, 2000)
    y = net.infer(torch.from_numpy(test).cuda()).cpu().numpy()
    assert np.mean(np.abs(y - test[:, 10:13])) < 0.05


def test_nrc_render_queries_and_trains():
    from paper_2407_19977_gb300 import api, scenes
    sc = scenes.pushbutton(width=320, height=180)
    g = api.Scene(sc)
    lo = sc.vertices.min(0) - 0.01
    hi = sc.vertices.max(0) + 0.01
    net = api.Nrc(seed=1, box=(tuple(lo), tuple(hi)))
    losses = []
    for f in range(12):
        acc = g.render(1, seed=f, mode=1, nrc=net, nrc_train=True)
        losses.append(net.last_loss())
    img = acc.image().cpu().numpy()
    st = g.stats()
    assert np.all(np.isfinite(img)) and img.mean() > 0
    # most pushbutton paths leave for the sky after one diffuse bounce: only a few reach a
    # second diffuse-ish vertex, where the cache answers
    assert st["nrc_queries"] > 0.005 * 320 * 180 * 12
    assert st["error_flags"] == 0
    assert np.mean(losses[-3:]) < np.mean(losses[:3])


def test_nrc_render_with_fuzz_materials():
    """The cached tracer on a scene with velvet boxes: queries and training run, the image is
    finite and its mean within 25 % of the plain tracer's (the cache is biased, not wrong by a
    factor)."""
    from paper_2407_19977_gb300 import api, scenes
    base = scenes.cornell_box(width=128, height=96, spp=1, max_depth=6)
    velvet = scenes.openpbr(base_color=(0.4, 0.4, 0.5), specular_roughness=0.5, fuzz_weight=1.0,
                            fuzz_color=(1.0, 0.8, 0.8), fuzz_roughness=0.4)
    mats = np.concatenate([np.asarray(base.materials, np.float32), velvet[None]])
    mid = np.asarray(base.material_ids, np.uint32).copy()
    mid[10:] = len(mats) - 1                # the boxes
    sc = scenes.Scene(base.name, base.vertices, base.indices, mid, mats, base.lights, base.env,
                      base.camera, base.spp, base.max_depth)
    g = api.Scene(sc)
    lo = sc.vertices.min(0) - 0.01
    hi = sc.vertices.max(0) + 0.01
    net = api.Nrc(seed=2, box=(tuple(lo), tuple(hi)))
    for f in range(24):
        acc = g.render(1, seed=f, mode=1, nrc=net, nrc_train=True)
    cached = g.render(16, seed=77, mode=1, nrc=net).image().cpu().numpy()
    plain = g.render(64, seed=78, mode=1).image().cpu().numpy()
    st = g.stats()
    assert st["error_flags"] == 0 and st["nrc_queries"] > 0
    assert np.all(np.isfinite(cached))
    assert abs(cached.mean() / plain.mean() - 1.0) < 0.25, (cached.mean(), plain.mean())


def test_nrc_frame_same_with_and_without_tail_kernel():
    """With the radiance cache on, the tail kernel ends paths at the same vertices, issues the
    same cache queries (in another order) and records the same training vertices: a frame
    rendered from two identical caches is bit-identical with and without it.  256x192 holds
    more paths than the training slots, so both kinds of path occur."""
    from paper_2407_19977_gb300 import api, scenes
    sc = scenes.cornell_box(width=256, height=192, spp=1, max_depth=8)
    g = api.Scene(sc)
    lo = sc.vertices.min(0) - 0.01
    hi = sc.vertices.max(0) + 0.01
    for train in (False, True):
        imgs, queries = [], []
        for tail in (-1, 1 << 30):
            net = api.Nrc(seed=3, box=(tuple(lo), tuple(hi)))
            b = g.stats()["nrc_queries"]
            acc = g.render(1, seed=4, mode=1, nrc=net, nrc_train=train, tail_paths=tail)
            torch.cuda.synchronize()
            queries.append(g.stats()["nrc_queries"] - b)
            imgs.append(acc.sum.clone())
        assert queries[0] == queries[1] > 0, (train, queries)
        assert torch.equal(imgs[0], imgs[1]), train


def test_nrc_graph_replay_equals_direct_launches():
    """Cached frames replayed from a captured graph against direct launches, from identical
    caches.  Without training the cache is fixed and every frame is bit-identical.  With
    training the first frame (its image is formed before the frame's training) is
    bit-identical; later frames follow caches trained with float atomics summing in no fixed
    order (Adam's first steps move a parameter by about the learning rate whatever its
    gradient's size), which differ between any two runs, so they are held to a valid
    estimate whose mean agrees within 5 %."""
    from paper_2407_19977_gb300 import api, scenes
    sc = scenes.cornell_box(width=256, height=192, spp=1, max_depth=8)
    g = api.Scene(sc)
    lo = sc.vertices.min(0) - 0.01
    hi = sc.vertices.max(0) + 0.01
    for train in (False, True):
        runs = []
        for use_graph in (False, True):
            net = api.Nrc(seed=3, box=(tuple(lo), tuple(hi)))
            acc = api.Accum(256, 192)
            out = []
            r0 = g.stats()["graph_replays"]
            for f in range(4):
                g.render(1, seed=4, accum=acc, mode=1, nrc=net, nrc_train=train, use_graph=use_graph)
                torch.cuda.synchronize()
                out.append(acc.sum.clone())
            runs.append(out)
            if use_graph:
                assert g.stats()["graph_replays"] - r0 >= 3
        direct, graph = runs
        assert torch.equal(direct[0], graph[0]), train
        for f in range(1, 4):
            if not train:
                assert torch.equal(direct[f], graph[f]), f
            else:
                assert torch.isfinite(graph[f]).all()
                assert abs(float(graph[f].mean()) / float(direct[f].mean()) - 1.0) < 0.05, f


def test_nrc_render_with_tcgen05_inference():
    """A rendered frame whose cache queries run on tcgen05 agrees with the mma.sync frame
    (same cache, same queries; the MLP sums in another order, so not bit for bit)."""
    from paper_2407_19977_gb300 import api, scenes
    sc = scenes.cornell_box(width=256, height=192, spp=1, max_depth=8)
    g = api.Scene(sc)
    lo = sc.vertices.min(0) - 0.01
    hi = sc.vertices.max(0) + 0.01
    imgs = []
    for tc in (False, True):
        net = api.Nrc(seed=3, box=(tuple(lo), tuple(hi)), tcgen05=tc)
        acc = g.render(4, seed=4, mode=1, nrc=net, nrc_train=False)
        torch.cuda.synchronize()
        imgs.append(acc.image().cpu().numpy().astype(np.float64))
        assert net.last_loss() == 0.0
    assert np.all(np.isfinite(imgs[1]))
    assert np.abs(imgs[1] - imgs[0]).max() <= 1e-3 * max(imgs[0].max(), 1e-6) + 1e-5


def test_nrc_gain_on_enclosed_scene():
    """What the trained cache gains: in a closed box most radiance arrives after several
    diffuse bounces; ending paths at their second diffuse vertex with the cache lowers the
    error at equal samples against a high-sample plain reference."""
    from paper_2407_19977_gb300 import api, scenes
    sc = scenes.cornell_box(width=128, height=128, spp=1, max_depth=8)
    g = api.Scene(sc)
    ref = api.Accum(128, 128)
    g.render(2048, seed=99, accum=ref, mode=1)
    ref_img = ref.image()
    net = api.Nrc(seed=2, box=((-0.01, -0.01, -0.01), (1.01, 1.01, 1.01)))
    for f in range(64):
        g.render(1, seed=1000 + f, mode=1, nrc=net, nrc_train=True)

    def relmse(img):
        d = img - ref_img
        return float((d * d / (ref_img * ref_img + 1e-2)).mean())

    plain = g.render(4, seed=5, mode=1)
    cached = g.render(4, seed=5, mode=1, nrc=net)
    e_plain, e_nrc = relmse(plain.image()), relmse(cached.image())
    assert e_nrc < 0.8 * e_plain, (e_nrc, e_plain)
