"""Host-side reader, structural check and quality measure of the exported 8-wide BVH.

The structure checks of Sec. 5.1.1 on the tree pt_bvh_export copies out:
decode_nodes() unpacks the 80-byte nodes (reference point, per-axis power-of-two scales,
8-bit child boxes); check() verifies that every node but the root has exactly one parent,
that every triangle sits in exactly one leaf, and that every decoded child box contains the
exact bounds of what lies below it; sah_cost() gives the surface-area measure of the tree's
quality: the box and triangle tests of a ray through the root box when every box it meets is
entered, with the chance of meeting a box taken as its area over the root's.

Everything is vectorised over nodes (one pass per tree level), so the 5.2-million-triangle
scene checks in seconds.
"""
from __future__ import annotations

import numpy as np


def _bytes8(lo, hi):
    b = np.empty((lo.shape[0], 8), dtype=np.uint32)
    for i in range(4):
        b[:, i] = (lo >> (8 * i)) & 0xFF
        b[:, 4 + i] = (hi >> (8 * i)) & 0xFF
    return b


def decode_nodes(nodes: np.ndarray):
    """nodes (n, 20) uint32 -> dict of per-node fields; lo/hi (n, 8, 3) float32 are the
    decoded child boxes p + q * scale (exact in float32: q < 256 times a power of two)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.uint32)
    p = nodes[:, 0:3].copy().view(np.float32)
    w = nodes[:, 3]
    e = np.stack([w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFF], 1).astype(np.uint32)
    scale = (e << 23).view(np.float32)
    imask = (w >> 24) & 0xFF
    meta = _bytes8(nodes[:, 6], nodes[:, 7])
    qlo = np.stack([_bytes8(nodes[:, 8], nodes[:, 9]), _bytes8(nodes[:, 10], nodes[:, 11]),
                    _bytes8(nodes[:, 12], nodes[:, 13])], -1)
    qhi = np.stack([_bytes8(nodes[:, 14], nodes[:, 15]), _bytes8(nodes[:, 16], nodes[:, 17]),
                    _bytes8(nodes[:, 18], nodes[:, 19])], -1)
    lo = p[:, None, :] + qlo.astype(np.float32) * scale[:, None, :]
    hi = p[:, None, :] + qhi.astype(np.float32) * scale[:, None, :]
    return dict(p=p, scale=scale, imask=imask, child_base=nodes[:, 4], tri_base=nodes[:, 5],
                meta=meta, lo=lo, hi=hi)


def _slots(D):
    """Flat lists of the used slots: internal (node, slot, child) and leaf (node, slot, first, count)."""
    n = D["meta"].shape[0]
    used = D["meta"] > 0
    internal = ((D["imask"][:, None] >> np.arange(8, dtype=np.uint32)[None, :]) & 1).astype(bool) & used
    rank = np.cumsum(internal, 1) - 1          # rank of an internal slot among the node's internal slots
    ni, si = np.nonzero(internal)
    child = D["child_base"][ni].astype(np.int64) + rank[ni, si]
    li, ls = np.nonzero(used & ~internal)
    m = D["meta"][li, ls]
    first = D["tri_base"][li].astype(np.int64) + (m & 31)
    count = (m >> 5).astype(np.int64)
    return dict(n=n, ni=ni, si=si, child=child, li=li, ls=ls, first=first, count=count)


def _area(lo, hi):
    d = np.maximum(hi - lo, 0.0)
    return 2.0 * (d[..., 0] * d[..., 1] + d[..., 1] * d[..., 2] + d[..., 2] * d[..., 0])


def _levels(S):
    """Node indices by depth from the root (node 0); child indices must be in range."""
    n = S["n"]
    order = np.argsort(S["ni"], kind="stable")
    ni, child = S["ni"][order], S["child"][order]
    start = np.searchsorted(ni, np.arange(n + 1))
    levels = [np.array([0], dtype=np.int64)]
    seen = 1
    while True:
        cur = levels[-1]
        cnt = start[cur + 1] - start[cur]
        if cnt.sum() == 0:
            break
        idx = np.repeat(start[cur], cnt) + (np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt))
        levels.append(child[idx])
        seen += len(idx)
        if seen > n or len(levels) > 4096:
            break
    return levels


def content_boxes(D, S, tris):
    """Exact bounds (float64) of the triangles below every node, bottom up, and of every slot."""
    n = S["n"]
    v = tris.reshape(-1, 3, 4)[:, :, :3].astype(np.float64)
    tlo, thi = v.min(1), v.max(1)
    # leaf slots: bounds of their triangle runs (counts are 1..7)
    rep = np.repeat(np.arange(len(S["first"])), S["count"])
    tidx = np.repeat(S["first"], S["count"]) + (np.arange(rep.size) - np.repeat(np.cumsum(S["count"]) - S["count"],
                                                                               S["count"]))
    leaf_lo = np.full((len(S["first"]), 3), np.inf)
    leaf_hi = np.full((len(S["first"]), 3), -np.inf)
    np.minimum.at(leaf_lo, rep, tlo[tidx])
    np.maximum.at(leaf_hi, rep, thi[tidx])
    node_lo = np.full((n, 3), np.inf)
    node_hi = np.full((n, 3), -np.inf)
    np.minimum.at(node_lo, S["li"], leaf_lo)
    np.maximum.at(node_hi, S["li"], leaf_hi)
    levels = _levels(S)
    parent = np.full(n, -1, dtype=np.int64)
    parent[S["child"]] = S["ni"]
    for lv in reversed(levels[1:]):
        np.minimum.at(node_lo, parent[lv], node_lo[lv])
        np.maximum.at(node_hi, parent[lv], node_hi[lv])
    return dict(leaf_lo=leaf_lo, leaf_hi=leaf_hi, node_lo=node_lo, node_hi=node_hi, levels=levels, tidx=tidx)


def check(nodes: np.ndarray, tris: np.ndarray):
    """Structural problems (list of strings, empty when the tree is sound) and statistics."""
    D = decode_nodes(nodes)
    S = _slots(D)
    n, n_tris = S["n"], tris.shape[0]
    problems = []
    if np.any(S["child"] >= n) or np.any(S["child"] <= 0):
        problems.append("child index out of range")
        return problems, {}
    if np.any(S["first"] + S["count"] > n_tris):
        problems.append("leaf triangle run out of range")
        return problems, {}
    parents = np.bincount(S["child"], minlength=n)
    if parents[0] != 0:
        problems.append("the root has a parent")
    if np.any(parents[1:] != 1):
        problems.append(f"{int((parents[1:] == 0).sum())} nodes without a parent, "
                        f"{int((parents[1:] > 1).sum())} with several")
    B = content_boxes(D, S, tris)
    seen = np.bincount(B["tidx"], minlength=n_tris)
    if np.any(seen != 1):
        problems.append(f"{int((seen == 0).sum())} triangles in no leaf, {int((seen > 1).sum())} in several")
    if sum(len(lv) for lv in B["levels"]) != n:
        problems.append("nodes unreachable from the root")
    # decoded boxes hold their contents exactly (the build rounds the 8-bit planes outward)
    llo = D["lo"][S["li"], S["ls"]].astype(np.float64)
    lhi = D["hi"][S["li"], S["ls"]].astype(np.float64)
    bad = np.any(llo > B["leaf_lo"], 1) | np.any(lhi < B["leaf_hi"], 1)
    if bad.any():
        problems.append(f"{int(bad.sum())} leaf boxes do not contain their triangles")
    ilo = D["lo"][S["ni"], S["si"]].astype(np.float64)
    ihi = D["hi"][S["ni"], S["si"]].astype(np.float64)
    bad = np.any(ilo > B["node_lo"][S["child"]], 1) | np.any(ihi < B["node_hi"][S["child"]], 1)
    if bad.any():
        problems.append(f"{int(bad.sum())} child boxes do not contain their subtrees")
    children = np.bincount(S["ni"], minlength=n) + np.bincount(S["li"], minlength=n)
    stats = dict(n_nodes=int(n), n_tris=int(n_tris), depth=len(B["levels"]),
                 mean_children=float(children.mean()), max_children=int(children.max()),
                 mean_leaf_size=float(S["count"].mean()),
                 max_leaf_size=int(S["count"].max()))
    return problems, stats


def sah_cost(nodes: np.ndarray, tris: np.ndarray):
    """Surface-area measures of the tree, with the probability of entering a box taken as
    its area over the root box's:
      node_visits  expected wide nodes entered (each entry tests all its child boxes),
      box_tests    expected child-box tests (node entries times the node's children),
      tri_tests    expected triangle tests (leaf areas times their triangle counts);
    '_exact' uses the exact bounds of each subtree, the plain keys the decoded 8-bit boxes
    the traversal actually tests."""
    D = decode_nodes(nodes)
    S = _slots(D)
    B = content_boxes(D, S, tris)
    n = S["n"]
    children = np.bincount(S["ni"], minlength=n) + np.bincount(S["li"], minlength=n)
    a_root = _area(B["node_lo"][0], B["node_hi"][0])
    out = {}
    # exact bounds
    a_node = _area(B["node_lo"], B["node_hi"]) / a_root
    a_leaf = _area(B["leaf_lo"], B["leaf_hi"]) / a_root
    out["node_visits_exact"] = float(a_node.sum())
    out["box_tests_exact"] = float((a_node * children).sum())
    out["tri_tests_exact"] = float((a_leaf * S["count"]).sum())
    # decoded boxes: a child node is entered through its parent's slot box
    a_slot_int = _area(D["lo"][S["ni"], S["si"]].astype(np.float64), D["hi"][S["ni"], S["si"]].astype(np.float64))
    a_slot_leaf = _area(D["lo"][S["li"], S["ls"]].astype(np.float64), D["hi"][S["li"], S["ls"]].astype(np.float64))
    a_enter = np.empty(n)
    a_enter[0] = 1.0
    a_enter[S["child"]] = a_slot_int / a_root
    out["node_visits"] = float(a_enter.sum())
    out["box_tests"] = float((a_enter * children).sum())
    out["tri_tests"] = float((a_slot_leaf / a_root * S["count"]).sum())
    return out
