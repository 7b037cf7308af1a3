"""BVH quality measures on the host (no GPU).

The oracle's reference tree (a binned surface-area-heuristic build, binary, leaves of at most
four triangles) is pinned against closed forms on hand-made geometry and against the cost of
the best tree found by exhaustive search on tiny inputs.  The device tree's checker
(bvh_check) is run on a hand-encoded 8-wide tree whose cost is worked out by hand, and on
copies of it with one planted defect each.
"""
import numpy as np
import pytest

import oracle
from paper_2407_19977_gb300 import bvh_check


def _tri(offset=(0.0, 0.0, 0.0)):
    """The unit right triangle in the z = 0 plane: box [0,1]x[0,1]x[0,0], surface area 2."""
    o = np.asarray(offset, float)
    return np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float) + o


def test_single_triangle_is_one_leaf():
    r = oracle.sah_reference(_tri()[None])
    assert r == {"box_tests": 0.0, "tri_tests": 1.0, "nodes": 1}


def test_coincident_triangles_above_the_leaf_limit_split_in_halves():
    # no centroid spread on any axis: 5 > 4 forces a split by list position, 2 + 3
    r = oracle.sah_reference(np.stack([_tri()] * 5))
    assert r == {"box_tests": 2.0, "tri_tests": 5.0, "nodes": 3}


def test_two_clusters_of_four():
    # root [0,101]x[0,1]x[0,0] has area 2*101 = 202; each cluster's box has area 2
    v = np.stack([_tri()] * 4 + [_tri((100, 0, 0))] * 4)
    r = oracle.sah_reference(v)
    assert r["nodes"] == 3
    assert r["box_tests"] == pytest.approx(2.0, abs=1e-15)
    assert r["tri_tests"] == pytest.approx(2 * 4 * 2 / 202, abs=1e-15)


def test_small_node_splits_when_the_split_is_cheaper_than_a_leaf():
    # four triangles fit one leaf (cost 4), but two pairs 100 apart cost 2 + 8/202 split
    v = np.stack([_tri()] * 2 + [_tri((100, 0, 0))] * 2)
    r = oracle.sah_reference(v)
    assert r["nodes"] == 3
    assert r["tri_tests"] == pytest.approx(2 * 2 * 2 / 202, abs=1e-15)
    # with the same pairs 0.1 apart, the leaf is cheaper: root [0,1.1]x[0,1]: area 2.2
    v = np.stack([_tri()] * 2 + [_tri((0.1, 0, 0))] * 2)
    assert oracle.sah_reference(v) == {"box_tests": 0.0, "tri_tests": 4.0, "nodes": 1}


def _box_area(v):
    d = v.reshape(-1, 3).max(0) - v.reshape(-1, 3).min(0)
    return 2.0 * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0])


def _optimal_cost(v, leaf_max=4):
    """The least (box + triangle tests) over every binary tree on the triangles, by search over
    all bipartitions of every subset (a leaf costs A * n, an internal node 2 A plus its
    children), divided by the root area."""
    n = len(v)
    memo = {}

    def best(mask):
        if mask in memo:
            return memo[mask]
        ids = [i for i in range(n) if mask >> i & 1]
        a = _box_area(v[ids])
        c = a * len(ids) if len(ids) <= leaf_max else np.inf
        low = mask & -mask
        sub = (mask - 1) & mask
        while sub:
            if sub & low:       # each bipartition once: the left part holds the lowest member
                c = min(c, 2 * a + best(sub) + best(mask ^ sub))
            sub = (sub - 1) & mask
        memo[mask] = c
        return c

    return best((1 << n) - 1) / _box_area(v)


def test_clustered_input_reaches_the_exhaustive_optimum():
    rng = np.random.default_rng(3)
    centres = [(0, 0, 0), (40, 0, 0), (0, 40, 0), (40, 40, 30)]
    v = np.stack([_tri(np.asarray(c) + rng.uniform(0, 0.5, 3)) for c in centres for _ in range(2)])
    r = oracle.sah_reference(v)
    assert r["box_tests"] + r["tri_tests"] == pytest.approx(_optimal_cost(v), rel=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_random_input_is_never_below_the_exhaustive_optimum(seed):
    rng = np.random.default_rng(seed)
    n = 7
    v = rng.uniform(0, 10, (n, 1, 3)) + rng.uniform(-1, 1, (n, 3, 3))
    r = oracle.sah_reference(v)
    opt = _optimal_cost(v)
    assert r["box_tests"] + r["tri_tests"] >= opt * (1 - 1e-12)
    # and each triangle is tested at least with the chance of meeting its own box
    own = sum(_box_area(t) for t in v) / _box_area(v)
    assert r["tri_tests"] >= own * (1 - 1e-12)
    assert r["tri_tests"] <= n


# ---- the device tree's checker on a hand-encoded tree ---------------------------------------

def _pack8(vals):
    vals = list(vals) + [0] * (8 - len(vals))
    lo = sum(int(vals[i]) << (8 * i) for i in range(4))
    hi = sum(int(vals[4 + i]) << (8 * i) for i in range(4))
    return lo, hi


def _node(p, slots, child_base, tri_base):
    """slots: (kind, box_lo, box_hi, count, offset) with kind 'i' (internal) or 'l' (leaf);
    scale 1 on every axis (exponent bias 127), boxes in integer units above p."""
    w = np.zeros(20, np.uint32)
    w[0:3] = np.asarray(p, np.float32).view(np.uint32)
    imask = sum(1 << j for j, s in enumerate(slots) if s[0] == "i")
    w[3] = 127 | (127 << 8) | (127 << 16) | (imask << 24)
    w[4], w[5] = child_base, tri_base
    meta = [1 if s[0] == "i" else (s[3] << 5) | s[4] for s in slots]
    w[6], w[7] = _pack8(meta)
    for a in range(3):
        w[8 + 2 * a], w[9 + 2 * a] = _pack8([s[1][a] for s in slots])
        w[14 + 2 * a], w[15 + 2 * a] = _pack8([s[2][a] for s in slots])
    return w


def _cube_pair(lo, size):
    """Two triangles whose joint bounds are the cube [lo, lo + size]^3."""
    l, h = float(lo), float(lo + size)
    a = [[l, l, l, 0], [h, l, l, 0], [l, h, h, 0]]
    b = [[h, h, h, 0], [l, h, l, 0], [h, l, l, 0]]
    return [a, b]


def _hand_tree():
    # root: a leaf over [0,2]^3 and an internal child over [10,20]^3; node 1: leaves over
    # [10,14]^3 and [16,20]^3, two triangles each
    tris = np.asarray(_cube_pair(0, 2) + _cube_pair(10, 4) + _cube_pair(16, 4), np.float32).reshape(6, 12)
    root = _node((0, 0, 0), [("l", (0, 0, 0), (2, 2, 2), 2, 0), ("i", (10, 10, 10), (20, 20, 20), 0, 0)], 1, 0)
    n1 = _node((10, 10, 10), [("l", (0, 0, 0), (4, 4, 4), 2, 0), ("l", (6, 6, 6), (10, 10, 10), 2, 2)], 0, 2)
    return np.stack([root, n1]), tris


def test_checker_accepts_the_hand_tree_and_costs_it():
    nodes, tris = _hand_tree()
    problems, stats = bvh_check.check(nodes, tris)
    assert problems == []
    assert stats["depth"] == 2 and stats["n_nodes"] == 2 and stats["max_leaf_size"] == 2
    c = bvh_check.sah_cost(nodes, tris)
    # areas: root [0,20]^3 2400, node 1 [10,20]^3 600, leaves 24, 96, 96
    assert c["node_visits_exact"] == pytest.approx(3000 / 2400, rel=1e-15)
    assert c["box_tests_exact"] == pytest.approx((2400 * 2 + 600 * 2) / 2400, rel=1e-15)
    assert c["tri_tests_exact"] == pytest.approx((24 * 2 + 96 * 2 + 96 * 2) / 2400, rel=1e-15)
    # the decoded boxes are exact here, so the two measures agree
    for k in ("node_visits", "box_tests", "tri_tests"):
        assert c[k] == pytest.approx(c[k + "_exact"], rel=1e-15)


def test_checker_finds_planted_defects():
    nodes, tris = _hand_tree()
    bad = nodes.copy()     # leaf box one unit short of its triangles
    bad[1] = _node((10, 10, 10), [("l", (0, 0, 0), (3, 4, 4), 2, 0), ("l", (6, 6, 6), (10, 10, 10), 2, 2)], 0, 2)
    assert any("leaf boxes" in p for p in bvh_check.check(bad, tris)[0])
    bad = nodes.copy()     # internal slot too small for its subtree
    bad[0] = _node((0, 0, 0), [("l", (0, 0, 0), (2, 2, 2), 2, 0), ("i", (10, 10, 10), (20, 19, 20), 0, 0)], 1, 0)
    assert any("child boxes" in p for p in bvh_check.check(bad, tris)[0])
    bad = nodes.copy()     # both leaves of node 1 over the same two triangles
    bad[1] = _node((10, 10, 10), [("l", (0, 0, 0), (10, 10, 10), 2, 0), ("l", (0, 0, 0), (10, 10, 10), 2, 0)], 0, 2)
    assert any("in no leaf" in p for p in bvh_check.check(bad, tris)[0])
    bad = np.stack([nodes[0], nodes[1], nodes[1]])   # a third node nobody points to
    assert any("without a parent" in p for p in bvh_check.check(bad, tris)[0])
