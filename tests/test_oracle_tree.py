"""Pins for the oracle's octree and interaction lists.

The strongest pin is coverage: for every (target leaf, source leaf) pair the
lists must account for the interaction exactly once, either directly (U), or
through exactly one (target ancestor, source ancestor) pair of the far-field
lists (V, X, W).  A wrong list definition double-counts or drops pairs.
"""
from collections import Counter

import numpy as np
import pytest

from oracle.kifmm import Octree, build_lists, surface_grid, _adjacent, _parent
from paper_2303_08394_gb300 import workloads as wl


def _ancestors_or_self(key):
    out = [key]
    while key[0] > 0:
        key = _parent(key)
        out.append(key)
    return out


def _leaves_below(tree, key, memo):
    if key in memo:
        return memo[key]
    if tree.leaf[key]:
        res = [key]
    else:
        res = []
        l, i, j, k = key
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    ch = (l + 1, 2 * i + cx, 2 * j + cy, 2 * k + cz)
                    if ch in tree.nonempty:
                        res.extend(_leaves_below(tree, ch, memo))
    memo[key] = res
    return res


def _coverage(tree, lists):
    U, V, W, X = lists
    memo = {}
    bad = 0
    for b in tree.leaves:
        cnt = Counter(U[b])
        for bp in _ancestors_or_self(b):
            for a in V.get(bp, ()):
                cnt.update(_leaves_below(tree, a, memo))
            cnt.update(X.get(bp, ()))
        for a in W.get(b, ()):
            cnt.update(_leaves_below(tree, a, memo))
        for a in tree.leaves:
            if cnt[a] != 1:
                bad += 1
        assert set(cnt) <= set(tree.leaves)
    return bad


CASES = [
    ("cube", 3000, 20),
    ("sphere", 3000, 8),
    ("gauss", 3000, 8),
]


@pytest.mark.parametrize("kind,n,ncrit", CASES)
@pytest.mark.parametrize("balance", [True, False])
def test_lists_cover_every_pair_once(kind, n, ncrit, balance):
    gen = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface,
           "gauss": wl.gaussian_mixture}[kind]
    x, _ = gen(n, 11)
    tree = Octree(x, ncrit, balance=balance)
    lists = build_lists(tree)
    assert _coverage(tree, lists) == 0


@pytest.mark.parametrize("kind,n,ncrit", CASES)
def test_balance_and_list_bounds(kind, n, ncrit, golden):
    bounds = {k: int(v) for k, v in golden("list_bounds.txt")}
    gen = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface,
           "gauss": wl.gaussian_mixture}[kind]
    x, _ = gen(n, 12)
    tree = Octree(x, ncrit, balance=True)
    # 2:1 balance over all leaves, empty ones included
    all_leaves = [k for k, v in tree.leaf.items() if v]
    by_level = {}
    for k in all_leaves:
        by_level.setdefault(k[0], []).append(k)
    for a in all_leaves:
        for lvl, ks in by_level.items():
            if abs(lvl - a[0]) > 1:
                assert not any(_adjacent(a, b) for b in ks), (a, lvl)
    U, V, W, X = build_lists(tree)
    for name, lst in (("U", U), ("V", V), ("W", W), ("X", X)):
        assert max((len(v) for v in lst.values()), default=0) <= bounds[name], name


def test_list_symmetries():
    x, _ = wl.sphere_surface(2500, 13)
    tree = Octree(x, 8)
    U, V, W, X = build_lists(tree)
    for b, lst in U.items():
        assert b in lst
        for a in lst:
            assert b in U[a]
    for b, lst in V.items():
        for a in lst:
            assert a[0] == b[0] and b in V[a] and not _adjacent(a, b)
    for b, lst in W.items():
        for a in lst:
            assert b in X[a] and a[0] > b[0]
            assert not _adjacent(a, b) and _adjacent(_parent(a), b)


def test_uniform_tree_shape():
    """10^4 uniform points with ncrit = 64 give the complete depth-3 tree
    (512 leaves); its V lists hold 56,448 pairs in total."""
    x, _ = wl.uniform_cube(10_000, 0)
    tree = Octree(x, 64)
    assert tree.depth == 3 and len(tree.leaves) == 512
    U, V, W, X = build_lists(tree)
    assert not W and not X
    # interior box at level 3 in an 8^3 grid: full 189-box V list
    assert len(V[(3, 3, 4, 3)]) == 189
    # count by geometry: all same-level pairs whose parents touch, minus
    # touching pairs, at levels 2 (4^3 grid) and 3 (8^3 grid)
    def v_pairs(m):
        c = np.arange(m)
        pc = c // 2
        par = (np.abs(pc[:, None] - pc[None, :]) <= 1).astype(np.int64)
        adj = (np.abs(c[:, None] - c[None, :]) <= 1).astype(np.int64)
        per_dim_par = par.sum()
        per_dim_adj = adj.sum()
        return per_dim_par ** 3 - per_dim_adj ** 3
    assert sum(len(v) for v in V.values()) == v_pairs(4) + v_pairs(8) == 56_448


def test_points_partitioned_and_under_ncrit():
    x, _ = wl.gaussian_mixture(4000, 14)
    tree = Octree(x, 16)
    seen = np.concatenate([tree.points[b] for b in tree.leaves])
    assert np.array_equal(np.sort(seen), np.arange(len(x)))
    for b in tree.leaves:
        assert len(tree.points[b]) <= 16
        lo = tree.box_centre(b) - tree.box_half_width(b[0])
        hi = tree.box_centre(b) + tree.box_half_width(b[0])
        pts = x[tree.points[b]]
        assert np.all(pts >= lo - 1e-12) and np.all(pts <= hi + 1e-12)


def test_surface_counts(golden):
    for p, n in golden("surface_counts.txt"):
        s = surface_grid(int(p))
        assert len(s) == int(n)
        assert np.allclose(np.abs(s).max(axis=1), 1.0)
        assert len(np.unique(s, axis=0)) == int(n)
