"""The level-synchronous tree builder, run on the host (FMM_TREE_LEVELS_HOST):
the same element steps and the same step sequence as the device builder, with
host sorts and prefix sums in place of the device ones.

* Against the oracle's octree and lists (bit-exact index work), balanced and
  not, on the three point distributions.
* Against the recursive host builder: every exported array and count equal,
  on the edge cases (one point, coincident points down to max_level,
  max_level 0 and 4, distinct targets, batches).
"""
import ctypes

import numpy as np
import pytest

from oracle import kifmm as ok
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl

from .test_abi_host import CASES, _csr, _plan_keys

ARRAYS = ("node_keys", "node_range", "leaf_flag", "perm", "u_ptr", "u_idx", "v_ptr", "v_idx",
          "w_ptr", "w_idx", "x_ptr", "x_idx", "root", "charge_row", "output_row", "node_problem")
COUNTS = ("n", "points", "nodes", "leaves", "depth", "u_pairs", "v_pairs", "w_pairs", "x_pairs",
          "p2p_pairs", "m2l_tiles", "m2l_entries")
GEN = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface, "gauss": wl.gaussian_mixture}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


def same_plan(A, B):
    for k in COUNTS:
        assert A.info(k) == B.info(k), k
    for nm in ARRAYS:
        a, b = A.array(nm), B.array(nm)
        assert a.dtype == b.dtype and a.shape == b.shape, nm
        np.testing.assert_array_equal(a, b, err_msg=nm)


@pytest.mark.parametrize("kind,n,ncrit,balance", CASES)
def test_level_builder_matches_oracle(kind, n, ncrit, balance):
    x, _ = GEN[kind](n, 31)
    P = FMMPlan(x, 4, ncrit, host_only=1, balance=int(balance), tree_build=N.TREE_LEVELS_HOST)
    tree = ok.Octree(x, ncrit, balance=balance)
    U, V, W, X = ok.build_lists(tree)
    keys = _plan_keys(P)
    assert set(keys) == tree.nonempty and len(keys) == len(set(keys))
    leaf = P.array("leaf_flag")
    assert {k for k, f in zip(keys, leaf) if f} == set(tree.leaves)
    rng = P.array("node_range").reshape(-1, 2)
    perm = P.array("perm")
    for k, (a, b) in zip(keys, rng):
        assert np.array_equal(np.sort(perm[a:b]), np.sort(tree.points[k]))
    for name, ref in (("u", U), ("v", V), ("w", W), ("x", X)):
        assert _csr(P, name, keys) == {k: sorted(v) for k, v in ref.items()}, name


EDGE = [
    ("cube", 4000, 24, 1, 16), ("sphere", 3000, 8, 0, 16), ("gauss", 20000, 16, 1, 16),
    ("gauss", 20000, 16, 0, 16), ("sphere", 30000, 32, 1, 16), ("cube", 1, 4, 1, 16),
    ("cube", 7, 4, 1, 16), ("gauss", 5000, 8, 1, 4), ("gauss", 5000, 8, 1, 0),
]


@pytest.mark.parametrize("kind,n,ncrit,balance,max_level", EDGE)
def test_level_builder_equals_recursive_builder(kind, n, ncrit, balance, max_level):
    x, _ = GEN[kind](n, 17)
    kw = dict(host_only=1, balance=balance, max_level=max_level)
    same_plan(FMMPlan(x, 4, ncrit, tree_build=N.TREE_HOST, **kw),
              FMMPlan(x, 4, ncrit, tree_build=N.TREE_LEVELS_HOST, **kw))


def test_coincident_points_and_distinct_targets():
    x = np.zeros((50, 3))
    x[25:] = 0.5  # two stacks of coincident points: both split to max_level
    A = FMMPlan(x, 4, 4, host_only=1, tree_build=N.TREE_HOST)
    B = FMMPlan(x, 4, 4, host_only=1, tree_build=N.TREE_LEVELS_HOST)
    assert B.info("depth") == 16
    same_plan(A, B)
    s, _ = wl.uniform_cube(3000, 5)
    t, _ = wl.gaussian_mixture(3000, 6)
    same_plan(FMMPlan(s, 4, 16, targets=t, host_only=1, tree_build=N.TREE_HOST),
              FMMPlan(s, 4, 16, targets=t, host_only=1, tree_build=N.TREE_LEVELS_HOST))


def test_batch_with_level_builder():
    sets = [GEN[k](n, 50 + i)[0] for i, (k, n) in
            enumerate([("cube", 900), ("sphere", 40), ("gauss", 2600), ("cube", 1)])]
    same_plan(FMMPlan.batch(sets, 4, 20, host_only=1, tree_build=N.TREE_HOST),
              FMMPlan.batch(sets, 4, 20, host_only=1, tree_build=N.TREE_LEVELS_HOST))


def test_tree_build_option_is_checked():
    x, _ = wl.uniform_cube(100, 3)
    L = N.lib()
    opts = N.Options()
    L.fmm_options_init(ctypes.byref(opts))
    assert opts.tree_build == N.TREE_AUTO
    pts = np.ascontiguousarray(x)
    h = ctypes.c_void_p()
    for tb, host_only in ((7, 1), (-1, 1), (N.TREE_DEVICE, 1)):
        opts.tree_build, opts.host_only = tb, host_only
        st = L.fmm_plan_create_ex(pts.ctypes.data, None, len(x), 4, 8, ctypes.byref(opts),
                                  ctypes.byref(h))
        assert st == N.FMM_ERR_INVALID_ARG and not h.value, tb
    # a host-only plan never builds on the device, whatever its size
    P = FMMPlan(wl.uniform_cube(70000, 4)[0], 4, 64, host_only=1)
    assert P.info("device_trees") == 0
