"""Parity of the device tree builder (FMM_TREE_DEVICE): level-synchronous
kernels with radix sorts and prefix sums on the GPU.

* Against the oracle's octree and lists (bit-exact index work).
* Against the recursive host builder: every exported array and count equal,
  including host and device input pointers, distinct targets, unbalanced
  trees, coincident points and batches; and the point data the arrays do not
  show (leaf-relative positions and their residuals) through evaluations
  that agree bit for bit.
* At the full size of the benchmark workload (10^6 uniform points, ncrit 150)
  and of the 4*10^6-point sphere: FMM_TREE_AUTO builds on the device and
  gives the host builder's plan.
"""
import numpy as np
import pytest

from oracle import kifmm as ok
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl

from .test_abi_host import CASES, _csr, _plan_keys
from .test_tree_levels import GEN, same_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def evaluate(plan, q):
    qd = torch.as_tensor(np.asarray(q, dtype=np.float32).reshape(len(q), -1), device="cuda")
    out = plan.evaluate(qd)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind,n,ncrit,balance", CASES)
def test_device_builder_matches_oracle(kind, n, ncrit, balance):
    x, _ = GEN[kind](n, 31)
    P = FMMPlan(x, 4, ncrit, balance=int(balance), tree_build=N.TREE_DEVICE)
    assert P.info("device_trees") == 1
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
    ("cube", 20000, 40, 1, 16), ("sphere", 30000, 16, 0, 16), ("gauss", 40000, 16, 1, 16),
    ("cube", 1, 4, 1, 16), ("cube", 7, 4, 1, 16), ("gauss", 5000, 8, 1, 4),
    ("gauss", 5000, 8, 1, 0),
]


@pytest.mark.parametrize("kind,n,ncrit,balance,max_level", EDGE)
def test_device_builder_equals_host_builder(kind, n, ncrit, balance, max_level):
    x, q = GEN[kind](n, 17)
    kw = dict(balance=balance, max_level=max_level)
    A = FMMPlan(x, 5, ncrit, tree_build=N.TREE_HOST, **kw)
    B = FMMPlan(x, 5, ncrit, tree_build=N.TREE_DEVICE, **kw)
    same_plan(A, B)
    # leaf-relative positions and residuals: identical evaluations
    np.testing.assert_array_equal(evaluate(A, q), evaluate(B, q))


def test_device_pointers_coincident_points_and_targets():
    x = np.zeros((50, 3))
    x[25:] = 0.5
    xd = torch.as_tensor(x, device="cuda")
    same_plan(FMMPlan(x, 4, 4, tree_build=N.TREE_HOST), FMMPlan(xd, 4, 4, tree_build=N.TREE_DEVICE))
    s, q = wl.uniform_cube(6000, 5)
    t, _ = wl.gaussian_mixture(6000, 6)
    A = FMMPlan(s, 5, 24, targets=t, tree_build=N.TREE_HOST, m2l_mode=N.M2L_BF16X3)
    B = FMMPlan(torch.as_tensor(s, device="cuda"), 5, 24, targets=torch.as_tensor(t, device="cuda"),
                tree_build=N.TREE_DEVICE, m2l_mode=N.M2L_BF16X3)
    same_plan(A, B)
    np.testing.assert_array_equal(evaluate(A, q), evaluate(B, q))


def test_batch_with_a_device_built_problem():
    sets = [wl.uniform_cube(70000, 3)[0], wl.sphere_surface(900, 4)[0],
            wl.gaussian_mixture(3000, 5)[0]]
    A = FMMPlan.batch(sets, 4, 32, tree_build=N.TREE_HOST)
    B = FMMPlan.batch(sets, 4, 32)  # auto: the 70000-point problem on the device
    assert B.info("device_trees") == 1 and A.info("device_trees") == 0
    same_plan(A, B)


@pytest.mark.parametrize("name", ["cube_n1e6_p6_ncrit150", "sphere_n4e6_p7_ncrit128"])
def test_full_size_workloads(name):
    w = wl.WORKLOADS[name]
    x, q = w.generate(0)
    B = FMMPlan(x, 4, w.ncrit)  # auto
    assert B.info("device_trees") == 1
    A = FMMPlan(x, 4, w.ncrit, tree_build=N.TREE_LEVELS_HOST)
    same_plan(A, B)
