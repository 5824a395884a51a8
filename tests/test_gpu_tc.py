"""GPU parity of the tensor-core M2L (tcgen05, split precision).

TF32x3 keeps the FP32 bar (<= 1e-6 against the oracle KIFMM).  BF16x3
carries about 16 significant bits in each operand product; its bar is
1e-5 against the oracle (prototype: 5.4e-6 at p = 6), the accuracy gate of
the benchmark metric.  Both are also compared with the FP32 CUDA-core M2L
on the same plan.
"""
import numpy as np
import pytest

from oracle.kifmm import KIFMM
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl
from tests.parity import check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BARS = {N.M2L_TF32X3: 1e-6, N.M2L_BF16X3: 1e-5}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def gpu_eval(plan, q):
    q = np.asarray(q, dtype=np.float32)
    out = plan.evaluate(torch.as_tensor(q.reshape(len(q), -1), device="cuda"))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", [N.M2L_TF32X3, N.M2L_BF16X3], ids=["tf32x3", "bf16x3"])
@pytest.mark.parametrize("gen,n,p,ncrit", [
    (wl.uniform_cube, 6000, 4, 32),
    (wl.uniform_cube, 12000, 6, 48),
    (wl.sphere_surface, 8000, 5, 16),
    (wl.sphere_surface, 6000, 7, 32),
], ids=["cube_p4", "cube_p6", "sphere_p5", "sphere_p7"])
def test_tc_m2l_matches_oracle(mode, gen, n, p, ncrit):
    x, q = gen(n, 61)
    q = q[:, 0]
    plan = FMMPlan(x, p, ncrit)
    simt = gpu_eval(plan, q)[:, 0]
    plan.set_m2l_mode(mode)
    tc = gpu_eval(plan, q)[:, 0]
    ora = KIFMM(x, p, ncrit).evaluate(q)
    assert rel(tc, ora) <= BARS[mode], (rel(tc, ora), rel(simt, ora))
    assert rel(tc, simt) <= BARS[mode]
    check(tc, ora, BARS[mode], what="tensor-core M2L vs oracle")
    check(tc, simt, BARS[mode], what="tensor-core M2L vs FP32 M2L")


@pytest.mark.parametrize("mode", [N.M2L_TF32X3, N.M2L_BF16X3], ids=["tf32x3", "bf16x3"])
def test_tc_nrhs_columns(mode):
    x, q = wl.gaussian_mixture(5000, 62, nrhs=3)
    plan = FMMPlan(x, 5, 20, m2l_mode=mode)
    multi = gpu_eval(plan, q)
    for r in range(3):
        single = gpu_eval(plan, q[:, r])[:, 0]
        np.testing.assert_allclose(multi[:, r], single, rtol=1e-12, atol=1e-12 * np.abs(single).max())


def test_tc_deep_adaptive_tree():
    x, q = wl.gaussian_mixture(7000, 63)
    x = np.concatenate([x, 0.5 + 1e-4 * np.random.default_rng(1).standard_normal((300, 3))])
    q = np.concatenate([q[:, 0], np.ones(300)])
    plan = FMMPlan(x, 4, 6, m2l_mode=N.M2L_TF32X3)
    phi = gpu_eval(plan, q)[:, 0]
    ora = KIFMM(x, 4, 6).evaluate(q)
    check(phi, ora, 1e-6, what="deep tree TF32x3 vs oracle")


# ---------------------------------------------------------------------------
# the pair-column kernel (operand width <= 128) against the oracle, the
# target-tile kernel and the FP32 path
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [N.M2L_TF32X3, N.M2L_BF16X3], ids=["tf32x3", "bf16x3"])
@pytest.mark.parametrize("gen,n,p,ncrit,nrhs", [
    (wl.uniform_cube, 6000, 4, 32, 1),     # kpad 64: one K chunk (BF16), zero rows 64..127
    (wl.sphere_surface, 8000, 5, 16, 1),   # kpad 112: a partial last K chunk
    (wl.gaussian_mixture, 7000, 5, 8, 3),  # deep adaptive tree, three columns
], ids=["cube_p4", "sphere_p5", "gauss_p5_nrhs3"])
def test_pair_column_m2l_matches_oracle_and_target_tiles(mode, gen, n, p, ncrit, nrhs):
    x, q = gen(n, 64, nrhs=nrhs)
    plan = FMMPlan(x, p, ncrit, m2l_mode=mode)
    plan.set_m2l_kernel(0)
    assert plan.info("m2l_kernel") == 2 and plan.info("m2l_windows") > 0
    pc = gpu_eval(plan, q)
    plan.set_m2l_kernel(1)
    assert plan.info("m2l_kernel") == 1
    tiles = gpu_eval(plan, q)
    ora = KIFMM(x, p, ncrit)
    for r in range(nrhs):
        ref = ora.evaluate(q[:, r])
        check(pc[:, r], ref, BARS[mode], what=f"pair columns vs oracle, column {r}")
        check(pc[:, r], tiles[:, r], BARS[mode], what=f"pair columns vs target tiles, column {r}")
    # repeat: the same bits (the summation order does not depend on timing)
    plan.set_m2l_kernel(0)
    np.testing.assert_array_equal(gpu_eval(plan, q), pc)


@pytest.mark.parametrize("mode", [N.M2L_TF32X3, N.M2L_BF16X3], ids=["tf32x3", "bf16x3"])
@pytest.mark.parametrize("gen,n,p,ncrit,eps", [
    (wl.uniform_cube, 30000, 6, 48, 5e-7),    # k = 127: operand width 128
    (wl.sphere_surface, 40000, 7, 32, 1e-6),  # k = 122: the sphere workload's width
], ids=["cube_p6", "sphere_p7"])
def test_pair_column_m2l_at_operand_width_128(mode, gen, n, p, ncrit, eps):
    """The compression of the benchmark workloads (operand width 128, so the
    pair-column kernel runs): against the FP32 path on the same plan (same
    compressed operators) and against the target-tile kernel."""
    x, q = gen(n, 65)
    q = q[:, 0]
    plan = FMMPlan(x, p, ncrit, eps_svd=eps)
    assert plan.info("rank_m2l") <= 128
    fp32 = gpu_eval(plan, q)[:, 0]
    plan.set_m2l_mode(mode)
    plan.set_m2l_kernel(0)
    assert plan.info("m2l_kernel") == 2
    pc = gpu_eval(plan, q)[:, 0]
    plan.set_m2l_kernel(1)
    tiles = gpu_eval(plan, q)[:, 0]
    check(pc, fp32, BARS[mode], what="pair columns vs FP32 M2L")
    check(pc, tiles, BARS[mode], what="pair columns vs target tiles")
