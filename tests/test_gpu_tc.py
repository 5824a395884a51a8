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
