"""GPU parity at the full sizes of the larger workloads, on sampled targets
against the FP64 direct sum of Eq. (1) (the oracle KIFMM does not reach
these sizes in test time):

* 4*10^6 points on the unit sphere, p = 7, ncrit = 128 (a strongly adaptive
  tree, 8 levels): every M2L mode;
* 10^6 uniform points with 64 charge columns, p = 6, ncrit = 150: every
  column, and columns against single-column evaluations;
* 1.6*10^7 points from eight Gaussians, p = 8, ncrit = 128, 8 columns
  (9 levels, kpad 176): BF16x3 M2L;
* gradients on the 4*10^6-point sphere against the FP64 direct gradient
  (measured 2.2e-7 in every M2L mode; bar 1e-6).

Bar: relative L2 error <= 1e-5 over the sampled targets (all columns),
the accuracy gate of the benchmark.
"""
import numpy as np
import pytest

from oracle.direct import direct_gradient, direct_sum
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl
from tests.parity import ELEM_C_DIRECT, ELEM_C_GRAD, check

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GATE = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _eval(plan, qd):
    out = plan.evaluate(qd)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_sphere_4m_p7_every_mode():
    w = wl.SPHERE_4M_P7
    x, q = w.generate(0)
    plan = FMMPlan(x, w.p, w.ncrit)
    assert plan.info("depth") >= 7 and plan.info("rank_m2l") > 144  # kpad 176
    idx = wl.sample_targets(w.n, w.error_samples, 0)
    ref = direct_sum(x, q[:, 0], x[idx])
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    errs = {}
    for mode in (N.M2L_FP32, N.M2L_TF32X3, N.M2L_BF16X3):
        plan.set_m2l_mode(mode)
        got = _eval(plan, qd)[idx, 0]
        errs[mode] = rel(got, ref)
        check(got, ref, GATE, c=ELEM_C_DIRECT, what=f"sphere 4e6 mode {mode} vs direct")
    assert max(errs.values()) <= GATE, errs
    # the split-precision forms stay near the plain FP32 path
    assert errs[N.M2L_TF32X3] <= 2 * errs[N.M2L_FP32] + 1e-7, errs


def test_cube_1m_p6_nrhs64():
    w = wl.CUBE_1M_P6_NRHS64
    x, q = w.generate(0)
    plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=N.M2L_BF16X3)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    phi = _eval(plan, qd)
    assert phi.shape == (w.n, 64)
    idx = wl.sample_targets(w.n, w.error_samples, 0)
    ref = direct_sum(x, q, x[idx])
    assert rel(phi[idx], ref) <= GATE
    # every column's targets against the gate over all columns (one column
    # alone may sit above the gate: measured 1.19e-5 for column 46)
    check(phi[idx], ref, GATE, c=ELEM_C_DIRECT, what="cube 1e6, 64 columns vs direct")
    # column r of the 64-column evaluation against a one-column evaluation
    for r in (0, 37, 63):
        one = _eval(plan, qd[:, r:r + 1].contiguous())
        check(phi[:, r], one[:, 0], 1e-6, what=f"column {r} vs one-column evaluation")
    plan.set_m2l_mode(N.M2L_FP32)
    phi32 = _eval(plan, qd)
    for r in (5, 63):
        np.testing.assert_array_equal(phi32[:, r], _eval(plan, qd[:, r:r + 1].contiguous())[:, 0])


def test_gauss_16m_p8_nrhs8():
    w = wl.GAUSS_16M_P8
    x, q = w.generate(0)
    plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=N.M2L_BF16X3)
    assert plan.info("depth") >= 8
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    phi = _eval(plan, qd)
    idx = wl.sample_targets(w.n, w.error_samples, 0)
    ref = direct_sum(x, q, x[idx])
    assert rel(phi[idx], ref) <= GATE
    check(phi[idx], ref, GATE, c=ELEM_C_DIRECT, what="gauss 1.6e7, 8 columns vs direct")


def test_sphere_4m_p7_gradient():
    w = wl.SPHERE_4M_P7
    x, q = w.generate(0)
    plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=N.M2L_BF16X3)
    qd = torch.as_tensor(q[:, 0].astype(np.float32), device="cuda")
    _, g = plan.evaluate_gradient(qd, potentials=False)
    torch.cuda.synchronize()
    idx = wl.sample_targets(w.n, w.error_samples, 0)
    ref = direct_gradient(x, q[:, 0], x[idx])
    check(g.cpu().numpy()[idx], ref, 1e-6, c=ELEM_C_GRAD, what="sphere gradient vs direct")
