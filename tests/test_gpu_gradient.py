"""GPU parity of fmm_evaluate_gradient: the gradient of the potential with
respect to the target position.

* Against the FP64 oracle KIFMM's gradient (same p, radii, cutoffs), every
  M2L mode, on the three distributions, to the bars of the potentials
  (1e-6 for FP32 and TF32x3, 1e-5 for BF16x3); and against the FP64 direct
  gradient within 1.5x the oracle's own error.
* The potentials the gradient call writes are those of fmm_evaluate, bit
  for bit; columns are independent of nrhs; host buffers and the
  gradients-only form give the same numbers.
* Distinct targets (tree on the union, targets uncharged) and batch plans.
* At the full size of the benchmark workload, sampled targets against the
  FP64 direct gradient.
"""
import numpy as np
import pytest

from oracle.direct import direct_gradient
from oracle.kifmm import KIFMM
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl
from tests.parity import ELEM_C_GRAD, check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEN = {"cube": wl.uniform_cube, "sphere": wl.sphere_surface, "gauss": wl.gaussian_mixture}
# measured: 1.9-2.9e-7 (FP32, TF32x3), 1.9-4.6e-7 (BF16x3) on these cases
BARS = {N.M2L_FP32: 1e-6, N.M2L_TF32X3: 1e-6, N.M2L_BF16X3: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def grad_eval(plan, q, potentials=True):
    qd = torch.as_tensor(np.asarray(q, dtype=np.float32).reshape(len(q), -1), device="cuda")
    phi, g = plan.evaluate_gradient(qd, potentials=potentials)
    torch.cuda.synchronize()
    return (phi.cpu().numpy() if phi is not None else None), g.cpu().numpy()


@pytest.mark.parametrize("mode", [N.M2L_FP32, N.M2L_TF32X3, N.M2L_BF16X3],
                         ids=["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("kind,n,p,ncrit", [("cube", 6000, 5, 32), ("gauss", 6000, 6, 24),
                                            ("sphere", 5000, 4, 16)])
def test_gradient_matches_oracle(mode, kind, n, p, ncrit):
    x, q = GEN[kind](n, 71)
    q = q[:, 0]
    plan = FMMPlan(x, p, ncrit, m2l_mode=mode)
    _, g = grad_eval(plan, q)
    _, g_ora = KIFMM(x, p, ncrit).evaluate(q, gradient=True)
    e_ora = rel(g[:, 0, :], g_ora)
    assert e_ora <= BARS[mode], e_ora
    ref = direct_gradient(x, q)
    e_gpu, e_fmm = rel(g[:, 0, :], ref), rel(g_ora, ref)
    assert e_gpu <= 1.5 * e_fmm + BARS[mode], (e_gpu, e_fmm)
    r1 = check(g[:, 0, :], g_ora, BARS[mode], c=ELEM_C_GRAD, what=f"{kind} gradient vs oracle")[1]
    r2 = check(g[:, 0, :], ref, 1.5 * e_fmm + BARS[mode], c=ELEM_C_GRAD,
               what=f"{kind} gradient vs direct")[1]
    print(kind, mode, "element ratios", r1, r2)


def test_potentials_columns_and_host_buffers():
    x, q = wl.gaussian_mixture(8000, 72, nrhs=3)
    plan = FMMPlan(x, 5, 24, m2l_mode=N.M2L_BF16X3)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    phi_eval = plan.evaluate(qd)
    torch.cuda.synchronize()
    phi, g = grad_eval(plan, q)
    np.testing.assert_array_equal(phi, phi_eval.cpu().numpy())
    for r in range(3):
        _, g1 = grad_eval(plan, q[:, r])
        np.testing.assert_array_equal(g1[:, 0, :], g[:, r, :])
    none, g_only = grad_eval(plan, q, potentials=False)
    assert none is None
    np.testing.assert_array_equal(g_only, g)
    phi_h, g_h = plan.evaluate_gradient(q.astype(np.float32))  # numpy in, numpy out
    np.testing.assert_array_equal(phi_h, phi)
    np.testing.assert_array_equal(g_h, g)


def test_distinct_targets_and_batches():
    x, q = wl.uniform_cube(4000, 73)
    y, _ = wl.gaussian_mixture(4000, 74)
    q = q[:, 0]
    plan = FMMPlan(x, 5, 24, targets=y)
    _, g = grad_eval(plan, q)
    ora = KIFMM(np.vstack([x, y]), 5, 24)
    _, g_ora = ora.evaluate(np.concatenate([q, np.zeros(len(y))]), gradient=True)
    check(g[:, 0, :], g_ora[len(x):], BARS[N.M2L_FP32], c=ELEM_C_GRAD,
          what="distinct targets gradient")
    sets = [wl.uniform_cube(n, 80 + n)[0] for n in (2500, 40, 1800)]
    qs = [wl.uniform_cube(len(s), 90 + len(s))[1][:, 0] for s in sets]
    B = FMMPlan.batch(sets, 4, 20)
    _, gb = grad_eval(B, np.concatenate(qs))
    parts = B.split(gb[:, 0, :])
    for s, qi, got in zip(sets, qs, parts):
        _, want = KIFMM(s, 4, 20).evaluate(qi, gradient=True)
        check(got, want, BARS[N.M2L_FP32], c=ELEM_C_GRAD,
              what=f"batch problem of {len(s)} points, gradient")


def test_benchmark_workload_sampled():
    w = wl.WORKLOADS["cube_n1e6_p6_ncrit150"]
    x, q = w.generate(0)
    plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=N.M2L_BF16X3, eps_svd=5e-7)
    _, g = grad_eval(plan, q[:, 0], potentials=False)
    idx = wl.sample_targets(w.n, w.error_samples, 0)
    ref = direct_gradient(x, q[:, 0], x[idx])
    check(g[idx, 0, :], ref, 2e-5, c=ELEM_C_GRAD, what="10^6 cube gradient")  # measured 9.9e-6
