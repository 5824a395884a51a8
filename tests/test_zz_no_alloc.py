"""fmm_evaluate_noalloc through the C ABI.

The entry point serves callers that may not allocate device memory while
they evaluate (their device memory belongs to another allocator, or a
cudaMalloc/cudaFree with its implicit device-wide synchronisation is not
acceptable in their loop).  It must return what fmm_evaluate returns,
within the parity tolerance of the GPU tests (per M2L mode), on two calls in
a row after another call left other data in the array (so a value a kernel
failed to write would show), and refuse
a workspace larger than its fixed 64 MiB array with a clear message.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl
from tests.parity import ELEM_C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative L2, the parity tolerance of the GPU tests


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def noalloc(plan, q, out):
    st = torch.cuda.current_stream().cuda_stream
    return N.lib().fmm_evaluate_noalloc(plan._h, q.data_ptr(), q.shape[1], out.data_ptr(),
                                        ctypes.c_void_p(st))


def _leave_other_data_in_the_array():
    """A no-alloc call on another plan with other charges and more columns,
    so the array holds different values when the call under test starts."""
    x, q = wl.gaussian_mixture(12_000, 53, nrhs=4)
    plan = FMMPlan(x, 4, 16, m2l_mode=N.M2L_BF16X3)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    out = torch.empty((len(x), 4), dtype=torch.float64, device="cuda")
    assert noalloc(plan, qd, out) == N.FMM_OK, N.lib().fmm_last_error()
    torch.cuda.synchronize()


MODES = [(N.M2L_FP32, TOL), (N.M2L_BF16X3, 1e-5), (N.M2L_TF32X3, TOL)]


@pytest.mark.parametrize("mode,tol", MODES, ids=["fp32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_evaluate_on_two_calls(nrhs, mode, tol):
    """Every M2L mode (the tensor-core modes also take their operand splits
    from the array), after another call left other data in the array, then
    twice in a row."""
    x, q = wl.sphere_surface(20_000, 51, nrhs=nrhs)
    plan = FMMPlan(x, 5, 24, m2l_mode=mode)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    ref = plan.evaluate(qd)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    _leave_other_data_in_the_array()
    out = torch.empty((len(x), nrhs), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        assert noalloc(plan, qd, out) == N.FMM_OK, N.lib().fmm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) <= tol
        assert np.max(np.abs(got - ref)) <= ELEM_C * tol * np.sqrt(np.mean(ref * ref))


def test_noalloc_keeps_the_callers_device():
    x, q = wl.uniform_cube(5_000, 54)
    plan = FMMPlan(x, 4, 32)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    out = torch.empty((len(x), 1), dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    assert noalloc(plan, qd, out) == N.FMM_OK, N.lib().fmm_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == before


def test_noalloc_refuses_oversized_workspace_and_host_buffers():
    x, q = wl.uniform_cube(20_000, 52, nrhs=16)
    plan = FMMPlan(x, 5, 24)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    out = torch.empty((len(x), 16), dtype=torch.float64, device="cuda")
    assert noalloc(plan, qd, out) == N.FMM_ERR_INVALID_ARG
    assert b"exceeds the fixed scratch" in N.lib().fmm_last_error()
    qh = np.ascontiguousarray(q[:, :1].astype(np.float32))
    oh = np.empty((len(x), 1))
    st = N.lib().fmm_evaluate_noalloc(plan._h, qh.ctypes.data, 1, oh.ctypes.data, None)
    assert st == N.FMM_ERR_INVALID_ARG
