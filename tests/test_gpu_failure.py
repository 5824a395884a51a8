"""Failure detection in the tensor-core M2L, made to happen without a fault.

Every wait inside the tensor-core M2L kernels (target tiles and pair
columns) is bounded; when one expires the block records
its role in the plan's mapped error word, drains what it issued, frees its
tensor memory and returns, and the host reports FMM_ERR_TIMEOUT.  The test
hook FMM_OPT_TEST_M2L_STALL makes block 0 wait on a barrier that nothing
completes (with a 0.1 s limit), so that path runs on every launch while the
option is on.  Nothing here traps, faults or hangs the GPU.
"""
import numpy as np
import pytest

from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def stall(plan, on):
    N.check(N.lib().fmm_plan_set_option(plan._h, N.OPT_TEST_M2L_STALL, 1.0 if on else 0.0))


@pytest.mark.parametrize("kernel", [0, 1], ids=["pair_columns", "target_tiles"])
@pytest.mark.parametrize("mode", [N.M2L_BF16X3, N.M2L_TF32X3], ids=["bf16x3", "tf32x3"])
def test_expired_wait_is_reported_and_the_plan_recovers(mode, kernel):
    x, q = wl.uniform_cube(20_000, 61, nrhs=2)
    plan = FMMPlan(x, 5, 24, m2l_mode=mode)
    plan.set_m2l_kernel(kernel)
    assert plan.info("m2l_kernel") == (2 if kernel == 0 else 1)
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    ref = plan.evaluate(qd)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()

    stall(plan, True)
    # host buffers: the call waits for its stream and reports the expiry
    with pytest.raises(N.FMMError) as e:
        plan.evaluate(np.asarray(q, dtype=np.float32))
    assert e.value.status == N.FMM_ERR_TIMEOUT
    assert "roles mask 32" in str(e.value)

    # device buffers on a side stream (captured into a graph): the call only
    # enqueues; once the work has finished the next call reports it
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.evaluate(qd)
    s.synchronize()
    stall(plan, False)
    with pytest.raises(N.FMMError) as e:
        plan.evaluate(qd)
    assert e.value.status == N.FMM_ERR_TIMEOUT

    # reported once; the plan and the context work as before, on both
    # paths, bit for bit
    got = plan.evaluate(qd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    with torch.cuda.stream(s):
        got = plan.evaluate(qd)
    s.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    np.testing.assert_array_equal(plan.evaluate(np.asarray(q, dtype=np.float32)), ref)


def test_stall_hook_has_no_effect_in_fp32_mode():
    x, q = wl.uniform_cube(8_000, 62)
    plan = FMMPlan(x, 4, 32, m2l_mode=N.M2L_FP32)
    qh = np.asarray(q, dtype=np.float32)
    ref = plan.evaluate(qh)
    stall(plan, True)
    np.testing.assert_array_equal(plan.evaluate(qh), ref)
    np.testing.assert_array_equal(plan.evaluate(qh), ref)
