"""GPU parity: the CUDA path against the FP64 oracle, through the C ABI.

Bars (FP32 path):
* against the oracle KIFMM run with the same p, radii and pseudo-inverse
  cutoff: relative L2 error <= 1e-6;
* against the FP64 direct sum: error <= 1.5x the oracle KIFMM's own error
  at the same p, plus an FP32 resolution floor of 3e-7 (where the FP64
  method is already more accurate than FP32 can resolve, e.g. p = 7, the
  FP32 path is held to that floor instead);
* column r of an nrhs evaluation equals the single-vector evaluation of
  charges[:, r] bit for bit (same FP32 operations in the same order);
* beside every relative L2 bar, every target's error is bounded by
  c * bar * rms(reference) (tests/parity.py: c = 8 against the oracle
  KIFMM, 16 against the direct sum).
"""
import numpy as np
import pytest

from oracle.direct import direct_sum
from oracle.kifmm import KIFMM
from paper_2303_08394_gb300 import FMMPlan, _native as N
from paper_2303_08394_gb300 import workloads as wl
from tests.parity import ELEM_C_DIRECT, check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative L2 resolution of an FP32 evaluation of the whole method
FP32_FLOOR = 3e-7


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def gpu_eval(plan, q):
    """Evaluate through the C ABI with device buffers; returns (n, nrhs)."""
    q = np.asarray(q, dtype=np.float32)
    qd = torch.as_tensor(q.reshape(len(q), -1), device="cuda")
    out = plan.evaluate(qd)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    # name, generator, n, p, ncrit
    ("cube10k_p4", wl.uniform_cube, 10_000, 4, 64),
    ("cube12k_p6", wl.uniform_cube, 12_000, 6, 48),
    ("sphere8k_p5", wl.sphere_surface, 8_000, 5, 16),
    ("gauss8k_p6", wl.gaussian_mixture, 8_000, 6, 24),
    ("sphere6k_p7", wl.sphere_surface, 6_000, 7, 32),
]


@pytest.mark.parametrize("name,gen,n,p,ncrit", CASES, ids=[c[0] for c in CASES])
def test_fmm_matches_oracle(name, gen, n, p, ncrit):
    x, q = gen(n, 41)
    q = q[:, 0]
    plan = FMMPlan(x, p, ncrit)
    phi = gpu_eval(plan, q)[:, 0]
    ora = KIFMM(x, p, ncrit)
    phi_o = ora.evaluate(q)
    ref = direct_sum(x, q)
    e_gpu_ora = rel(phi, phi_o)
    e_gpu, e_ora = rel(phi, ref), rel(phi_o, ref)
    assert e_gpu_ora <= 1e-6, (e_gpu_ora, e_gpu, e_ora)
    assert e_gpu <= 1.5 * e_ora + FP32_FLOOR, (e_gpu, e_ora)
    r1 = check(phi, phi_o, 1e-6, what=f"{name} vs oracle")[1]
    r2 = check(phi, ref, 1.5 * e_ora + FP32_FLOOR, c=ELEM_C_DIRECT,
               what=f"{name} vs direct")[1]
    print(name, "element ratios", r1, r2)
    # the lists the GPU ran on are the oracle's lists
    assert plan.info("v_pairs") == sum(len(v) for v in ora.V.values())
    assert plan.info("u_pairs") == sum(len(v) for v in ora.U.values())


@pytest.mark.parametrize("mode", [N.M2L_FP32, N.M2L_BF16X3], ids=["fp32", "bf16x3"])
def test_w_and_x_through_surfaces_match_oracle(mode):
    """direct_wx = 0: every W box through M2P and every X list through P2L
    (the paper's form), against the oracle run the same way, on clustered
    points where both lists are used; and the two forms against each other
    within the method's error."""
    x, q = wl.gaussian_mixture(8000, 46, nrhs=2)
    plan0 = FMMPlan(x, 5, 16, direct_wx=0, m2l_mode=mode)
    plan1 = FMMPlan(x, 5, 16, m2l_mode=mode)
    assert plan0.info("wx_direct_pairs") == 0 and plan1.info("wx_direct_pairs") > 0
    assert plan0.info("surf_pairs") > plan1.info("surf_pairs")
    phi0, phi1 = gpu_eval(plan0, q), gpu_eval(plan1, q)
    ora = KIFMM(x, 5, 16, direct_wx=False).evaluate(q)
    bar = 1e-6 if mode == N.M2L_FP32 else 1e-5
    for r in range(2):
        check(phi0[:, r], ora[:, r], bar, what=f"surface W/X column {r} vs oracle")
    ref = direct_sum(x, q[:, 0])
    e0, e1 = rel(phi0[:, 0], ref), rel(phi1[:, 0], ref)
    assert e1 <= 1.2 * e0 + FP32_FLOOR, (e1, e0)


@pytest.mark.parametrize("nrhs", [3, 8, 21])
def test_nrhs_columns_equal_single_vector(nrhs):
    x, q = wl.gaussian_mixture(5000, 42, nrhs=nrhs)
    plan = FMMPlan(x, 5, 20)
    multi = gpu_eval(plan, q)
    for r in (0, nrhs // 2, nrhs - 1):
        single = gpu_eval(plan, q[:, r])[:, 0]
        np.testing.assert_array_equal(multi[:, r], single)


def test_single_leaf_equals_direct_sum():
    x, q = wl.uniform_cube(120, 43)
    plan = FMMPlan(x, 4, 200)
    assert plan.info("depth") == 0
    phi = gpu_eval(plan, q[:, 0])[:, 0]
    ref = direct_sum(x, q[:, 0])
    check(phi, ref, 1e-6, what="single leaf vs direct")


def test_one_point_and_coincident_points():
    plan = FMMPlan(np.array([[0.5, 0.5, 0.5]]), 4, 8)
    assert gpu_eval(plan, [2.0])[0, 0] == 0.0
    x, q = wl.uniform_cube(3000, 44)
    x[10] = x[11]
    x[200:205] = x[300]
    plan = FMMPlan(x, 5, 16)
    phi = gpu_eval(plan, q[:, 0])[:, 0]
    ref = direct_sum(x, q[:, 0])
    ora = KIFMM(x, 5, 16).evaluate(q[:, 0])
    check(phi, ora, 1e-6, what="coincident points vs oracle")
    assert np.all(np.isfinite(phi))


def test_ragged_tiles_and_deep_tree():
    """Adaptive tree with many levels, partly filled M2L tiles and W/X lists."""
    x, q = wl.gaussian_mixture(7000, 45)
    x = np.concatenate([x, 0.5 + 1e-4 * np.random.default_rng(0).standard_normal((300, 3))])
    q = np.concatenate([q[:, 0], np.ones(300)])
    plan = FMMPlan(x, 4, 6)
    assert plan.info("depth") >= 9
    assert plan.info("w_pairs") > 0 and plan.info("x_pairs") > 0
    phi = gpu_eval(plan, q)[:, 0]
    ora = KIFMM(x, 4, 6).evaluate(q)
    check(phi, ora, 1e-6, what="deep tree vs oracle")


def test_host_buffers_match_device_buffers():
    x, q = wl.uniform_cube(6000, 46, nrhs=2)
    plan = FMMPlan(x, 4, 32)
    dev = gpu_eval(plan, q)
    host = plan.evaluate(np.asarray(q, dtype=np.float32))
    np.testing.assert_array_equal(host, dev)
    pinned_q = torch.tensor(np.asarray(q, dtype=np.float32)).pin_memory()
    pinned_out = torch.empty((len(x), 2), dtype=torch.float64).pin_memory()
    plan.evaluate(pinned_q, out=pinned_out)
    np.testing.assert_array_equal(pinned_out.numpy(), dev)


def test_evaluate_on_a_side_stream_and_repeat():
    x, q = wl.uniform_cube(8000, 47)
    plan = FMMPlan(x, 4, 40)
    qd = torch.as_tensor(q[:, 0].astype(np.float32), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = plan.evaluate(qd)
        b = plan.evaluate(qd)
    s.synchronize()
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert plan.info("last_launches") >= 5


def test_graph_replay_matches_direct_launches():
    """On a non-default stream an evaluation is captured into a CUDA graph and
    replayed; the result is bit-identical to launching the kernels directly,
    and new buffers, a new nrhs or a new M2L mode re-capture."""
    x, q = wl.gaussian_mixture(9000, 48, nrhs=3)
    plan = FMMPlan(x, 5, 30)
    plan.set_graph(False)
    direct = gpu_eval(plan, q)
    plan.set_graph(True)
    s = torch.cuda.Stream()
    qd = torch.as_tensor(q.astype(np.float32), device="cuda")
    outs = []
    with torch.cuda.stream(s):
        for _ in range(3):
            outs.append(plan.evaluate(qd).clone())
        out1 = plan.evaluate(qd[:, :1].contiguous())      # new nrhs and buffers
        plan.set_m2l_mode(N.M2L_TF32X3)
        tc = plan.evaluate(qd)                             # new mode
        plan.set_m2l_mode(N.M2L_FP32)
        back = plan.evaluate(qd)
    s.synchronize()
    for o in outs + [back]:
        np.testing.assert_array_equal(o.cpu().numpy(), direct)
    np.testing.assert_array_equal(out1.cpu().numpy()[:, 0], direct[:, 0])
    check(tc.cpu().numpy(), direct, 1e-6, what="tf32x3 vs fp32")


@pytest.mark.parametrize("mode", [N.M2L_FP32, N.M2L_BF16X3], ids=["fp32", "bf16x3"])
def test_autotuned_tile_shapes_are_bit_identical(mode):
    """The first evaluation times every tile shape of each level product and
    keeps the fastest; every shape computes the same bits, so the tuned
    result equals the result of any forced shape and of tuning off."""
    x, q = wl.gaussian_mixture(20000, 49, nrhs=2)
    plan = FMMPlan(x, 6, 40, m2l_mode=mode)
    tuned = gpu_eval(plan, q)
    shapes = plan.array("gemm_shapes")
    assert len(shapes) > 0 and set(shapes.tolist()) <= {0, 1, 2, 3, 4}
    np.testing.assert_array_equal(gpu_eval(plan, q), tuned)       # replay of the choice
    for sh in range(5):
        plan.set_gemm_shape(sh)
        np.testing.assert_array_equal(gpu_eval(plan, q), tuned)
    plan.set_gemm_shape(-1)
    plan.set_autotune(False)
    np.testing.assert_array_equal(gpu_eval(plan, q), tuned)


@pytest.mark.parametrize("mode", [N.M2L_BF16X3, N.M2L_FP32], ids=["bf16x3", "fp32"])
def test_tuned_m2l_schedule_and_leaf_order_are_bit_identical(mode):
    """The autotuner's other two choices (the target-tile M2L's block
    schedule, the leaf pass's launch order) change no summation order: the
    tuned result equals every forced combination, and the choices are
    exported."""
    x, q = wl.sphere_surface(300_000, 57, nrhs=2)
    plan = FMMPlan(x, 4, 16, m2l_mode=mode)
    assert plan.info("m2l_tiles") >= 152  # the block schedule exists
    tuned = gpu_eval(plan, q)
    knobs = plan.array("tuned_knobs")
    assert len(knobs) == 2 and set(knobs.tolist()) <= {0, 1}
    for k in range(4):
        plan.set_knobs(k)
        np.testing.assert_array_equal(gpu_eval(plan, q), tuned)
        assert plan.array("tuned_knobs").tolist() == [k & 1, k >> 1]
    plan.set_knobs(-1)
    np.testing.assert_array_equal(gpu_eval(plan, q), tuned)
    # the gradient pass takes the same leaf launch order
    q0 = np.ascontiguousarray(q[:, 0], dtype=np.float32)
    g_tuned = plan.evaluate_gradient(q0)[1]
    plan.set_knobs(2)
    np.testing.assert_array_equal(plan.evaluate_gradient(q0)[1], g_tuned)


@pytest.mark.slow
def test_million_point_workload_sampled_against_direct_sum():
    """The 10^6-point uniform workload at p=6, ncrit=150 (the benchmark's
    workload and launch configuration): relative L2 error on 1,000 sampled
    targets against the FP64 direct sum stays within 1e-5."""
    w = wl.CUBE_1M_P6
    x, q = w.generate(0)
    plan = FMMPlan(x, w.p, w.ncrit)
    phi = gpu_eval(plan, q[:, 0])[:, 0]
    idx = wl.sample_targets(w.n, w.error_samples, 0)
    # the zero-distance self pair is skipped, so these are Eq. (1) potentials
    ref = direct_sum(x, q[:, 0], targets=x[idx])
    check(phi[idx], ref, 1e-5, c=ELEM_C_DIRECT, what="10^6 cube vs direct")


@pytest.mark.parametrize("p,n,ncrit", [(2, 3000, 16), (10, 1500, 32)], ids=["p2", "p10"])
def test_extreme_orders_every_mode(p, n, ncrit):
    """The smallest and largest expansion orders the ABI accepts: p = 2 (the
    eight corners of the cube, M2L rank 8, one 16-wide tensor-core K step)
    and p = 10 (488 surface points: the widest P2M and P2L blocks and the
    largest M2L rank), in every M2L mode, against the oracle and the direct
    sum with the bars above."""
    x, q = wl.uniform_cube(n, 70)
    q = q[:, 0]
    ora = KIFMM(x, p, ncrit).evaluate(q)
    ref = direct_sum(x, q)
    e_ora = rel(ora, ref)
    plan = FMMPlan(x, p, ncrit)
    errs = {}
    bars = {"fp32": 1e-6, "tf32x3": 1e-6, "bf16x3": 1e-5}
    for mode, name in ((N.M2L_FP32, "fp32"), (N.M2L_TF32X3, "tf32x3"), (N.M2L_BF16X3, "bf16x3")):
        plan.set_m2l_mode(mode)
        phi = gpu_eval(plan, q)[:, 0]
        errs[name] = (rel(phi, ora), rel(phi, ref))
        check(phi, ora, bars[name], what=f"p={p} {name} vs oracle")
        if name == "fp32":
            check(phi, ref, 1.5 * e_ora + FP32_FLOOR, c=ELEM_C_DIRECT, what=f"p={p} fp32 vs direct")
    print(p, "k", plan.info("rank_m2l"), "oracle vs direct", e_ora, errs)
    assert errs["fp32"][0] <= 1e-6 and errs["tf32x3"][0] <= 1e-6, (e_ora, errs)
    assert errs["bf16x3"][0] <= 1e-5, (e_ora, errs)
    assert errs["fp32"][1] <= 1.5 * e_ora + FP32_FLOOR, (e_ora, errs)


def test_tuned_shapes_are_kept_per_nrhs():
    """The autotuner keeps its choice per nrhs: a caller that alternates the
    number of charge columns tunes once per count, and every evaluation with
    a count returns the bits of the first one."""
    x, q = wl.gaussian_mixture(20000, 50, nrhs=3)
    plan = FMMPlan(x, 5, 40)
    first = {1: gpu_eval(plan, q[:, :1]), 3: gpu_eval(plan, q)}
    assert plan.info("tunings") == 2
    s = torch.cuda.Stream()
    for r in (1, 3, 1, 3):
        np.testing.assert_array_equal(gpu_eval(plan, q[:, :r]), first[r])
        with torch.cuda.stream(s):   # graph replay for both counts
            got = plan.evaluate(torch.as_tensor(q[:, :r].astype(np.float32), device="cuda"))
        s.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), first[r])
    assert plan.info("tunings") == 2
