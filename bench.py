#!/usr/bin/env python
"""Benchmark: Laplace KIFMM points/s on one GB300 (or N independent ones).

Workload (default): 10^6 points uniform in the unit cube, charges uniform in
[-1, 1], p = 6, ncrit = 150, adaptive octree; M2L compression tolerance
eps_svd = 5e-7 (rank k = 127, operand width 128; the error against the
direct sum is set by p: 5.26e-6 here against 5.24e-6 at eps_svd = 1e-7, k = 143).  One step is one full
``fmm_evaluate`` (every operator, the M2L and P2P hot path included) with
inputs resident in device memory, replayed as a CUDA graph on a side
stream; L2 is flushed (256 MB write) before every timed step, outside the
timed events.  The headline runs the M2L in BF16x3 split precision on the
tensor cores (mixed); the plain FP32 path is timed on the same plan with
the same protocol and reported beside it.

Printed: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Laplace FMM points/s at rel L2 err \u22641e-5, mixed vs FP32; M2L % tensor peak"
UNIT = "points/s"
FP32_LANES_PER_SM = 128
NUM_SMS = 152
CPU_SAMPLE_N = 40_000
# --impl reference: the whole run (warm-up + timed steps) is held to about
# this many seconds by shrinking each step's sample as the step count grows
# (the oracle evaluates about 1e4 points/s on one host core at p = 6), with
# at least REF_MIN_N points so the sample still has a level-2 M2L
REF_BUDGET_S = 150.0
REF_MIN_N = 4_000


def reference_sample_n(reps):
    return max(REF_MIN_N, min(CPU_SAMPLE_N, int(REF_BUDGET_S * 1e4 / max(reps, 1))))
# DRAM bytes (read + write) of one launch, from the ncu captures summarised
# in profiles/ (k_m2l_tc_cube_n1e6_p6_bf16x3.md, k_eval_cube_n1e6_p6.md).
# Keyed by kernel, workload, M2L mode and M2L operand width (kpad; the leaf
# kernel does not depend on it: None); any other combination reports null.
TRAFFIC = {
    # dram read + write of one launch (profiles/k_m2l_tc_cube_n1e6_p6_bf16x3.md)
    ("k_m2l_tc", "cube_n1e6_p6_ncrit150", "bf16x3", 128): 77.2e6,
    # the leaf pass: its four width-group launches together
    ("k_eval", "cube_n1e6_p6_ncrit150", "bf16x3", None): 90.6e6,
    # the gradient variant (profiles/k_eval_gradient_cube_n1e6_p6.md)
    ("k_eval_grad", "cube_n1e6_p6_ncrit150", "bf16x3", None): 117.1e6,
    ("k_eval", "cube_n1e6_p6_ncrit150", "fp32", None): 90.6e6,
    ("k_eval", "cube_n1e6_p6_ncrit150", "tf32x3", None): 90.6e6,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="cube_n1e6_p6_ncrit150")
    ap.add_argument("--m2l", default="bf16x3", choices=["fp32", "bf16x3", "tf32x3"])
    ap.add_argument("--eps-svd", type=float, default=5e-7,
                    help="M2L compression tolerance (rank: singular values above eps * max)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error-check", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only: no CPU baseline, error gate or e2e leg")
    a = ap.parse_args()
    if a.quick:
        a.no_cpu_baseline = a.no_error_check = True
    return a


def max_over_ranks(value, world, device="cpu"):
    """The largest of every rank's `value` (all ranks get it); the timed
    region of a multi-rank run is its slowest rank's."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, steps, world, seconds):
    """Whole-job throughput: the units every rank processed over the time of
    the slowest rank."""
    return units_per_rank * steps * world / seconds


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
_ORACLE_STEP = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle.kifmm import KIFMM
from paper_2303_08394_gb300 import workloads as wl
w = wl.WORKLOADS[{workload!r}]
gen = {{"cube": wl.uniform_cube, "sphere": wl.sphere_surface, "gauss": wl.gaussian_mixture}}[w.kind]
x, q = gen({n}, 0, w.nrhs)
f = KIFMM(x, w.p, w.ncrit)
times = []
for i in range({reps}):
    t0 = time.perf_counter()
    f.evaluate(q)
    times.append(time.perf_counter() - t0)
print(json.dumps({{"times": times, "n": {n}, "nrhs": w.nrhs}}))
"""


def run_oracle(workload, n, reps):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = _ORACLE_STEP.format(root=ROOT, workload=workload, n=n, reps=reps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode:
        raise RuntimeError("oracle run failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(workload, w, reps=1):
    res = run_oracle(workload, CPU_SAMPLE_N, reps)
    t = statistics.median(res["times"])
    return {"value": res["n"] * res["nrhs"] / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"FP64 numpy KIFMM (dense M2L) evaluate on {res['n']:,} points of the "
                       f"same distribution, p={w.p}, ncrit={w.ncrit}; tree and operator setup "
                       f"excluded; {t:.2f} s per evaluate")}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# accuracy gate: FP64 direct sum of Eq. (1) on sampled targets (numpy)
# ---------------------------------------------------------------------------
def direct_sum_sampled(x, q, idx, block=4):
    import numpy as np
    out = np.zeros((len(idx), q.shape[1]))
    for s in range(0, len(idx), block):
        t = idx[s:s + block]
        d = x[None, :, :] - x[t][:, None, :]
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        with np.errstate(divide="ignore"):
            inv = np.where(r > 0, 1.0 / r, 0.0)
        out[s:s + block] = inv @ q
    return out / (4 * np.pi)


def direct_gradient_sampled(x, q, idx, block=4):
    """FP64 gradient of the direct sum at the sampled targets (numpy)."""
    import numpy as np
    out = np.zeros((len(idx), 3))
    for s in range(0, len(idx), block):
        t = idx[s:s + block]
        d = x[None, :, :] - x[t][:, None, :]
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        with np.errstate(divide="ignore"):
            w3 = np.where(r > 0, 1.0 / r ** 3, 0.0) * q[None, :]
        out[s:s + block] = np.einsum("ij,ijk->ik", w3, d)
    return out / (4 * np.pi)


# ---------------------------------------------------------------------------
def time_mode(plan, qd, out, flush, stream, steps, warmup, world, call=None):
    """Warm up, then time `steps` evaluations (CUDA events on `stream`, L2
    flushed before each step outside the events); returns per-step ms, the
    per-phase ms of every step and the launches of one evaluation.  `call`
    replaces the evaluation (default: potentials into `out`)."""
    import torch
    import torch.distributed as dist
    if call is None:
        def call():
            plan.evaluate(qd, out=out, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            call()
    torch.cuda.synchronize()
    launches = plan.info("last_launches")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    phases = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            call()
            ends[i].record(stream)
            phases.append(plan.phase_ms())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)], phases, launches


def main():
    a = parse()
    rank, world, local = dist_env()
    from paper_2303_08394_gb300 import workloads as wl
    w = wl.WORKLOADS[a.workload]
    config = {"workload": w.name, "n": w.n, "p": w.p, "ncrit": w.ncrit, "nrhs": w.nrhs,
              "points": w.kind, "m2l": a.m2l, "eps_svd": a.eps_svd,
              "graph": "CUDA graph replay on a side stream",
              "l2_flush": "256 MB write before every step",
              "per_rank": "independent problem (seed = rank)"}

    if a.impl == "reference":
        if rank != 0:
            return
        reps = a.warmup + a.steps
        res = run_oracle(a.workload, reference_sample_n(reps), reps)
        times = res["times"][a.warmup:]
        total = sum(times)
        value = res["n"] * res["nrhs"] * len(times) / total
        line = {"impl": "reference", "metric": METRIC, "value": value,
                "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"FP64 numpy KIFMM evaluate on {res['n']:,} points "
                                           f"of the workload's distribution per step"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    os.environ["FMM_TIMING"] = "1"
    from paper_2303_08394_gb300 import FMMPlan, build, _native as N
    if not os.path.exists(N.LIB_PATH):
        build.build()
    modes = {"fp32": N.M2L_FP32, "bf16x3": N.M2L_BF16X3, "tf32x3": N.M2L_TF32X3}
    x, q = w.generate(rank)
    t0 = time.perf_counter()
    plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=modes[a.m2l], eps_svd=a.eps_svd)
    plan_s = time.perf_counter() - t0
    qd = torch.as_tensor(q.astype(np.float32), device=dev)
    out = torch.empty((w.n, w.nrhs), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.perf_counter()
    step_ms, phases, launches_per_step = time_mode(plan, qd, out, flush, stream, a.steps,
                                                   a.warmup, world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / a.steps
    value = job_value(w.n * w.nrhs, a.steps, world, total_ms / 1e3)

    # accuracy gate on sampled targets (FP64 direct sum)
    err = None
    idx = ref = None
    if not a.no_error_check and rank == 0:
        idx = wl.sample_targets(w.n, w.error_samples or 1000, 0)
        ref = direct_sum_sampled(x, q, idx)
        got = out.cpu().numpy()[idx]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    # the plain FP32 path on the same plan, same protocol ("mixed vs FP32")
    fp32 = None
    if a.m2l != "fp32" and not a.quick:
        plan.set_m2l_mode(N.M2L_FP32)
        f_ms, f_ph, _ = time_mode(plan, qd, out, flush, stream, a.steps, a.warmup, world)
        f_tot = max_over_ranks(sum(f_ms), world, dev)
        fp32 = {"value": job_value(w.n * w.nrhs, a.steps, world, f_tot / 1e3),
                "ms_per_step": f_tot / a.steps,
                "m2l_ms": statistics.mean(ph["m2l"] for ph in f_ph)}
        if ref is not None:
            got = out.cpu().numpy()[idx]
            fp32["rel_l2_err"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        fp32["mixed_over_fp32"] = value / fp32["value"]
        plan.set_m2l_mode(modes[a.m2l])

    # gradients of the potentials (fmm_evaluate_gradient), same protocol, the
    # gradients only
    gradient = None
    if not a.quick and w.nrhs == 1:
        gout = torch.empty((w.n, 1, 3), dtype=torch.float64, device=dev)
        g_steps = min(a.steps, 100)
        g_ms, g_ph, g_launch = time_mode(
            plan, qd, out, flush, stream, g_steps, a.warmup, world,
            call=lambda: plan.evaluate_gradient(qd, grad_out=gout, potentials=False,
                                                stream=stream))
        g_tot = max_over_ranks(sum(g_ms), world, dev)
        gradient = {"value": job_value(w.n, g_steps, world, g_tot / 1e3), "unit": UNIT,
                    "ms_per_step": g_tot / g_steps, "steps": g_steps,
                    "phase_ms": {k: statistics.mean(ph[k] for ph in g_ph) for k in g_ph[0]},
                    "gpu_launches": g_launch * g_steps}
        if idx is not None:
            got = gout.cpu().numpy()[idx, 0, :]
            gref = direct_gradient_sampled(x, q[:, 0], idx)
            gradient["rel_l2_err"] = float(np.linalg.norm(got - gref) / np.linalg.norm(gref))

    # rooflines from the library's per-phase CUDA events (each phase below is
    # one kernel launch on `stream`)
    peaks, peak_src = load_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s
    k = plan.info("rank_m2l")
    kpad = (k + 15) // 16 * 16
    v_pairs = plan.info("v_pairs")
    p2p_pairs = plan.info("p2p_pairs")
    m2l_ms = statistics.mean(ph["m2l"] for ph in phases)
    leaf_ms = statistics.mean(ph["leaf"] for ph in phases)
    m2l_flops = 2.0 * k * k * v_pairs * w.nrhs
    m2l_tf = m2l_flops / (m2l_ms / 1e3) / 1e12
    near_flops = (8.0 + 2.0 * w.nrhs) * p2p_pairs
    leaf_tf = near_flops / (leaf_ms / 1e3) / 1e12
    if a.m2l == "fp32":
        m2l_roof = {"kernel": "k_m2l_simt", "bound": "alu", "achieved": m2l_tf,
                    "peak": fp32_peak, "unit": "TFLOP/s", "frac": m2l_tf / fp32_peak,
                    "traffic": TRAFFIC.get(("k_m2l_simt", w.name, a.m2l, kpad)),
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz",
                    "flops_per_launch": m2l_flops, "ms_per_launch": m2l_ms}
    else:
        tc_peak = peaks["bf16_tflops"] * (1.0 if a.m2l == "bf16x3" else 0.5)
        issued = 3 * m2l_flops
        m2l_roof = {"kernel": "k_m2l_tc", "bound": "tensor",
                    "achieved": issued / (m2l_ms / 1e3) / 1e12,
                    "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": issued / (m2l_ms / 1e3) / 1e12 / tc_peak,
                    "traffic": TRAFFIC.get(("k_m2l_tc", w.name, a.m2l, kpad)),
                    "peak_source": f"bf16_tflops of {peak_src}" +
                                   ("" if a.m2l == "bf16x3" else " x 1/2 (tf32)"),
                    "flops_per_launch": issued, "useful_flops_per_launch": m2l_flops,
                    "useful_frac_of_bf16_peak": m2l_flops / (m2l_ms / 1e3) / 1e12 /
                    peaks["bf16_tflops"],
                    "ms_per_launch": m2l_ms}
    leaf_roof = {"kernel": "k_eval", "bound": "alu", "achieved": leaf_tf, "peak": fp32_peak,
                 "unit": "TFLOP/s", "frac": leaf_tf / fp32_peak,
                 "traffic": TRAFFIC.get(("k_eval", w.name, a.m2l, None)),
                 "flops_per_launch": near_flops, "ms_per_launch": leaf_ms,
                 "note": "near-field pair flops only (8 + 2 nrhs per pair); L2P/M2P work "
                         "uncounted; one leaf pass = one launch per leaf width group (T = 1..4 "
                         "targets per lane), timed and counted together"}
    dominant = m2l_roof if m2l_ms >= leaf_ms else leaf_roof
    if gradient is not None:
        # potential + gradient: 8 (r^2, as above) + 2 (potential) + 3 (q / r^3)
        # + 6 (three FMAs) flops per near-field pair
        g_leaf = gradient["phase_ms"]["leaf"]
        g_flops = 19.0 * p2p_pairs
        g_tf = g_flops / (g_leaf / 1e3) / 1e12
        gradient["roofline"] = {"kernel": "k_eval (gradient variant)", "bound": "alu",
                                "achieved": g_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                                "frac": g_tf / fp32_peak,
                                "traffic": TRAFFIC.get(("k_eval_grad", w.name, a.m2l, None)),
                                "flops_per_launch": g_flops, "ms_per_launch": g_leaf,
                                "note": "near-field pair flops only (19 per pair); one leaf "
                                        "pass = one launch per leaf width group"}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not a.quick:
        e2e = run_e2e(plan, q, w, a, world, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f32" if a.m2l == "fp32" else f"f32 (M2L {a.m2l} split on tensor cores)",
                "data": "synthetic", "config": config,
                "rel_l2_err": err, "error_gate_1e-5": (err is not None and err <= 1e-5),
                "fp32": fp32, "gradient": gradient,
                "roofline": dominant, "rooflines": {"m2l": m2l_roof, "leaf": leaf_roof},
                "phase_ms": {k2: statistics.mean(ph[k2] for ph in phases) for k2 in phases[0]},
                "e2e": e2e,
                "gpu_launches": launches_per_step * a.steps, "clocks": clk,
                "plan_s": plan_s, "wall_s_timed_region": wall,
                "tree": {key: plan.info(key) for key in
                         ("nodes", "leaves", "depth", "rank_m2l", "v_pairs", "u_pairs",
                          "p2p_pairs", "m2l_tiles")},
                "peaks": peak_src}
        if world == 1 and not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(a.workload, w)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(plan, q, w, a, world, dev):
    import numpy as np
    import torch
    import torch.distributed as dist
    qh = torch.tensor(q.astype(np.float32)).pin_memory()
    oh = torch.empty((w.n, w.nrhs), dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream(device=dev)
    # host buffers: the library copies charges in, replays its graph and
    # copies potentials out on `stream`, and returns when they have landed
    plan.evaluate(qh, out=oh, stream=stream)
    steps = max(3, a.steps // 2)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.evaluate(qh, out=oh, stream=stream)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    return {"value": job_value(w.n * w.nrhs, steps, world, e2e_s), "unit": UNIT,
            "h2d_bytes_per_step": w.n * w.nrhs * 4, "d2h_bytes_per_step": w.n * w.nrhs * 8,
            "steps": steps}


if __name__ == "__main__":
    main()
