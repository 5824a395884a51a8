#!/usr/bin/env python
"""Benchmark: Laplace KIFMM points/s on one GB300 (or N independent ones).

Workload (default): 4*10^6 points uniform on the unit sphere (a strongly
adaptive octree), charges N(0, 1), p = 7, ncrit = 128; M2L compression
tolerance eps_svd = 1e-6 (rank k = 122, operand width 128; the error against
the direct sum is set by p).  One step is one full ``fmm_evaluate`` (every
operator, the M2L and P2P hot path included) with inputs resident in device
memory, replayed as a CUDA graph on a side stream; L2 is flushed (256 MB
write) before every timed step, outside the timed events.  The headline
runs the M2L in BF16x3 split precision on the tensor cores (mixed); the
plain FP32 path and the TF32x3 split (FP32-like accuracy) are timed on the
same plan with the same protocol and reported beside it, each with its
relative L2 error against the FP64 direct sum on 1,000 sampled targets.

``--workload cube_n1e6_p6_ncrit150`` (and the other named workloads) runs
another configuration.  Printed: one JSON line (rank 0).  ``--impl
reference`` times the FP64 CPU oracle on bounded samples of the same
workload on every host core instead.
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

METRIC = "Laplace FMM points/s at rel L2 err ≤1e-5, mixed vs FP32; M2L % tensor peak"
UNIT = "points/s"
FP32_LANES_PER_SM = 128
NUM_SMS = 152
DEFAULT_WORKLOAD = "sphere_n4e6_p7_ncrit128"
# the batched-problems workload reported beside every full run
BATCH_WORKLOAD = "batch256_cube_p6_ncrit150"
# M2L compression tolerance per workload: the largest that keeps the error
# against the direct sum where p puts it and gives an operand width of 128
# (k = 127 at p = 6, 122 at p = 7, 124 at p = 8)
EPS_SVD = {"cube_n1e6_p6_ncrit150": 5e-7, "cube_n1e6_p6_ncrit150_nrhs64": 5e-7,
           "sphere_n4e6_p7_ncrit128": 1e-6, "gauss8_n1.6e7_p8_ncrit128_nrhs8": 1e-6,
           "batch256_cube_p6_ncrit150": 5e-7}
# CPU oracle samples: points per worker process (one process per host core)
CPU_SAMPLE_N = 20_000
# --impl reference: the whole run (warm-up + timed steps) is held to about
# this many seconds by shrinking each step's sample as the step count grows
# (the oracle evaluates about 4e3-1e4 points/s per core), with at least
# REF_MIN_N points so the sample still has a level-2 M2L
REF_BUDGET_S = 120.0
REF_MIN_N = 4_000


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_sample_n(reps, rate=4e3):
    return max(REF_MIN_N, min(CPU_SAMPLE_N, int(REF_BUDGET_S * rate / max(reps, 1))))


# DRAM bytes (read + write) of one launch, from the ncu captures summarised
# in profiles/ (the leaf pass: the sum over its width-group launches, each
# captured cold).  Keyed by kernel, workload, M2L mode and M2L operand width
# (kpad; the leaf kernel does not depend on it: None); any other combination
# reports null.
TRAFFIC = {
    ("k_m2l_tc", "sphere_n4e6_p7_ncrit128", "bf16x3", 128): 138.7e6 + 32.4e6,
    ("k_eval", "sphere_n4e6_p7_ncrit128", "bf16x3", None): 1415.6e6 + 62.3e6,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--m2l", default="bf16x3", choices=["fp32", "bf16x3", "tf32x3"])
    ap.add_argument("--m2l-kernel", default="tiles", choices=["tiles", "pairs"],
                    help="tensor-core M2L kernel: target tiles or pair columns")
    ap.add_argument("--eps-svd", type=float, default=None,
                    help="M2L compression tolerance (rank: singular values above eps * max); "
                         "default per workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error-check", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only: no other legs, CPU baseline, error gate or e2e")
    a = ap.parse_args()
    if a.quick:
        a.no_cpu_baseline = a.no_error_check = True
    if a.eps_svd is None:
        a.eps_svd = EPS_SVD.get(a.workload, 1e-7)
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
# CPU oracle legs (cpu_baseline and --impl reference).  The oracle runs as
# it stands: one single-threaded process per host core, each evaluating its
# own seeded sample of the workload's distribution; they start their timed
# evaluations together (a barrier on stdin) and the throughput is the points
# all of them evaluated over the wall time until the last one finished.
# ---------------------------------------------------------------------------
_ORACLE_WORKER = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle.kifmm import KIFMM
from paper_2303_08394_gb300 import workloads as wl
w = wl.WORKLOADS[{workload!r}]
gen = {{"cube": wl.uniform_cube, "sphere": wl.sphere_surface, "gauss": wl.gaussian_mixture,
        "batch": wl.uniform_cube}}[w.kind]
x, q = gen({n}, {seed}, w.nrhs)
f = KIFMM(x, w.p, w.ncrit)
out = {{"n": {n}, "nrhs": w.nrhs, "depth": f.tree.depth, "warm": [], "timed": []}}
for phase, reps in (("warm", {warm}), ("timed", {reps})):
    print("ready", flush=True)
    sys.stdin.readline()
    for i in range(reps):
        t0 = time.perf_counter()
        f.evaluate(q)
        out[phase].append(time.perf_counter() - t0)
print(json.dumps(out), flush=True)
"""


def run_oracle_workers(workload, n, warm, reps, workers):
    """`workers` concurrent oracle processes (seeds 0..workers-1), `warm`
    untimed then `reps` timed evaluations each; returns (wall seconds of the
    timed evaluations, per-worker results)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    procs = []
    for s in range(workers):
        code = _ORACLE_WORKER.format(root=ROOT, workload=workload, n=n, seed=s, warm=warm,
                                     reps=reps)
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True, env=env))

    def barrier():
        for p in procs:
            line = p.stdout.readline()
            if line.strip() != "ready":
                err = p.stderr.read()
                for q in procs:
                    q.kill()
                raise RuntimeError("oracle worker failed:\n" + (line + err)[-2000:])
        t = time.perf_counter()
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        return t

    barrier()            # setup done: warm-up evaluations
    t0 = barrier()       # warm-up done: timed evaluations
    results = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode:
            raise RuntimeError("oracle worker failed:\n" + err[-2000:])
        results.append(json.loads(out.strip().splitlines()[-1]))
    return time.perf_counter() - t0, results


_DIRECT_WORKER = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import direct
from paper_2303_08394_gb300 import workloads as wl
w = wl.WORKLOADS[{workload!r}]
direct.build()
if w.kind == "batch":
    # each sampled target sums over its own problem (the bench's samples)
    sets = w.problem_sets(0)
    parts, t, pairs = [], 0.0, 0
    for i, (xi, qi) in enumerate(sets):
        loc = wl.sample_targets(len(xi), min({m}, len(xi)), i)
        t0 = time.perf_counter()
        parts.append(direct.direct_sum(xi, qi, targets=xi[loc]))
        t += time.perf_counter() - t0
        pairs += len(loc) * len(xi)
    phi = np.concatenate(parts)
    idx = np.arange(len(phi))
else:
    x, q = w.generate(0)
    idx = wl.sample_targets(w.n, {m}, 0)
    t0 = time.perf_counter()
    phi = direct.direct_sum(x, q, targets=x[idx])
    t = time.perf_counter() - t0
    pairs = len(idx) * w.n
np.save({out!r}, phi)
print(json.dumps({{"seconds": t, "threads": direct.num_threads(), "targets": len(idx),
                  "pairs": pairs}}))
"""


def cpu_baseline(workload, w, ref_sampled=None):
    """The oracle KIFMM on every host core (one process per core), plus the
    oracle's OpenMP direct sum of Eq. (1) on the sampled targets of the full
    workload (checked against the bench's own FP64 reference)."""
    import numpy as np
    cores = host_cores()
    wall, res = run_oracle_workers(workload, CPU_SAMPLE_N, 0, 1, cores)
    pts = sum(r["n"] * r["nrhs"] * len(r["timed"]) for r in res)
    per = statistics.median(t for r in res for t in r["timed"])
    line = {"value": pts / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{cores} concurrent single-threaded processes of the FP64 numpy KIFMM "
                       f"(dense M2L), each evaluating its own {CPU_SAMPLE_N:,}-point sample of "
                       f"the workload's distribution (seeds 0..{cores - 1}, p={w.p}, "
                       f"ncrit={w.ncrit}, tree depth {res[0]['depth']} against the full "
                       f"workload's deeper tree); tree and operator setup excluded; "
                       f"{per:.2f} s per evaluate, {wall:.2f} s wall for all")}
    m = w.error_samples or 1000
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "phi.npy")
        env = dict(os.environ)
        env["OMP_NUM_THREADS"] = str(cores)
        r = subprocess.run([sys.executable, "-c", _DIRECT_WORKER.format(
            root=ROOT, workload=workload, m=m, out=out)], capture_output=True, text=True, env=env)
        if r.returncode == 0:
            d = json.loads(r.stdout.strip().splitlines()[-1])
            phi = np.load(out)
            # a batch's targets each see their own problem's sources only
            d["sources"] = w.n
            d["pairs_per_s"] = d["pairs"] / d["seconds"]
            d["targets_per_s"] = d["targets"] / d["seconds"]
            d["what"] = ("oracle/direct.c, FP64 O(N) sum per sampled target over all N sources "
                         "(a batch: over its own problem's), OpenMP over targets")
            if ref_sampled is not None:
                d["max_rel_diff_vs_bench_reference"] = float(
                    np.max(np.abs(phi - ref_sampled)) / np.max(np.abs(ref_sampled)))
            line["direct_sum"] = d
        else:
            line["direct_sum"] = {"error": r.stderr[-500:]}
    return line


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
# accuracy gate: FP64 direct sum of Eq. (1) on sampled targets, computed with
# plain torch FP64 operations on the GPU (sources in chunks); the CPU
# baseline's OpenMP direct sum is checked against it
# ---------------------------------------------------------------------------
def _direct_sampled(x, q, idx, dev, gradient=False, chunk=1 << 15):
    import numpy as np
    import torch
    xs = torch.as_tensor(x, dtype=torch.float64, device=dev)
    qs = torch.as_tensor(np.asarray(q, dtype=np.float64).reshape(len(x), -1), device=dev)
    xt = xs[torch.as_tensor(idx, device=dev)]
    out = torch.zeros((len(idx), 3 if gradient else qs.shape[1]), dtype=torch.float64,
                      device=dev)
    for s in range(0, len(x), chunk):
        d = xs[None, s:s + chunk, :] - xt[:, None, :]          # (targets, sources, 3)
        r = torch.sqrt((d * d).sum(-1))
        inv = torch.where(r > 0, 1.0 / r, torch.zeros_like(r))
        if gradient:
            w3 = inv ** 3 * qs[s:s + chunk, 0][None, :]
            out += torch.einsum("ij,ijk->ik", w3, d)
        else:
            out += inv @ qs[s:s + chunk]
        del d, r, inv
    return (out / (4 * np.pi)).cpu().numpy()


def _batch_samples(sets, per):
    """`per` sampled targets of every problem of a batch, as indices into the
    concatenated points."""
    import numpy as np
    from paper_2303_08394_gb300 import workloads as wl
    out, base = [], 0
    for i, (xi, _) in enumerate(sets):
        out.append(base + wl.sample_targets(len(xi), min(per, len(xi)), i))
        base += len(xi)
    return np.concatenate(out)


def _reference(x, q, idx, dev, sets=None, gradient=False):
    """FP64 direct sum at the points idx; for a batch, each point's sum runs
    over its own problem's sources only."""
    import numpy as np
    if sets is None:
        return _direct_sampled(x, q, idx, dev, gradient=gradient)
    parts, base = [], 0
    for xi, qi in sets:
        sel = idx[(idx >= base) & (idx < base + len(xi))] - base
        if len(sel):
            parts.append(_direct_sampled(xi, qi, sel, dev, gradient=gradient))
        base += len(xi)
    return np.concatenate(parts)


def rel_l2(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


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


def run_batch_leg(a, world, rank, dev, flush, stream):
    """The 256-problem batch (one forest plan: every problem's boxes in the
    same level products, M2L tiles and leaf launches, one graph per
    evaluation) timed with the main line's protocol, its error over each
    sampled target's own problem."""
    import numpy as np
    import torch
    from paper_2303_08394_gb300 import FMMPlan, _native as N
    from paper_2303_08394_gb300 import workloads as wl
    w = wl.WORKLOADS[BATCH_WORKLOAD]
    modes = {"fp32": N.M2L_FP32, "bf16x3": N.M2L_BF16X3, "tf32x3": N.M2L_TF32X3}
    sets = w.problem_sets(rank)
    x, q = w.generate(rank)
    n = len(x)
    t0 = time.perf_counter()
    plan = FMMPlan.batch([xi for xi, _ in sets], w.p, w.ncrit, m2l_mode=modes[a.m2l],
                         eps_svd=EPS_SVD[BATCH_WORKLOAD])
    plan_s = time.perf_counter() - t0
    qd = torch.as_tensor(q.astype(np.float32), device=dev)
    out = torch.empty((n, w.nrhs), dtype=torch.float64, device=dev)
    steps = min(a.steps, 30)
    ms, ph, launches = time_mode(plan, qd, out, flush, stream, steps, a.warmup, world)
    tot = max_over_ranks(sum(ms), world, dev)
    leg = {"workload": w.name, "problems": len(sets), "n": n, "p": w.p, "ncrit": w.ncrit,
           "m2l": a.m2l, "value": job_value(n * w.nrhs, steps, world, tot / 1e3),
           "unit": UNIT, "ms_per_step": tot / steps, "steps": steps,
           "phase_ms": mean_phases(ph), "gpu_launches_per_step": launches,
           "plan_s": plan_s}
    if not a.no_error_check and rank == 0:
        idx = _batch_samples(sets, w.error_samples)
        leg["rel_l2_err"] = rel_l2(out.cpu().numpy()[idx], _reference(x, q, idx, dev, sets))
        leg["error_samples"] = len(idx)
    del plan
    return leg


def run_trials(a, w, dev, flush, stream, value0, err0, seeds=(1, 2, 3, 4)):
    """The same workload on further seeds (new points and charges, a new
    plan each), with the main line's protocol but fewer steps: the spread of
    points/s and error over seeds 0..4 (seed 0 is the main run)."""
    import numpy as np
    import torch
    from paper_2303_08394_gb300 import FMMPlan, _native as N
    from paper_2303_08394_gb300 import workloads as wl
    modes = {"fp32": N.M2L_FP32, "bf16x3": N.M2L_BF16X3, "tf32x3": N.M2L_TF32X3}
    steps = min(a.steps, 20)
    values, errs = [value0], [err0]
    for seed in seeds:
        x, q = w.generate(seed)
        n = len(x)
        plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=modes[a.m2l], eps_svd=a.eps_svd)
        qd = torch.as_tensor(q.astype(np.float32), device=dev)
        out = torch.empty((n, w.nrhs), dtype=torch.float64, device=dev)
        ms, _, _ = time_mode(plan, qd, out, flush, stream, steps, a.warmup, 1)
        values.append(job_value(n * w.nrhs, steps, 1, sum(ms) / 1e3))
        err = None
        if err0 is not None:
            idx = wl.sample_targets(n, w.error_samples or 1000, seed)
            err = rel_l2(out.cpu().numpy()[idx], _reference(x, q, idx, dev))
        errs.append(err)
        del plan, qd, out
    res = {"seeds": [0, *seeds], "value": values, "unit": UNIT,
           "value_mean": statistics.mean(values), "value_std": statistics.stdev(values),
           "steps_per_seed": steps, "rel_l2_err": errs}
    if all(e is not None for e in errs):
        res["rel_l2_err_mean"] = statistics.mean(errs)
        res["rel_l2_err_std"] = statistics.stdev(errs)
    return res


def mean_phases(phases):
    return {k: statistics.mean(ph[k] for ph in phases) for k in phases[0]}


def reference_arm(a, w, config):
    """--impl reference: the FP64 oracle KIFMM, as it stands, on every host
    core (one process per core, each on its own bounded sample)."""
    cores = host_cores()
    n = reference_sample_n(a.warmup + a.steps)
    wall, res = run_oracle_workers(a.workload, n, a.warmup, a.steps, cores)
    pts = sum(r["n"] * r["nrhs"] * len(r["timed"]) for r in res)
    value = pts / wall
    sample = (f"{cores} concurrent single-threaded processes of the FP64 numpy KIFMM (dense "
              f"M2L), each evaluating its own {n:,}-point sample of the workload's "
              f"distribution per step (seeds 0..{cores - 1}); tree and operator setup "
              f"excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * wall / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def m2l_roofline(plan, mode, w, m2l_ms, peaks, peak_src, fp32_peak, sm_mhz):
    """Roofline object of the M2L launch.  Useful flops: 2 k^2 per V pair and
    right-hand side; the tensor-core modes issue three split products per
    pair (counted in `achieved`), over tiles whose rows are not all filled
    (`fill`: V pairs / rows the MMAs process; `mma_flops_per_launch` counts
    the padded rows and the operand width kpad)."""
    import numpy as np
    k = plan.info("rank_m2l")
    kpad = (k + 15) // 16 * 16
    v_pairs = plan.info("v_pairs")
    useful = 2.0 * k * k * v_pairs * w.nrhs
    pairs_kernel = mode != "fp32" and plan.info("m2l_kernel") == 2
    if pairs_kernel:
        # pair columns: M = 128 coefficient rows, N = the item's pairs rounded to 16
        cols = np.diff(plan.array("m2l_item_pair_ptr").astype(np.int64))
        padded = float(((cols + 15) // 16 * 16).sum())
        fill = v_pairs / max(1.0, padded)
        mma_rows = padded * 128.0 / kpad   # in units of kpad-wide rows, as below
    else:
        entries = plan.info("m2l_entries")
        fill = v_pairs / max(1, entries * 128)
        mma_rows = entries * 128.0
    if mode == "fp32":
        tf = useful / (m2l_ms / 1e3) / 1e12
        return {"kernel": "k_m2l_simt", "bound": "alu", "achieved": tf,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak,
                "traffic": TRAFFIC.get(("k_m2l_simt", w.name, mode, kpad)),
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz",
                "flops_per_launch": useful, "ms_per_launch": m2l_ms, "fill": fill}
    tc_peak = peaks["bf16_tflops"] * (1.0 if mode == "bf16x3" else 0.5)
    issued = 3 * useful
    mma = 3 * 2.0 * kpad * kpad * mma_rows * w.nrhs
    return {"kernel": "k_m2l_pc" if pairs_kernel else "k_m2l_tc", "bound": "tensor",
            "achieved": issued / (m2l_ms / 1e3) / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
            "frac": issued / (m2l_ms / 1e3) / 1e12 / tc_peak,
            "traffic": TRAFFIC.get(("k_m2l_tc", w.name, mode, kpad)),
            "peak_source": f"bf16_tflops of {peak_src} (burst)" +
                           ("" if mode == "bf16x3" else " x 1/2 (tf32)"),
            "flops_per_launch": issued, "useful_flops_per_launch": useful,
            "useful_frac_of_bf16_peak": useful / (m2l_ms / 1e3) / 1e12 / peaks["bf16_tflops"],
            "fill": fill, "mma_flops_per_launch": mma,
            "mma_frac": mma / (m2l_ms / 1e3) / 1e12 / tc_peak,
            "ms_per_launch": m2l_ms}


def main():
    a = parse()
    rank, world, local = dist_env()
    from paper_2303_08394_gb300 import workloads as wl
    w = wl.WORKLOADS[a.workload]
    config = {"workload": w.name, "n": w.n, "p": w.p, "ncrit": w.ncrit, "nrhs": w.nrhs,
              "points": w.kind, "m2l": a.m2l, "m2l_kernel": a.m2l_kernel, "eps_svd": a.eps_svd,
              "graph": "CUDA graph replay on a side stream",
              "l2_flush": "256 MB write before every step",
              "per_rank": "independent problem (seed = rank)"}

    if a.impl == "reference":
        if rank == 0:
            reference_arm(a, w, config)
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
    sets = w.problem_sets(rank) if w.kind == "batch" else None
    x, q = w.generate(rank)
    n = len(x)  # a batch's total depends on the seed
    t0 = time.perf_counter()
    if sets is not None:
        plan = FMMPlan.batch([xi for xi, _ in sets], w.p, w.ncrit, m2l_mode=modes[a.m2l],
                             eps_svd=a.eps_svd)
    else:
        plan = FMMPlan(x, w.p, w.ncrit, m2l_mode=modes[a.m2l], eps_svd=a.eps_svd)
    plan.set_m2l_kernel(0 if a.m2l_kernel == "pairs" else 1)
    plan_s = time.perf_counter() - t0
    qd = torch.as_tensor(q.astype(np.float32), device=dev)
    out = torch.empty((n, w.nrhs), dtype=torch.float64, device=dev)
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
    value = job_value(n * w.nrhs, a.steps, world, total_ms / 1e3)

    # accuracy gate on sampled targets (FP64 direct sum; for a batch, over
    # each target's own problem)
    err = idx = ref = None
    if not a.no_error_check and rank == 0:
        idx = (_batch_samples(sets, w.error_samples) if sets is not None
               else wl.sample_targets(n, w.error_samples or 1000, 0))
        got = out.cpu().numpy()[idx]
        ref = _reference(x, q, idx, dev, sets)
        err = rel_l2(got, ref)

    # the other M2L modes on the same plan, same protocol: the plain FP32
    # path ("mixed vs FP32") and TF32x3 (FP32-like accuracy)
    legs = {}
    if not a.quick:
        for name in ("fp32", "tf32x3", "bf16x3"):
            if name == a.m2l:
                continue
            plan.set_m2l_mode(modes[name])
            l_ms, l_ph, _ = time_mode(plan, qd, out, flush, stream, a.steps, a.warmup, world)
            l_tot = max_over_ranks(sum(l_ms), world, dev)
            leg = {"value": job_value(n * w.nrhs, a.steps, world, l_tot / 1e3),
                   "ms_per_step": l_tot / a.steps, "phase_ms": mean_phases(l_ph)}
            if ref is not None:
                leg["rel_l2_err"] = rel_l2(out.cpu().numpy()[idx], ref)
            leg["value_over_this_leg"] = value / leg["value"]
            legs[name] = leg
        plan.set_m2l_mode(modes[a.m2l])

    # gradients of the potentials (fmm_evaluate_gradient), same protocol, the
    # gradients only
    gradient = None
    if not a.quick and w.nrhs == 1:
        gout = torch.empty((n, 1, 3), dtype=torch.float64, device=dev)
        g_steps = min(a.steps, 50)
        g_ms, g_ph, g_launch = time_mode(
            plan, qd, out, flush, stream, g_steps, a.warmup, world,
            call=lambda: plan.evaluate_gradient(qd, grad_out=gout, potentials=False,
                                                stream=stream))
        g_tot = max_over_ranks(sum(g_ms), world, dev)
        gradient = {"value": job_value(n, g_steps, world, g_tot / 1e3), "unit": UNIT,
                    "ms_per_step": g_tot / g_steps, "steps": g_steps,
                    "phase_ms": mean_phases(g_ph), "gpu_launches": g_launch * g_steps}
        if idx is not None:
            got = gout.cpu().numpy()[idx, 0, :]
            gref = _reference(x, q, idx, dev, sets, gradient=True)
            gradient["rel_l2_err"] = rel_l2(got, gref)

    # rooflines from the library's per-phase CUDA events (each phase is
    # timed on `stream`, the stream its kernels run on)
    peaks, peak_src = load_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s
    p2p_pairs = plan.info("p2p_pairs")
    surf_pairs = plan.info("surf_pairs")
    wx_pairs = plan.info("wx_direct_pairs")
    ph = mean_phases(phases)
    m2l_roof = m2l_roofline(plan, a.m2l, w, ph["m2l"], peaks, peak_src, fp32_peak, sm_mhz)
    leaf_ms = ph["leaf"]
    # every (target, source) pair the leaf kernel evaluates: the near field
    # over U, the small W / X leaves taken directly, L2P from the leaf's own
    # downward surface and M2P from the other W surfaces; the same
    # arithmetic per pair
    leaf_pairs = p2p_pairs + wx_pairs + surf_pairs
    near_flops = (8.0 + 2.0 * w.nrhs) * leaf_pairs
    leaf_tf = near_flops / (leaf_ms / 1e3) / 1e12
    leaf_roof = {"kernel": "k_eval", "bound": "alu", "achieved": leaf_tf, "peak": fp32_peak,
                 "unit": "TFLOP/s", "frac": leaf_tf / fp32_peak,
                 "traffic": TRAFFIC.get(("k_eval", w.name, a.m2l, None)),
                 "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz "
                                "(derived; no measured FP32 figure)",
                 "flops_per_launch": near_flops, "ms_per_launch": leaf_ms,
                 "pairs": {"near_field": p2p_pairs, "direct_w_x": wx_pairs,
                           "l2p_m2p": surf_pairs},
                 "note": "8 + 2 nrhs flops per evaluated pair (near field, direct W/X "
                         "leaves, L2P, M2P); "
                         "the leaf pass (its width-group launches) is timed as one phase"}
    dominant = m2l_roof if ph["m2l"] >= leaf_ms else leaf_roof
    for name, leg in legs.items():
        leg["roofline_m2l"] = m2l_roofline(plan, name, w, leg["phase_ms"]["m2l"], peaks,
                                           peak_src, fp32_peak, sm_mhz)
    if gradient is not None:
        # potential + gradient: 8 (r^2, as above) + 2 (potential) + 3 (q / r^3)
        # + 6 (three FMAs) flops per near-field pair
        g_leaf = gradient["phase_ms"]["leaf"]
        g_flops = 19.0 * leaf_pairs
        g_tf = g_flops / (g_leaf / 1e3) / 1e12
        gradient["roofline"] = {"kernel": "k_eval (gradient variant)", "bound": "alu",
                                "achieved": g_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                                "frac": g_tf / fp32_peak,
                                "traffic": TRAFFIC.get(("k_eval_grad", w.name, a.m2l, None)),
                                "flops_per_launch": g_flops, "ms_per_launch": g_leaf,
                                "note": "19 flops per evaluated pair (near field, direct "
                                        "W/X leaves, L2P, M2P)"}

    # the same workload on seeds 1..4 (one rank only): mean and spread
    trials = None
    if not a.quick and world == 1 and w.kind != "batch":
        trials = run_trials(a, w, dev, flush, stream, value, err)

    # the batch of 256 independent problems, same protocol
    batch = None
    if not a.quick and w.kind != "batch":
        batch = run_batch_leg(a, world, rank, dev, flush, stream)

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
                "legs": legs, "fp32": legs.get("fp32"), "gradient": gradient,
                "batch": batch, "trials": trials,
                "roofline": dominant, "rooflines": {"m2l": m2l_roof, "leaf": leaf_roof},
                "phase_ms": ph, "e2e": e2e,
                "gpu_launches": launches_per_step * a.steps, "clocks": clk,
                "plan_s": plan_s, "wall_s_timed_region": wall,
                "tree": {key: plan.info(key) for key in
                         ("nodes", "leaves", "depth", "rank_m2l", "v_pairs", "u_pairs",
                          "p2p_pairs", "wx_direct_pairs", "surf_pairs", "m2l_tiles",
                          "m2l_entries")},
                "peaks": peak_src}
        if world == 1 and not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(a.workload, w, ref)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(plan, q, w, a, world, dev):
    import numpy as np
    import torch
    import torch.distributed as dist
    n = len(q)
    qh = torch.tensor(q.astype(np.float32)).pin_memory()
    oh = torch.empty((n, w.nrhs), dtype=torch.float64).pin_memory()
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
    return {"value": job_value(n * w.nrhs, steps, world, e2e_s), "unit": UNIT,
            "h2d_bytes_per_step": n * w.nrhs * 4, "d2h_bytes_per_step": n * w.nrhs * 8,
            "steps": steps}


if __name__ == "__main__":
    main()
