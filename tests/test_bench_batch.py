"""The bench's batch workload helpers on CPU: each sampled target of a batch
is compared with the direct sum over its own problem only."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def test_batch_samples_and_reference_stay_within_each_problem():
    import bench
    from oracle.direct import direct_sum
    from paper_2303_08394_gb300 import workloads as wl
    sets = wl.batch_problems(4, 3, lo=40, hi=300)
    x = np.concatenate([a for a, _ in sets])
    q = np.concatenate([b for _, b in sets])
    idx = bench._batch_samples(sets, 5)
    sizes = np.array([len(a) for a, _ in sets])
    starts = np.concatenate([[0], np.cumsum(sizes)])
    # five distinct targets inside every problem, in order
    for i in range(len(sets)):
        sel = idx[(idx >= starts[i]) & (idx < starts[i + 1])]
        assert len(sel) == 5 and len(np.unique(sel)) == 5
    assert np.all(np.diff(idx) > 0)
    ref = bench._reference(x, q, idx, torch.device("cpu"), sets)
    want = np.concatenate([
        direct_sum(a, b, targets=a[idx[(idx >= s0) & (idx < s1)] - s0])
        for (a, b), s0, s1 in zip(sets, starts[:-1], starts[1:])]).reshape(ref.shape)
    np.testing.assert_allclose(ref, want, rtol=1e-12, atol=0)
    # and not against the whole concatenation
    whole = direct_sum(x, q, targets=x[idx]).reshape(ref.shape)
    assert np.max(np.abs(whole - want)) > 1e-3 * np.max(np.abs(want))


def test_batch_leg_names_a_batch_workload_with_its_tolerance():
    import bench
    from paper_2303_08394_gb300 import workloads as wl
    w = wl.WORKLOADS[bench.BATCH_WORKLOAD]
    assert w.kind == "batch" and w.problems == 256
    assert bench.BATCH_WORKLOAD in bench.EPS_SVD
    assert callable(bench.run_batch_leg)


def test_trials_use_four_more_seeds_of_the_same_workload():
    import inspect
    import bench
    sig = inspect.signature(bench.run_trials)
    assert sig.parameters["seeds"].default == (1, 2, 3, 4)
