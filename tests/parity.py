"""Parity checks shared by the GPU tests: a relative L2 bar over all targets
and, beside it, a bound on every single target.

A norm over all targets hides a localized mistake: one wrong leaf of 64
targets among 10^4 moves the relative L2 error by only about 0.08 times that
leaf's own relative error.  So every comparison also bounds each target:

    max_j |got_j - ref_j|  <=  c * bar * rms(ref)

with rms(ref) the root mean square of the reference over the compared
targets.  A leaf whose targets are off by 10x the bar (relative to their own
potentials, which sit near rms(ref)) fails it whenever c < 10.

c is set from the error distributions measured on the CPU oracle itself
(max |error| / rms(error) of the FP64 KIFMM against the FP64 direct sum on
the test cases: 6.7 (cube, p = 4), 10.4 (cube, p = 6), 14.0 (sphere,
p = 5), 9.0 (Gaussians, p = 6), 7.6 (sphere, p = 7)):

* ELEM_C = 8 against the oracle KIFMM or another GPU evaluation: the
  difference is FP32 rounding spread over the whole pipeline, whose tail is
  that of a sum of many small terms, and the measured relative errors sit
  at a third of the bars or below;
* ELEM_C_DIRECT = 16 against the FP64 direct sum: the difference is then
  the method's truncation error, whose tail reaches 14 times its own rms;
* ELEM_C_GRAD = 24 for gradients of the potential: their magnitudes are
  heavy-tailed (|grad phi| grows as q / r^2 near close pairs, and the error
  of a target scales with its own gradient), so the tails are longer: the
  oracle's gradient against the FP64 direct gradient has max / rms error
  ratios of 17.6 (cube, p = 5), 19.6 (Gaussians, p = 6) and 13.7 (sphere,
  p = 4); the GPU gradient against the oracle's measured 8.3-13.6 x bar.
"""
from __future__ import annotations

import numpy as np

ELEM_C = 8.0
ELEM_C_DIRECT = 16.0
ELEM_C_GRAD = 24.0


def rel(a, b):
    """Relative L2 error of a against b."""
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def elem_ratio(got, ref, bar):
    """max_j |got_j - ref_j| / (bar * rms(ref))."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rms = float(np.sqrt(np.mean(ref * ref)))
    return float(np.max(np.abs(got - ref))) / (bar * rms)


def check(got, ref, bar, c=ELEM_C, what=""):
    """Assert rel(got, ref) <= bar and every target within c * bar * rms(ref);
    returns (relative L2 error, element ratio) for printing."""
    e = rel(got, ref)
    r = elem_ratio(got, ref, bar)
    assert e <= bar, f"{what}: relative L2 {e:.3e} > bar {bar:.1e}"
    assert r <= c, (f"{what}: worst target off by {r:.2f} x bar x rms(ref) "
                    f"(limit {c}); relative L2 {e:.3e}")
    return e, r
