"""The element-wise parity check (tests/parity.py) catches what a norm over
all targets misses: one leaf of 64 targets off by 10x the bar among 10^4
targets, while the relative L2 error stays under the bar."""
import numpy as np
import pytest

from tests.parity import ELEM_C, check, elem_ratio, rel


def test_localized_error_fails_only_the_element_bound():
    rng = np.random.default_rng(5)
    ref = rng.standard_normal(10_000)
    bar = 1e-6
    got = ref + 0.3 * bar * rng.standard_normal(10_000) * np.abs(ref)
    e, r = check(got, ref, bar)           # ordinary rounding noise passes
    assert e < bar and r < ELEM_C
    bad = got.copy()
    bad[640:704] = ref[640:704] * (1 + 10 * bar)   # one wrong leaf
    assert rel(bad, ref) < bar                     # the norm alone misses it
    assert elem_ratio(bad, ref, bar) > ELEM_C
    with pytest.raises(AssertionError, match="worst target"):
        check(bad, ref, bar)


def test_relative_l2_bar_still_applies():
    ref = np.ones(100)
    with pytest.raises(AssertionError, match="relative L2"):
        check(ref * (1 + 2e-6), ref, 1e-6)
