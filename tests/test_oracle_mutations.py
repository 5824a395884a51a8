"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in a copy of the oracle (on the CPU) and checks
that the accuracy or coverage pin it should trip does trip.
"""
import numpy as np

from oracle import kifmm
from oracle.direct import direct_sum
from paper_2303_08394_gb300 import workloads as wl


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sphere():
    x, q = wl.sphere_surface(2500, 21)
    return x, q[:, 0], direct_sum(x, q[:, 0])


def test_correct_oracle_passes_the_bar():
    x, q, ref = _sphere()
    assert rel(kifmm.fmm(x, q, p=5, ncrit=12), ref) < 3e-5


def test_swapped_surface_radii_fail():
    x, q, ref = _sphere()
    bad = kifmm.fmm(x, q, p=5, ncrit=12, alpha_inner=2.95, alpha_outer=1.05)
    assert rel(bad, ref) > 1e-3


def test_transposed_m2l_fails():
    class T(kifmm.KIFMM):
        def _m2l_matrix(self, b, a):
            return super()._m2l_matrix(b, a).T
    x, q, ref = _sphere()
    assert rel(T(x, 5, 12).evaluate(q), ref) > 1e-3


def test_dropped_lists_fail():
    x, q, ref = _sphere()
    for name in ("X", "W", "V"):
        f = kifmm.KIFMM(x, 5, 12)
        setattr(f, name, {})
        assert rel(f.evaluate(q), ref) > 1e-3, name


def test_wrong_v_definition_breaks_coverage():
    """V lists that also keep adjacent children double-count pairs that U
    already holds; the coverage pin sees it."""
    from tests.test_oracle_tree import _coverage
    x, _ = wl.uniform_cube(1500, 22)
    tree = kifmm.Octree(x, 16)
    U, V, W, X = kifmm.build_lists(tree)
    bad_v = {}
    for b in tree.nonempty:
        if b[0] < 2:
            continue
        out = []
        for col in kifmm._colleagues(tree, kifmm._parent(b)):
            if not tree.leaf[col]:
                out += [c for c in kifmm._children(col)
                        if c in tree.nonempty and c != b]
        bad_v[b] = out
    assert _coverage(tree, (U, V, W, X)) == 0
    assert _coverage(tree, (U, bad_v, W, X)) > 0


def test_gradient_kernel_sign_fails(monkeypatch):
    """A sign error in the kernel's target-gradient: the KIFMM gradient then
    disagrees with the direct gradient (itself pinned by central
    differences of the direct potential)."""
    from oracle.direct import direct_gradient
    x, q, _ = _sphere()
    ref = direct_gradient(x, q)
    f = kifmm.KIFMM(x, 5, 12)
    _, good = f.evaluate(q, gradient=True)
    assert rel(good, ref) < 3e-4
    flipped = kifmm.laplace_gradient_kernel
    monkeypatch.setattr(kifmm, "laplace_gradient_kernel", lambda t, s: -flipped(t, s))
    _, bad = f.evaluate(q, gradient=True)
    assert rel(bad, ref) > 1e-1


def test_dropped_l2l_fails(monkeypatch):
    """Every box's parent reported at level 1 during the evaluation: the
    downward pass loses every L2L term below level 2."""
    x, q, ref = _sphere()
    f = kifmm.KIFMM(x, 5, 12)       # tree and lists built with the true parents
    monkeypatch.setattr(kifmm, "_parent", lambda key: (1, 0, 0, 0))
    assert rel(f.evaluate(q), ref) > 1e-3


def test_wrong_level_width_fails(monkeypatch):
    """Surfaces sized for the level below (half the box): the check and
    equivalent surfaces no longer enclose what they represent."""
    x, q, ref = _sphere()
    f = kifmm.KIFMM(x, 5, 12)
    true_width = kifmm.Octree.box_half_width
    monkeypatch.setattr(kifmm.Octree, "box_half_width",
                        lambda self, level: true_width(self, level + 1))
    assert rel(f.evaluate(q), ref) > 1e-3
