"""Pins for the FP64 KIFMM oracle.

Against the direct sum (itself pinned to closed forms): the single-leaf case
equals it to round-off and the error falls with p.  Against the mathematics:
linearity in the charges, invariance under dyadic translation, 1/s scaling.
Per operator: each equivalent density reproduces the field it stands for,
so a swapped radius, a transposed matrix or a dropped term fails here.
"""
import numpy as np
import pytest

from oracle.direct import direct_sum
from oracle.kifmm import KIFMM, laplace_kernel, fmm, _parent, _children
from paper_2303_08394_gb300 import workloads as wl


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_single_leaf_is_direct_sum():
    x, q = wl.uniform_cube(90, 1)
    phi = fmm(x, q, p=4, ncrit=100)
    np.testing.assert_allclose(phi, direct_sum(x, q), rtol=1e-13, atol=0)


def test_error_falls_with_p():
    x, q = wl.uniform_cube(2000, 2)
    ref = direct_sum(x, q)
    errs = [rel(fmm(x, q, p=p, ncrit=24), ref) for p in (3, 4, 5, 6, 7, 8)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    # roughly geometric: each order gains at least a factor 1.5 up to p=7
    assert all(e2 < e1 / 1.5 for e1, e2 in zip(errs[:-1], errs[1:-1])), errs
    assert errs[0] < 3e-3 and errs[-1] < 5e-7, errs


def test_adaptive_tree_accuracy():
    x, q = wl.sphere_surface(4000, 3)
    f = KIFMM(x, 6, 16)
    assert f.W and f.X, "sphere tree must exercise M2P and P2L"
    assert rel(f.evaluate(q), direct_sum(x, q)) < 2e-5


def test_linearity_in_charges():
    x, q = wl.gaussian_mixture(2000, 4, nrhs=2)
    f = KIFMM(x, 5, 16)
    a, b = 0.75, -2.5
    lhs = f.evaluate(a * q[:, 0] + b * q[:, 1])
    rhs = a * f.evaluate(q[:, 0]) + b * f.evaluate(q[:, 1])
    # exact up to rounding amplified by the kept condition number (~1e7)
    assert rel(lhs, rhs) < 1e-9
    both = f.evaluate(q)
    np.testing.assert_allclose(both[:, 1], f.evaluate(q[:, 1]), rtol=1e-9,
                               atol=1e-9 * np.abs(both).max())


def test_translation_and_scaling():
    x, q = wl.sphere_surface(1500, 5)
    phi = fmm(x, q, p=5, ncrit=12)
    shifted = fmm(x + np.array([0.5, -0.25, 2.0]), q, p=5, ncrit=12)
    assert rel(shifted, phi) < 1e-9
    scaled = fmm(2.0 * x, q, p=5, ncrit=12)
    assert rel(scaled, phi / 2.0) < 1e-9


def test_single_charge_far_field():
    x, _ = wl.uniform_cube(2000, 6)
    q = np.zeros(len(x))
    q[17] = 1.5
    phi = fmm(x, q, p=6, ncrit=20)
    r = np.linalg.norm(x - x[17], axis=1)
    far = r > 0.5
    np.testing.assert_allclose(phi[far], 1.5 / (4 * np.pi * r[far]), rtol=1e-5)


def _far_points(centre, h, count=64, radius=4.0):
    rng = np.random.default_rng(0)
    d = rng.standard_normal((count, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return centre + radius * h * d


def test_upward_densities_reproduce_source_field():
    """P2M and M2M: the upward equivalent density of a box, evaluated outside
    its upward check surface, equals the field of the points it holds."""
    x, q = wl.gaussian_mixture(3000, 7)
    q = q[:, 0]
    f = KIFMM(x, 6, 16)
    f.evaluate(q)
    t = f.tree
    checked = 0
    for b, dens in f.up.items():
        if checked >= 40:
            break
        c, h = t.box_centre(b), t.box_half_width(b[0])
        y = _far_points(c, h)
        ue = c + f.alpha_inner * h * f.surf
        approx = laplace_kernel(y, ue) @ dens[:, 0]
        idx = t.points[b]
        exact = laplace_kernel(y, x[idx]) @ q[idx]
        assert rel(approx, exact) < 1e-4, (b, t.leaf[b])
        checked += 1


def _far_sources_of_leaf(f, b):
    """Indices of the points whose field reaches leaf b through its local
    (downward) expansion: all points except those of U(b) leaves and of the
    boxes in W(b), and -- when b takes its X list directly (a leaf with no
    more points than a surface, under direct_wx) -- of the X(b) leaves."""
    t = f.tree
    excl = set()
    for a in f.U[b]:
        excl.update(t.points[a].tolist())
    for a in f.W.get(b, ()):
        excl.update(t.points[a].tolist())
    if f.direct_wx and len(t.points[b]) <= len(f.surf):
        for a in f.X.get(b, ()):
            excl.update(t.points[a].tolist())
    return np.array(sorted(set(range(len(t.x))) - excl), dtype=np.int64)


@pytest.mark.parametrize("direct_wx", [True, False])
def test_downward_density_reproduces_far_field(direct_wx):
    """M2L, P2L and L2L together: a leaf's downward density evaluated at its
    own points equals the direct field of its far sources."""
    x, q = wl.sphere_surface(3000, 8)
    q = q[:, 0]
    f = KIFMM(x, 6, 12, direct_wx=direct_wx)
    f.evaluate(q)
    t = f.tree
    leaves = [b for b in t.leaves if b[0] >= 2]
    rng = np.random.default_rng(1)
    for b in rng.choice(len(leaves), size=25, replace=False):
        b = leaves[b]
        tidx = t.points[b]
        src = _far_sources_of_leaf(f, b)
        exact = laplace_kernel(x[tidx], x[src]) @ q[src]
        de = t.box_centre(b) + f.alpha_outer * t.box_half_width(b[0]) * f.surf
        approx = laplace_kernel(x[tidx], de) @ f.down[b][:, 0]
        assert rel(approx, exact) < 1e-4, b


def test_near_plus_far_split():
    x, q = wl.uniform_cube(2000, 9)
    q = q[:, 0]
    f = KIFMM(x, 5, 20)
    phi = f.evaluate(q)
    np.testing.assert_allclose(phi, (f.near + f.far)[:, 0])
    # near field alone is the direct sum over U-list leaves, checked by brute force
    t = f.tree
    b = t.leaves[3]
    src = np.concatenate([t.points[a] for a in f.U[b]])
    tidx = t.points[b]
    np.testing.assert_allclose(f.near[tidx, 0],
                               direct_sum(x[src], q[src], targets=x[tidx]),
                               rtol=1e-12)


def test_duplicate_points_and_tiny_inputs():
    x, q = wl.uniform_cube(400, 10)
    x[5] = x[6]                     # coincident pair
    phi = fmm(x, q, p=5, ncrit=10)
    assert rel(phi, direct_sum(x, q)) < 1e-4
    one = fmm(np.array([[0.2, 0.3, 0.4]]), np.array([1.0]), p=4, ncrit=1)
    assert one.shape == (1,) and one[0] == 0.0


def test_direct_wx_rule_is_exact_for_its_terms():
    """The direct_wx reading: small W boxes and the X lists of small leaves
    interact through their points.  On clustered points (W and X lists in
    use, many small leaves) both forms stay within the method's error of the
    direct sum, the direct form is no less accurate, and the leaf step's W
    part changes only where the rule applies."""
    x, q = wl.gaussian_mixture(3000, 21)
    q = q[:, 0]
    ref = direct_sum(x, q)
    f1 = KIFMM(x, 5, 16, direct_wx=True)
    f0 = KIFMM(x, 5, 16, direct_wx=False)
    phi1, phi0 = f1.evaluate(q), f0.evaluate(q)
    t = f1.tree
    ne = len(f1.surf)
    small_w = sum(1 for b in t.leaves for a in f1.W.get(b, ())
                  if t.is_leaf(a) and len(t.points[a]) <= ne)
    small_x = sum(len(f1.X.get(b, ())) for b in t.leaves if len(t.points[b]) <= ne)
    assert small_w > 0 and small_x > 0
    e1, e0 = rel(phi1, ref), rel(phi0, ref)
    assert e0 < 1e-4 and e1 <= e0 * 1.02, (e1, e0)
    # identical near field; the far parts differ by at most the method's error
    np.testing.assert_array_equal(f1.near, f0.near)
    assert rel(f1.far[:, 0], f0.far[:, 0]) < 1e-3
