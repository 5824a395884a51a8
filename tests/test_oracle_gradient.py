"""Pins of the FP64 gradient oracles (direct sum and KIFMM leaf step): the
gradient of the potential of Eq. (1) with respect to the target position.

Each pin comes from outside the gradient code: a hand-worked value, central
differences of the potential routines, symmetry, the vanishing Laplacian of
a harmonic potential, and the shell theorem; for the KIFMM, the one-leaf
reduction to the direct sum, convergence in p, linearity, and central
differences of its own L2P and M2P potentials.
"""
import numpy as np
import pytest

from oracle.direct import direct_gradient, direct_sum
from oracle import kifmm as ok
from paper_2303_08394_gb300 import workloads as wl


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_worked_value_one_charge():
    # q = 3 at the origin, target (0, 0, 2): phi = 3 / (8 pi), and moving the
    # target away lowers it: d phi / dz = -3 / (16 pi)
    g = direct_gradient(np.zeros((1, 3)), np.array([3.0]), np.array([[0.0, 0.0, 2.0]]))
    np.testing.assert_allclose(g[0], [0.0, 0.0, -3.0 / (16.0 * np.pi)], rtol=1e-15, atol=1e-18)
    # target (1, 2, 2), |r| = 3: gradient = -q r / (4 pi 27)
    g = direct_gradient(np.zeros((1, 3)), np.array([3.0]), np.array([[1.0, 2.0, 2.0]]))
    np.testing.assert_allclose(g[0], np.array([-1.0, -2.0, -2.0]) / (36.0 * np.pi), rtol=1e-15)


def test_central_differences_of_the_potential():
    x, q = wl.uniform_cube(400, 3, nrhs=2)
    y = np.random.default_rng(4).uniform(1.5, 2.5, size=(50, 3))  # away from every source
    g = direct_gradient(x, q, y)
    h = 1e-4
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (direct_sum(x, q, y + e) - direct_sum(x, q, y - e)) / (2 * h)
        np.testing.assert_allclose(g[:, :, k], fd, rtol=1e-6, atol=1e-9)


def test_symmetry_and_columns():
    x = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    g = direct_gradient(x, np.array([1.0, 1.0]), np.array([[0.0, 0.0, 0.0], [0.7, 0.0, 0.0]]))
    np.testing.assert_array_equal(g[0], [0.0, 0.0, 0.0])  # midpoint of two equal charges
    assert g[1, 0] < 0 and g[1, 1] == 0.0 and g[1, 2] == 0.0
    xs, q = wl.gaussian_mixture(300, 5, nrhs=3)
    G = direct_gradient(xs, q)
    for r in range(3):
        np.testing.assert_array_equal(G[:, r, :], direct_gradient(xs, q[:, r]))


def test_laplacian_vanishes_away_from_charges():
    x, q = wl.uniform_cube(300, 6)
    q = q[:, 0]
    y = np.random.default_rng(7).uniform(2.0, 3.0, size=(20, 3))
    h = 1e-3
    div = np.zeros(len(y))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        div += (direct_gradient(x, q, y + e)[:, k] - direct_gradient(x, q, y - e)[:, k]) / (2 * h)
    scale = np.abs(direct_gradient(x, q, y)).max()
    assert np.abs(div).max() <= 1e-5 * scale


def test_shell_theorem():
    # equal charges on a Fibonacci sphere of radius 1: no field inside, the
    # field of the total charge at the centre outside
    n = 4000
    k = np.arange(n) + 0.5
    th = np.arccos(1 - 2 * k / n)
    ph = np.pi * (1 + 5 ** 0.5) * k
    x = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], axis=1)
    q = np.full(n, 1.0 / n)
    outside = np.array([[0.0, 0.0, 3.0], [2.0, 2.0, 1.0]])
    g = direct_gradient(x, q, outside)
    r = np.linalg.norm(outside, axis=1)
    want = -outside / (4 * np.pi * r[:, None] ** 3)
    # a 4000-point shell matches the point charge to ~2e-6 outside
    np.testing.assert_allclose(g, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())
    inside = np.array([[0.0, 0.0, 0.0], [0.2, -0.1, 0.3]])
    assert np.abs(direct_gradient(x, q, inside)).max() <= 1e-3 / (4 * np.pi)


def test_kifmm_single_leaf_is_direct():
    x, q = wl.uniform_cube(50, 8)
    phi, g = ok.KIFMM(x, 4, 64).evaluate(q[:, 0], gradient=True)
    np.testing.assert_allclose(g, direct_gradient(x, q[:, 0]), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(phi, direct_sum(x, q[:, 0]), rtol=1e-12)


def test_kifmm_gradient_converges_with_p():
    x, q = wl.uniform_cube(2000, 9)
    ref = direct_gradient(x, q[:, 0])
    errs = [rel(ok.KIFMM(x, p, 32).evaluate(q[:, 0], gradient=True)[1], ref) for p in (3, 4, 5, 6)]
    assert all(b < 0.4 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-5


def test_kifmm_gradient_linearity_and_columns():
    x, q = wl.gaussian_mixture(1500, 10, nrhs=2)
    fmm = ok.KIFMM(x, 4, 16)
    _, g2 = fmm.evaluate(q, gradient=True)
    _, ga = fmm.evaluate(q[:, 0], gradient=True)
    _, gb = fmm.evaluate(q[:, 1], gradient=True)
    # (the BLAS products of one and two columns round differently)
    np.testing.assert_allclose(g2[:, 0, :], ga, rtol=1e-9, atol=1e-10 * np.abs(ga).max())
    _, gs = fmm.evaluate(2.0 * q[:, 0] - 3.0 * q[:, 1], gradient=True)
    np.testing.assert_allclose(gs, 2.0 * ga - 3.0 * gb, rtol=1e-9, atol=1e-9 * np.abs(gs).max())


def test_kifmm_leaf_gradients_are_derivatives_of_leaf_potentials():
    """The L2P and M2P gradients at a leaf's points equal central
    differences of the same surfaces' potentials (the potential kernel moved
    by +-h), for every leaf with a downward density or a W list."""
    x, q = wl.gaussian_mixture(3000, 11)
    fmm = ok.KIFMM(x, 5, 12)
    fmm.evaluate(q[:, 0])
    t = fmm.tree
    h = 1e-5
    checked = 0
    for b in t.leaves:
        xt = t.x[t.points[b]]
        pieces = []
        if b[0] >= 2:
            pieces.append((fmm._surface(b, fmm.alpha_outer), fmm.down[b]))
        for a in fmm.W.get(b, ()):
            pieces.append((fmm._surface(a, fmm.alpha_inner), fmm.up[a]))
        for srf, dens in pieces:
            g = np.einsum("ijk,jr->irk", ok.laplace_gradient_kernel(xt, srf), dens)
            for k in range(3):
                e = np.zeros(3)
                e[k] = h
                fd = (ok.laplace_kernel(xt + e, srf) @ dens - ok.laplace_kernel(xt - e, srf) @ dens) / (2 * h)
                np.testing.assert_allclose(g[:, :, k], fd, rtol=1e-5, atol=1e-7 * np.abs(g).max())
            checked += 1
    assert checked > 50
