"""Pins for the FP64 direct-sum oracle of Eq. (1).

Each test checks the oracle against something other than its own formula:
closed forms, Newton's shell theorem, symmetry and homogeneity of the kernel,
and a pure-Python enumeration on tiny inputs.
"""
import math

import numpy as np
import pytest

from oracle.direct import direct_sum


def test_cube_vertex_closed_form(golden):
    vals = {k: float(v) for k, v in golden("cube_charges.txt")}
    x = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)],
                 dtype=np.float64)
    phi = direct_sum(x, np.ones(8))
    np.testing.assert_allclose(phi, vals["vertex"], rtol=1e-15)
    centre = direct_sum(x, np.ones(8), targets=np.array([[0.5, 0.5, 0.5]]))
    np.testing.assert_allclose(centre, vals["centre"], rtol=1e-15)


def test_single_charge_closed_form():
    src = np.array([[0.1, -0.2, 0.3]])
    tgt = np.array([[1.1, -0.2, 0.3], [0.1, 2.2, 0.3], [0.1, -0.2, -3.7]])
    phi = direct_sum(src, [2.5], targets=tgt)
    np.testing.assert_allclose(phi, 2.5 / (4 * np.pi * np.array([1.0, 2.4, 4.0])),
                               rtol=1e-15)


def _fibonacci_sphere(n, radius):
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    phi = np.pi * (1.0 + 5 ** 0.5) * k
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def test_shell_theorem():
    """A uniformly charged shell acts outside as a point charge at its centre
    and is at constant potential Q/(4 pi R) inside."""
    n, radius, total = 20000, 0.7, 3.0
    shell = _fibonacci_sphere(n, radius)
    q = np.full(n, total / n)
    outside = np.array([[2.0, 0.0, 0.0], [0.0, -1.5, 0.5], [1.0, 1.0, 1.0]])
    inside = np.array([[0.0, 0.0, 0.0], [0.2, -0.1, 0.05]])
    d = np.linalg.norm(outside, axis=1)
    np.testing.assert_allclose(direct_sum(shell, q, targets=outside),
                               total / (4 * np.pi * d), rtol=1e-6)
    np.testing.assert_allclose(direct_sum(shell, q, targets=inside),
                               total / (4 * np.pi * radius), rtol=1e-4)


def test_brute_force_enumeration():
    rng = np.random.default_rng(7)
    x = rng.random((9, 3))
    q = rng.standard_normal((9, 2))
    ref = np.zeros((9, 2))
    for j in range(9):
        for i in range(9):
            if i != j:
                ref[j] += q[i] / (4 * math.pi * math.dist(x[i], x[j]))
    np.testing.assert_allclose(direct_sum(x, q), ref, rtol=1e-13, atol=1e-15)


def test_self_and_coincident_points_skipped():
    x = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    phi = direct_sum(x, [1.0, 2.0, 4.0])
    # each of the two coincident points sees only the charge at distance 1
    np.testing.assert_allclose(phi[:2], 4.0 / (4 * np.pi), rtol=1e-15)
    np.testing.assert_allclose(phi[2], 3.0 / (4 * np.pi), rtol=1e-15)


def test_homogeneity_translation_and_symmetry():
    rng = np.random.default_rng(3)
    x = rng.random((200, 3))
    q = rng.uniform(-1, 1, 200)
    phi = direct_sum(x, q)
    np.testing.assert_allclose(direct_sum(2.0 * x, q), phi / 2.0, rtol=1e-13)
    np.testing.assert_allclose(direct_sum(x + np.array([0.25, -8.0, 3.5]), q), phi,
                               rtol=1e-10)
    # pair symmetry: G(a, b) = G(b, a)
    a, b = x[:1], x[1:2]
    assert direct_sum(a, [1.0], targets=b)[0] == direct_sum(b, [1.0], targets=a)[0]


def test_columns_are_independent():
    rng = np.random.default_rng(5)
    x = rng.random((300, 3))
    q = rng.standard_normal((300, 3))
    phi = direct_sum(x, q)
    for r in range(3):
        np.testing.assert_array_equal(phi[:, r], direct_sum(x, q[:, r]))


@pytest.mark.parametrize("n", [1, 2])
def test_tiny(n):
    x = np.zeros((n, 3))
    x[-1, 0] = 1.0
    phi = direct_sum(x, np.ones(n))
    assert phi.shape == (n,)
    if n == 1:
        assert phi[0] == 0.0
    else:
        np.testing.assert_allclose(phi, 1 / (4 * np.pi), rtol=1e-15)
