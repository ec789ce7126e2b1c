"""Pins for oracle/rules.py: Jacobi polynomials, Gauss-Jacobi rules, Lagrange bases.

References are library routines (scipy.special, scipy.integrate) and textbook
closed forms, never the oracle itself.
"""

import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

from oracle.rules import gauss_jacobi, gauss_legendre, jacobi, jacobi_deriv, lagrange


@pytest.mark.parametrize("alpha", [0, 1, 2, 3, 5, 9, 17])
@pytest.mark.parametrize("n", [0, 1, 2, 5, 9])
def test_jacobi_matches_scipy(n, alpha):
    x = np.linspace(-1, 1, 41)
    np.testing.assert_allclose(jacobi(n, alpha, 0, x), scipy.special.eval_jacobi(n, alpha, 0, x), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("alpha", [0, 2, 7])
@pytest.mark.parametrize("n", [1, 3, 6])
def test_jacobi_derivative_by_finite_difference(n, alpha):
    x = np.linspace(-0.9, 0.9, 13)
    h = 1e-6
    fd = (scipy.special.eval_jacobi(n, alpha, 0, x + h) - scipy.special.eval_jacobi(n, alpha, 0, x - h)) / (2 * h)
    np.testing.assert_allclose(jacobi_deriv(n, alpha, 0, x), fd, rtol=1e-7, atol=1e-6)


@pytest.mark.parametrize("ab", [(0, 0), (1, 0), (2, 0), (5, 0), (11, 0)])
@pytest.mark.parametrize("n", [1, 2, 4, 8, 10])
def test_gauss_jacobi_matches_scipy(n, ab):
    x, w = gauss_jacobi(n, *ab)
    xs, ws = scipy.special.roots_jacobi(n, *ab)
    np.testing.assert_allclose(x, xs, atol=1e-13)
    np.testing.assert_allclose(w, ws, rtol=1e-12)


@pytest.mark.parametrize("ab", [(0, 0), (1, 0), (2, 0)])
@pytest.mark.parametrize("n", [1, 3, 6])
def test_gauss_jacobi_exact_to_degree_2n_minus_1(n, ab):
    alpha, beta = ab
    x, w = gauss_jacobi(n, alpha, beta)
    for m in range(2 * n):
        exact, _ = scipy.integrate.quad(lambda t: (1 - t) ** alpha * (1 + t) ** beta * t ** m, -1, 1, epsabs=1e-14)
        assert abs(np.dot(w, x ** m) - exact) < 1e-12


def test_gauss_legendre_closed_forms():
    x, w = gauss_legendre(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [1, 1], atol=1e-14)
    x, w = gauss_legendre(3)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 5])
def test_lagrange_nodal_and_derivative(n):
    nodes, _ = gauss_legendre(n)
    L, _ = lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(n), atol=1e-14)
    x = np.linspace(-1, 1, 9)
    h = 1e-6
    _, dL = lagrange(nodes, x)
    Lp, _ = lagrange(nodes, x + h)
    Lm, _ = lagrange(nodes, x - h)
    np.testing.assert_allclose(dL, (Lp - Lm) / (2 * h), atol=1e-6)
    # reproduces polynomials of degree n-1
    f = lambda t: 0.3 + 0.7 * t ** (n - 1) - (1.2 * t if n >= 2 else 0.0)
    np.testing.assert_allclose(lagrange(nodes, x)[0] @ f(nodes), f(x), atol=1e-13)
