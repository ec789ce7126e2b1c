"""Jacobi polynomials and Gauss-Jacobi rules (oracle; test infrastructure only).

Sec. 2 builds every basis and cubature from Jacobi polynomials P_n^{(alpha,beta)}
with the standard normalisation P_n^{(alpha,beta)}(1) = binom(n+alpha, n). The
rules here come from the Golub-Welsch eigenvalue method.

Pinned by tests/test_oracle_rules.py against scipy.special (a library routine)
and by exactness on monomials.
"""

from __future__ import annotations

import math

import numpy as np


def jacobi(n, alpha, beta, x):
    """P_n^{(alpha,beta)}(x) by the three-term recurrence (standard normalisation)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = 0.5 * (alpha - beta + (alpha + beta + 2.0) * x)
    for m in range(2, n + 1):
        s = 2.0 * m + alpha + beta
        a1 = 2.0 * m * (m + alpha + beta) * (s - 2.0)
        a2 = (s - 1.0) * (alpha * alpha - beta * beta)
        a3 = (s - 2.0) * (s - 1.0) * s
        a4 = 2.0 * (m + alpha - 1.0) * (m + beta - 1.0) * s
        p0, p1 = p1, ((a2 + a3 * x) * p1 - a4 * p0) / a1
    return p1


def jacobi_deriv(n, alpha, beta, x):
    """d/dx P_n^{(alpha,beta)}(x) = (n+alpha+beta+1)/2 * P_{n-1}^{(alpha+1,beta+1)}(x)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + alpha + beta + 1.0) * jacobi(n - 1, alpha + 1.0, beta + 1.0, x)


def gauss_jacobi(n, alpha=0.0, beta=0.0):
    """n-point Gauss-Jacobi rule for weight (1-x)^alpha (1+x)^beta on [-1, 1].

    Golub-Welsch: nodes are the eigenvalues of the symmetric tridiagonal
    matrix of the monic recurrence; weights are mu0 times the squared first
    components of the normalised eigenvectors. Exact for degree 2n-1.
    Returns (nodes ascending, weights).
    """
    alpha = float(alpha)
    beta = float(beta)
    diag = np.empty(n)
    off = np.empty(max(n - 1, 0))
    for m in range(n):
        s = 2.0 * m + alpha + beta
        if m == 0:
            diag[m] = (beta - alpha) / (alpha + beta + 2.0)
        else:
            diag[m] = (beta * beta - alpha * alpha) / (s * (s + 2.0))
        if m >= 1:
            num = 4.0 * m * (m + alpha) * (m + beta) * (m + alpha + beta)
            den = s * s * (s + 1.0) * (s - 1.0)
            off[m - 1] = math.sqrt(num / den)
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    nodes, vecs = np.linalg.eigh(T)
    mu0 = 2.0 ** (alpha + beta + 1.0) * math.gamma(alpha + 1.0) * math.gamma(beta + 1.0) / math.gamma(alpha + beta + 2.0)
    weights = mu0 * vecs[0, :] ** 2
    order = np.argsort(nodes)
    return nodes[order], weights[order]


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1]."""
    return gauss_jacobi(n, 0.0, 0.0)


def lagrange(nodes, x):
    """Lagrange basis l_i(x) on the given nodes and its derivative.

    Returns (L, dL), each of shape (len(x), len(nodes)); written out as the
    plain product formula and its product-rule derivative.
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    L = np.ones((x.size, n))
    dL = np.zeros((x.size, n))
    for i in range(n):
        for m in range(n):
            if m != i:
                L[:, i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
        for l in range(n):
            if l == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[l]))
            for m in range(n):
                if m != i and m != l:
                    term *= (x - nodes[m]) / (nodes[i] - nodes[m])
            dL[:, i] += term
    return L, dL
