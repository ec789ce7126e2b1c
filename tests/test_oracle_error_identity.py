"""The identity behind the error norm from coefficients, checked with the oracle alone.

For the error rule's inner product <.,.>_Q ((N+3)-point rules) and the projection P onto
an element's polynomial space under it, U_h - P U_ex lies in the space and P U_ex - U_ex
is <.,.>_Q-orthogonal to it, so
    |U_h - U_ex|_Q^2 = (u - s)^T M^Q (u - s) + |P U_ex - U_ex|_Q^2,
with s the coefficients of P U_ex and M^Q the element mass matrix under that rule. The
exact fields are S(x) times a time factor, so s and the second term scale with it. The
oracle's pointwise error and this decomposition are compared here in its own basis psi
(dense M^Q), and M^Q of the semi-nodal basis is checked to be diagonal (Lemma 3) under
the same rule, which lets the library use the diagonal."""

import numpy as np
import pytest

from oracle.basis import abc_to_rst, phi, psi, reference_rule
from oracle.dg import PyramidDG, exact_solution
from oracle.geometry import map_points
from paper_1502_07703_gb300.mesh import make_pyramid_mesh, random_state


def _rule_data(dg):
    a, b, c, w = reference_rule(dg.N + 3)
    r, s, t = abc_to_rst(a, b, c)
    X, Jac = map_points(dg.ev, r, s, t)
    W = w[None, :] * np.linalg.det(Jac)  # (K, Q^3) weights w J
    return a, b, c, X, W


@pytest.mark.parametrize("bc,N", [("wall", 2), ("wall", 3), ("free", 3)])
def test_pythagorean_split_matches_pointwise_error(bc, N):
    lo, hi = (0.0, 1.0) if bc == "wall" else (-1.0, 1.0)
    v, e = make_pyramid_mesh(2, delta=0.05, seed=4, domain=(lo, hi))
    dg = PyramidDG(v, e, N, bc=bc)
    U = random_state(dg.K, dg.Np, 8)
    t = 0.41
    err_abs, _ = dg.error(U, t)
    a, b, c, X, W = _rule_data(dg)
    V = psi(N, a, b, c)[0]                                   # (Q^3, Np)
    Ue = exact_solution(bc, X[..., 0], X[..., 1], X[..., 2], t)  # (K, Q^3, 4)
    M = np.einsum("kq,qi,qj->kij", W, V, V)                  # dense M^Q per element
    rhs = np.einsum("kq,qi,kqc->kic", W, V, Ue)
    s = np.linalg.solve(M, rhs)                              # (K, Np, 4): coefficients of P U_ex
    d = np.transpose(U, (0, 2, 1)) - s
    part1 = np.einsum("kic,kij,kjc->", d, M, d)
    part2 = np.einsum("kq,kqc->", W, (np.einsum("qi,kic->kqc", V, s) - Ue) ** 2)
    assert part1 > 0 and part2 > 0
    np.testing.assert_allclose(np.sqrt(part1 + part2), err_abs, rtol=1e-11)


def test_time_factor_separates():
    """P is linear and the exact fields are S(x) T(t), so P U_ex(t) = T(t) P S."""
    v, e = make_pyramid_mesh(2, delta=0.05, seed=4)
    dg = PyramidDG(v, e, 2)
    a, b, c, X, W = _rule_data(dg)
    V = psi(2, a, b, c)[0]
    M = np.einsum("kq,qi,qj->kij", W, V, V)
    proj = lambda F: np.linalg.solve(M, np.einsum("kq,qi,kqc->kic", W, V, F))
    t1, t2 = 0.13, 0.77
    U1 = exact_solution("wall", X[..., 0], X[..., 1], X[..., 2], t1)
    U2 = exact_solution("wall", X[..., 0], X[..., 1], X[..., 2], t2)
    w = np.sqrt(3.0) * np.pi
    T1 = np.array([np.cos(w * t1)] + [np.sin(w * t1)] * 3)
    T2 = np.array([np.cos(w * t2)] + [np.sin(w * t2)] * 3)
    np.testing.assert_allclose(proj(U1) / T1, proj(U2) / T2, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_seminodal_mass_diagonal_under_error_rule(N):
    v, e = make_pyramid_mesh(2, delta=0.05, seed=4)
    dg = PyramidDG(v, e, N)
    a, b, c, X, W = _rule_data(dg)
    Vp = phi(N, a, b, c)[0]
    M = np.einsum("kq,qi,qj->kij", W, Vp, Vp)
    off = M - np.einsum("kii->ki", M)[:, :, None] * np.eye(dg.Np)[None]
    assert np.abs(off).max() < 1e-13 * np.abs(M).max()
