"""Pins for oracle/basis.py: counts, orthonormality, derivatives, Lemma 2, Lemma 4."""

import numpy as np
import pytest

from oracle.basis import abc_to_rst, num_modes, phi, phi_indices, psi, psi_indices, reference_rule
from oracle.rules import gauss_legendre, jacobi

GOLDEN_NP = {1: 5, 2: 14, 3: 30, 4: 55, 5: 91, 6: 140, 7: 204, 8: 285}


def _rst_to_abc(r, s, t):
    return 2 * (1 + r) / (1 - t) - 1, 2 * (1 + s) / (1 - t) - 1, t


@pytest.mark.parametrize("N", range(1, 9))
def test_counts(N):
    # Lemma 4 counts sum_k (k+1)^2 = (N+1)(N+2)(2N+3)/6 (tests/golden/np_counts.txt)
    assert num_modes(N) == GOLDEN_NP[N]
    assert len(psi_indices(N)) == GOLDEN_NP[N]
    assert len(phi_indices(N)) == GOLDEN_NP[N]


def test_golden_np_file():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "np_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for N, Np in rows:
        assert num_modes(int(N)) == int(Np)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_psi_orthonormal_on_reference(N):
    # Eq. (1): orthonormal over the reference pyramid. Check with a rule two points finer.
    a, b, c, w = reference_rule(N + 3)
    V = psi(N, a, b, c)[0]
    G = np.einsum("q,qi,qj->ij", w, V, V)
    np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-12)


@pytest.mark.parametrize("basis", [psi, phi])
@pytest.mark.parametrize("N", [1, 3, 4])
def test_rst_derivatives_by_finite_difference(basis, N):
    rng = np.random.default_rng(5)
    a, b, c = rng.uniform(-0.9, 0.9, (3, 20))
    r, s, t = abc_to_rst(a, b, c)
    _, Vr, Vs, Vt = basis(N, a, b, c)
    h = 1e-6
    for D, dr in ((Vr, (h, 0, 0)), (Vs, (0, h, 0)), (Vt, (0, 0, h))):
        Vp = basis(N, *_rst_to_abc(r + dr[0], s + dr[1], t + dr[2]))[0]
        Vm = basis(N, *_rst_to_abc(r - dr[0], s - dr[1], t - dr[2]))[0]
        np.testing.assert_allclose(D, (Vp - Vm) / (2 * h), atol=2e-5 * (1 + np.abs(D).max()))


@pytest.mark.parametrize("N", range(0, 9))
def test_lemma2_constant(N):
    """Lemma 2 at i = j, after the index change of the paper: the c-integral of
    ((1-c)/2)^{2+2k} (P_{N-k}^{(2k+3,0)})^2 equals 2/(2k+3) for every N.

    The printed C^N_i = (N+2)/(2^{2(N+1-i)}(2N+3-2i)) fails already at N = 0
    (1/6 against the integral 2/3); the value pinned here is the integral itself,
    by a 60-point Gauss-Legendre rule (exact), and the closed form 2/(2k+3)
    (tests/golden/lemma2_constants.txt)."""
    xg, wg = gauss_legendre(60)
    for k in range(N + 1):
        val = np.sum(wg * ((1 - xg) / 2) ** (2 + 2 * k) * jacobi(N - k, 2 * k + 3, 0, xg) ** 2)
        assert abs(val - 2.0 / (2 * k + 3)) < 1e-13
    if N == 0:
        printed = (N + 2) / (2 ** (2 * (N + 1)) * (2 * N + 3))
        assert abs(printed - 2.0 / 3.0) > 0.4


def test_golden_lemma2_file():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "lemma2_constants.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    xg, wg = gauss_legendre(60)
    for k, num, den in rows:
        k = int(k)
        val = np.sum(wg * ((1 - xg) / 2) ** (2 + 2 * k) * jacobi(3, 2 * k + 3, 0, xg) ** 2)
        assert abs(val - int(num) / int(den)) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_lemma4_same_span(N):
    """Lemma 4: span(phi) = span(psi). Least-squares fit of every phi_n by psi at
    random points leaves no residual, and the stacked matrix has rank Np."""
    rng = np.random.default_rng(N)
    a, b, c = rng.uniform(-1, 1, (3, 4 * num_modes(N)))
    Vpsi = psi(N, a, b, c)[0]
    Vphi = phi(N, a, b, c)[0]
    coef, *_ = np.linalg.lstsq(Vpsi, Vphi, rcond=None)
    assert np.max(np.abs(Vpsi @ coef - Vphi)) < 1e-10
    assert np.linalg.matrix_rank(np.hstack([Vpsi, Vphi]), tol=1e-9) == num_modes(N)
