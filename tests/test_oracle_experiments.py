"""Sec. 3 basis comparisons (oracle/experiments.py), pinned against closed forms and the paper's
statements: Chebyshev iteration on the psi mass matrix with the Corollary 1 bounds (Sec. 3.1)
and LSC-DG against the semi-nodal basis for the L2 projection of cosh(x+y+z) (Sec. 3.2)."""

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from oracle.experiments import (chebyshev, chebyshev_bound, chebyshev_on_warped_pyramid, level_jacobian_range,
                                projection_errors, psi_mass, warped_pyramid)
from paper_1502_07703_gb300.mesh import make_pyramid_mesh


def _cheb_T(k, x):
    return npcheb.chebval(x, [0.0] * k + [1.0])


def test_chebyshev_iteration_error_is_the_chebyshev_polynomial():
    """On a diagonal matrix each eigen-component of the error after k steps is
    T_k((theta - lambda)/delta) / T_k(theta/delta) (numpy's Chebyshev series as the reference),
    which at the end points of the interval is the classical bound 2 tau^k / (1 + tau^(2k))."""
    lmin, lmax = 0.7, 1.9
    lam = np.array([lmin, 0.9, 1.3, 1.75, lmax])
    A = np.diag(lam)
    x = np.array([1.0, -2.0, 0.5, 3.0, -1.5])
    X = chebyshev(A, A @ x, lmin, lmax, 12)
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    for k in range(13):
        want = _cheb_T(k, (theta - lam) / delta) / _cheb_T(k, theta / delta)
        np.testing.assert_allclose((X[k] - x) / (-x), want, rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(abs(want[0]), chebyshev_bound(k, lmin, lmax), rtol=1e-10)


def test_chebyshev_on_the_reference_pyramid_is_one_step():
    """gamma = 0 is the reference pyramid: J = 1, M_psi = I, one point spectrum."""
    r = chebyshev_on_warped_pyramid(0.0, 3, max_iters=3)
    assert r["lmin"] == pytest.approx(1.0, abs=1e-14) and r["lmax"] == pytest.approx(1.0, abs=1e-14)
    assert r["iters"] == 1


@pytest.mark.parametrize("N", [2, 4])
@pytest.mark.parametrize("gamma", [0.2, 0.5, 1.0])
def test_corollary1_bounds_and_chebyshev_rate_on_warped_pyramids(gamma, N):
    """The level-grid Jacobian range is the extreme eigenvalues of M_psi (Corollary 1), and every
    Chebyshev iterate obeys the bound of Sec. 3.1 with those bounds."""
    ev = warped_pyramid(gamma)
    eig = np.linalg.eigvalsh(psi_mass(ev, N))
    lmin, lmax = level_jacobian_range(ev, N)
    np.testing.assert_allclose([eig.min(), eig.max()], [lmin, lmax], rtol=1e-12)
    r = chebyshev_on_warped_pyramid(gamma, N, max_iters=60)
    assert np.all(r["err"] <= r["bound"] * (1 + 1e-9) + 1e-13)


def test_chebyshev_iteration_counts_on_warped_pyramids():
    """Sec. 3.1: the count grows with the warping and hardly with N; already above ten
    iterations at gamma = 1 (tolerance 1e-8 on the error)."""
    counts = {(g, N): chebyshev_on_warped_pyramid(g, N)["iters"] for g in (0.2, 0.5, 1.0) for N in (2, 4, 6)}
    for N in (2, 4, 6):
        assert counts[(0.2, N)] < counts[(0.5, N)] < counts[(1.0, N)], counts
        assert counts[(1.0, N)] > 10, counts
    for g in (0.2, 0.5, 1.0):
        assert max(counts[(g, N)] for N in (2, 4, 6)) - min(counts[(g, N)] for N in (2, 4, 6)) <= 2, counts


def test_projections_reproduce_polynomials_where_the_space_holds_them():
    """The semi-nodal space holds P_N in physical coordinates on any vertex-mapped pyramid; the
    LSC-DG space only where J is constant (parallelogram base)."""
    rng = np.random.default_rng(4)
    cf = rng.standard_normal(10)

    def quad(X):  # a random physical polynomial of degree 2
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return (cf[0] + cf[1] * x + cf[2] * y + cf[3] * z + cf[4] * x * x + cf[5] * y * y + cf[6] * z * z
                + cf[7] * x * y + cf[8] * y * z + cf[9] * x * z)

    flat = warped_pyramid(0.0).copy()
    flat[4] += np.array([0.3, -0.2, 0.1])  # apex moved: an affine pyramid, J constant
    sn, lsc, nrm = projection_errors(flat[None], 2, quad)
    assert sn <= 1e-13 * nrm and lsc <= 1e-13 * nrm, (sn, lsc)
    sn, lsc, nrm = projection_errors(warped_pyramid(0.5)[None], 2, quad)
    assert sn <= 1e-13 * nrm, sn
    assert lsc > 1e-4 * nrm, lsc


@pytest.mark.parametrize("gamma", [0.2, 0.5, 1.0])
def test_lsc_dg_stalls_under_n_refinement_on_a_warped_pyramid(gamma):
    """Sec. 3.2: L2 projection of cosh(x+y+z) on the warped pyramid for N = 2..6. The semi-nodal
    error keeps falling (by more than 1000x over the range); the LSC-DG error stalls (falls by
    less than 2x per degree at the top) and ends more than 100x above the semi-nodal one."""
    ev = warped_pyramid(gamma)[None]
    errs = np.array([projection_errors(ev, N)[:2] for N in range(2, 7)])
    sn, lsc = errs[:, 0], errs[:, 1]
    assert np.all(sn[1:] < sn[:-1]) and sn[0] > 1000 * sn[-1], sn
    assert lsc[-2] / lsc[-1] < 2.0, lsc
    assert sn[-2] / sn[-1] > 10.0, sn
    assert lsc[-1] > 100 * sn[-1], (sn, lsc)


@pytest.mark.parametrize("N", [2, 3])
def test_lsc_dg_stalls_under_h_refinement(N):
    """Sec. 3.2: the bi-unit cube cut into K1D^3 hexes x 6 pyramids, vertices perturbed
    (+-0.1h, seed 3). Between K1D = 4 and 8 the semi-nodal error converges at about the optimal
    rate N+1; the LSC-DG error does not converge (rate below 0.5)."""
    errs = {}
    for n in (4, 8):
        v, e = make_pyramid_mesh(n, delta=0.1, seed=3, domain=(-1.0, 1.0))
        ev = np.asarray(v)[np.asarray(e)]
        errs[n] = projection_errors(ev, N)
    rate_sn = np.log2(errs[4][0] / errs[8][0])
    rate_lsc = np.log2(errs[4][1] / errs[8][1])
    assert rate_sn > N + 0.5, rate_sn
    assert rate_lsc < 0.5, rate_lsc
