"""Pins for oracle/advection.py (Sec. 4.1 advection with the alpha-flux, periodic box)."""

import numpy as np
import pytest

from oracle.advection import PyramidAdvection, exact_advection
from paper_1502_07703_gb300.mesh import make_pyramid_mesh


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_energy_identity_and_stability(alpha):
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=3)
    ad = PyramidAdvection(v, e, 3, beta=(1.0, 0.3, -0.2), alpha=alpha)
    U = np.random.default_rng(2).standard_normal((ad.K, 1, ad.Np))
    dEdt = np.einsum("ki,kij,kj->", U[:, 0], ad.dg.M, ad.rhs(U)[:, 0])
    D = ad.dissipation(U)
    assert abs(dEdt + D) < 1e-11 * max(1.0, abs(np.einsum("ki,kj,kij->", U[:, 0], U[:, 0], np.abs(ad.Sb))))
    if alpha == 0.0:
        assert D == 0.0
    else:
        assert D > 0.0


def test_periodic_matching_is_complete():
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    ad = PyramidAdvection(v, e, 2)
    assert np.all(ad.dg.interior)
    X = ad.dg.Xf.reshape(-1, 3)
    d = np.mod(X[ad.dg.mapP] - X + 0.5, 1.0) - 0.5  # coincide modulo the unit period
    assert np.max(np.abs(d)) < 1e-12


def test_constant_is_steady_and_exact_solution_is_a_solution():
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    ad = PyramidAdvection(v, e, 2, beta=(1.0, 0.5, 0.25))
    U = ad.dg.project(lambda X: np.ones(X.shape[:-1] + (4,)))[:, :1]
    assert np.max(np.abs(ad.rhs(U))) < 1e-11
    rng = np.random.default_rng(0)
    x, y, z, t = rng.uniform(0, 1, (4, 10))
    h = 1e-6
    b = np.array([1.0, 0.5, 0.25])
    ut = (exact_advection(x, y, z, t + h, b) - exact_advection(x, y, z, t - h, b)) / (2 * h)
    ux = (exact_advection(x + h, y, z, t, b) - exact_advection(x - h, y, z, t, b)) / (2 * h)
    uy = (exact_advection(x, y + h, z, t, b) - exact_advection(x, y - h, z, t, b)) / (2 * h)
    uz = (exact_advection(x, y, z + h, t, b) - exact_advection(x, y, z - h, t, b)) / (2 * h)
    np.testing.assert_allclose(ut + b[0] * ux + b[1] * uy + b[2] * uz, 0.0, atol=1e-7)


@pytest.mark.parametrize("N", [1, 2])
def test_advection_converges(N):
    errs = []
    for n in (4, 8):  # u0 has wavenumber 2 pi: 2^3 hexes are still pre-asymptotic
        v, e = make_pyramid_mesh(n, delta=0.05, seed=1)
        ad = PyramidAdvection(v, e, N)
        T = 0.05
        steps = int(np.ceil(T / ad.dt_cfl(0.5)))
        U = ad.lsrk4(ad.project_exact(0.0), T / steps, steps)
        errs.append(ad.error(U, T)[0])
    rate = np.log2(errs[0] / errs[1])
    assert rate > N + 0.5, (errs, rate)
