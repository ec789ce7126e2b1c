"""Pins for oracle/dg.py against what the paper and the mathematics fix.

* Lemma 3: the semi-nodal mass matrix on a vertex-mapped pyramid is diagonal,
  M = J(a_i^k, b_j^k) w_i^k w_j^k C_k with C_k = 2/(2k+3); checked against a
  dense assembly with a finer (non-minimal) rule, i.e. by brute force.
* Corollary 1 (strengthened): the eigenvalues of the psi-basis mass matrix are
  exactly the values J(a_i^k, b_j^k); its diagonal is constant, J(0,0)
  (the observation of Sec. 3.1).
* Polynomial reproduction: physical polynomials of degree N lie in the space;
  projection and M^{-1} S^x reproduce them and their x-derivative exactly.
* Integration by parts with the minimal rules (Sec. 4.1): S^m + S^m^T equals
  the face matrix of n_m.
* Semi-discrete energy identity of the Sec. 4.3 flux: dE/dt equals minus the
  flux dissipation, zero for the central flux.
* Convergence: projection and evolution errors fall at the optimal rate N+1
  (Sec. 4.3).
* Spectral radius (Sec. 4.3): rho(A) ~ 2(N+1)(N+3)/3 * |dK|/|K|, and the CFL
  time step lies in the LSRK4 stability region.
"""

import numpy as np
import pytest

from oracle.basis import abc_to_rst, num_modes, phi, phi_indices, psi
from oracle.dg import LSRK_A, LSRK_B, PyramidDG, exact_solution
from oracle.geometry import REF_VERTICES, map_points
from oracle.rules import gauss_legendre
from paper_1502_07703_gb300.mesh import make_pyramid_mesh


def _warped_single(seed, amp=0.25):
    rng = np.random.default_rng(seed)
    v = REF_VERTICES + rng.uniform(-amp, amp, (5, 3))
    return v, np.array([[0, 1, 2, 3, 4]], dtype=np.int32)


def _level_jacobians(ev, N):
    """J at the level-k Gauss points (a_i^k, b_j^k), phi storage order, and the mass diagonal."""
    Jv, Mdiag = [], []
    for (i, j, k) in phi_indices(N):
        xk, wk = gauss_legendre(k + 1)
        r, s, t = abc_to_rst(np.array([xk[i]]), np.array([xk[j]]), np.array([0.3]))
        J = np.linalg.det(map_points(ev[None], r, s, t)[1][0, 0])
        Jv.append(J)
        Mdiag.append(J * wk[i] * wk[j] * 2.0 / (2 * k + 3))
    return np.array(Jv), np.array(Mdiag)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_lemma3_semi_nodal_mass_is_diagonal(N):
    v, e = _warped_single(N)
    dg = PyramidDG(v, e, N)
    # brute force: dense assembly with a rule two points finer than the minimal one
    from oracle.basis import reference_rule
    a, b, c, w = reference_rule(N + 3)
    X, Jac = map_points(dg.ev, *abc_to_rst(a, b, c))
    J = np.linalg.det(Jac)[0]
    Vphi = phi(N, a, b, c)[0]
    M = np.einsum("q,q,qi,qj->ij", w, J, Vphi, Vphi)
    _, Mdiag = _level_jacobians(dg.ev[0], N)
    np.testing.assert_allclose(M, np.diag(Mdiag), atol=1e-13 * Mdiag.max())
    # and the minimal rule of Sec. 4.1 gives the same matrix
    Vphi_min = phi(N, *dg.vol_abc)[0]
    Mmin = np.einsum("q,q,qi,qj->ij", dg.w, dg.J[0], Vphi_min, Vphi_min)
    np.testing.assert_allclose(Mmin, M, atol=1e-13 * Mdiag.max())


@pytest.mark.parametrize("N", [2, 3, 5])
def test_corollary1_psi_mass_spectrum_and_constant_diagonal(N):
    v, e = _warped_single(10 + N)
    dg = PyramidDG(v, e, N)
    Jv, _ = _level_jacobians(dg.ev[0], N)
    eig = np.linalg.eigvalsh(dg.M[0])
    np.testing.assert_allclose(np.sort(eig), np.sort(Jv), rtol=1e-12)
    r, s, t = abc_to_rst(np.zeros(1), np.zeros(1), np.zeros(1))
    J00 = np.linalg.det(map_points(dg.ev, r, s, t)[1][0, 0])
    np.testing.assert_allclose(np.diag(dg.M[0]), J00, rtol=1e-12)


def _physical_poly(N, seed):
    rng = np.random.default_rng(seed)
    terms = [(i, j, k) for i in range(N + 1) for j in range(N + 1) for k in range(N + 1) if i + j + k <= N]
    coef = rng.standard_normal(len(terms))

    def f(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return sum(cf * x ** i * y ** j * z ** k for cf, (i, j, k) in zip(coef, terms))

    def fx(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return sum(cf * i * x ** max(i - 1, 0) * y ** j * z ** k for cf, (i, j, k) in zip(coef, terms) if i > 0)

    return f, fx


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_polynomial_reproduction_and_exact_derivative(N):
    v, e = make_pyramid_mesh(2, 1, 1, delta=0.15, seed=7)
    dg = PyramidDG(v, e, N)
    f, fx = _physical_poly(N, N)
    U = dg.project(lambda X: np.repeat(f(X)[..., None], 4, axis=-1))
    rng = np.random.default_rng(3)
    a, b, c = rng.uniform(-1, 1, (3, 25))
    Vp = psi(N, a, b, c)[0]
    X, _ = map_points(dg.ev, *abc_to_rst(a, b, c))
    scale = np.max(np.abs(f(X)))
    np.testing.assert_allclose(np.einsum("qn,kn->kq", Vp, U[:, 0]), f(X), atol=1e-11 * scale)
    dU = np.einsum("kij,kjl,kl->ki", dg.Minv, dg.S[:, 0], U[:, 0])
    np.testing.assert_allclose(np.einsum("qn,kn->kq", Vp, dU), fx(X), atol=1e-10 * max(1.0, np.max(np.abs(fx(X)))))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_integration_by_parts_with_minimal_rules(N):
    v, e = make_pyramid_mesh(1, delta=0.0)
    v = v + np.random.default_rng(2).uniform(-0.08, 0.08, v.shape) * (np.abs(v - 0.5) < 0.49).all(axis=1)[:, None]
    dg = PyramidDG(v, e, N)
    W = dg.fw[None] * dg.sJ
    for m in range(3):
        E = np.einsum("kfq,kfq,fqi,fqj->kij", W, dg.nrm[..., m], dg.Vf, dg.Vf)
        Sm = dg.S[:, m]
        np.testing.assert_allclose(Sm + Sm.transpose(0, 2, 1), E, atol=1e-12 * np.abs(E).max())


def test_face_matching_counts_and_coincidence():
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    dg = PyramidDG(v, e, 3)
    nf = 16
    assert (~dg.interior).sum() == 24 * nf  # 6 box faces x 4 hex faces
    inter = np.nonzero(dg.interior)[0]
    X = dg.Xf.reshape(-1, 3)
    W = (dg.fw[None] * dg.sJ).reshape(-1)
    np.testing.assert_allclose(X[inter], X[dg.mapP[inter]], atol=1e-13)
    np.testing.assert_allclose(W[inter], W[dg.mapP[inter]], rtol=1e-12)
    n = dg.nrm.reshape(-1, 3)
    np.testing.assert_allclose(n[inter], -n[dg.mapP[inter]], atol=1e-12)


@pytest.mark.parametrize("bc", ["wall", "free"])
def test_free_stream(bc):
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    dg = PyramidDG(v, e, 3, bc=bc)
    U = dg.project(lambda X: np.stack([np.ones(X.shape[:-1])] + [np.zeros(X.shape[:-1])] * 3, axis=-1))
    R = dg.rhs(U)
    if bc == "wall":
        assert np.max(np.abs(R)) < 1e-11
    else:  # p = 1 is not a steady state of the free-surface problem, u = 0 with p = 0 is
        U[:, 0] = 0.0
        assert np.max(np.abs(dg.rhs(U))) < 1e-14


@pytest.mark.parametrize("bc", ["wall", "free"])
@pytest.mark.parametrize("tau", [0.0, 1.0])
def test_energy_identity(bc, tau):
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=3)
    dg = PyramidDG(v, e, 3, tau=tau, bc=bc)
    U = np.random.default_rng(9).standard_normal((dg.K, 4, dg.Np))
    dEdt = np.einsum("kci,kij,kcj->", U, dg.M, dg.rhs(U))
    D = dg.dissipation(U)
    scale = np.abs(np.einsum("kci,kcj,kij->", U, U, np.abs(dg.S).sum(axis=1)))
    assert abs(dEdt + D) < 1e-12 * scale
    if tau == 0.0:
        assert D == 0.0
    else:
        assert D > 0.0


def test_exact_solution_satisfies_pde_and_bc():
    rng = np.random.default_rng(0)
    h = 1e-5
    for bc, lo, hi in (("wall", 0.0, 1.0), ("free", -1.0, 1.0)):
        x, y, z = rng.uniform(lo, hi, (3, 20))
        t = rng.uniform(0, 1, 20)
        d = lambda ax: (exact_solution(bc, *[q + (h if i == ax else 0) for i, q in enumerate((x, y, z, t))])
                        - exact_solution(bc, *[q - (h if i == ax else 0) for i, q in enumerate((x, y, z, t))])) / (2 * h)
        dx, dy, dz, dt = d(0), d(1), d(2), d(3)
        np.testing.assert_allclose(dt[:, 0] + dx[:, 1] + dy[:, 2] + dz[:, 3], 0, atol=1e-7)
        np.testing.assert_allclose(dt[:, 1:] + np.stack([dx[:, 0], dy[:, 0], dz[:, 0]], 1), 0, atol=1e-7)
        side = np.full(20, lo)
        if bc == "wall":  # n.u = 0 on x = lo and x = hi
            assert np.max(np.abs(exact_solution(bc, side, y, z, t)[:, 1])) < 1e-15
            assert np.max(np.abs(exact_solution(bc, side + (hi - lo), y, z, t)[:, 1])) < 1e-15
        else:  # p = 0 on the boundary
            assert np.max(np.abs(exact_solution(bc, side, y, z, t)[:, 0])) < 1e-15


@pytest.mark.parametrize("N", [1, 2, 3])
def test_projection_converges_at_optimal_rate(N):
    errs = []
    for n in (2, 4):
        v, e = make_pyramid_mesh(n, delta=0.1, seed=1)
        dg = PyramidDG(v, e, N)
        errs.append(dg.error(dg.project_exact(0.3), 0.3)[0])
    rate = np.log2(errs[0] / errs[1])
    assert rate > N + 0.6, (errs, rate)


@pytest.mark.parametrize("N", [1, 2])
def test_evolution_converges_at_optimal_rate(N):
    errs = []
    T = 0.1
    for n in (2, 4):
        v, e = make_pyramid_mesh(n, delta=0.05, seed=1)
        dg = PyramidDG(v, e, N)
        dt0 = dg.dt_cfl(0.5)
        steps = int(np.ceil(T / dt0))
        U = dg.lsrk4(dg.project_exact(0.0), T / steps, steps)
        errs.append(dg.error(U, T)[0])
    rate = np.log2(errs[0] / errs[1])
    assert rate > N + 0.5, (errs, rate)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_spectral_radius_fit_and_cfl_stability(N):
    v, e = make_pyramid_mesh(2, 1, 1, delta=0.05, seed=0)
    dg = PyramidDG(v, e, N)
    n = dg.K * 4 * dg.Np
    A = np.empty((n, n))
    for col in range(n):
        x = np.zeros(n)
        x[col] = 1.0
        A[:, col] = dg.rhs(x.reshape(dg.K, 4, dg.Np)).ravel()
    lam = np.linalg.eigvals(A)
    rho = np.max(np.abs(lam))
    CN = 2.0 * (N + 1) * (N + 3) / 3.0
    ratio = rho / (CN * np.max(dg.surface_areas() / dg.volumes()))
    assert 0.2 < ratio < 1.5, ratio
    assert np.max(lam.real) < 1e-9 * rho  # upwind: no growing modes
    dt = dg.dt_cfl(0.5)
    y = np.ones_like(lam)
    res = np.zeros_like(lam)
    for s in range(5):
        res = LSRK_A[s] * res + dt * lam * y
        y = y + LSRK_B[s] * res
    assert np.max(np.abs(y)) <= 1.0 + 1e-12


def _golden_cfl_constants():
    """C_N of the Sec. 4.3 spectral-radius fit, read from tests/golden/spectral_radius_constants.txt
    (tabulated as the numerator over 3)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "spectral_radius_constants.txt")
    out = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            n, num = line.split()
            out[int(n)] = int(num) / 3.0
    return out


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_dt_cfl_uses_the_papers_constant(N):
    """dt = CFL / (C_N max_K |dK|/|K|) with C_N from the golden table, on unperturbed meshes,
    where every pyramid (a cube face as base, the cube centre as apex) has |K| = h^3/6 and
    |dK| = h^2 (1 + sqrt 2) in closed form, so max |dK|/|K| = 6 (1 + sqrt 2) / h. A slip in the
    oracle's constant (say (N+2) for (N+3)) or in its area or volume sums fails here."""
    CN = _golden_cfl_constants()
    assert sorted(CN) == list(range(1, 8))
    for n_hex in (1, 2):
        v, e = make_pyramid_mesh(n_hex, delta=0.0)
        dg = PyramidDG(v, e, N)
        aov = 6.0 * (1.0 + np.sqrt(2.0)) * n_hex
        np.testing.assert_allclose(dg.volumes(), 1.0 / (6 * n_hex ** 3), rtol=1e-13)
        np.testing.assert_allclose(dg.surface_areas(), (1.0 + np.sqrt(2.0)) / n_hex ** 2, rtol=1e-13)
        for cfl in (0.5, 0.25):
            np.testing.assert_allclose(dg.dt_cfl(cfl), cfl / (CN[N] * aov), rtol=1e-13)


def test_worst_element_measure_sees_a_single_element_fault():
    """The worst-element parity measure at full size for a fault in one element, where the
    mesh-wide relative L2 is diluted by about sqrt(K); the chunked large-mesh comparison gives
    the same two numbers as the dense oracle's."""
    from oracle.dg import phi_states_l2_diff
    from paper_1502_07703_gb300.mesh import random_state
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    N = 3
    dg = PyramidDG(v, e, N)
    B = random_state(dg.K, dg.Np, 5)
    A = B.copy()
    A[17, 2] *= 1.0 + 1e-4  # one field of one element off by 1e-4
    Av, Bv = dg.values_phi(A), dg.values_phi(B)
    rel, worst = dg.rel_l2_points(Av, Bv), dg.worst_element_rel(Av, Bv)
    assert worst > 3e-5 and rel < worst / 3, (rel, worst)
    assert dg.worst_element_rel(Bv, Bv) == 0.0
    r2, w2 = phi_states_l2_diff(v, e, N, A, B, chunk=5)
    np.testing.assert_allclose([r2, w2], [rel, worst], rtol=1e-12)
    # a single row with its element index gives that element's own relative difference
    w1 = dg.worst_element_rel(Av[17:18], Bv[17:18], elems=[17])
    wJ = dg.w * dg.J[17]
    own = np.sqrt(np.einsum("q,qc->", wJ, (Av[17] - Bv[17]) ** 2) / np.einsum("q,qc->", wJ, Bv[17] ** 2))
    np.testing.assert_allclose(w1, own, rtol=1e-12)
