"""Basis comparisons of Sec. 3 (oracle-side; test infrastructure only, plain FP64 numpy).

Sec. 3.1: the mass matrix of the rational orthonormal basis psi (Eq. (1)) on a vertex-mapped
pyramid is not diagonal, so an explicit scheme would have to invert it; Chebyshev iteration
with the spectral bounds of Corollary 1 (the eigenvalues lie between the smallest and the
largest Jacobian on the level grids) converges at the rate of the classical bound
    |x - x_k| <= 2 tau^k / (1 + tau^(2k)) |x - x_0|,
    tau = (1 - sqrt(lmin/lmax)) / (1 + sqrt(lmin/lmax)),
which on a warped pyramid already needs more than ten iterations.

Sec. 3.2: Low-Storage Curvilinear DG (LSC-DG) uses psi_i / sqrt(J), whose mass matrix is the
reference one (the identity for orthonormal psi). On pyramids with non-parallelogram bases
J depends on (a, b), so the weighted space contains no polynomials beyond constants times
1/sqrt(J) and its L2 projection error stalls under h- and N-refinement, while the semi-nodal
space (which contains P_N in physical coordinates) converges at the optimal rate.

The warped pyramid of Sec. 3.1 is drawn only in a figure; the reading taken here is the
reference pyramid whose base corners are moved along t by +gamma/2 (v1, v3) and -gamma/2
(v2, v4): a bilinear twist of the base of magnitude gamma, so that J varies with (a, b).
"""

from __future__ import annotations

import numpy as np

from .basis import abc_to_rst, phi, psi, reference_rule
from .geometry import REF_VERTICES, jacobian_and_inverse, map_points
from .rules import gauss_legendre


def warped_pyramid(gamma):
    """Vertices (5, 3) of the reference pyramid with its base twisted by gamma (module doc)."""
    v = REF_VERTICES.copy()
    v[0, 2] += 0.5 * gamma
    v[2, 2] += 0.5 * gamma
    v[1, 2] -= 0.5 * gamma
    v[3, 2] -= 0.5 * gamma
    return v


def psi_mass(ev, N, nq=None):
    """Dense mass matrix int_K psi_i psi_j of one element (ev: (5, 3)) with an nq-point rule."""
    nq = N + 1 if nq is None else nq
    a, b, c, w = reference_rule(nq)
    r, s, t = abc_to_rst(a, b, c)
    J = jacobian_and_inverse(map_points(ev[None], r, s, t)[1])[0][0]
    V = psi(N, a, b, c)[0]
    return np.einsum("q,qi,qj->ij", w * J, V, V)


def level_jacobian_range(ev, N):
    """Smallest and largest J(a_i^k, b_j^k) over the level grids k = 0..N: the bounds of the
    psi mass spectrum (Corollary 1)."""
    vals = []
    for k in range(N + 1):
        xk, _ = gauss_legendre(k + 1)
        A, B = np.meshgrid(xk, xk, indexing="ij")
        r, s, t = abc_to_rst(A.ravel(), B.ravel(), np.zeros(A.size))
        vals.append(np.linalg.det(map_points(ev[None], r, s, t)[1][0]))
    vals = np.concatenate(vals)
    return float(vals.min()), float(vals.max())


def chebyshev(A, b, lmin, lmax, iters, x0=None):
    """Chebyshev iteration for A x = b with the spectrum of the SPD matrix A in [lmin, lmax]:
    the iterates x_0 .. x_iters (array (iters+1, n)). With theta, delta the centre and
    half-width of the interval, the error after k steps is T_k((theta - A)/delta) /
    T_k(theta/delta) times the initial error; the three-term Chebyshev recurrence gives the
    updates."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    out = [x.copy()]
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    r = b - A @ x
    if delta <= 0.0:  # one point spectrum: A = theta I on the relevant space
        for _ in range(iters):
            x = x + r / theta
            r = b - A @ x
            out.append(x.copy())
        return np.array(out)
    sigma = theta / delta
    rho = 1.0 / sigma
    d = r / theta
    for _ in range(iters):
        x = x + d
        r = r - A @ d
        rho_next = 1.0 / (2.0 * sigma - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * r
        rho = rho_next
        out.append(x.copy())
    return np.array(out)


def chebyshev_bound(k, lmin, lmax):
    """2 tau^k / (1 + tau^(2k)) with tau = (1 - sqrt(lmin/lmax)) / (1 + sqrt(lmin/lmax))."""
    q = np.sqrt(lmin / lmax)
    tau = (1.0 - q) / (1.0 + q)
    k = np.asarray(k, dtype=np.float64)
    return 2.0 * tau ** k / (1.0 + tau ** (2.0 * k))


def chebyshev_on_warped_pyramid(gamma, N, tol=1e-8, max_iters=200, seed=0):
    """Solve M_psi x = b (random b) on the pyramid warped by gamma with the Corollary 1 bounds.

    Returns dict: bounds, per-iteration relative errors |x - x_k| / |x - x_0|, the classical
    bound at each k, and the first k whose relative error is <= tol."""
    ev = warped_pyramid(gamma)
    M = psi_mass(ev, N)
    lmin, lmax = level_jacobian_range(ev, N)
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(M.shape[0])
    x = np.linalg.solve(M, b)
    X = chebyshev(M, b, lmin, lmax, max_iters)
    err = np.linalg.norm(X - x[None], axis=1) / np.linalg.norm(x)
    hit = np.nonzero(err <= tol)[0]
    return {"lmin": lmin, "lmax": lmax, "err": err, "bound": chebyshev_bound(np.arange(max_iters + 1), lmin, lmax),
            "iters": int(hit[0]) if hit.size else None}


def cosh_sum(X):
    """f(x, y, z) = cosh(x + y + z), the test function of Sec. 3.2."""
    return np.cosh(X[..., 0] + X[..., 1] + X[..., 2])


def _rule_data(ev, N, nq):
    a, b, c, w = reference_rule(nq)
    r, s, t = abc_to_rst(a, b, c)
    X, Jac = map_points(ev, r, s, t)
    J = np.linalg.det(Jac)
    if np.any(J <= 0.0):
        raise ValueError("non-positive Jacobian")
    return a, b, c, w, X, J


def projection_errors(ev, N, f=cosh_sum, nq=None):
    """L2 projection errors of f onto each element's space, for the semi-nodal space
    span{phi_ijk} (Lemma 3) and the LSC-DG space span{psi_i / sqrt(J)}; ev: (K, 5, 3).

    Both projections and the errors use an nq-point rule per direction (default N + 4, so the
    semi-nodal mass matrix is exact and the smooth integrands are resolved well past the
    errors compared). Returns (semi-nodal error, LSC-DG error, |f|), each the L2 norm over all
    elements."""
    nq = N + 4 if nq is None else nq
    a, b, c, w, X, J = _rule_data(ev, N, nq)
    fv = f(X)
    wJ = w[None, :] * J
    # semi-nodal: M c = V^T W f per element
    V = phi(N, a, b, c)[0]
    M = np.einsum("kq,qi,qj->kij", wJ, V, V)
    rhs = np.einsum("kq,qi,kq->ki", wJ, V, fv)
    coef = np.linalg.solve(M, rhs[..., None])[..., 0]
    e_sn = fv - np.einsum("qi,ki->kq", V, coef)
    # LSC-DG: basis psi_i / sqrt(J), mass = reference mass of psi (identity up to the rule)
    P = psi(N, a, b, c)[0]
    sq = np.sqrt(J)
    Mref = np.einsum("q,qi,qj->ij", w, P, P)
    rhs_l = np.einsum("kq,qi,kq->ki", wJ / sq, P, fv)
    coef_l = np.linalg.solve(Mref, rhs_l.T).T
    e_lsc = fv - np.einsum("qi,ki->kq", P, coef_l) / sq
    nrm = np.sqrt(np.sum(wJ * fv ** 2))
    return float(np.sqrt(np.sum(wJ * e_sn ** 2))), float(np.sqrt(np.sum(wJ * e_lsc ** 2))), float(nrm)
