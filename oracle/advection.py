"""Scalar advection on pyramids (oracle; test infrastructure only).

Sec. 4.1: u_t + div(beta u) = 0 on a periodic box, beta constant, with the
alpha-flux of Sec. 4.1 (alpha = 1 upwind, 0 central). The printed surface term
((beta_n - alpha |beta_n|)/2) v [[u]] with [[u]] = u- - u+ grows energy; the
reading taken is the standard upwind-weighted term with the jump u+ - u-:
    M du/dt = -( S^beta u + L^f F ),   F = ((beta_n - alpha |beta_n|)/2) (u+ - u-),
S^beta = sum_m beta_m S^m. Its semi-discrete energy identity,
dE/dt = -sum_interior faces (alpha |beta_n| / 2) int [[u]]^2, is pinned in
tests/test_oracle_advection.py. Same dense-matrix route as oracle/dg.py, whose
geometry, matrices and (periodic) face matching are reused.
"""

from __future__ import annotations

import numpy as np

from .dg import LSRK_A, LSRK_B, PyramidDG


def exact_advection(x, y, z, t, beta, lo=0.0, hi=1.0):
    """u0(x - beta t) with u0 = sin(2 pi X) cos(2 pi Y) sin(2 pi Z), X = (x - lo)/(hi - lo)."""
    L = hi - lo
    k = 2.0 * np.pi / L
    return (np.sin(k * (x - beta[0] * t - lo)) * np.cos(k * (y - beta[1] * t - lo))
            * np.sin(k * (z - beta[2] * t - lo)))


class PyramidAdvection:
    """Dense-matrix DG for u_t + div(beta u) = 0 on a periodic pyramid mesh (state (K, 1, Np), psi basis)."""

    def __init__(self, vertices, EToV, N, beta=(1.0, 0.0, 0.0), alpha=1.0, box=(0.0, 1.0)):
        self.dg = PyramidDG(vertices, EToV, N, tau=0.0, bc="wall", periodic=box)
        if not np.all(self.dg.interior):
            raise ValueError("advection needs a fully periodic mesh (every face matched)")
        self.beta = np.asarray(beta, dtype=np.float64)
        self.alpha = float(alpha)
        self.box = box
        self.N = N
        self.Np = self.dg.Np
        self.K = self.dg.K
        self.Sb = np.einsum("m,kmij->kij", self.beta, self.dg.S)
        self.bn = np.einsum("m,kfqm->kfq", self.beta, self.dg.nrm)

    def rhs(self, U):
        dg = self.dg
        um = np.einsum("fqn,kn->kfq", dg.Vf, U[:, 0])
        up = um.reshape(-1)[dg.mapP].reshape(um.shape)
        F = 0.5 * (self.bn - self.alpha * np.abs(self.bn)) * (up - um)
        W = dg.fw[None] * dg.sJ
        r = np.einsum("kij,kj->ki", self.Sb, U[:, 0]) + np.einsum("fqi,kfq->ki", dg.Vf, W * F)
        return -np.einsum("kij,kj->ki", dg.Minv, r)[:, None, :]

    def lsrk4(self, U, dt, nsteps):
        U = U.copy()
        res = np.zeros_like(U)
        for _ in range(nsteps):
            for s in range(5):
                res = LSRK_A[s] * res + dt * self.rhs(U)
                U = U + LSRK_B[s] * res
        return U

    def project_exact(self, t):
        lo, hi = self.box
        return self.dg.project(lambda X: np.repeat(exact_advection(X[..., 0], X[..., 1], X[..., 2], t, self.beta,
                                                                   lo, hi)[..., None], 4, axis=-1))[:, :1]

    def energy(self, U):
        return 0.5 * np.einsum("ki,kij,kj->", U[:, 0], self.dg.M, U[:, 0])

    def dissipation(self, U):
        """-dE/dt predicted by the flux: alpha |beta_n| / 4 [[u]]^2 per point side, weighted w sJ."""
        dg = self.dg
        um = np.einsum("fqn,kn->kfq", dg.Vf, U[:, 0])
        up = um.reshape(-1)[dg.mapP].reshape(um.shape)
        W = dg.fw[None] * dg.sJ
        return np.sum(W * 0.25 * self.alpha * np.abs(self.bn) * (up - um) ** 2)

    def error(self, U, t, nq=None):
        """L2 error against the exact solution with the (N+3)-point rule; (abs, rel)."""
        from .basis import abc_to_rst, psi, reference_rule
        from .geometry import map_points
        nq = self.N + 3 if nq is None else nq
        a, b, c, w = reference_rule(nq)
        V = psi(self.N, a, b, c)[0]
        X, Jac = map_points(self.dg.ev, *abc_to_rst(a, b, c))
        J = np.linalg.det(Jac)
        uh = np.einsum("qn,kn->kq", V, U[:, 0])
        lo, hi = self.box
        ue = exact_advection(X[..., 0], X[..., 1], X[..., 2], t, self.beta, lo, hi)
        e2 = np.einsum("q,kq,kq->", w, J, (uh - ue) ** 2)
        n2 = np.einsum("q,kq,kq->", w, J, ue ** 2)
        return np.sqrt(e2), np.sqrt(e2 / n2)

    def dt_cfl(self, cfl=0.5):
        return self.dg.dt_cfl(cfl) / max(1e-300, np.linalg.norm(self.beta))
