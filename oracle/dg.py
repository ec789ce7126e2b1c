"""Plain FP64 DG solver for the acoustic wave system on pyramids (oracle; test infrastructure only).

Follows Sec. 4.3 of the paper with rho = kappa = 1 (so c = 1 and
tau_p = tau_u = tau): for each element,
    M dp/dt   = -( sum_m S^m u_m + L^f F_p ),
    M du_m/dt = -( S^m p          + L^f F_{u_m} ),
with S^m_ij = int phi_i d(phi_j)/dx_m, L^f the face integrals, and the flux of
Sec. 4.3 read with jumps [[q]] = q+ - q-:
    F_p = 1/2 ( n.[[u]] - tau [[p]] ),   F_u = 1/2 n ( [[p]] - tau n.[[u]] ).
(The printed ODE system has rho where 1/rho belongs and S^k u_k in the velocity
equation where S^k p belongs; with rho = kappa = 1 the first is moot and the
second is read as S^k p.)

Everything is done the plain way, in the orthonormal rational basis psi of
Eq. (1): dense per-element M, S^m and face matrices from the cubature of
Sec. 4.1 (Nc = (N+1)^3 points: Gauss-Legendre in a and b, Gauss-Jacobi (2,0)
in c), dense inverse of M. Faces use a rule the paper does not state (Sec. 4.2
only counts "N_c^f points over all faces"); the reading taken is
    base quad:  (N+1)^2 Gauss-Legendre points in (a, b) at c = -1,
    triangles:  (N+1) Gauss-Legendre points along the base edge times (N+1)
                Gauss-Jacobi (1,0) points toward the apex,
which integrates products of traces exactly. Neighbours are found by matching
the physical coordinates of face points, so any conforming mesh whose shared
faces carry coincident points works.

Boundary conditions: 'wall' (rigid wall n.u = 0 by the mirror state p+ = p-,
u+ = u- - 2 (n.u-) n) and 'free' (free surface p = 0 of Sec. 4.3 by p+ = -p-,
u+ = u-). Exact standing-wave solutions for both are in ``exact_solution``.

Time stepping: the 5-stage 2N-storage fourth-order Runge-Kutta method of
Carpenter and Kennedy that Sec. 4.1 cites (its coefficients are not printed in
the paper; the published values are used).

Pinned by tests/test_oracle_dg.py (polynomial reproduction, free stream, the
semi-discrete energy identity, h-convergence, brute-force mass) and
tests/test_oracle_lsrk.py (order conditions).
"""

from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .basis import abc_to_rst, num_modes, phi, psi, reference_rule
from .geometry import jacobian_and_inverse, map_points
from .rules import gauss_jacobi, gauss_legendre

# Carpenter & Kennedy (1994), 5-stage 2N-storage RK4: res = A_s res + dt f; u += B_s res.
LSRK_A = np.array([
    0.0,
    -567301805773.0 / 1357537059087.0,
    -2404267990393.0 / 2016746695238.0,
    -3550918686646.0 / 2091501179385.0,
    -1275806237668.0 / 842570457699.0,
])
LSRK_B = np.array([
    1432997174477.0 / 9575080441755.0,
    5161836677717.0 / 13612068292357.0,
    1720146321549.0 / 2090206949498.0,
    3134564353537.0 / 4481467310338.0,
    2277821191437.0 / 14882151754819.0,
])
LSRK_C = np.array([
    0.0,
    1432997174477.0 / 9575080441755.0,
    2526269341429.0 / 6820363962896.0,
    2006345519317.0 / 3224310063776.0,
    2802321613138.0 / 2924317926251.0,
])


def exact_solution(bc, x, y, z, t):
    """Standing-wave solutions of p_t + div u = 0, u_t + grad p = 0.

    'wall': on [0,1]^3 with n.u = 0,
        p = cos(pi x) cos(pi y) cos(pi z) cos(sqrt(3) pi t),
        u = sin(pi x) cos(pi y) cos(pi z) sin(sqrt(3) pi t) / sqrt(3), cyclic.
    'free': the resonant cavity of Sec. 4.3 on [-1,1]^3 with p = 0,
        p = cos(pi x/2) cos(pi y/2) cos(pi z/2) cos(sqrt(3) pi t / 2),
        u = sin(pi x/2) cos(pi y/2) cos(pi z/2) sin(sqrt(3) pi t / 2) / sqrt(3), cyclic.
    Returns an array (..., 4) of (p, u, v, w).
    """
    k = np.pi if bc == "wall" else np.pi / 2.0
    om = np.sqrt(3.0) * k
    cx, cy, cz = np.cos(k * x), np.cos(k * y), np.cos(k * z)
    sx, sy, sz = np.sin(k * x), np.sin(k * y), np.sin(k * z)
    ct, st = np.cos(om * t), np.sin(om * t)
    s3 = np.sqrt(3.0)
    return np.stack([
        cx * cy * cz * ct,
        sx * cy * cz * st / s3,
        cx * sy * cz * st / s3,
        cx * cy * sz * st / s3,
    ], axis=-1)


def face_rules(N):
    """Reference face points and weights (see module docstring).

    Returns a list of 5 dicts with cube coordinates a, b, c (each (N+1)^2,
    first index fastest) and weights w for the face's own area measure:
    face 0 base t = -1 (params r, s); face 1 s = -1; face 2 r = -t;
    face 3 s = -t; face 4 r = -1 (params along the base edge and t).
    """
    n = N + 1
    xg, wg = gauss_legendre(n)
    xj, wj = gauss_jacobi(n, 1.0, 0.0)
    G2, G1 = np.meshgrid(xg, xg, indexing="ij")
    W2, W1 = np.meshgrid(wg, wg, indexing="ij")
    base = dict(a=G1.ravel(), b=G2.ravel(), c=-np.ones(n * n), w=(W1 * W2).ravel())
    C, E = np.meshgrid(xj, xg, indexing="ij")
    WC, WE = np.meshgrid(wj, wg, indexing="ij")
    e, cc, wt = E.ravel(), C.ravel(), (WE * WC).ravel() / 2.0  # (1-c)/2 of the collapse
    one = np.ones(n * n)
    return [
        base,
        dict(a=e, b=-one, c=cc, w=wt),
        dict(a=one, b=e, c=cc, w=wt),
        dict(a=e, b=one, c=cc, w=wt),
        dict(a=-one, b=e, c=cc, w=wt),
    ]


def _face_tangents(f, Jac):
    """Two tangent vectors of reference face f, from dx/d(r,s,t)."""
    Xr, Xs, Xt = Jac[..., 0], Jac[..., 1], Jac[..., 2]
    if f == 0:
        return Xr, Xs
    if f == 1:
        return Xr, Xt
    if f == 2:
        return Xs, Xt - Xr
    if f == 3:
        return Xr, Xt - Xs
    return Xs, Xt


class PyramidDG:
    """Dense-matrix DG discretisation on a pyramid mesh (state arrays (K, 4, Np), psi basis)."""

    def __init__(self, vertices, EToV, N, tau=1.0, bc="wall", chunk=512, periodic=None, threads=1):
        self.N = int(N)
        # threads > 1: the per-element contractions of traces / residual / rhs run on element
        # chunks in a thread pool (numpy releases the GIL in einsum); each element's arithmetic
        # is the same as with one thread. Used to time the oracle on all host cores.
        self.threads = max(1, int(threads))
        self._pool = None
        self.Np = num_modes(self.N)
        self.tau = float(tau)
        self.bc = bc
        ev = np.asarray(vertices, dtype=np.float64)[np.asarray(EToV)]
        self.ev = ev
        K = self.K = ev.shape[0]
        Np = self.Np

        # volume cubature (Sec. 4.1)
        a, b, c, w = reference_rule(self.N + 1)
        r, s, t = abc_to_rst(a, b, c)
        self.vol_abc = (a, b, c)
        self.w = w
        V, Vr, Vs, Vt = psi(self.N, a, b, c)
        self.V = V
        dref = np.stack([Vr, Vs, Vt], axis=1)  # (q, d, n)

        self.M = np.empty((K, Np, Np))
        self.S = np.empty((K, 3, Np, Np))
        self.J = np.empty((K, w.size))
        self.X = np.empty((K, w.size, 3))
        for k0 in range(0, K, chunk):
            sl = slice(k0, min(K, k0 + chunk))
            X, Jac = map_points(ev[sl], r, s, t)
            J, inv = jacobian_and_inverse(Jac)
            if np.any(J <= 0.0):
                raise ValueError("non-positive Jacobian at a volume cubature point")
            self.J[sl] = J
            self.X[sl] = X
            Dphys = np.einsum("kqdm,qdn->kqmn", inv, dref, optimize=True)  # d psi_n / d x_m
            wJ = w[None, :] * J
            self.M[sl] = np.einsum("kq,qi,qj->kij", wJ, V, V, optimize=True)
            self.S[sl] = np.einsum("kq,qi,kqmj->kmij", wJ, V, Dphys, optimize=True)
        self.Minv = np.linalg.inv(self.M)

        # faces
        self.frules = face_rules(self.N)
        nf = (self.N + 1) ** 2
        self.nf = nf
        self.Vf = np.empty((5, nf, Np))
        self.Xf = np.empty((K, 5, nf, 3))
        self.nrm = np.empty((K, 5, nf, 3))
        self.sJ = np.empty((K, 5, nf))
        centroid = ev.mean(axis=1)
        for f, fr in enumerate(self.frules):
            self.Vf[f] = psi(self.N, fr["a"], fr["b"], fr["c"])[0]
            rf, sf, tf = abc_to_rst(fr["a"], fr["b"], fr["c"])
            X, Jac = map_points(ev, rf, sf, tf)
            T1, T2 = _face_tangents(f, Jac)
            ns = np.cross(T1, T2)
            outward = np.einsum("kqm,kqm->k", ns, X - centroid[:, None, :])
            ns = ns * np.where(outward > 0.0, 1.0, -1.0)[:, None, None]
            sJ = np.linalg.norm(ns, axis=-1)
            self.Xf[:, f] = X
            self.sJ[:, f] = sJ
            self.nrm[:, f] = ns / sJ[..., None]
        self.fw = np.stack([fr["w"] for fr in self.frules])  # (5, nf)

        # connectivity: match face points by physical coordinates; with periodic = (lo, hi)
        # the box [lo, hi]^3 is a torus and points are matched modulo its period
        pts = self.Xf.reshape(-1, 3)
        hmin = np.cbrt(np.min(np.einsum("q,kq->k", w, self.J)))
        tol = 1e-8 * hmin
        if periodic is not None:
            lo, hi = float(periodic[0]), float(periodic[1])
            L = hi - lo
            pts = np.mod(pts - lo, L)
            pts = np.where(pts > L - 1e-9 * L, 0.0, pts)
            tree = cKDTree(pts, boxsize=L)
        else:
            tree = cKDTree(pts)
        dist, idx = tree.query(pts, k=2)
        mapP = np.where(dist[:, 1] < tol, idx[:, 1], -1)
        # the nearest point is the point itself unless two coincide exactly
        same = idx[:, 0] != np.arange(pts.shape[0])
        mapP = np.where(same & (dist[:, 0] < tol), idx[:, 0], mapP)
        inter = mapP >= 0
        if np.any(mapP[mapP[inter]] != np.nonzero(inter)[0]):
            raise ValueError("face point matching is not symmetric")
        per_face = inter.reshape(K, 5, nf)
        if np.any(per_face.any(axis=2) != per_face.all(axis=2)):
            raise ValueError("a face is only partly matched")
        self.mapP = mapP
        self.interior = inter

    # ------------------------------------------------------------------ operators
    def _per_element(self, fn, *arrays):
        """fn(*arrays) where every array's first axis runs over the elements: on one thread, or
        on contiguous element chunks in the thread pool, concatenated in element order."""
        if self.threads == 1 or self.K < 2 * self.threads:
            return fn(*arrays)
        if self._pool is None:
            from concurrent.futures import ThreadPoolExecutor
            self._pool = ThreadPoolExecutor(self.threads)
        bounds = np.linspace(0, self.K, self.threads + 1).astype(int)
        parts = self._pool.map(lambda i: fn(*(a[bounds[i]:bounds[i + 1]] for a in arrays)), range(self.threads))
        return np.concatenate(list(parts), axis=0)

    def traces(self, U):
        """Values of the four fields at every face point, (K, 5, nf, 4)."""
        return self._per_element(lambda u: np.einsum("fqn,kcn->kfqc", self.Vf, u), U)

    def exterior(self, Uf):
        """Neighbour (or boundary mirror) values at every face point, same shape as Uf."""
        flat = Uf.reshape(-1, 4)
        plus = np.empty_like(flat)
        inter = self.interior
        plus[inter] = flat[self.mapP[inter]]
        bnd = ~inter
        n = self.nrm.reshape(-1, 3)[bnd]
        um = flat[bnd]
        if self.bc == "wall":
            un = np.einsum("qm,qm->q", n, um[:, 1:])
            plus[bnd, 0] = um[:, 0]
            plus[bnd, 1:] = um[:, 1:] - 2.0 * un[:, None] * n
        elif self.bc == "free":
            plus[bnd, 0] = -um[:, 0]
            plus[bnd, 1:] = um[:, 1:]
        else:
            raise ValueError(self.bc)
        return plus.reshape(Uf.shape)

    def fluxes(self, U):
        """Flux of Sec. 4.3 at every face point: (F_p, F_u) of shapes (K,5,nf), (K,5,nf,3)."""
        Um = self.traces(U)
        Up = self.exterior(Um)
        dp = Up[..., 0] - Um[..., 0]
        du = Up[..., 1:] - Um[..., 1:]
        nd = np.einsum("kfqm,kfqm->kfq", self.nrm, du)
        Fp = 0.5 * (nd - self.tau * dp)
        Fu = 0.5 * self.nrm * (dp - self.tau * nd)[..., None]
        return Fp, Fu, Um, Up

    def residual(self, U):
        """sum_m S^m u_m + L F_p and S^m p + L F_{u_m}: the bracket of Sec. 4.3, (K, 4, Np)."""
        p = U[:, 0]
        u = U[:, 1:]
        Fp, Fu, _, _ = self.fluxes(U)
        W = self.fw[None] * self.sJ  # (K, 5, nf)

        def part(S, p, u, WFp, WFu):
            out = np.empty((S.shape[0],) + U.shape[1:])
            out[:, 0] = np.einsum("kmij,kmj->ki", S, u) + np.einsum("fqi,kfq->ki", self.Vf, WFp)
            out[:, 1:] = np.einsum("kmij,kj->kmi", S, p) + np.einsum("fqi,kfqm->kmi", self.Vf, WFu)
            return out

        return self._per_element(part, self.S, p, u, W * Fp, W[..., None] * Fu)

    def rhs(self, U):
        """dU/dt = -M^{-1} (volume + surface terms), dense inverse per element."""
        return self._per_element(lambda Mi, R: -np.einsum("kij,kcj->kci", Mi, R), self.Minv, self.residual(U))

    def lsrk4(self, U, dt, nsteps):
        """Advance nsteps of the 2N-storage RK4 with fixed dt; returns the new state."""
        U = U.copy()
        res = np.zeros_like(U)
        for _ in range(nsteps):
            for s in range(5):
                res = LSRK_A[s] * res + dt * self.rhs(U)
                U = U + LSRK_B[s] * res
        return U

    # ------------------------------------------------------------- projections
    def project(self, fn):
        """L2 projection of fn(X) -> (K, Nc, 4) onto the element spaces (volume rule)."""
        vals = fn(self.X)
        b = np.einsum("q,kq,qi,kqc->kci", self.w, self.J, self.V, vals)
        return np.einsum("kij,kcj->kci", self.Minv, b)

    def project_exact(self, t):
        return self.project(lambda X: exact_solution(self.bc, X[..., 0], X[..., 1], X[..., 2], t))

    def energy(self, U):
        """E = 1/2 sum_K U^T M_K U over the four fields."""
        return 0.5 * np.einsum("kci,kij,kcj->", U, self.M, U)

    def dissipation(self, U):
        """-dE/dt predicted by the flux: tau/4 (dp^2 + (n.du)^2) per interior point side,
        tau (n.u-)^2 at wall points, tau (p-)^2 at free-surface points; weighted w sJ."""
        _, _, Um, Up = self.fluxes(U)
        W = self.fw[None] * self.sJ
        dp = Up[..., 0] - Um[..., 0]
        nd = np.einsum("kfqm,kfqm->kfq", self.nrm, Up[..., 1:] - Um[..., 1:])
        inter = self.interior.reshape(W.shape)
        d_int = 0.25 * self.tau * (dp ** 2 + nd ** 2)
        if self.bc == "wall":
            d_bnd = self.tau * np.einsum("kfqm,kfqm->kfq", self.nrm, Um[..., 1:]) ** 2
        else:
            d_bnd = self.tau * Um[..., 0] ** 2
        return np.sum(W * np.where(inter, d_int, d_bnd))

    def volumes(self):
        return np.einsum("q,kq->k", self.w, self.J)

    def surface_areas(self):
        return np.einsum("fq,kfq->k", self.fw, self.sJ)

    def dt_cfl(self, cfl=0.5):
        """dt = CFL / (C_N max_K |dK|/|K|), C_N = 2(N+1)(N+3)/3 (Sec. 4.3 spectral-radius fit)."""
        CN = 2.0 * (self.N + 1) * (self.N + 3) / 3.0
        return cfl / (CN * np.max(self.surface_areas() / self.volumes()))

    # ------------------------------------------------------------ evaluation
    def error(self, U, t, nq=None):
        """L2 error against the exact solution with an (N+3)-point rule; returns (abs, rel)."""
        nq = self.N + 3 if nq is None else nq
        a, b, c, w = reference_rule(nq)
        r, s, tt = abc_to_rst(a, b, c)
        V = psi(self.N, a, b, c)[0]
        X, Jac = map_points(self.ev, r, s, tt)
        J = np.linalg.det(Jac)
        Uh = np.einsum("qn,kcn->kqc", V, U)
        Ue = exact_solution(self.bc, X[..., 0], X[..., 1], X[..., 2], t)
        e2 = np.einsum("q,kq,kqc->", w, J, (Uh - Ue) ** 2)
        n2 = np.einsum("q,kq,kqc->", w, J, Ue ** 2)
        return np.sqrt(e2), np.sqrt(e2 / n2)

    def psi_from_phi(self, Uphi):
        """Convert semi-nodal (Lemma 3) coefficients to psi coefficients.

        psi is orthonormal on the reference pyramid, so its coefficients are
        reference inner products, computed with a rule exact for psi*phi."""
        a, b, c, w = reference_rule(self.N + 1)
        Vpsi = psi(self.N, a, b, c)[0]
        Vphi = phi(self.N, a, b, c)[0]
        T = np.einsum("q,qi,qj->ij", w, Vpsi, Vphi)
        return np.einsum("ij,kcj->kci", T, Uphi)

    def values_psi(self, U):
        """Values of a psi-coefficient state at the volume cubature points, (K, Nc, 4)."""
        return np.einsum("qn,kcn->kqc", self.V, U)

    def values_phi(self, Uphi):
        """Values of a semi-nodal coefficient state at the volume cubature points, (K, Nc, 4)."""
        Vphi = phi(self.N, *self.vol_abc)[0]
        return np.einsum("qn,kcn->kqc", Vphi, Uphi)

    def rel_l2_points(self, A, B):
        """Quadrature-weighted relative L2 difference of two point-value arrays (K, Nc, 4)."""
        wJ = self.w[None, :] * self.J
        d2 = np.einsum("kq,kqc->", wJ, (A - B) ** 2)
        n2 = np.einsum("kq,kqc->", wJ, B ** 2)
        return np.sqrt(d2 / n2)

    def worst_element_rel(self, A, B, elems=None):
        """The worst element of two point-value arrays (K', Nc, 4) whose rows are the elements
        `elems` (default: all K, in order): max over elements of the quadrature-weighted L2
        difference on that element, divided by the larger of that element's norm of B and the
        root-mean-square element norm of B over the rows.

        A fault confined to one element (or one face of it) shows here at full size, where the
        mesh-wide relative L2 dilutes it by the square root of the element count; the floor at
        the mean element norm keeps elements where B nearly vanishes from dividing by ~0."""
        J = self.J if elems is None else self.J[np.asarray(elems)]
        if J.shape[0] != A.shape[0] or A.shape != B.shape:
            raise ValueError("point arrays and element list disagree")
        wJ = self.w[None, :] * J
        d2 = np.einsum("kq,kqc->k", wJ, (A - B) ** 2)
        n2 = np.einsum("kq,kqc->k", wJ, B ** 2)
        floor = np.mean(n2)
        return float(np.sqrt(np.max(d2 / np.maximum(n2, floor))))


def phi_states_l2_diff(vertices, EToV, N, A, B, chunk=4096):
    """Compare two semi-nodal coefficient states (K, 4, Np) of one mesh by their values at every
    element's volume cubature points, without the dense element matrices (large meshes):
    returns (mesh-wide quadrature-weighted relative L2 of A - B against B, worst element), the
    worst element as in PyramidDG.worst_element_rel."""
    ev = np.asarray(vertices, dtype=np.float64)[np.asarray(EToV)]
    a, b, c, w = reference_rule(N + 1)
    r, s, t = abc_to_rst(a, b, c)
    V = phi(N, a, b, c)[0]
    K = ev.shape[0]
    d2 = np.empty(K)
    n2 = np.empty(K)
    for k0 in range(0, K, chunk):
        sl = slice(k0, min(K, k0 + chunk))
        _, Jac = map_points(ev[sl], r, s, t)
        wJ = w[None, :] * np.linalg.det(Jac)
        Av = np.einsum("qn,kcn->kqc", V, np.asarray(A[sl], dtype=np.float64))
        Bv = np.einsum("qn,kcn->kqc", V, np.asarray(B[sl], dtype=np.float64))
        d2[sl] = np.einsum("kq,kqc->k", wJ, (Av - Bv) ** 2)
        n2[sl] = np.einsum("kq,kqc->k", wJ, Bv ** 2)
    rel = float(np.sqrt(d2.sum() / n2.sum()))
    worst = float(np.sqrt(np.max(d2 / np.maximum(n2, np.mean(n2)))))
    return rel, worst
