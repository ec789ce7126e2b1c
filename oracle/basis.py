"""Pyramid bases on the collapsed cube (oracle; test infrastructure only).

Coordinates (Sec. 2): the reference pyramid is r, s in [-1, -t], t in [-1, 1];
the Duffy-type map from the cube (a, b, c) in [-1, 1]^3 is
    r = (1+a)(1-c)/2 - 1,   s = (1+b)(1-c)/2 - 1,   t = c.
Derivatives with respect to (r, s, t) follow by the chain rule
    d/dr = 2/(1-c) d/da,  d/ds = 2/(1-c) d/db,
    d/dt = (1+a)/2 d/dr + (1+b)/2 d/ds + d/dc,
with the powers of (1-c)/2 carried by each basis function cancelling 2/(1-c)
exactly, so no division by (1-c) is performed.

Two bases:
  * ``psi``: the rational orthonormal basis of Eq. (1), read (garbled print)
    as P_i(a) P_j(b) ((1-c)/2)^mu P_k^{(2mu+2,0)}(c), mu = max(i, j),
    0 <= i, j <= N, 0 <= k <= N - mu; normalised numerically on the reference
    pyramid. This is the oracle's working basis.
  * ``phi``: the semi-nodal basis of Lemma 3,
    l_i^k(a) l_j^k(b) ((1-c)/2)^k P_{N-k}^{(2k+3,0)}(c), 0 <= i, j <= k <= N,
    read with degree N-k and weights (2k+3, 0) for the c factor. The oracle
    uses it only to pin Lemma 3 and to read the CUDA path's coefficient
    arrays, ordered n = k(k+1)(2k+1)/6 + j(k+1) + i.

Pinned by tests/test_oracle_basis.py: reference Gram matrix of psi is the
identity; the counts equal (N+1)(N+2)(2N+3)/6; derivatives agree with finite
differences of the values; span(phi) = span(psi) (Lemma 4).
"""

from __future__ import annotations

import numpy as np

from .rules import gauss_jacobi, gauss_legendre, jacobi, jacobi_deriv, lagrange


def num_modes(N):
    """Number of basis functions, (N+1)(N+2)(2N+3)/6 (the count of Lemma 4)."""
    return (N + 1) * (N + 2) * (2 * N + 3) // 6


def abc_to_rst(a, b, c):
    """Duffy-type map of Sec. 2 from the cube to the reference pyramid."""
    r = (1.0 + a) * (1.0 - c) / 2.0 - 1.0
    s = (1.0 + b) * (1.0 - c) / 2.0 - 1.0
    return r, s, np.asarray(c, dtype=np.float64).copy()


def psi_indices(N):
    """(i, j, k) triples of Eq. (1): mu = max(i, j), k <= N - mu."""
    out = []
    for i in range(N + 1):
        for j in range(N + 1):
            mu = max(i, j)
            for k in range(N - mu + 1):
                out.append((i, j, k))
    return out


def _psi_raw(N, a, b, c):
    """Unnormalised psi and its (r, s, t) derivatives at cube points."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    idx = psi_indices(N)
    npts = a.size
    V = np.empty((npts, len(idx)))
    Vr = np.empty_like(V)
    Vs = np.empty_like(V)
    Vt = np.empty_like(V)
    h = (1.0 - c) / 2.0
    for n, (i, j, k) in enumerate(idx):
        mu = max(i, j)
        Pa, dPa = jacobi(i, 0, 0, a), jacobi_deriv(i, 0, 0, a)
        Pb, dPb = jacobi(j, 0, 0, b), jacobi_deriv(j, 0, 0, b)
        Pc = jacobi(k, 2 * mu + 2, 0, c)
        dPc = jacobi_deriv(k, 2 * mu + 2, 0, c)
        hm = h ** mu
        V[:, n] = Pa * Pb * hm * Pc
        hm1 = h ** (mu - 1) if mu >= 1 else np.zeros_like(h)
        dr = dPa * Pb * hm1 * Pc  # 2/(1-c) d/da, with (1-c)/2 cancelled
        ds = Pa * dPb * hm1 * Pc
        dc = Pa * Pb * (-(mu / 2.0) * hm1 * Pc + hm * dPc)
        Vr[:, n] = dr
        Vs[:, n] = ds
        Vt[:, n] = (1.0 + a) / 2.0 * dr + (1.0 + b) / 2.0 * ds + dc
    return V, Vr, Vs, Vt


def reference_rule(n):
    """Tensor rule on the reference pyramid: n-point Gauss-Legendre in a and b,
    n-point Gauss-Jacobi (2,0) in c; weights include the Duffy factor
    ((1-c)/2)^2 = (1-c)^2/4 (Sec. 4.1). Returns (a, b, c, w), a fastest."""
    xa, wa = gauss_legendre(n)
    xc, wc = gauss_jacobi(n, 2.0, 0.0)
    C, B, A = np.meshgrid(xc, xa, xa, indexing="ij")
    WC, WB, WA = np.meshgrid(wc, wa, wa, indexing="ij")
    return A.ravel(), B.ravel(), C.ravel(), (WA * WB * WC).ravel() / 4.0


def psi_norms(N):
    """Reference-pyramid L2 norms of the unnormalised psi (by an exact rule)."""
    a, b, c, w = reference_rule(N + 2)
    V, _, _, _ = _psi_raw(N, a, b, c)
    return np.sqrt(np.einsum("q,qn,qn->n", w, V, V))


def psi(N, a, b, c):
    """Orthonormal psi of Eq. (1) and its (r, s, t) derivatives; arrays (npts, Np)."""
    nrm = psi_norms(N)
    V, Vr, Vs, Vt = _psi_raw(N, a, b, c)
    return V / nrm, Vr / nrm, Vs / nrm, Vt / nrm


def phi_indices(N):
    """(i, j, k) of the semi-nodal basis in storage order (i fastest, then j, then k)."""
    return [(i, j, k) for k in range(N + 1) for j in range(k + 1) for i in range(k + 1)]


def phi(N, a, b, c):
    """Semi-nodal basis of Lemma 3 and its (r, s, t) derivatives; arrays (npts, Np)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    h = (1.0 - c) / 2.0
    cols = []
    for k in range(N + 1):
        xk, _ = gauss_legendre(k + 1)
        La, dLa = lagrange(xk, a)
        Lb, dLb = lagrange(xk, b)
        Pc = jacobi(N - k, 2 * k + 3, 0, c)
        dPc = jacobi_deriv(N - k, 2 * k + 3, 0, c)
        hk = h ** k
        hk1 = h ** (k - 1) if k >= 1 else np.zeros_like(h)
        for j in range(k + 1):
            for i in range(k + 1):
                v = La[:, i] * Lb[:, j] * hk * Pc
                dr = dLa[:, i] * Lb[:, j] * hk1 * Pc
                ds = La[:, i] * dLb[:, j] * hk1 * Pc
                dc = La[:, i] * Lb[:, j] * (-(k / 2.0) * hk1 * Pc + hk * dPc)
                dt = (1.0 + a) / 2.0 * dr + (1.0 + b) / 2.0 * ds + dc
                cols.append((v, dr, ds, dt))
    V = np.stack([t[0] for t in cols], axis=1)
    Vr = np.stack([t[1] for t in cols], axis=1)
    Vs = np.stack([t[2] for t in cols], axis=1)
    Vt = np.stack([t[3] for t in cols], axis=1)
    return V, Vr, Vs, Vt
