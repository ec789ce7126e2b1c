"""Nodal set and change of basis for the nodal variant of Sec. 4.4.1 (oracle; test infrastructure only).

Sec. 4.4.1 switches to a Lagrange basis at Np distinct points of the pyramid, with the face
points distributed like those of the neighbouring element types, so that a triangle face
carries (N+1)(N+2)/2 points and the quadrilateral face (N+1)^2. The paper takes its point
sets from a survey it cites; the reading taken here is the layered set
    layer m = 0..N at c = the m-th of the N+1 Gauss-Lobatto-Legendre (GLL) points (ascending),
    carrying the (N+1-m) x (N+1-m) grid of GLL points in (a, b); the apex layer is one node,
ordered by layer, then the b index, then the a index. The base (layer 0) is the (N+1)^2 GLL
grid; each triangle face gets, per layer, the GLL points along its edge, (N+1)(N+2)/2 in
all, symmetric under the edge reversal that matches two triangle faces sharing an apex.

The Lagrange basis at these nodes spans the pyramid's approximation space (the nodes are
unisolvent: the Vandermonde matrix is invertible, pinned in tests/test_oracle_nodal.py), so a
nodal state is the same function as its psi (or phi) coefficients; the oracle converts with
its own Vandermonde of the orthonormal basis psi at the nodes and solves the same dense
discretisation as for the modal basis.
"""

from __future__ import annotations

import numpy as np

from .basis import psi
from .rules import gauss_jacobi


def gll(n):
    """The n Gauss-Lobatto-Legendre points on [-1, 1] (ascending): the end points and the
    zeros of P'_{n-1}, which are the Gauss-Jacobi (1,1) points; n = 1 gives the midpoint 0."""
    if n == 1:
        return np.array([0.0])
    if n == 2:
        return np.array([-1.0, 1.0])
    x, _ = gauss_jacobi(n - 2, 1.0, 1.0)
    return np.concatenate([[-1.0], np.sort(x), [1.0]])


def nodal_points(N):
    """(Np, 3) collapsed coordinates (a, b, c) of the layered nodal set, state order."""
    cl = gll(N + 1)
    out = []
    for m in range(N + 1):
        nm = N + 1 - m
        xs = gll(nm) if nm > 1 else np.array([0.0])
        for q in range(nm):
            for p in range(nm):
                out.append((xs[p], xs[q], cl[m]))
    return np.array(out)


def psi_vandermonde(N):
    """V[i, n] = psi_n(node i): nodal values = V @ psi coefficients."""
    X = nodal_points(N)
    return psi(N, X[:, 0], X[:, 1], X[:, 2])[0]


def psi_from_nodal(N, U):
    """psi coefficients (K, nf, Np) of a nodal state (K, nf, Np)."""
    V = psi_vandermonde(N)
    K, nf, Np = U.shape
    return np.linalg.solve(V, U.reshape(K * nf, Np).T).T.reshape(K, nf, Np)


def nodal_from_psi(N, C):
    """Nodal values (K, nf, Np) of a psi-coefficient state."""
    return np.einsum("in,kcn->kci", psi_vandermonde(N), C)
