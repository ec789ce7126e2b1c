"""Vertex map of a pyramid from Bedrosian's vertex functions (oracle; test infrastructure only).

Sec. 2 maps the reference pyramid to a physical one by F(r,s,t) = sum_i V_i v_i(r,s,t).
The printed v_2, v_3, v_4 are garbled (v_3 = -v_1 as printed, and v_2/v_4 do not
vanish at the right vertices). Read as the nodal set of the five vertices
(-1,-1,-1), (1,-1,-1), (1,1,-1), (-1,1,-1), (-1,-1,1):
    v1 =  (r+t)(s+t) / (2(1-t))
    v2 = -(r+1)(s+t) / (2(1-t))
    v3 =  (r+1)(s+1) / (2(1-t))
    v4 = -(r+t)(s+1) / (2(1-t))
    v5 =  (1+t)/2
Each is 1 at its own vertex and 0 at the other four, and they sum to 1.

Pinned by tests/test_oracle_geometry.py: nodality and partition of unity; the
identity map on the reference pyramid gives J = 1; Lemma 1 (J is bilinear in
(a, b) and constant in c), checked by sampling; sum of element volumes equals
the box volume; finite-difference check of the analytic derivatives.
"""

from __future__ import annotations

import numpy as np

REF_VERTICES = np.array(
    [[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [1.0, 1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]]
)


def vertex_functions(r, s, t):
    """Values and (r, s, t)-gradients of v1..v5; shapes (npts, 5) and (npts, 5, 3)."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    D = 2.0 * (1.0 - t)
    # numerators N_i and their partial derivatives; v_i = N_i / D, dD/dt = -2
    Nv = [(r + t) * (s + t), -(r + 1.0) * (s + t), (r + 1.0) * (s + 1.0), -(r + t) * (s + 1.0)]
    Nr = [s + t, -(s + t), s + 1.0, -(s + 1.0)]
    Ns = [r + t, -(r + 1.0), r + 1.0, -(r + t)]
    Nt = [(r + t) + (s + t), -(r + 1.0), np.zeros_like(t), -(s + 1.0)]
    vals = np.empty(r.shape + (5,))
    grads = np.empty(r.shape + (5, 3))
    for i in range(4):
        vals[..., i] = Nv[i] / D
        grads[..., i, 0] = Nr[i] / D
        grads[..., i, 1] = Ns[i] / D
        grads[..., i, 2] = Nt[i] / D + 2.0 * Nv[i] / (D * D)
    vals[..., 4] = (1.0 + t) / 2.0
    grads[..., 4, 0] = 0.0
    grads[..., 4, 1] = 0.0
    grads[..., 4, 2] = 0.5
    return vals, grads


def map_points(elem_verts, r, s, t):
    """Physical points x = F(r,s,t) and Jacobian matrices dx/d(r,s,t).

    elem_verts: (K, 5, 3). Returns X (K, npts, 3) and Jac (K, npts, 3, 3) with
    Jac[..., m, d] = d x_m / d (r, s, t)_d.
    """
    vals, grads = vertex_functions(r, s, t)
    X = np.einsum("pi,kim->kpm", vals, elem_verts)
    Jac = np.einsum("pid,kim->kpmd", grads, elem_verts)
    return X, Jac


def jacobian_and_inverse(Jac):
    """J = det(dx/drst) and the inverse matrix d(r,s,t)/dx (rows: grad r, grad s, grad t)."""
    J = np.linalg.det(Jac)
    inv = np.linalg.inv(Jac)
    return J, inv
