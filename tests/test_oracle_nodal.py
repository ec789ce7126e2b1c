"""The layered nodal set of the nodal variant (oracle/nodal.py, Sec. 4.4.1), pinned by its
defining properties: GLL points (library Legendre polynomials, exactness of the GLL rule),
node counts on every face as Sec. 4.4.1 asks, unisolvency, coincident face nodes across shared
faces of a mesh, and the host builder's nodes against this definition."""

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle.basis import abc_to_rst, num_modes
from oracle.geometry import map_points
from oracle.nodal import gll, nodal_from_psi, nodal_points, psi_from_nodal, psi_vandermonde
from paper_1502_07703_gb300.mesh import make_pyramid_mesh


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8])
def test_gll_points_and_rule(n):
    """End points and the zeros of P'_{n-1} (numpy's Legendre series); the weights
    2 / (n(n-1) P_{n-1}(x)^2) integrate x^k exactly for k <= 2n - 3."""
    x = gll(n)
    assert x[0] == -1.0 and x[-1] == 1.0 and np.all(np.diff(x) > 0)
    dP = npleg.legder([0.0] * (n - 1) + [1.0])
    np.testing.assert_allclose(npleg.legval(x[1:-1], dP), 0.0, atol=1e-11)
    P = npleg.legval(x, [0.0] * (n - 1) + [1.0])
    w = 2.0 / (n * (n - 1) * P ** 2)
    for k in range(2 * n - 2):
        np.testing.assert_allclose(np.sum(w * x ** k), (2.0 / (k + 1)) if k % 2 == 0 else 0.0, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_nodal_set_counts_on_faces_and_unisolvency(N):
    X = nodal_points(N)
    a, b, c = X[:, 0], X[:, 1], X[:, 2]
    assert X.shape == (num_modes(N), 3)
    apex = c == 1.0
    assert np.count_nonzero(apex) == 1
    assert np.count_nonzero(c == -1.0) == (N + 1) ** 2  # the quadrilateral face
    tri = (N + 1) * (N + 2) // 2
    for on_face in (a == -1.0, a == 1.0, b == -1.0, b == 1.0):
        assert np.count_nonzero(on_face & ~apex) + 1 == tri
    # layers: (N+1-m)^2 nodes at the m-th GLL height
    heights, counts = np.unique(c, return_counts=True)
    np.testing.assert_allclose(heights, gll(N + 1))
    assert list(counts) == [(N + 1 - m) ** 2 for m in range(N + 1)]
    # unisolvent: the Vandermonde of the orthonormal basis is well conditioned
    assert np.linalg.cond(psi_vandermonde(N)) < 1e3
    rng = np.random.default_rng(N)
    C = rng.standard_normal((2, 4, num_modes(N)))
    np.testing.assert_allclose(psi_from_nodal(N, nodal_from_psi(N, C)), C, atol=1e-12)


def _face_nodes(N, face):
    X = nodal_points(N)
    a, b, c = X[:, 0], X[:, 1], X[:, 2]
    sel = {0: c == -1.0, 1: (b == -1.0) | (c == 1.0), 2: (a == 1.0) | (c == 1.0),
           3: (b == 1.0) | (c == 1.0), 4: (a == -1.0) | (c == 1.0)}[face]
    return X[sel]


@pytest.mark.parametrize("N", [2, 4])
def test_shared_faces_carry_coincident_nodes(N):
    """Every face shared by two pyramids of a perturbed 2x2x1-hex mesh (triangles inside a hex,
    quadrilaterals between hexes) carries the same physical nodes from both sides."""
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=4)
    ev = np.asarray(v)[np.asarray(e)]
    faces = ((0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (3, 2, 4), (0, 3, 4))
    owner, shared = {}, 0
    for k, row in enumerate(np.asarray(e)):
        for f, fv in enumerate(faces):
            key = tuple(sorted(int(row[i]) for i in fv))
            if key in owner:
                k2, f2 = owner.pop(key)
                pts = []
                for kk, ff in ((k, f), (k2, f2)):
                    Y = _face_nodes(N, ff)
                    cy = np.minimum(Y[:, 2], 1.0 - 1e-13)  # the map's (r,s,t) form is 0/0 at the apex itself
                    Xp, _ = map_points(ev[kk:kk + 1], *abc_to_rst(Y[:, 0], Y[:, 1], cy))
                    assert np.all(np.isfinite(Xp))
                    pts.append(Xp[0][np.lexsort(np.round(Xp[0], 9).T)])
                np.testing.assert_allclose(pts[0], pts[1], atol=1e-12)
                shared += 1
            else:
                owner[key] = (k, f)
    assert shared == 24 * 2 + 4  # 12 triangles in each of the 4 hexes, 4 inner hex faces


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_library_nodal_points_match_the_definition(N):
    from paper_1502_07703_gb300.binding import host_nodal_points
    np.testing.assert_allclose(host_nodal_points(N), nodal_points(N), atol=1e-14)
