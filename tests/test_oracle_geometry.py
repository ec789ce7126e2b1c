"""Pins for oracle/geometry.py: Bedrosian vertex functions and Lemma 1."""

import numpy as np
import pytest

from oracle.basis import abc_to_rst
from oracle.geometry import REF_VERTICES, map_points, vertex_functions
from paper_1502_07703_gb300.mesh import make_pyramid_mesh


def _random_abc(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.95, 0.95, (3, n))


def test_nodal_and_partition_of_unity():
    r, s, t = REF_VERTICES[:, 0], REF_VERTICES[:, 1], np.minimum(REF_VERTICES[:, 2], 1 - 1e-12)
    vals, _ = vertex_functions(r, s, t)
    np.testing.assert_allclose(vals, np.eye(5), atol=1e-10)
    a, b, c = _random_abc(50, 1)
    vals, grads = vertex_functions(*abc_to_rst(a, b, c))
    np.testing.assert_allclose(vals.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(grads.sum(axis=1), 0.0, atol=1e-13)


def test_gradients_by_finite_difference():
    a, b, c = _random_abc(30, 2)
    r, s, t = abc_to_rst(a, b, c)
    _, g = vertex_functions(r, s, t)
    h = 1e-6
    for d in range(3):
        dp = [r, s, t]
        dm = [r, s, t]
        dp = [x + (h if i == d else 0) for i, x in enumerate(dp)]
        dm = [x - (h if i == d else 0) for i, x in enumerate(dm)]
        fd = (vertex_functions(*dp)[0] - vertex_functions(*dm)[0]) / (2 * h)
        np.testing.assert_allclose(g[..., d], fd, atol=1e-7)


def test_identity_map_has_unit_jacobian():
    a, b, c = _random_abc(40, 3)
    r, s, t = abc_to_rst(a, b, c)
    X, Jac = map_points(REF_VERTICES[None], r, s, t)
    np.testing.assert_allclose(X[0], np.stack([r, s, t], axis=1), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(Jac[0]), 1.0, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma1_jacobian_bilinear_in_ab_constant_in_c(seed):
    """Lemma 1: for a vertex-mapped pyramid (non-planar base allowed) J in Q_{1,1,0}."""
    rng = np.random.default_rng(seed)
    verts = REF_VERTICES + rng.uniform(-0.3, 0.3, (5, 3))
    a, b, c = _random_abc(60, 10 + seed)
    J = np.linalg.det(map_points(verts[None], *abc_to_rst(a, b, c))[1][0])
    A = np.stack([np.ones_like(a), a, b, a * b], axis=1)
    coef, *_ = np.linalg.lstsq(A, J, rcond=None)
    assert np.max(np.abs(A @ coef - J)) < 1e-12 * np.max(np.abs(J))
    J2 = np.linalg.det(map_points(verts[None], *abc_to_rst(a, b, -c))[1][0])
    np.testing.assert_allclose(J, J2, rtol=1e-12)


def test_mesh_volume_and_positive_jacobian():
    from oracle.dg import PyramidDG
    v, e = make_pyramid_mesh(3, 2, 2, delta=0.1, seed=4)
    dg = PyramidDG(v, e, 2)
    assert np.all(dg.J > 0)
    assert abs(dg.volumes().sum() - 1.0) < 1e-13
    # an unperturbed hex cut into 6 pyramids: each has volume h^3/6
    v, e = make_pyramid_mesh(2, delta=0.0)
    dg = PyramidDG(v, e, 1)
    np.testing.assert_allclose(dg.volumes(), (0.5 ** 3) / 6, rtol=1e-13)
