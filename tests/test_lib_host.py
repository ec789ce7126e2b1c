"""Host-side tests of libpyrdg.so that need no GPU: the library loads, exports
every function include/pyrdg.h declares, its FP64 builder produces the right
Gauss rules and face connectivity, and setup rejects bad input before any
device work."""

import ctypes
import os
import re

import numpy as np
import pytest
import scipy.special

from oracle.basis import abc_to_rst
from oracle.geometry import map_points
from paper_1502_07703_gb300 import binding
from paper_1502_07703_gb300.mesh import make_pyramid_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1502_07703_gb300 import build
    build.build()


def test_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "pyrdg.h")).read()
    names = set(re.findall(r"\b(pyr_dg_\w+)\s*\(", header))
    assert len(names) >= 15
    L = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("ab", [(0, 0), (1, 0), (2, 0), (9, 0)])
@pytest.mark.parametrize("n", [1, 2, 4, 8, 10])
def test_builder_gauss_jacobi_matches_scipy(n, ab):
    x, w = binding.gauss_jacobi(n, *ab)
    xs, ws = scipy.special.roots_jacobi(n, *ab)
    np.testing.assert_allclose(x, xs, atol=2e-15)
    np.testing.assert_allclose(w, ws, rtol=2e-13)


def _face_abc(N, face, idx):
    """Cube coordinates of face point idx, as include/pyrdg.h documents them."""
    n1 = N + 1
    xg, _ = scipy.special.roots_jacobi(n1, 0, 0)
    xf, _ = scipy.special.roots_jacobi(n1, 1, 0)
    e, m = idx % n1, idx // n1
    return {0: (xg[e], xg[m], -1.0), 1: (xg[e], -1.0, xf[m]), 2: (1.0, xg[e], xf[m]),
            3: (xg[e], 1.0, xf[m]), 4: (-1.0, xg[e], xf[m])}[face]


@pytest.mark.parametrize("N", [1, 3, 4])
def test_connectivity_symmetric_and_coincident(N):
    v, e = make_pyramid_mesh(3, 2, 2, delta=0.1, seed=3)
    mapP, nb = binding.connectivity(v, e, N)
    K = e.shape[0]
    n2 = (N + 1) ** 2
    Nfc = 5 * n2
    assert nb == 2 * (3 * 2 + 3 * 2 + 2 * 2)  # hex faces on the box boundary
    g = np.arange(K * Nfc)
    assert np.all(mapP[mapP] == g)
    bnd = mapP == g
    assert bnd.sum() == nb * n2
    # physical coordinates of every point and of its match, by the oracle's vertex map
    abc = np.array([_face_abc(N, f, i) for f in range(5) for i in range(n2)])
    X, _ = map_points(v[e], *abc_to_rst(abc[:, 0], abc[:, 1], abc[:, 2]))
    X = X.reshape(-1, 3)
    np.testing.assert_allclose(X[mapP], X, atol=1e-13)


def test_connectivity_rejects_nonconforming_and_bad_index():
    v, e = make_pyramid_mesh(1, delta=0.0)
    # two pyramids glued along a triangle whose collapse vertex differs on the two sides
    bad = e.copy()
    bad[1] = [bad[1][4], bad[1][1], bad[1][2], bad[1][3], bad[1][0]]
    with pytest.raises(binding.PyrDGError):
        binding.connectivity(v, bad, 2)
    oob = e.copy()
    oob[0, 0] = len(v)
    with pytest.raises(binding.PyrDGError, match="BAD_MESH"):
        binding.connectivity(v, oob, 2)


def test_setup_rejects_bad_input_before_device_work():
    v, e = make_pyramid_mesh(1, delta=0.0)
    with pytest.raises(binding.PyrDGError, match="UNSUPPORTED_N"):
        binding.Solver(v, e, 0)
    with pytest.raises(binding.PyrDGError, match="UNSUPPORTED_N"):
        binding.Solver(v, e, 8)
    inv = e.copy()
    inv[:, [1, 3]] = inv[:, [3, 1]]  # mirror the base order: J < 0
    with pytest.raises(binding.PyrDGError, match="BAD_MESH"):
        binding.Solver(v, inv, 2)
    with pytest.raises(binding.PyrDGError, match="BAD_ARG"):
        binding.Solver(v, e, 2, tau=-1.0)


def test_raw_abi_null_and_range_checks():
    L = binding.lib()
    h = ctypes.c_void_p()
    assert L.pyr_dg_setup(None, 0, None, 0, 3, None, ctypes.byref(h)) == -1
    assert L.pyr_dg_step(None, 1, 0.1) == -1
    assert L.pyr_dg_error(None, None, None) == -1
    assert L.pyr_dg_set_error_cache(None, 1) == -1
    assert b"null" in L.pyr_dg_last_error()
    x = np.empty(4)
    assert L.pyr_dg_host_gauss_jacobi(0, 0.0, 0.0, x.ctypes.data_as(binding._c_dp), x.ctypes.data_as(binding._c_dp)) == -1


def test_periodic_connectivity_matches_every_face():
    N = 2
    v, e = make_pyramid_mesh(3, 2, 2, delta=0.1, seed=8)
    mapP, nb = binding.connectivity_periodic(v, e, N, box=(0.0, 1.0))
    assert nb == 0
    g = np.arange(mapP.size)
    assert np.all(mapP[mapP] == g) and np.all(mapP != g)
    n2 = (N + 1) ** 2
    abc = np.array([_face_abc(N, f, i) for f in range(5) for i in range(n2)])
    X, _ = map_points(v[e], *abc_to_rst(abc[:, 0], abc[:, 1], abc[:, 2]))
    X = X.reshape(-1, 3)
    d = np.mod(X[mapP] - X + 0.5, 1.0) - 0.5
    assert np.max(np.abs(d)) < 1e-13


def test_advection_setup_requires_periodic_box():
    v, e = make_pyramid_mesh(1)
    with pytest.raises(binding.PyrDGError, match="BAD_ARG"):
        binding.Solver(v, e, 2, equation="advection")


def test_setup_rejects_empty_and_degenerate_meshes():
    v, e = make_pyramid_mesh(1, delta=0.0)
    with pytest.raises(binding.PyrDGError, match="BAD_ARG"):
        binding.Solver(v, e[:0], 2)                # no elements
    with pytest.raises(binding.PyrDGError, match="BAD_ARG"):
        binding.Solver(v[:4], e[:0], 2)            # fewer than 5 vertices
    flat = e.copy()
    flat[:, 4] = flat[:, 0]                        # apex on a base vertex: J = 0
    with pytest.raises(binding.PyrDGError, match="BAD_MESH"):
        binding.Solver(v, flat, 2)
    bad = e.copy()
    bad[0, 2] = v.shape[0]                         # vertex index out of range
    with pytest.raises(binding.PyrDGError, match="BAD"):
        binding.Solver(v, bad, 2)


def test_newer_calls_check_their_arguments_on_the_host():
    """Null handles and out-of-range arguments of the nodal, tensor-core, L2-distance and batch
    launch-mode calls are refused before any device work."""
    L = binding.lib()
    assert L.pyr_dg_l2_diff(None, None, None, None, None) == -1
    assert L.pyr_dg_set_tensor_mixing(None, 1) == -1
    assert L.pyr_dg_batch_launch_mode(None, None, None) == -1
    assert L.pyr_dg_batch_set_launch_mode(None, 1) == -1
    x = np.empty(3 * 100)
    assert L.pyr_dg_host_nodal_points(0, x.ctypes.data_as(binding._c_dp)) == -3
    assert L.pyr_dg_host_nodal_points(8, x.ctypes.data_as(binding._c_dp)) == -3
    assert L.pyr_dg_host_nodal_points(3, None) == -1
    v, e = make_pyramid_mesh(1)
    for kw in ({"precision": "f32"}, {"equation": "advection", "periodic": (0.0, 1.0)}):
        with pytest.raises(binding.PyrDGError, match="BAD_ARG"):
            binding.Solver(v, e, 2, basis="nodal", **kw)
    o = binding.Opts()
    L.pyr_dg_default_opts(ctypes.byref(o))
    assert o.basis == binding.PYR_DG_MODAL
    o.basis = 7
    V = np.ascontiguousarray(v, dtype=np.float64)
    E = np.ascontiguousarray(e, dtype=np.int32)
    h = ctypes.c_void_p()
    assert L.pyr_dg_setup(V.ctypes.data_as(binding._c_dp), V.shape[0], E.ctypes.data_as(binding._c_i32p),
                          E.shape[0], 2, ctypes.byref(o), ctypes.byref(h)) == -1
    assert b"basis" in L.pyr_dg_last_error()


def test_setup_refuses_sizes_beyond_its_index_range():
    """Element counts whose face-point index K * 5(N+1)^2 or grid size would overflow 32 bits are
    refused before the arrays are read (a one-element array stands in for the claimed size)."""
    L = binding.lib()
    v, e = make_pyramid_mesh(1)
    V = np.ascontiguousarray(v, dtype=np.float64)
    E = np.ascontiguousarray(e[:1], dtype=np.int32)
    h = ctypes.c_void_p()
    for K, N in ((2 ** 31 // 125 + 1, 4), (2 ** 31 // 320 + 1, 7), (2 ** 31, 1)):
        rc = L.pyr_dg_setup(V.ctypes.data_as(binding._c_dp), V.shape[0], E.ctypes.data_as(binding._c_i32p), K, N,
                            None, ctypes.byref(h))
        assert rc == -1 and not h.value, (K, N, rc)
        assert b"exceeds" in L.pyr_dg_last_error()
