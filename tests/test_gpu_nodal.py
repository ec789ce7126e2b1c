"""GPU parity of the nodal variant (Sec. 4.4.1): the state holds nodal values at the layered
nodal set, M^{-1} goes through the change of basis to the semi-nodal basis, the triangle faces
are integrated with nodal face mass matrices. The discrete solution is the modal one, so the
CUDA path is compared with the FP64 oracle (dense psi-basis solver) after converting nodal
values to psi coefficients with the oracle's own Vandermonde (oracle/nodal.py), by point values
at every volume cubature point (mesh-wide and worst element), FP64 <= 1e-12."""

import numpy as np
import pytest

from _parity import TOL, check
from oracle.dg import PyramidDG
from oracle.nodal import nodal_from_psi, psi_from_nodal
from paper_1502_07703_gb300.mesh import make_pyramid_mesh, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_07703_gb300 import build
    build.build()
    return torch


def _solver(v, e, N, **kw):
    from paper_1502_07703_gb300.binding import Solver
    return Solver(v, e, N, precision="f64", basis="nodal", **kw)


def _rhs_parity(torch, v, e, N, bc="wall", tau=1.0, seed=0):
    dg = PyramidDG(v, e, N, tau=tau, bc=bc)
    U = random_state(dg.K, dg.Np, seed)  # nodal values
    with _solver(v, e, N, bc=bc, tau=tau) as s:
        R = s.rhs(torch.tensor(U, device="cuda")).cpu().numpy()
    R_or = dg.rhs(psi_from_nodal(N, U))
    check(dg, dg.values_psi(psi_from_nodal(N, R)), dg.values_psi(R_or), TOL["f64"], (N, bc, tau))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_nodal_rhs_parity_all_degrees(torch_cuda, N):
    v, e = make_pyramid_mesh(3, 2, 1, delta=0.1, seed=5)
    _rhs_parity(torch_cuda, v, e, N, seed=200 + N)


@pytest.mark.parametrize("bc,tau", [("wall", 0.0), ("free", 1.0), ("wall", 0.5)])
def test_nodal_rhs_flux_and_boundary_variants(torch_cuda, bc, tau):
    v, e = make_pyramid_mesh(2, 2, 2, delta=0.08, seed=6, domain=(0.0, 1.0) if bc == "wall" else (-1.0, 1.0))
    _rhs_parity(torch_cuda, v, e, 3, bc, tau, seed=9)


def test_nodal_rhs_single_element_and_partial_hex(torch_cuda):
    """A single pyramid (every face, triangles too, on the boundary) and a 2x1x1-hex mesh with
    one pyramid dropped (its neighbours' triangle faces become boundary faces)."""
    rng = np.random.default_rng(1)
    ref = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    v = ref + rng.uniform(-0.2, 0.2, ref.shape)
    for N in (1, 4):
        _rhs_parity(torch_cuda, v, np.array([[0, 1, 2, 3, 4]], dtype=np.int32), N, seed=N)
    v, e = make_pyramid_mesh(2, 1, 1, delta=0.1, seed=8)
    _rhs_parity(torch_cuda, v, e[:-1], 3, seed=3)


def test_nodal_evolution_error_norm_and_modal_equivalence(torch_cuda):
    """Config 1's mesh (2^3 hexes, +-0.05h, seed 0), N = 3, 10 LSRK4 steps from the projected
    standing wave: against the oracle, the error norm against the oracle's, and against the
    modal path (the same function in another basis)."""
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    N = 3
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 10)
    with _solver(v, e, N) as s:
        s.project(0.0)
        P = s.get_state()
        s.step(10, dt)
        Un = s.get_state()
        err = s.error()
        err_again = s.error()
        err_stored = s.error()
    check(dg, dg.values_psi(psi_from_nodal(N, P)), dg.values_psi(dg.project_exact(0.0)), 1e-13, "projection")
    check(dg, dg.values_psi(psi_from_nodal(N, Un)), dg.values_psi(U_or), TOL["f64"], "10 steps")
    for er in (err, err_again, err_stored):
        np.testing.assert_allclose(er, dg.error(U_or, 10 * dt), rtol=1e-9)
    with Solver(v, e, N, precision="f64") as m:
        m.project(0.0)
        m.step(10, dt)
        Um = m.get_state()
    check(dg, dg.values_psi(psi_from_nodal(N, Un)), dg.values_phi(Um), TOL["f64"], "nodal vs modal")


def test_nodal_state_roundtrip_and_rejections(torch_cuda):
    from paper_1502_07703_gb300.binding import PyrDGError, Solver
    v, e = make_pyramid_mesh(1, 1, 1, delta=0.05, seed=2)
    with _solver(v, e, 2) as s:
        U = nodal_from_psi(2, random_state(s.K, s.Np, 3))
        s.set_state(U, t=0.1)
        np.testing.assert_array_equal(s.get_state(), U)
    for kw in ({"precision": "f32"}, {"equation": "advection", "periodic": (0.0, 1.0)}):
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            Solver(v, e, 2, basis="nodal", **kw)


def test_nodal_full_size_sampled(torch_cuda):
    """The bench's mesh (32^3 hexes x 6 = 196,608 pyramids, +-0.05h, seed 1) at N = 4 in the
    nodal basis: one LSRK4 step from the projected standing wave, checked on sampled elements
    whose 6-hop neighbourhood the oracle advances (influence crosses one face per stage)."""
    from _parity import face_neighbours, patch as _patch
    v, e = make_pyramid_mesh(32, delta=0.05, seed=1)
    K, N = e.shape[0], 4
    nbrs = face_neighbours(e)
    rng = np.random.default_rng(23)
    samples = [int(x) for x in rng.choice(K, 2, replace=False)] + [K - 1]
    dt = PyramidDG(v, e[:6], N).dt_cfl(0.5)
    with _solver(v, e, N) as s:
        s.project(0.0)
        s.step(1, dt)
        U1 = s.get_state()
    for c in samples:
        patch = _patch(nbrs, c, 6)
        dg = PyramidDG(v, e[patch], N)
        i = patch.index(c)
        Up = dg.lsrk4(dg.project_exact(0.0), dt, 1)
        check(dg, dg.values_psi(psi_from_nodal(N, U1[patch]))[i:i + 1], dg.values_psi(Up)[i:i + 1], TOL["f64"], c,
              elems=[i])
