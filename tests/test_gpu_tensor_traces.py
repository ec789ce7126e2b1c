"""FP32 face traces on the tensor cores (the element-batched tcgen05 product T = U Phi_f^T,
TF32 3-term split, FP32 accumulation in tensor memory): the stepped state against the FP64
oracle (mesh-wide and worst element, 1e-5) and against the stage kernel's own traces, at every
degree; on a mesh of several tiles per CTA with a ragged last tile for every buffering and
operator-piece configuration; together with the tensor-core level mixing; and the handles it
is not built for."""

import numpy as np
import pytest

from _parity import TOL, check
from oracle.dg import PyramidDG
from paper_1502_07703_gb300.mesh import make_pyramid_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_07703_gb300 import build
    build.build()
    return torch


def _run(v, e, N, dt, nsteps, traces, mixing=False):
    from paper_1502_07703_gb300.binding import Solver
    with Solver(v, e, N, precision="f32") as s:
        s.set_tensor_traces(traces)  # explicit either way: the default depends on the degree
        if mixing:
            s.set_tensor_mixing(True)
        s.project(0.0)
        for _ in range(nsteps):
            s.step(1, dt)
        s.sync()  # raises TIMEOUT if a tensor-core completion wait gave up
        return s.get_state().astype(np.float64)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_tensor_traces_match_oracle_and_stage_kernel_traces(torch_cuda, N):
    """24 pyramids: one tile of 32 rows x 4 fields, 8 of its element slots past the mesh."""
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=90 + N)
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 5)
    tc = _run(v, e, N, dt, 5, True)
    cc = _run(v, e, N, dt, 5, False)
    check(dg, dg.values_phi(tc), dg.values_psi(U_or), TOL["f32"], ("tensor traces", N))
    rel = np.linalg.norm(tc - cc) / np.linalg.norm(cc)
    assert rel <= 2e-6, rel


@pytest.mark.parametrize("N", [4, 5, 6, 7])
def test_tensor_traces_several_tiles_per_cta(torch_cuda, N):
    """11^3 hexes = 7986 pyramids = 249 full tiles and one of 18 elements, over at most one CTA
    per SM: the persistent loop, the next tile's prefetch (N <= 5), the operator in one piece
    (N = 4) or streamed per tile in 2, 3 or 7 pieces (N = 5, 6, 7). 10 steps against the
    stage kernel's own traces."""
    v, e = make_pyramid_mesh(11, delta=0.05, seed=3)
    from paper_1502_07703_gb300.binding import Solver
    with Solver(v, e, N, precision="f32") as s:
        dt = s.dt_cfl(0.5)
    tc = _run(v, e, N, dt, 10, True)
    cc = _run(v, e, N, dt, 10, False)
    rel = np.linalg.norm(tc - cc) / np.linalg.norm(cc)
    assert rel <= 2e-6, rel


@pytest.mark.parametrize("N,nelem", [(2, 1), (5, 1), (7, 1), (3, 33), (6, 33)])
def test_tensor_traces_ragged_tiles(torch_cuda, N, nelem):
    """A single pyramid (one tile holding one element) and 33 pyramids (a full tile and one
    element), 4 steps against the oracle."""
    v, e = make_pyramid_mesh(3, 2, 1, delta=0.06, seed=60 + N)
    e = e[:nelem]
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 4)
    tc = _run(v, e, N, dt, 4, True)
    check(dg, dg.values_phi(tc), dg.values_psi(U_or), TOL["f32"], ("tensor traces, ragged", N, nelem))


def test_tensor_traces_with_tensor_mixing(torch_cuda):
    N = 5
    v, e = make_pyramid_mesh(2, 2, 2, delta=0.1, seed=7)
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 3)
    both = _run(v, e, N, dt, 3, True, mixing=True)
    check(dg, dg.values_phi(both), dg.values_psi(U_or), TOL["f32"], ("tensor traces + mixing", N))


def test_tensor_traces_rejections_and_switching_off(torch_cuda):
    from paper_1502_07703_gb300.binding import PyrDGError, Solver
    v, e = make_pyramid_mesh(2, delta=0.05, seed=2)
    with Solver(v, e, 5, precision="f64") as s:  # FP64 has them at N = 2..4 only
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            s.set_tensor_traces(True)
    with Solver(v, e, 3, precision="f32", equation="advection", periodic=(0.0, 1.0)) as s:
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            s.set_tensor_traces(True)
    with Solver(v, e, 4, precision="f32") as s:  # on, then off again: the stage kernel's own traces
        dt = s.dt_cfl(0.5)
        s.set_tensor_traces(True)
        s.set_tensor_traces(False)
        s.project(0.0)
        s.step(3, dt)
        off = s.get_state().astype(np.float64)
    assert np.array_equal(off, _run(v, e, 4, dt, 3, False))
