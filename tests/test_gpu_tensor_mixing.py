"""FP32 stage kernel with the level mixing on the tensor cores (tcgen05.mma kind::tf32, 3-term
split, FP32 accumulation in tensor memory): against the FP64 oracle (mesh-wide and worst
element, 1e-5) and against the CUDA-core FP32 kernel, at every degree it is built for."""

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


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_tensor_mixing_matches_oracle_and_cuda_core_path(torch_cuda, N):
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=80 + N)
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 5)
    states = {}
    for tc in (False, True):
        with Solver(v, e, N, precision="f32") as s:
            if tc:
                s.set_tensor_mixing(True)
            s.project(0.0)
            for _ in range(3):
                s.step(1, dt)
            s.step(2, dt)
            s.sync()  # raises TIMEOUT if a tensor-core completion wait gave up
            states[tc] = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(states[True]), dg.values_psi(U_or), TOL["f32"], ("tensor cores", N))
    rel = np.linalg.norm(states[True] - states[False]) / np.linalg.norm(states[False])
    assert rel <= 2e-6, rel


def test_tensor_mixing_on_a_larger_mesh_and_rejections(torch_cuda):
    """N = 7 on 8^3 hexes (3072 pyramids, many CTAs per SM, persistent loop over elements),
    10 steps against the CUDA-core kernel; handles it is not built for are refused."""
    from paper_1502_07703_gb300.binding import PyrDGError, Solver
    v, e = make_pyramid_mesh(8, delta=0.05, seed=1)
    N = 7
    out = {}
    for tc in (False, True):
        with Solver(v, e, N, precision="f32") as s:
            if tc:
                s.set_tensor_mixing(True)
            dt = s.dt_cfl(0.5)
            s.project(0.0)
            s.step(10, dt)
            s.sync()
            out[tc] = s.get_state().astype(np.float64)
    rel = np.linalg.norm(out[True] - out[False]) / np.linalg.norm(out[False])
    assert rel <= 2e-6, rel
    v1, e1 = make_pyramid_mesh(1, delta=0.05, seed=2)
    with Solver(v1, e1, 4, precision="f64") as s:
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            s.set_tensor_mixing(True)


@pytest.mark.parametrize("N", [1, 2, 5])
def test_tensor_mixing_single_element(torch_cuda, N):
    """One pyramid, every face on the wall: the persistent grid has one CTA and one element."""
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(1, delta=0.0)
    e = e[:1]
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 4)
    with Solver(v, e, N, precision="f32") as s:
        s.set_tensor_mixing(True)
        s.project(0.0)
        s.step(4, dt)
        s.sync()
        Ug = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f32"], N)
