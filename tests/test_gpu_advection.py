"""GPU parity for scalar advection (Sec. 4.1) on a periodic pyramid mesh: the
CUDA path against the FP64 oracle (oracle/advection.py)."""

import numpy as np
import pytest

from _parity import TOL, check
from oracle.advection import PyramidAdvection
from paper_1502_07703_gb300.mesh import make_pyramid_mesh, random_state

pytestmark = pytest.mark.gpu

BETA = (1.0, 0.3, -0.2)


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
    return Solver(v, e, N, equation="advection", periodic=(0.0, 1.0), beta=BETA, **kw)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_advection_rhs_parity(torch_cuda, N, precision):
    torch = torch_cuda
    v, e = make_pyramid_mesh(3, 2, 2, delta=0.1, seed=30)
    for alpha in (1.0, 0.0):
        ad = PyramidAdvection(v, e, N, beta=BETA, alpha=alpha)
        U = random_state(ad.K, ad.Np, 50 + N)[:, :1]
        with _solver(v, e, N, precision=precision, tau=alpha) as s:
            assert s.nf == 1
            R = s.rhs(torch.tensor(U, dtype=s.torch_dtype, device="cuda")).double().cpu().numpy()
        Uin = U.astype(np.float32).astype(np.float64) if precision == "f32" else U
        Ro = ad.rhs(ad.dg.psi_from_phi(Uin))
        check(ad.dg, ad.dg.values_phi(R), ad.dg.values_psi(Ro), TOL[precision], alpha)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_advection_evolution_projection_and_error(torch_cuda, precision):
    v, e = make_pyramid_mesh(3, 3, 2, delta=0.05, seed=31)
    N = 3
    ad = PyramidAdvection(v, e, N, beta=BETA)
    dt = ad.dt_cfl(0.5)
    U0 = ad.project_exact(0.0)
    U10 = ad.lsrk4(U0, dt, 10)
    with _solver(v, e, N, precision=precision) as s:
        assert abs(s.dt_cfl(0.5) - dt) <= 1e-12 * dt
        s.project(0.0)
        P = s.get_state().astype(np.float64)
        s.step(10, dt)
        G = s.get_state().astype(np.float64)
        err = s.error()
    check(ad.dg, ad.dg.values_phi(P), ad.dg.values_psi(U0), 1e-13 if precision == "f64" else 1e-6, "projection")
    check(ad.dg, ad.dg.values_phi(G), ad.dg.values_psi(U10), TOL[precision], "10 steps")
    eo = ad.error(U10, 10 * dt)
    np.testing.assert_allclose(err, eo, rtol=1e-9 if precision == "f64" else 1e-3)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_advection_f32_stage_kernel_all_degrees(torch_cuda, N):
    """The single-launch FP32 advection kernel (several elements per CTA, ping-pong
    traces) at every degree: 6 steps from the projected field, taken in calls of 1, 2
    and 3 steps, against the oracle. 3x3x1 hexes give 54 pyramids, so with 4 or 8
    elements per CTA the last group runs past the end of the mesh."""
    v, e = make_pyramid_mesh(3, 3, 1, delta=0.1, seed=70 + N)
    ad = PyramidAdvection(v, e, N, beta=BETA)
    dt = ad.dt_cfl(0.5)
    U6 = ad.lsrk4(ad.project_exact(0.0), dt, 6)
    with _solver(v, e, N, precision="f32") as s:
        assert s.K == 54
        s.project(0.0)
        s.step(1, dt)
        s.step(2, dt)
        s.step(3, dt)
        G = s.get_state().astype(np.float64)
    check(ad.dg, ad.dg.values_phi(G), ad.dg.values_psi(U6), TOL["f32"])
