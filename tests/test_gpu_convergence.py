"""Properties that hold at full size: optimal h-convergence of the FP64 path and
the FP32 error floor.

Sec. 4.3 reports optimal O(h^{N+1}) L2 convergence for the resonant cavity, and
that single precision follows the same rates until the L2 error stalls near
1e-6. Here the 8^3 -> 16^3 -> 32^3 hex sweep at N = 4 (the benchmark's mesh
family, up to 196,608 pyramids) is advanced to the same final time on the GPU,
and the errors against the exact standing wave give the observed rates."""

import numpy as np
import pytest

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


def _run(nx, N, precision, T):
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(nx, delta=0.05, seed=1)
    with Solver(v, e, N, precision=precision) as s:
        dt0 = s.dt_cfl(0.5)
        steps = int(np.ceil(T / dt0))
        s.project(0.0)
        s.step(steps, T / steps)
        return s.error()


def test_fp64_h_convergence_rate_n4(torch_cuda):
    T = 0.02
    errs = [_run(nx, 4, "f64", T)[0] for nx in (8, 16, 32)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates >= 4.5), (errs, rates)


def test_fp32_error_floor_near_1e6(torch_cuda):
    """FP32 on the finest mesh: the discretisation error (FP64) is ~1e-10, the FP32
    run's error sits at the rounding floor, between 1e-8 and 1e-5 relative."""
    T = 0.005
    e64 = _run(32, 4, "f64", T)[1]
    e32 = _run(32, 4, "f32", T)[1]
    assert e64 < 1e-8
    assert 1e-8 < e32 < 1e-5, e32
