"""FP64 face traces on the tensor cores with FP64 accuracy (the trace map and each state row cut
into eight exact balanced BF16 digits, the level sums accumulated exactly in FP32 in tensor
memory, recombined with integer operations): the stepped state against the FP64 oracle (1e-12)
and against the CUDA-core FP64 trace kernel at every degree it is built for; several tiles per
CTA with a ragged last tile; single-element and one-past-a-tile meshes; states at the ends of
the exponent range and rows spanning many binades; the handles it is not built for."""

import numpy as np
import pytest

from _parity import TOL, check
from oracle.dg import PyramidDG
from paper_1502_07703_gb300.mesh import make_pyramid_mesh

pytestmark = pytest.mark.gpu

# the two trace paths differ by rounding only (both FP64-accurate)
TOL_PATHS = 1e-13


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_07703_gb300 import build
    build.build()
    return torch


def _run(v, e, N, dt, nsteps, traces, q0=None):
    from paper_1502_07703_gb300.binding import Solver
    with Solver(v, e, N, precision="f64") as s:
        s.set_tensor_traces(traces)
        if q0 is None:
            s.project(0.0)
        else:
            s.set_state(q0)
        s.step(nsteps, dt)
        s.sync()  # raises TIMEOUT if a tensor-core completion wait gave up
        return s.get_state()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N", [2, 3, 4])
def test_fp64_tensor_traces_match_oracle_and_trace_kernel(torch_cuda, N):
    """24 pyramids: three full tiles of 8 elements x 4 fields."""
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=90 + N)
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 5)
    tc = _run(v, e, N, dt, 5, True)
    cc = _run(v, e, N, dt, 5, False)
    check(dg, dg.values_phi(tc), dg.values_psi(U_or), TOL["f64"], ("fp64 tensor traces", N))
    assert _rel(tc, cc) <= TOL_PATHS


@pytest.mark.parametrize("N", [2, 3, 4])
def test_fp64_tensor_traces_several_tiles_per_cta(torch_cuda, N):
    """11^3 hexes = 7986 pyramids = 998 full tiles and one of 2 elements over one CTA per SM
    (the persistent loop, both accumulators and state slots, the exponent ring); 10 steps."""
    v, e = make_pyramid_mesh(11, delta=0.05, seed=3)
    from paper_1502_07703_gb300.binding import Solver
    with Solver(v, e, N, precision="f64") as s:
        dt = s.dt_cfl(0.5)
    assert _rel(_run(v, e, N, dt, 10, True), _run(v, e, N, dt, 10, False)) <= TOL_PATHS


@pytest.mark.parametrize("N,nelem", [(2, 1), (4, 1), (3, 9), (4, 9)])
def test_fp64_tensor_traces_ragged_tiles(torch_cuda, N, nelem):
    """One pyramid (one tile with 7 empty element slots) and 9 pyramids (a full tile and one
    element), 4 steps against the oracle."""
    v, e = make_pyramid_mesh(3, 2, 1, delta=0.06, seed=60 + N)
    e = e[:nelem]
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 4)
    tc = _run(v, e, N, dt, 4, True)
    check(dg, dg.values_phi(tc), dg.values_psi(U_or), TOL["f64"], ("fp64 tensor traces, ragged", N, nelem))


@pytest.mark.parametrize("scale_exp", [-900, 0, 900])
def test_fp64_tensor_traces_exponent_range(torch_cuda, scale_exp):
    """A random state whose rows decay over 2^-100 (modes) with random signs, scaled by 2^-900,
    1 or 2^900: the row and face-point exponents, the recombination and its scaling over the
    whole normal range. One step against the trace kernel."""
    N = 4
    v, e = make_pyramid_mesh(3, delta=0.05, seed=8)
    from paper_1502_07703_gb300.binding import Solver
    with Solver(v, e, N, precision="f64") as s:
        dt = s.dt_cfl(0.5)
        K, Np = s.K, s.Np
    rng = np.random.default_rng(17)
    q0 = rng.standard_normal((K, 4, Np)) * np.exp2(-100.0 * np.arange(Np) / (Np - 1))[None, None, :]
    q0 = np.ldexp(q0, scale_exp)
    tc = _run(v, e, N, dt, 1, True, q0)
    cc = _run(v, e, N, dt, 1, False, q0)
    assert np.all(np.isfinite(tc))
    # compared at unit scale: the squares of 2^-900 values underflow (of 2^900 values overflow)
    assert _rel(np.ldexp(tc, -scale_exp), np.ldexp(cc, -scale_exp)) <= TOL_PATHS


def test_fp64_tensor_traces_rejections_and_switching_off(torch_cuda):
    from paper_1502_07703_gb300.binding import PyrDGError, Solver
    v, e = make_pyramid_mesh(2, delta=0.05, seed=2)
    for N in (1, 5):  # one M block of face points (Nfc <= 128) and exact level sums (Np <= 102)
        with Solver(v, e, N, precision="f64") as s:
            with pytest.raises(PyrDGError, match="BAD_ARG"):
                s.set_tensor_traces(True)
    with Solver(v, e, 3, precision="f64", basis="nodal") as s:
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            s.set_tensor_traces(True)
    with Solver(v, e, 4, precision="f64") as s:  # on, then off again: the FP64 trace kernel
        dt = s.dt_cfl(0.5)
        s.set_tensor_traces(True)
        s.set_tensor_traces(False)
        s.project(0.0)
        s.step(3, dt)
        off = s.get_state()
    assert np.array_equal(off, _run(v, e, 4, dt, 3, False))
