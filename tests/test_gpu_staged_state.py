"""pyr_dg_stage_state: the next step's input copied in while the current step runs.

A caller that feeds a new state every step (a serving loop, the end-to-end bench line)
stages it from host memory on the handle's copy stream; the next pyr_dg_step waits for
that copy on the device and makes it the state. These tests check, through the C ABI, that
a staged state steps to exactly what pyr_dg_set_state + pyr_dg_step give, that calls made
between staging and the step still see the current state, that the buffer rotation keeps
its order over several steps in a row from page-locked memory, and that set_state drops a
staged state and a later stage replaces an earlier one.
"""

import numpy as np
import pytest

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


def _solver(kind, precision):
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(3, 3, 2, delta=0.08, seed=41)
    if kind == "advection":
        return Solver(v, e, 3, precision=precision, equation="advection", periodic=(0.0, 1.0))
    return Solver(v, e, 3, precision=precision)


def _state(s, seed):
    return random_state(s.K, s.Np, seed)[:, : s.shape[1], :].astype(s.np_dtype)


def _stepped(s, U, t, dt, nsteps=1):
    s.set_state(U, t)
    s.step(nsteps, dt)
    return s.get_state(), s.time


@pytest.mark.parametrize("kind,precision", [("wave", "f64"), ("wave", "f32"), ("advection", "f64")])
def test_staged_state_steps_like_set_state(torch_cuda, kind, precision):
    with _solver(kind, precision) as s:
        dt = s.dt_cfl(0.4)
        U = _state(s, 7)
        ref, tref = _stepped(s, U, 0.25, dt, 2)
        s.project(0.0)
        s.step(1, dt)
        s.stage_state(U, 0.25)
        s.step(2, dt)
        out = s.get_state()
        assert np.array_equal(out, ref)
        assert s.time == pytest.approx(tref, rel=0, abs=1e-15)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_staged_copy_overlaps_and_rotates(torch_cuda, precision):
    """Inputs U_i staged from page-locked memory while step i-1 runs; error() and get_state()
    between staging and stepping see step i-1's result; four steps in a row rotate the two
    buffers (each copy waits for the previous state's last reader)."""
    torch = torch_cuda
    with _solver("wave", precision) as s:
        dt = s.dt_cfl(0.4)
        Us = [_state(s, 100 + i) for i in range(4)]
        refs = [_stepped(s, U, 0.0, dt) for U in Us]
        errs = []
        for U in Us:
            s.set_state(U, 0.0)
            s.step(1, dt)
            errs.append(s.error())
        pinned = [torch.from_numpy(U.copy()).pin_memory() for U in Us]
        s.stage_state_host_ptr(pinned[0].data_ptr(), 0.0)
        for i in range(4):
            s.step(1, dt)
            if i + 1 < 4:
                s.stage_state_host_ptr(pinned[i + 1].data_ptr(), 0.0)
            assert s.error() == pytest.approx(errs[i], rel=1e-10), i  # stored or direct error rule
            out = s.get_state()
            assert np.array_equal(out, refs[i][0]), i
        s.sync()


def test_set_state_drops_and_later_stage_replaces(torch_cuda):
    with _solver("wave", "f64") as s:
        dt = s.dt_cfl(0.4)
        U1, U2 = _state(s, 1), _state(s, 2)
        r1, _ = _stepped(s, U1, 0.0, dt)
        r2, _ = _stepped(s, U2, 0.0, dt)
        s.stage_state(U2, 0.0)
        s.set_state(U1, 0.0)
        s.step(1, dt)
        assert np.array_equal(s.get_state(), r1)
        s.stage_state(U1, 0.0)
        s.stage_state(U2, 0.0)
        s.step(1, dt)
        assert np.array_equal(s.get_state(), r2)
        s.stage_state(U1, 0.0)
        s.project(0.0)
        s.step(1, dt)
        p = s.get_state()
        s.project(0.0)
        s.step(1, dt)
        assert np.array_equal(s.get_state(), p)


def test_stage_state_rejects_bad_arguments(torch_cuda):
    from paper_1502_07703_gb300 import binding
    bad_arg = -1  # PYR_DG_ERR_BAD_ARG
    with _solver("wave", "f64") as s:
        L = binding.lib()
        assert L.pyr_dg_stage_state(s._h, None, 0.0) == bad_arg
        buf = np.zeros(s.shape)
        assert L.pyr_dg_stage_state(s._h, buf.ctypes.data, float("nan")) == bad_arg
