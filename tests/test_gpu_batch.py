"""Batched form: many independent meshes of different sizes and degrees in one
batch (one launch per degree per stage, CUDA-graph replay, per-mesh dt).

Each mesh's result must equal what a single-mesh solver computes for it (the
per-element arithmetic is the same), and one mesh per degree is also checked
against the FP64 oracle."""

import numpy as np
import pytest

from _parity import check
from oracle.dg import PyramidDG
from paper_1502_07703_gb300.mesh import make_pyramid_mesh

pytestmark = pytest.mark.gpu

SHAPES = [((2, 1, 1), 2, 0.05, 1), ((2, 2, 1), 3, 0.1, 2), ((1, 1, 1), 2, 0.0, 3), ((2, 2, 2), 4, 0.08, 4),
          ((3, 1, 1), 3, 0.05, 5), ((1, 2, 1), 5, 0.1, 6), ((2, 1, 2), 4, 0.05, 7)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_07703_gb300 import build
    build.build()
    return torch


def _meshes():
    out = []
    for (nx, ny, nz), n, delta, seed in SHAPES:
        v, e = make_pyramid_mesh(nx, ny, nz, delta=delta, seed=seed)
        out.append((v, e, n))
    return out


@pytest.mark.parametrize("precision,tol_single,tol_oracle", [("f64", 1e-14, 1e-12), ("f32", 1e-6, 1e-5)])
def test_batch_matches_single_mesh_runs_and_oracle(torch_cuda, precision, tol_single, tol_oracle):
    from paper_1502_07703_gb300.binding import Batch, Solver
    meshes = _meshes()
    with Batch(meshes, precision=precision) as b:
        assert b.ngroups == len({n for _, _, n in meshes})
        dt = b.dt_cfl(0.5)
        b.project(0.0)
        b.step(3, dt)          # capture
        b.step(3, dt)          # replay
        dt2 = dt * 0.8
        b.step(2, dt2)         # new dt and new step count: upload + recapture
        states = [b.get_state(i).astype(np.float64) for i in range(b.nmesh)]
        err_abs, err_rel = b.error()
    seen = set()
    for i, (v, e, n) in enumerate(meshes):
        with Solver(v, e, n, precision=precision) as s:
            s.project(0.0)
            s.step(3, dt[i])
            s.step(3, dt[i])
            s.step(2, dt2[i])
            U = s.get_state().astype(np.float64)
            ea, er = s.error()
        rel = np.linalg.norm(states[i] - U) / np.linalg.norm(U)
        assert rel <= tol_single, (i, rel)
        # | |U_b - U_ex| - |U_s - U_ex| | <= |U_b - U_s| (triangle inequality, one norm): the
        # relative error norms differ by at most about the states' relative distance. FP32
        # batches may run the single-launch kernel (CUDA-core traces) while single meshes use
        # the tensor-core traces, so the two FP32 results round differently.
        assert abs(err_rel[i] - er) <= 2 * tol_single, (i, err_rel[i], er)
        if precision == "f64":
            np.testing.assert_allclose([err_abs[i], err_rel[i]], [ea, er], rtol=1e-6)
        if n not in seen:
            seen.add(n)
            dg = PyramidDG(v, e, n)
            # the 2N-storage residual restarts at every step (A_1 = 0), so steps compose
            Ur = dg.lsrk4(dg.lsrk4(dg.project_exact(0.0), dt[i], 6), dt2[i], 2)
            check(dg, dg.values_phi(states[i]), dg.values_psi(Ur), tol_oracle, i)


def test_batch_autotuned_elements_per_block(torch_cuda):
    """Degree groups of at least 4096 pyramids are autotuned at setup over elements per
    CTA and grid size. Grouping does not change the per-element arithmetic, so each
    mesh's FP32 state equals the single-mesh run's (which uses the default grouping)."""
    from paper_1502_07703_gb300.binding import Batch, Solver
    meshes = []
    for (nx, ny, nz), n, seed in (((10, 10, 7), 1, 11), ((9, 9, 9), 2, 12), ((1, 2, 1), 3, 13)):
        v, e = make_pyramid_mesh(nx, ny, nz, delta=0.05, seed=seed)
        meshes.append((v, e, n))
    with Batch(meshes, precision="f32") as b:
        info = {g["N"]: g for g in b.groups()}
        for g in info.values():
            assert g["elems_per_block"] in (1, 2, 4, 8)
            assert 1 <= g["stage_blocks"] <= -(-g["K"] // g["elems_per_block"])
        dt = b.dt_cfl(0.5)
        b.project(0.0)
        b.step(3, dt)
        states = [b.get_state(i) for i in range(b.nmesh)]
    for i, (v, e, n) in enumerate(meshes):
        with Solver(v, e, n, precision="f32") as s:
            s.project(0.0)
            s.step(3, dt[i])
            U = s.get_state()
        rel = np.linalg.norm(states[i].astype(np.float64) - U) / np.linalg.norm(U.astype(np.float64))
        assert rel <= 1e-6, (i, rel)


@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_batch_lowest_and_highest_degrees(torch_cuda, precision, tol):
    """A batch of N = 1, 6 and 7 meshes (FP32: 8 elements per CTA at N = 1, one at 6 and 7)
    against the oracle after 3 steps of each mesh's own dt."""
    from paper_1502_07703_gb300.binding import Batch
    meshes = []
    for (nx, ny, nz), n, seed in (((3, 1, 1), 1, 21), ((1, 2, 1), 6, 22), ((1, 1, 1), 7, 23)):
        v, e = make_pyramid_mesh(nx, ny, nz, delta=0.08, seed=seed)
        meshes.append((v, e, n))
    with Batch(meshes, precision=precision) as b:
        dt = b.dt_cfl(0.5)
        b.project(0.0)
        b.step(3, dt)
        states = [b.get_state(i).astype(np.float64) for i in range(b.nmesh)]
    for i, (v, e, n) in enumerate(meshes):
        dg = PyramidDG(v, e, n)
        Ur = dg.lsrk4(dg.project_exact(0.0), dt[i], 3)
        check(dg, dg.values_phi(states[i]), dg.values_psi(Ur), tol, n)


def test_batch_oracle_parity_fixed_dt(torch_cuda):
    """Every mesh of a mixed-degree FP64 batch against the oracle over 4 steps."""
    from paper_1502_07703_gb300.binding import Batch
    meshes = _meshes()[:4]
    with Batch(meshes, precision="f64") as b:
        dt = b.dt_cfl(0.4)
        b.project(0.0)
        b.step(4, dt)
        states = [b.get_state(i) for i in range(b.nmesh)]
    for i, (v, e, n) in enumerate(meshes):
        dg = PyramidDG(v, e, n)
        Ur = dg.lsrk4(dg.project_exact(0.0), dt[i], 4)
        check(dg, dg.values_phi(states[i]), dg.values_psi(Ur), 1e-12, i)


def test_batch_rejects_bad_input(torch_cuda):
    from paper_1502_07703_gb300.binding import Batch, PyrDGError
    v, e = make_pyramid_mesh(1)
    with pytest.raises(PyrDGError, match="UNSUPPORTED_N"):
        Batch([(v, e, 2), (v, e, 9)])
    with Batch([(v, e, 2)]) as b:
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            b.step(1, np.array([-1.0]))


def test_batch_replays_alternate_trace_halves(torch_cuda):
    """FP32 batch graphs keep the face traces in a ping-pong pair across replays: one step
    flips the current half five times, so consecutive single-step replays alternate between
    the two captured graphs. Five replays, a projection (traces recomputed), then steps of 1 and
    2, against single-mesh runs of the same sequence (same arithmetic: 1e-6 in FP32)."""
    from paper_1502_07703_gb300.binding import Batch, Solver
    meshes = _meshes()[:4]
    with Batch(meshes, precision="f32") as b:
        assert b.ngroups == 3
        dt = b.dt_cfl(0.5)
        b.project(0.0)
        for _ in range(5):
            b.step(1, dt)
        mid = [b.get_state(i).astype(np.float64) for i in range(b.nmesh)]
        b.project(0.0)
        b.step(1, dt)
        b.step(2, dt)
        b.step(1, dt)
        end = [b.get_state(i).astype(np.float64) for i in range(b.nmesh)]
    for i, (v, e, n) in enumerate(meshes):
        with Solver(v, e, n, precision="f32") as s:
            s.project(0.0)
            for _ in range(5):
                s.step(1, dt[i])
            U5 = s.get_state().astype(np.float64)
            s.project(0.0)
            s.step(1, dt[i])
            s.step(2, dt[i])
            s.step(1, dt[i])
            U4 = s.get_state().astype(np.float64)
        for got, want in ((mid[i], U5), (end[i], U4)):
            rel = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert rel <= 1e-6, (i, rel)


@pytest.mark.parametrize("single", [True, False])
def test_batch_launch_modes_against_single_meshes_and_oracle(torch_cuda, single):
    """Both ways of running an FP32 batch stage: one kernel for every degree group (CTAs
    split between the groups) and one launch per group on graph branches. Steps, replays and a
    projection against single-mesh runs (1e-6) and one mesh per degree against the oracle."""
    from paper_1502_07703_gb300.binding import Batch, Solver
    meshes = _meshes()
    with Batch(meshes, precision="f32") as b:
        b.set_launch_mode(single)
        assert b.launch_mode() == (single, 1 if single else b.ngroups)
        dt = b.dt_cfl(0.5)
        b.project(0.0)
        b.step(2, dt)
        b.step(1, dt)
        b.step(1, dt)
        states = [b.get_state(i).astype(np.float64) for i in range(b.nmesh)]
    seen = set()
    for i, (v, e, n) in enumerate(meshes):
        with Solver(v, e, n, precision="f32") as s:
            s.project(0.0)
            s.step(4, dt[i])
            U = s.get_state().astype(np.float64)
        rel = np.linalg.norm(states[i] - U) / np.linalg.norm(U)
        assert rel <= 1e-6, (i, rel)
        if n not in seen:
            seen.add(n)
            dg = PyramidDG(v, e, n)
            check(dg, dg.values_phi(states[i]), dg.values_psi(dg.lsrk4(dg.project_exact(0.0), dt[i], 4)), 1e-5,
                  (single, n))


def test_batch_single_launch_refused_where_unavailable(torch_cuda):
    from paper_1502_07703_gb300.binding import Batch, PyrDGError
    v, e = make_pyramid_mesh(1, delta=0.05, seed=3)
    with Batch([(v, e, 2), (v, e, 3)], precision="f64") as b:
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            b.set_launch_mode(True)
        b.set_launch_mode(False)
    with Batch([(v, e, 2), (v, e, 2)], precision="f32") as b:  # one degree group
        with pytest.raises(PyrDGError, match="BAD_ARG"):
            b.set_launch_mode(True)


def test_full_size_config4_sampled(torch_cuda):
    """Config 4 as the bench runs it: 256 meshes (sizes log-uniform 48..49,152 pyramids, seed 2;
    mesh i perturbed +-0.05h with seed 1000+i), degrees 2..6, FP32, each mesh at its own CFL
    step, in the launch mode the setup autotuner picks. One step from the projected standing
    wave, checked against the oracle on sampled elements of sampled meshes (one per degree,
    the largest mesh among them) over their 6-hop neighbourhoods."""
    from _parity import face_neighbours, patch
    from paper_1502_07703_gb300.binding import Batch
    from paper_1502_07703_gb300.mesh import batch_mesh_shapes
    shapes = batch_mesh_shapes(count=256, seed=2)
    meshes = []
    for i, (nx, ny, nz, n) in enumerate(shapes):
        v, e = make_pyramid_mesh(nx, ny, nz, delta=0.05, seed=1000 + i)
        meshes.append((v, e, n))
    with Batch(meshes, precision="f32") as b:
        assert b.nmesh == 256 and b.ngroups == 5
        dt = b.dt_cfl(0.5)
        b.project(0.0)
        b.step(1, dt)
        picks = {}
        for i, (_, e, n) in enumerate(meshes):
            if n not in picks or e.shape[0] > meshes[picks[n]][1].shape[0]:
                picks[n] = i
        states = {i: b.get_state(i).astype(np.float64) for i in picks.values()}
    rng = np.random.default_rng(29)
    for n, i in sorted(picks.items()):
        v, e, _ = meshes[i]
        nbrs = face_neighbours(e)
        for c in (int(rng.integers(e.shape[0])), e.shape[0] - 1):
            p = patch(nbrs, c, 6)
            dg = PyramidDG(v, e[p], n)
            j = p.index(c)
            Up = dg.lsrk4(dg.project_exact(0.0), dt[i], 1)
            check(dg, dg.values_phi(states[i][p])[j:j + 1], dg.values_psi(Up)[j:j + 1], 1e-5, (n, i, c), elems=[j])
