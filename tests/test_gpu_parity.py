"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

The two sides share only the seeded inputs (mesh, random coefficient states).
The oracle works in the psi basis with dense matrices; the CUDA path in the
semi-nodal basis with the diagonal mass of Lemma 3. States are compared by
their values at every element's volume cubature points, as a
quadrature-weighted relative L2 difference over all four fields, and on the
worst element (tests/_parity.py): FP64 <= 1e-12, FP32 <= 1e-5 (the tolerances
the target states).
"""

import numpy as np
import pytest

from _parity import TOL, check, face_neighbours as _face_neighbours, patch as _patch, record
from oracle.dg import PyramidDG
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


def _domain(bc):
    return (0.0, 1.0) if bc == "wall" else (-1.0, 1.0)


def _solver(v, e, N, **kw):
    from paper_1502_07703_gb300.binding import Solver
    return Solver(v, e, N, **kw)


def _rhs_case(torch, v, e, N, bc, tau, precision, seed):
    dg = PyramidDG(v, e, N, tau=tau, bc=bc)
    U = random_state(dg.K, dg.Np, seed)
    with _solver(v, e, N, precision=precision, bc=bc, tau=tau) as s:
        q = torch.tensor(U, dtype=s.torch_dtype, device="cuda")
        R_gpu = s.rhs(q).double().cpu().numpy()
    # the oracle gets the same input function: the coefficients as rounded to the device precision
    Uin = U.astype(np.float32).astype(np.float64) if precision == "f32" else U
    R_or = dg.rhs(dg.psi_from_phi(Uin))
    return dg, dg.values_phi(R_gpu), dg.values_psi(R_or)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_rhs_parity_all_degrees(torch_cuda, N, precision):
    v, e = make_pyramid_mesh(3, 2, 1, delta=0.1, seed=5)
    check(*_rhs_case(torch_cuda, v, e, N, "wall", 1.0, precision, seed=100 + N), TOL[precision], N)


@pytest.mark.parametrize("bc,tau", [("wall", 0.0), ("free", 1.0), ("free", 0.0), ("wall", 0.5)])
def test_rhs_parity_flux_and_boundary_variants(torch_cuda, bc, tau):
    v, e = make_pyramid_mesh(2, 2, 2, delta=0.08, seed=6, domain=_domain(bc))
    check(*_rhs_case(torch_cuda, v, e, 3, bc, tau, "f64", seed=7), TOL["f64"], (bc, tau))


def test_rhs_single_element_all_boundary(torch_cuda):
    rng = np.random.default_rng(1)
    ref = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    v = ref + rng.uniform(-0.2, 0.2, ref.shape)
    e = np.array([[0, 1, 2, 3, 4]], dtype=np.int32)
    for N in (1, 4, 7):
        check(*_rhs_case(torch_cuda, v, e, N, "wall", 1.0, "f64", seed=N), TOL["f64"], N)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_projection_parity(torch_cuda, precision):
    v, e = make_pyramid_mesh(3, 3, 2, delta=0.1, seed=2)
    dg = PyramidDG(v, e, 4)
    with _solver(v, e, 4, precision=precision) as s:
        s.project(0.3)
        Ug = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(Ug), dg.values_psi(dg.project_exact(0.3)), 1e-13 if precision == "f64" else 1e-6)


def test_config1_evolution_and_error_norm(torch_cuda):
    """48 pyramids (2x2x2 hexes, +-0.05h, seed 0), N = 3, upwind, wall, 10 LSRK4 steps at CFL 0.5."""
    v, e = make_pyramid_mesh(2, delta=0.05, seed=0)
    dg = PyramidDG(v, e, 3)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 10)
    with _solver(v, e, 3) as s:
        s.project(0.0)
        s.step(10, dt)
        Ug = s.get_state()
        err_gpu = s.error()
        assert abs(s.time - 10 * dt) < 1e-15
        assert abs(s.dt_cfl(0.5) - dt) <= 1e-12 * dt
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f64"])
    err_or = dg.error(U_or, 10 * dt)
    np.testing.assert_allclose(err_gpu, err_or, rtol=1e-9)


def test_f32_evolution_matches_oracle(torch_cuda):
    v, e = make_pyramid_mesh(2, 2, 2, delta=0.05, seed=1)
    N = 5
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 40)
    with _solver(v, e, N, precision="f32") as s:
        s.project(0.0)
        s.step(40, dt)
        Ug = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f32"])


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 7])
def test_f32_stage_kernel_all_degrees(torch_cuda, N):
    """The single-launch FP32 stage kernel (ping-pong traces) at every degree:
    5 steps taken one call at a time, against the oracle."""
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=40 + N)
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 5)
    with _solver(v, e, N, precision="f32") as s:
        s.project(0.0)
        for _ in range(5):
            s.step(1, dt)
        Ug = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f32"])


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_f32_stage_kernel_partial_last_group(torch_cuda, N):
    """At low degree the FP32 stage kernel works on 2 to 8 elements per CTA. A mesh of
    23 pyramids (one of a 2x2x1-hex mesh dropped: its faces become boundary) leaves the
    last group partly past the end of the mesh; 5 steps against the oracle."""
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=60 + N)
    e = e[:-1]
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 5)
    with _solver(v, e, N, precision="f32") as s:
        assert s.K == 23
        s.project(0.0)
        s.step(5, dt)
        Ug = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f32"])


@pytest.mark.parametrize("bc,tau", [("wall", 0.0), ("free", 1.0)])
def test_f32_stage_kernel_invalidation_and_variants(torch_cuda, bc, tau):
    """Traces stay consistent when stepping is interleaved with rhs (which uses the
    trace buffer as scratch) and with set_state (which replaces the state)."""
    torch = torch_cuda
    v, e = make_pyramid_mesh(2, 2, 2, delta=0.08, seed=9, domain=_domain(bc))
    N = 3
    dg = PyramidDG(v, e, N, tau=tau, bc=bc)
    dt = dg.dt_cfl(0.5)
    U0 = random_state(dg.K, dg.Np, 77).astype(np.float32)
    U_or = dg.lsrk4(dg.psi_from_phi(U0.astype(np.float64)), dt, 4)
    with _solver(v, e, N, precision="f32", bc=bc, tau=tau) as s:
        s.project(0.0)
        s.step(2, dt)                      # traces of the projected state become valid
        s.set_state(U0)                    # must invalidate them
        s.step(1, dt)
        s.rhs(torch.zeros(s.shape, dtype=s.torch_dtype, device="cuda"))  # scratch use of the trace buffer
        s.step(1, dt)
        s.step(2, dt)
        Ug = s.get_state().astype(np.float64)
    # set_state zeroes the residual, so the reference restarts the 2N-storage scheme too
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f32"])


def test_state_roundtrip_host_and_device(torch_cuda):
    torch = torch_cuda
    v, e = make_pyramid_mesh(2, 1, 1, delta=0.1, seed=3)
    for prec in ("f64", "f32"):
        with _solver(v, e, 2, precision=prec) as s:
            U = random_state(s.K, s.Np, 4).astype(s.np_dtype)
            s.set_state(U, t=0.25)
            assert s.time == 0.25
            np.testing.assert_array_equal(s.get_state(), U)
            d = s.get_state(device=True)
            s.set_state(d * 2, t=0.0)
            np.testing.assert_array_equal(s.get_state(), 2 * U)
            np.testing.assert_array_equal(d.cpu().numpy(), U)


def test_full_size_config2_sampled(torch_cuda):
    """Config of the benchmark: 32^3 hexes x 6 = 196,608 pyramids, +-0.05h (seed 1), N = 4, FP64,
    stepping with the face traces on the tensor cores (the handle's default at this size).

    (1) rhs of a random state, checked on sampled elements: the oracle runs on
    the sample's face neighbourhood; (2) one LSRK4 step from the projected
    standing wave, checked on sampled elements whose 6-hop neighbourhood the
    oracle advances (influence travels one face per stage, 5 stages)."""
    torch = torch_cuda
    v, e = make_pyramid_mesh(32, delta=0.05, seed=1)
    K, N = e.shape[0], 4
    assert K == 196608
    nbrs = _face_neighbours(e)
    rng = np.random.default_rng(11)
    samples = [int(x) for x in rng.choice(K, 3, replace=False)] + [0, K - 1]
    U = random_state(K, 55, 12)
    with _solver(v, e, N) as s:
        assert s.tensor_traces  # the stepping path the bench times: FP64 traces on the tensor cores
        R = s.rhs(torch.tensor(U, device="cuda")).cpu().numpy()
        dt_or = PyramidDG(v, e[:6], N).dt_cfl(0.5)  # a fixed dt from one hex's pyramids
        s.project(0.0)
        s.step(1, dt_or)
        U1 = s.get_state()
    for c in samples:
        patch = _patch(nbrs, c, 1)
        dg = PyramidDG(v, e[patch], N)
        i = patch.index(c)
        Rp = dg.rhs(dg.psi_from_phi(U[patch]))
        check(dg, dg.values_phi(R[patch])[i:i + 1], dg.values_psi(Rp)[i:i + 1], TOL["f64"], c, elems=[i])
    for c in samples[:2]:
        patch = _patch(nbrs, c, 6)
        dg = PyramidDG(v, e[patch], N)
        i = patch.index(c)
        Up = dg.lsrk4(dg.project_exact(0.0), dt_or, 1)
        check(dg, dg.values_phi(U1[patch])[i:i + 1], dg.values_psi(Up)[i:i + 1], TOL["f64"], c, elems=[i])


def test_full_size_config5_f32_sampled(torch_cuda):
    """Config of the large run: 64^3 hexes x 6 = 1,572,864 pyramids, +-0.1h (seed 3), N = 5,
    FP32, through the single-launch stage kernel as the bench launches it. One LSRK4 step
    from the projected standing wave, checked on sampled elements whose 6-hop
    neighbourhood the oracle advances."""
    v, e = make_pyramid_mesh(64, delta=0.1, seed=3)
    K, N = e.shape[0], 5
    assert K == 1572864
    nbrs = _face_neighbours(e)
    rng = np.random.default_rng(13)
    samples = [int(x) for x in rng.choice(K, 2, replace=False)] + [K - 1]
    dt_or = PyramidDG(v, e[:6], N).dt_cfl(0.5)
    with _solver(v, e, N, precision="f32") as s:
        s.project(0.0)
        s.step(1, dt_or)
        U1 = s.get_state().astype(np.float64)
    for c in samples:
        patch = _patch(nbrs, c, 6)
        dg = PyramidDG(v, e[patch], N)
        i = patch.index(c)
        Up = dg.lsrk4(dg.project_exact(0.0), dt_or, 1)
        check(dg, dg.values_phi(U1[patch])[i:i + 1], dg.values_psi(Up)[i:i + 1], TOL["f32"], c, elems=[i])


@pytest.mark.parametrize("N", [1, 2, 5])
def test_f32_stage_kernel_single_element(torch_cuda, N):
    """One pyramid, all faces on the wall: with several elements per CTA the only group
    is one element and copies of it (stores skipped); 4 steps against the oracle."""
    v, e = make_pyramid_mesh(1, delta=0.0)
    e = e[:1]
    dg = PyramidDG(v, e, N)
    dt = dg.dt_cfl(0.5)
    U_or = dg.lsrk4(dg.project_exact(0.0), dt, 4)
    with _solver(v, e, N, precision="f32") as s:
        assert s.K == 1
        s.project(0.0)
        s.step(4, dt)
        Ug = s.get_state().astype(np.float64)
    check(dg, dg.values_phi(Ug), dg.values_psi(U_or), TOL["f32"])


@pytest.mark.parametrize("nx,bc", [(8, "wall"), (16, "wall"), (16, "free")])
def test_error_norm_fine_meshes(torch_cuda, nx, bc):
    """The FP64 error norm of a random state at t = 0.3 against the oracle's. On fine meshes
    the kernel evaluates the exact fields along each c line by angle addition from the
    (a, b) point (16^3 hexes: everywhere; 8^3: at some points), elsewhere with sincospi."""
    from oracle.dg import PyramidDG as DG
    v, e = make_pyramid_mesh(nx, delta=0.05, seed=5, domain=_domain(bc))
    N = 2
    dg = DG(v, e, N, bc=bc)
    U = random_state(dg.K, dg.Np, 21)
    with _solver(v, e, N, bc=bc) as s:
        s.set_state(U, t=0.3)
        err_gpu = s.error()  # exact fields evaluated in the kernel
        err_stored = s.error()  # the second call stores their spatial factors
        err_again = s.error()
    err_or = dg.error(dg.psi_from_phi(U), 0.3)
    for err in (err_gpu, err_stored, err_again):
        np.testing.assert_allclose(err, err_or, rtol=1e-12)


@pytest.mark.parametrize("precision,N", [("f64", 3), ("f32", 3), ("f64", 1), ("f64", 5), ("f32", 7), ("f64", 4)])
def test_error_norm_store_matches_direct(torch_cuda, precision, N):
    """The error norm from coefficients (the error rule's projection of the exact fields'
    spatial factors, stored at the second call) equals the direct kernel's at several times
    (the time factors come from the host), and the store takes the device memory the header
    states and gives it back when switched off."""
    import torch
    # 16^3 hexes at N = 4: a store of 54 MB, large enough for the device-memory checks
    # (small stores come out of already-mapped pages)
    v, e = make_pyramid_mesh(16 if N == 4 else 6 if N <= 5 else 3, delta=0.05, seed=7)
    with _solver(v, e, N, precision=precision) as s:
        U = random_state(s.K, s.Np, 31).astype(s.np_dtype)
        store = s.K * 5 * s.Np * 8
        for t in (0.0, 0.37, 1.9):
            s.set_state(U, t=t)
            s.set_error_cache(False)
            direct = s.error()
            free0 = torch.cuda.mem_get_info()[0]
            s.set_error_cache(True)
            np.testing.assert_allclose(s.error(), direct, rtol=1e-12)  # no store at one call
            big = store >= 16 << 20
            assert not big or free0 - torch.cuda.mem_get_info()[0] < store
            stored = s.error()
            free1 = torch.cuda.mem_get_info()[0]
            assert not big or free0 - free1 >= store, (free0, free1, store)
            np.testing.assert_allclose(s.error(), direct, rtol=1e-12)
            np.testing.assert_allclose(stored, direct, rtol=1e-12)
        s.set_error_cache(False)
        assert not big or torch.cuda.mem_get_info()[0] - free1 >= store


@pytest.mark.parametrize("bc", ["wall", "free"])
def test_error_norm_store_converged_state(torch_cuda, bc):
    """On an evolved standing wave the error is small against the fields, and both of its
    parts matter: sum M (u - T s)^2 and the projection error T^2 |PS - S|^2. The stored path
    and the direct kernel agree to the digits that survive the cancellation in U_h - U_ex."""
    v, e = make_pyramid_mesh(8, delta=0.05, seed=3, domain=_domain(bc))
    N = 3
    with _solver(v, e, N, bc=bc) as s:
        dt = s.dt_cfl(0.5)
        s.project(0.0)
        s.step(20, dt)
        direct = s.error()
        s.error()  # stores
        stored = s.error()
    assert 1e-9 < direct[1] < 1e-4, direct
    np.testing.assert_allclose(stored, direct, rtol=1e-6)


@pytest.mark.parametrize("nx,N", [(32, 5), (16, 7)])
def test_config3_f32_200_steps(torch_cuda, nx, N):
    """Config 3 (the precision form): the FP32 single-launch stage kernel from the projected
    standing wave.

    (1) One LSRK4 step against the oracle on sampled elements whose 6-hop neighbourhood the
    oracle advances. (2) 200 LSRK4 steps in FP32 against the same 200 steps in FP64, compared
    by point values at every volume cubature point with the quadrature weight (mesh-wide
    relative L2 and the worst element); the FP64 path matches the oracle to 1e-12 (tests
    above and the sampled check below), so it stands in for the oracle over 200 steps of the
    whole mesh. Both stay close to the exact solution."""
    from oracle.dg import phi_states_l2_diff
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(nx, delta=0.05, seed=1)
    K = e.shape[0]
    nbrs = _face_neighbours(e)
    rng = np.random.default_rng(17 + N)
    samples = [int(x) for x in rng.choice(K, 2, replace=False)] + [K - 1]
    states, errs, oracle = {}, {}, {}
    for prec in ("f64", "f32"):
        with Solver(v, e, N, precision=prec) as s:
            dt = s.dt_cfl(0.5) if prec == "f64" else dt
            s.project(0.0)
            s.step(1, dt)
            U1 = s.get_state().astype(np.float64)
            for c in samples:
                if c not in oracle:
                    patch = _patch(nbrs, c, 6)
                    dg = PyramidDG(v, e[patch], N)
                    oracle[c] = (patch, dg, dg.values_psi(dg.lsrk4(dg.project_exact(0.0), dt, 1)))
                patch, dg, Bv = oracle[c]
                i = patch.index(c)
                check(dg, dg.values_phi(U1[patch])[i:i + 1], Bv[i:i + 1], TOL[prec], (prec, c), elems=[i])
            s.step(199, dt)
            states[prec] = s.get_state().astype(np.float64)
            errs[prec] = s.error()[1]
    rel, worst = phi_states_l2_diff(v, e, N, states["f32"], states["f64"])
    record(rel, worst, TOL["f32"], "200 steps f32 vs f64")
    assert errs["f64"] < 1e-6 and errs["f32"] < 1e-5, errs


def test_dt_cfl_library_uses_the_papers_constant(torch_cuda):
    """pyr_dg_dt_cfl and pyr_dg_batch_dt_cfl against C_N of the golden table (the Sec. 4.3
    spectral-radius fit) on unperturbed meshes, where max |dK|/|K| = 6 (1 + sqrt 2) / h."""
    import os
    from paper_1502_07703_gb300.binding import Batch, Solver
    CN = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "spectral_radius_constants.txt")):
        if line.strip() and not line.startswith("#"):
            n, num = line.split()
            CN[int(n)] = int(num) / 3.0
    meshes = []
    for N in range(1, 8):
        n_hex = 1 + N % 2
        v, e = make_pyramid_mesh(n_hex, delta=0.0)
        meshes.append((v, e, N))
        with Solver(v, e, N) as s:
            np.testing.assert_allclose(s.dt_cfl(0.5), 0.5 / (CN[N] * 6.0 * (1.0 + np.sqrt(2.0)) * n_hex),
                                       rtol=1e-13)
    with Batch(meshes, precision="f32") as b:
        want = [0.5 / (CN[N] * 6.0 * (1.0 + np.sqrt(2.0)) * (1 + N % 2)) for N in range(1, 8)]
        np.testing.assert_allclose(b.dt_cfl(0.5), want, rtol=1e-13)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_l2_diff_is_the_quadrature_norm(torch_cuda, precision):
    """pyr_dg_l2_diff (mass-weighted coefficient sums) against the oracle's quadrature L2
    norms of the point values: equal because the semi-nodal mass matrix is diagonal (Lemma 3)
    and the volume rule integrates it exactly."""
    torch = torch_cuda
    from oracle.dg import PyramidDG
    v, e = make_pyramid_mesh(2, 2, 1, delta=0.1, seed=8)
    N = 4
    dg = PyramidDG(v, e, N)
    A = random_state(dg.K, dg.Np, 51)
    B = random_state(dg.K, dg.Np, 52)
    with _solver(v, e, N, precision=precision) as s:
        qa = torch.tensor(A, dtype=s.torch_dtype, device="cuda")
        qb = torch.tensor(B, dtype=s.torch_dtype, device="cuda")
        d, nb = s.l2_diff(qa, qb)
        A = qa.double().cpu().numpy()
        B = qb.double().cpu().numpy()
    wJ = dg.w[None, :] * dg.J
    Va, Vb = dg.values_phi(A), dg.values_phi(B)
    d_or = np.sqrt(np.einsum("kq,kqc->", wJ, (Va - Vb) ** 2))
    n_or = np.sqrt(np.einsum("kq,kqc->", wJ, Vb ** 2))
    tol = 1e-12 if precision == "f64" else 1e-6  # FP32 handles keep M^{-1} in float
    np.testing.assert_allclose([d, nb], [d_or, n_or], rtol=tol)
