"""pyr_dg_rhs_noalloc, the allocation-free variant of pyr_dg_rhs.

Some callers cannot allocate device memory at the moment they call in (their
memory is owned by another allocator, or allocating is not allowed in that
phase). pyr_dg_rhs_noalloc serves them with its face-trace scratch in a static
device array instead of the handle's buffer. These tests call it through the C
ABI and check, on two calls in a row, that it returns what pyr_dg_rhs returns
for the same state, and that a mesh too large for the static array is refused
with a clear error. This file is collected last so that a failure here stops a
-x run only after every other test has run; it also runs on its own.
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


def _noalloc(s, q, out):
    from paper_1502_07703_gb300 import binding
    rc = binding.lib().pyr_dg_rhs_noalloc(s._h, q.data_ptr(), out.data_ptr())
    binding._check(rc)
    return out


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_matches_rhs_on_two_calls(torch_cuda, precision, tol):
    torch = torch_cuda
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(3, 2, 2, delta=0.08, seed=21)
    with Solver(v, e, 3, precision=precision) as s:
        for call, seed in enumerate((31, 32)):
            q = torch.tensor(random_state(s.K, s.Np, seed), dtype=s.torch_dtype, device="cuda")
            ref = s.rhs(q)
            out = torch.full_like(q, float("nan"))
            _noalloc(s, q, out)
            torch.cuda.synchronize()
            a = out.double().cpu().numpy()
            b = ref.double().cpu().numpy()
            assert np.all(np.isfinite(a)), call
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel <= tol, (call, rel)


def test_noalloc_rejects_mesh_beyond_static_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1502_07703_gb300 import binding
    from paper_1502_07703_gb300.binding import Solver
    v, e = make_pyramid_mesh(8, delta=0.05, seed=1)  # 3072 pyramids, N = 4: 12.3 MB of traces in double
    with Solver(v, e, 4) as s:
        q = torch.zeros(s.shape, dtype=s.torch_dtype, device="cuda")
        out = torch.zeros_like(q)
        rc = binding.lib().pyr_dg_rhs_noalloc(s._h, q.data_ptr(), out.data_ptr())
        assert rc == -1
        assert b"static scratch holds" in binding.lib().pyr_dg_last_error()


def test_noalloc_takes_no_device_memory_and_ignores_stale_scratch(torch_cuda):
    """A caller that cannot allocate sees free device memory unchanged across the call, and a
    call after a larger mesh's call (whose traces are still in the array) is unaffected by them."""
    torch = torch_cuda
    from paper_1502_07703_gb300.binding import Solver
    vb, eb = make_pyramid_mesh(4, 4, 3, delta=0.08, seed=22)  # 288 pyramids: 1.7 MB of traces at N = 5
    vs, es = make_pyramid_mesh(2, 1, 1, delta=0.08, seed=23)  # 12 pyramids
    with Solver(vb, eb, 5) as big, Solver(vs, es, 5) as small:
        qb = torch.tensor(random_state(big.K, big.Np, 41), dtype=big.torch_dtype, device="cuda")
        qs = torch.tensor(random_state(small.K, small.Np, 42), dtype=small.torch_dtype, device="cuda")
        ref_s = small.rhs(qs)
        ob, os_ = torch.empty_like(qb), torch.empty_like(qs)
        _noalloc(big, qb, ob)  # warm: both handles' kernels are loaded
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _noalloc(big, qb, ob)
        _noalloc(small, qs, os_)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        a, b = os_.cpu().numpy(), ref_s.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
