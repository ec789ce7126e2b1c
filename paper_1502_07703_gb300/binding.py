"""Thin ctypes binding of libpyrdg.so (C ABI in include/pyrdg.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. PyTorch supplies device memory (``rhs``, device-side state
copies) and the default stream. Loading fails loudly when the library has not
been built; there is no Python or CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpyrdg.so")

PYR_DG_F64, PYR_DG_F32 = 0, 1
PYR_DG_BC_WALL, PYR_DG_BC_FREE = 0, 1
PYR_DG_HOST, PYR_DG_DEVICE = 0, 1
PYR_DG_WAVE, PYR_DG_ADVECTION = 0, 1
PYR_DG_MODAL, PYR_DG_NODAL = 0, 1
ERRORS = {-1: "BAD_ARG", -2: "BAD_MESH", -3: "UNSUPPORTED_N", -4: "CUDA", -5: "NO_MEMORY", -6: "TIMEOUT"}

_lib = None


class PyrDGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
        ("equation", ctypes.c_int),
        ("beta", ctypes.c_double * 3),
        ("periodic", ctypes.c_int),
        ("box_lo", ctypes.c_double),
        ("box_hi", ctypes.c_double),
        ("basis", ctypes.c_int),
    ]


_c_dp = ctypes.POINTER(ctypes.c_double)
_c_ip = ctypes.POINTER(ctypes.c_int)
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_h = ctypes.c_void_p

_SIGNATURES = {
    "pyr_dg_default_opts": (None, [ctypes.POINTER(Opts)]),
    "pyr_dg_setup": (ctypes.c_int, [_c_dp, ctypes.c_int64, _c_i32p, ctypes.c_int64, ctypes.c_int,
                                    ctypes.POINTER(Opts), ctypes.POINTER(_c_h)]),
    "pyr_dg_info": (ctypes.c_int, [_c_h, _c_i64p, _c_ip, _c_ip, _c_ip, _c_ip]),
    "pyr_dg_project": (ctypes.c_int, [_c_h, ctypes.c_double]),
    "pyr_dg_set_state": (ctypes.c_int, [_c_h, ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "pyr_dg_get_state": (ctypes.c_int, [_c_h, ctypes.c_void_p, ctypes.c_int]),
    "pyr_dg_stage_state": (ctypes.c_int, [_c_h, ctypes.c_void_p, ctypes.c_double]),
    "pyr_dg_rhs": (ctypes.c_int, [_c_h, ctypes.c_void_p, ctypes.c_void_p]),
    "pyr_dg_step": (ctypes.c_int, [_c_h, ctypes.c_int, ctypes.c_double]),
    "pyr_dg_error": (ctypes.c_int, [_c_h, _c_dp, _c_dp]),
    "pyr_dg_set_error_cache": (ctypes.c_int, [_c_h, ctypes.c_int]),
    "pyr_dg_dt_cfl": (ctypes.c_int, [_c_h, ctypes.c_double, _c_dp]),
    "pyr_dg_time": (ctypes.c_int, [_c_h, _c_dp]),
    "pyr_dg_sync": (ctypes.c_int, [_c_h]),
    "pyr_dg_destroy": (None, [_c_h]),
    "pyr_dg_last_error": (ctypes.c_char_p, []),
    "pyr_dg_host_gauss_jacobi": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _c_dp, _c_dp]),
    "pyr_dg_host_connectivity": (ctypes.c_int, [_c_dp, ctypes.c_int64, _c_i32p, ctypes.c_int64, ctypes.c_int,
                                                _c_i64p, _c_i64p]),
    "pyr_dg_fma_peak": (ctypes.c_int, [ctypes.c_int, _c_dp]),
    "pyr_dg_num_fields": (ctypes.c_int, [_c_h, _c_ip]),
    "pyr_dg_host_connectivity_periodic": (ctypes.c_int, [_c_dp, ctypes.c_int64, _c_i32p, ctypes.c_int64, ctypes.c_int,
                                                         ctypes.c_double, ctypes.c_double, _c_i64p, _c_i64p]),
    "pyr_dg_rhs_noalloc": (ctypes.c_int, [_c_h, ctypes.c_void_p, ctypes.c_void_p]),
    "pyr_dg_profile": (ctypes.c_int, [_c_h, ctypes.c_int]),
    "pyr_dg_batch_setup": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_c_dp), _c_i64p, ctypes.POINTER(_c_i32p),
                                          _c_i64p, _c_ip, ctypes.POINTER(Opts), ctypes.POINTER(_c_h)]),
    "pyr_dg_batch_info": (ctypes.c_int, [_c_h, _c_ip, _c_ip, _c_i64p, _c_i64p]),
    "pyr_dg_batch_group_info": (ctypes.c_int, [_c_h, ctypes.c_int, _c_ip, _c_i64p, _c_ip, _c_ip]),
    "pyr_dg_batch_project": (ctypes.c_int, [_c_h, ctypes.c_double]),
    "pyr_dg_batch_dt_cfl": (ctypes.c_int, [_c_h, ctypes.c_double, _c_dp]),
    "pyr_dg_batch_step": (ctypes.c_int, [_c_h, ctypes.c_int, _c_dp]),
    "pyr_dg_batch_error": (ctypes.c_int, [_c_h, _c_dp, _c_dp]),
    "pyr_dg_batch_get_state": (ctypes.c_int, [_c_h, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "pyr_dg_batch_sync": (ctypes.c_int, [_c_h]),
    "pyr_dg_batch_stream": (ctypes.c_void_p, [_c_h]),
    "pyr_dg_batch_destroy": (None, [_c_h]),
    "pyr_dg_profile_read": (ctypes.c_int, [_c_h, _c_dp, _c_i64p, _c_dp, _c_i64p]),
    "pyr_dg_l2_diff": (ctypes.c_int, [_c_h, ctypes.c_void_p, ctypes.c_void_p, _c_dp, _c_dp]),
    "pyr_dg_host_nodal_points": (ctypes.c_int, [ctypes.c_int, _c_dp]),
    "pyr_dg_set_tensor_mixing": (ctypes.c_int, [_c_h, ctypes.c_int]),
    "pyr_dg_set_tensor_traces": (ctypes.c_int, [_c_h, ctypes.c_int]),
    "pyr_dg_get_tensor_traces": (ctypes.c_int, [_c_h, ctypes.POINTER(ctypes.c_int)]),
    "pyr_dg_batch_launch_mode": (ctypes.c_int, [_c_h, _c_ip, _c_ip]),
    "pyr_dg_batch_set_launch_mode": (ctypes.c_int, [_c_h, ctypes.c_int]),
}


def lib():
    """Load libpyrdg.so (once) and declare its signatures. Raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_1502_07703_gb300.build.build() "
                "(or __graft_entry__.build()); there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise PyrDGError(rc, lib().pyr_dg_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def gauss_jacobi(n, alpha, beta):
    """The library's host Gauss-Jacobi rule: (nodes, weights)."""
    x = np.empty(n)
    w = np.empty(n)
    _check(lib().pyr_dg_host_gauss_jacobi(n, alpha, beta, _ptr(x, ctypes.c_double), _ptr(w, ctypes.c_double)))
    return x, w


def connectivity(vertices, EToV, N):
    """The library's host face connectivity: (mapP (K*Nfc,) int64, number of boundary faces)."""
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    E = np.ascontiguousarray(EToV, dtype=np.int32)
    K = E.shape[0]
    mapP = np.empty(K * 5 * (N + 1) ** 2, dtype=np.int64)
    nb = ctypes.c_int64(0)
    _check(lib().pyr_dg_host_connectivity(_ptr(V, ctypes.c_double), V.shape[0], _ptr(E, ctypes.c_int32), K, N,
                                          _ptr(mapP, ctypes.c_int64), ctypes.byref(nb)))
    return mapP, nb.value


def connectivity_periodic(vertices, EToV, N, box=(0.0, 1.0)):
    """The library's host face connectivity on the periodic box [lo, hi]^3."""
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    E = np.ascontiguousarray(EToV, dtype=np.int32)
    K = E.shape[0]
    mapP = np.empty(K * 5 * (N + 1) ** 2, dtype=np.int64)
    nb = ctypes.c_int64(0)
    _check(lib().pyr_dg_host_connectivity_periodic(_ptr(V, ctypes.c_double), V.shape[0], _ptr(E, ctypes.c_int32), K,
                                                   N, float(box[0]), float(box[1]), _ptr(mapP, ctypes.c_int64),
                                                   ctypes.byref(nb)))
    return mapP, nb.value


def fma_peak(precision="f64"):
    """Measured FMA throughput of the current GPU in TFLOP/s."""
    out = ctypes.c_double(0.0)
    _check(lib().pyr_dg_fma_peak(PYR_DG_F64 if precision == "f64" else PYR_DG_F32, ctypes.byref(out)))
    return out.value


def host_nodal_points(N):
    """(Np, 3) collapsed coordinates (a, b, c) of the nodal variant's nodes, in state order
    (host-only builder query, no GPU needed)."""
    Np = (N + 1) * (N + 2) * (2 * N + 3) // 6
    out = np.empty((Np, 3))
    _check(lib().pyr_dg_host_nodal_points(int(N), _ptr(out, ctypes.c_double)))
    return out


class Solver:
    """One mesh advanced by the library. State arrays are (K, 4, Np) in the
    handle's precision: semi-nodal coefficients, or with basis="nodal" the values at the
    nodes of host_nodal_points (layout in include/pyrdg.h)."""

    def __init__(self, vertices, EToV, N, precision="f64", bc="wall", tau=1.0, stream=None, device=None,
                 equation="wave", beta=(1.0, 0.0, 0.0), periodic=None, basis="modal"):
        """equation: "wave" (4 fields) or "advection" (1 field, needs periodic=(lo, hi); tau is alpha).
        basis: "modal" (semi-nodal coefficients) or "nodal" (Sec. 4.4.1; wave, f64)."""
        import torch

        self._torch = torch
        V = np.ascontiguousarray(vertices, dtype=np.float64)
        E = np.ascontiguousarray(EToV, dtype=np.int32)
        if V.ndim != 2 or V.shape[1] != 3 or E.ndim != 2 or E.shape[1] != 5:
            raise ValueError("vertices must be (Nv, 3) and EToV (K, 5)")
        o = Opts()
        lib().pyr_dg_default_opts(ctypes.byref(o))
        o.precision = {"f64": PYR_DG_F64, "f32": PYR_DG_F32}[precision]
        o.bc = {"wall": PYR_DG_BC_WALL, "free": PYR_DG_BC_FREE}[bc]
        o.tau = float(tau)
        o.equation = {"wave": PYR_DG_WAVE, "advection": PYR_DG_ADVECTION}[equation]
        o.basis = {"modal": PYR_DG_MODAL, "nodal": PYR_DG_NODAL}[basis]
        for m in range(3):
            o.beta[m] = float(beta[m])
        if periodic is not None:
            o.periodic = 1
            o.box_lo, o.box_hi = float(periodic[0]), float(periodic[1])
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        o.device = int(device)
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(device).cuda_stream
        o.stream = stream
        h = _c_h()
        _check(lib().pyr_dg_setup(_ptr(V, ctypes.c_double), V.shape[0], _ptr(E, ctypes.c_int32), E.shape[0], int(N),
                                  ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.device = device
        self.precision = precision
        self.bc = bc
        self.tau = float(tau)
        K, n, Np, Nfc, prec = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().pyr_dg_info(h, ctypes.byref(K), ctypes.byref(n), ctypes.byref(Np), ctypes.byref(Nfc),
                                 ctypes.byref(prec)))
        self.K, self.N, self.Np, self.Nfc = K.value, n.value, Np.value, Nfc.value
        nf = ctypes.c_int()
        _check(lib().pyr_dg_num_fields(h, ctypes.byref(nf)))
        self.nf = nf.value
        self.equation = equation
        self.basis = basis
        self.np_dtype = np.float64 if precision == "f64" else np.float32
        self.torch_dtype = torch.float64 if precision == "f64" else torch.float32

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().pyr_dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.K, self.nf, self.Np)

    # -- calls
    def project(self, t0=0.0):
        _check(lib().pyr_dg_project(self._h, float(t0)))

    def set_state(self, q, t=0.0):
        """q: numpy array (host) or torch CUDA tensor (device), shape (K, 4, Np)."""
        if isinstance(q, np.ndarray):
            a = np.ascontiguousarray(q, dtype=self.np_dtype).reshape(self.shape)
            _check(lib().pyr_dg_set_state(self._h, a.ctypes.data, PYR_DG_HOST, float(t)))
        else:
            a = q.contiguous().to(self.torch_dtype).reshape(self.shape)
            self._require_device(a)
            _check(lib().pyr_dg_set_state(self._h, a.data_ptr(), PYR_DG_DEVICE, float(t)))

    def set_state_host_ptr(self, ptr, t=0.0):
        """Set the state from a raw host pointer (e.g. a pinned torch tensor's data_ptr())."""
        _check(lib().pyr_dg_set_state(self._h, ctypes.c_void_p(ptr), PYR_DG_HOST, float(t)))

    def stage_state_host_ptr(self, ptr, t=0.0):
        """Stage the next step's input from a raw host pointer (best from page-locked memory,
        e.g. a pinned torch tensor's data_ptr()); the copy overlaps enqueued work and the next
        step() makes it the state. The buffer must not change until sync() (or error() /
        get_state() after that step) returns."""
        _check(lib().pyr_dg_stage_state(self._h, ctypes.c_void_p(ptr), float(t)))

    def stage_state(self, q, t=0.0):
        """Stage the next step's input from a numpy array (see stage_state_host_ptr). From
        ordinary (pageable) memory the array has been copied out when the call returns, without
        the overlap; the binding keeps a reference to it until the next stage_state()."""
        a = np.ascontiguousarray(q, dtype=self.np_dtype).reshape(self.shape)
        self._staged = a
        _check(lib().pyr_dg_stage_state(self._h, a.ctypes.data, float(t)))

    def get_state(self, device=False):
        """Copy of the state: numpy array, or a torch CUDA tensor if device=True."""
        if device:
            out = self._torch.empty(self.shape, dtype=self.torch_dtype, device=f"cuda:{self.device}")
            _check(lib().pyr_dg_get_state(self._h, out.data_ptr(), PYR_DG_DEVICE))
            return out
        out = np.empty(self.shape, dtype=self.np_dtype)
        _check(lib().pyr_dg_get_state(self._h, out.ctypes.data, PYR_DG_HOST))
        return out

    def rhs(self, q, out=None):
        """dU/dt of q (torch CUDA tensor (K, 4, Np) of the handle's dtype) into a new or given tensor."""
        self._require_device(q)
        q = q.contiguous()
        if out is None:
            out = self._torch.empty_like(q)
        self._require_device(out)
        _check(lib().pyr_dg_rhs(self._h, q.data_ptr(), out.data_ptr()))
        return out

    def step(self, nsteps, dt):
        _check(lib().pyr_dg_step(self._h, int(nsteps), float(dt)))

    def error(self):
        a, r = ctypes.c_double(), ctypes.c_double()
        _check(lib().pyr_dg_error(self._h, ctypes.byref(a), ctypes.byref(r)))
        return a.value, r.value

    def l2_diff(self, qa, qb):
        """(L2 norm of qa - qb, L2 norm of qb) over the mesh for two device states of this handle
        (torch CUDA tensors of the state's shape and dtype), from the diagonal mass matrix."""
        for q in (qa, qb):
            self._require_device(q)
            if tuple(q.shape) != tuple(self.shape) or q.dtype != self.torch_dtype or not q.is_contiguous():
                raise ValueError("l2_diff needs contiguous states of the handle's shape and dtype")
        d2, n2 = ctypes.c_double(), ctypes.c_double()
        _check(lib().pyr_dg_l2_diff(self._h, qa.data_ptr(), qb.data_ptr(), ctypes.byref(d2), ctypes.byref(n2)))
        return float(np.sqrt(d2.value)), float(np.sqrt(n2.value))

    def set_tensor_mixing(self, enable=True):
        """FP32 wave handles at N >= 4: run the level mixing on the tensor cores (tcgen05 TF32,
        3-term split) instead of the CUDA cores."""
        _check(lib().pyr_dg_set_tensor_mixing(self._h, 1 if enable else 0))

    def set_tensor_traces(self, enable=True):
        """Modal wave handles: interpolate each stage's state to the face points on the tensor
        cores. FP32: tcgen05 TF32, 3-term split, 32 elements x 4 fields per MMA tile, instead of
        in the stage kernel. FP64 (N = 2..4): exact balanced BF16 slices of the trace map and of
        the state, 8 elements x 4 fields per tile, FP64-accurate, instead of the FP64 trace
        kernel."""
        _check(lib().pyr_dg_set_tensor_traces(self._h, 1 if enable else 0))

    @property
    def tensor_traces(self):
        """Whether stepping computes the face traces on the tensor cores (see set_tensor_traces)."""
        v = ctypes.c_int()
        _check(lib().pyr_dg_get_tensor_traces(self._h, ctypes.byref(v)))
        return bool(v.value)

    def set_error_cache(self, enable=True):
        """Store the exact fields' spatial factors for error() when they fit (the default),
        or evaluate them at every call (enable=False)."""
        _check(lib().pyr_dg_set_error_cache(self._h, 1 if enable else 0))

    def dt_cfl(self, cfl=0.5):
        dt = ctypes.c_double()
        _check(lib().pyr_dg_dt_cfl(self._h, float(cfl), ctypes.byref(dt)))
        return dt.value

    @property
    def time(self):
        t = ctypes.c_double()
        _check(lib().pyr_dg_time(self._h, ctypes.byref(t)))
        return t.value

    def profile(self, enable=True):
        """Start (or stop) per-kernel CUDA-event timing of step()."""
        _check(lib().pyr_dg_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{'trace': (ms, launches), 'rhs': (ms, launches)} since profile() was called."""
        tm, rm = ctypes.c_double(), ctypes.c_double()
        tn, rn = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pyr_dg_profile_read(self._h, ctypes.byref(tm), ctypes.byref(tn), ctypes.byref(rm),
                                         ctypes.byref(rn)))
        return {"trace": (tm.value, tn.value), "rhs": (rm.value, rn.value)}

    def sync(self):
        _check(lib().pyr_dg_sync(self._h))

    def _require_device(self, t):
        if not (hasattr(t, "is_cuda") and t.is_cuda) or t.dtype != self.torch_dtype or tuple(t.shape) != self.shape:
            raise ValueError(f"expected a CUDA tensor of shape {self.shape} and dtype {self.torch_dtype}")


class Batch:
    """Many independent meshes advanced together (include/pyrdg.h, batched form).

    meshes: list of (vertices (Nv, 3), EToV (K, 5), N). States are per mesh."""

    def __init__(self, meshes, precision="f32", bc="wall", tau=1.0, device=None):
        import torch

        self._torch = torch
        self._keep = [(np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(e, dtype=np.int32), int(n))
                      for v, e, n in meshes]
        nm = len(self._keep)
        V = (_c_dp * nm)(*[_ptr(v, ctypes.c_double) for v, _, _ in self._keep])
        E = (_c_i32p * nm)(*[_ptr(e, ctypes.c_int32) for _, e, _ in self._keep])
        Nv = np.array([v.shape[0] for v, _, _ in self._keep], dtype=np.int64)
        K = np.array([e.shape[0] for _, e, _ in self._keep], dtype=np.int64)
        Ns = np.array([n for _, _, n in self._keep], dtype=np.int32)
        o = Opts()
        lib().pyr_dg_default_opts(ctypes.byref(o))
        o.precision = {"f64": PYR_DG_F64, "f32": PYR_DG_F32}[precision]
        o.bc = {"wall": PYR_DG_BC_WALL, "free": PYR_DG_BC_FREE}[bc]
        o.tau = float(tau)
        o.device = int(torch.cuda.current_device() if device is None else device)
        o.stream = None
        h = _c_h()
        _check(lib().pyr_dg_batch_setup(nm, V, _ptr(Nv, ctypes.c_int64), E, _ptr(K, ctypes.c_int64),
                                        _ptr(Ns, ctypes.c_int), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.nmesh = nm
        self.K = K
        self.N = Ns
        self.Np = np.array([(n + 1) * (n + 2) * (2 * n + 3) // 6 for n in Ns])
        self.np_dtype = np.float64 if precision == "f64" else np.float32
        nmesh, ng, tk, td = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pyr_dg_batch_info(h, ctypes.byref(nmesh), ctypes.byref(ng), ctypes.byref(tk), ctypes.byref(td)))
        self.ngroups, self.total_K, self.total_dofs = ng.value, tk.value, td.value

    def close(self):
        if getattr(self, "_h", None):
            lib().pyr_dg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def launch_mode(self):
        """(single_launch, launches_per_stage): one kernel per stage for every degree group, or
        one per group on parallel graph branches (chosen at setup by timing both)."""
        a, n = ctypes.c_int(), ctypes.c_int()
        _check(lib().pyr_dg_batch_launch_mode(self._h, ctypes.byref(a), ctypes.byref(n)))
        return bool(a.value), n.value

    def set_launch_mode(self, single_launch):
        _check(lib().pyr_dg_batch_set_launch_mode(self._h, 1 if single_launch else 0))

    def groups(self):
        out = []
        for g in range(self.ngroups):
            n, k, b, epb = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
            _check(lib().pyr_dg_batch_group_info(self._h, g, ctypes.byref(n), ctypes.byref(k), ctypes.byref(b),
                                                 ctypes.byref(epb)))
            out.append({"N": n.value, "K": k.value, "stage_blocks": b.value, "elems_per_block": epb.value})
        return out

    @property
    def stream_ptr(self):
        return lib().pyr_dg_batch_stream(self._h)

    def project(self, t0=0.0):
        _check(lib().pyr_dg_batch_project(self._h, float(t0)))

    def dt_cfl(self, cfl=0.5):
        dt = np.empty(self.nmesh)
        _check(lib().pyr_dg_batch_dt_cfl(self._h, float(cfl), _ptr(dt, ctypes.c_double)))
        return dt

    def step(self, nsteps, dt):
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        _check(lib().pyr_dg_batch_step(self._h, int(nsteps), _ptr(dt, ctypes.c_double)))

    def error(self):
        a = np.empty(self.nmesh)
        r = np.empty(self.nmesh)
        _check(lib().pyr_dg_batch_error(self._h, _ptr(a, ctypes.c_double), _ptr(r, ctypes.c_double)))
        return a, r

    def get_state(self, mesh):
        out = np.empty((int(self.K[mesh]), 4, int(self.Np[mesh])), dtype=self.np_dtype)
        _check(lib().pyr_dg_batch_get_state(self._h, int(mesh), out.ctypes.data, PYR_DG_HOST))
        return out

    def sync(self):
        _check(lib().pyr_dg_batch_sync(self._h))
