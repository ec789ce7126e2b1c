// Internal definition of the pyr_dg handle and helpers shared by the C-ABI
// translation units (api.cu, batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pyrdg.h"
#include "launch.h"

// Carpenter & Kennedy (1994) 5-stage 2N-storage RK4 (cited in Sec. 4.1).
extern const double kRkA[5];
extern const double kRkB[5];

struct pyr_dg {
  int device = 0;
  cudaStream_t stream = nullptr;
  int N = 0, Np = 0, Nfc = 0, precision = 0, bc = 0;
  int equation = PYR_DG_WAVE;  // PYR_DG_WAVE or PYR_DG_ADVECTION
  int nf = 4;                  // fields per element in the state
  double beta[3] = {1.0, 0.0, 0.0};
  double box_lo = 0.0, box_hi = 1.0;
  bool use_stage32 = false;    // FP32 handle: single-launch stage kernel (wave or advection)
  double tau = 1.0;
  int64_t K = 0;
  size_t tsize = 8;
  double t = 0.0;
  double max_aov = 0.0;
  int err_blocks = 0;
  const pyrdg::Launchers* L = nullptr;
  void *q = nullptr, *res = nullptr, *tr = nullptr, *geo = nullptr, *gface = nullptr, *invM = nullptr,
       *tab = nullptr;
  double *tabd = nullptr, *gtab = nullptr, *ev = nullptr, *partial = nullptr;
  int32_t* mapP = nullptr;
  // FP32 handles: second trace buffer; {tr, tr2}[tr_cur] holds the traces of q when tr_valid
  void* tr2 = nullptr;
  int tr_cur = 0;
  bool tr_valid = false;
  bool use_tc = false;          // FP32 stage with the tensor-core level mixing (pyr_dg_set_tensor_mixing)
  bool use_tctr = false;        // traces on the tensor cores (pyr_dg_set_tensor_traces)
  void* tctr_op = nullptr;      // their operator (FP32: the trace map's TF32 hi/lo parts;
                                // FP64: its exact BF16 slices and row exponents)
  int tctr_blocks = 0;          // their persistent grid
  int stage_blocks = 0;         // persistent grid of the FP32 stage kernel
  int stage_epb = 1;            // elements per CTA of the FP32 stage kernel
  // per-element time step (device, K elements of the handle's type) when the handle
  // holds several batched meshes; null for a single mesh
  void* dt_elem = nullptr;
  // pyr_dg_error's store: the error rule's projection of the exact fields' spatial factors
  // (K x 4 x Np doubles), the mass diagonal in double (K x Np), then 4 sums per error block;
  // ecache_sum: |PS_p - S_p|^2, sum_m |PS_m - S_m|^2, |S_p|^2, sum_m |S_m|^2 over the mesh.
  // ecache_mode: 1 store when it fits (default), 0 never. ecache_state: 0 no call yet,
  // 2 one call made without the store, 1 stored, -1 not stored (too large, or mode 0).
  double* ecache = nullptr;
  double ecache_sum[4] = {0.0, 0.0, 0.0, 0.0};
  int ecache_mode = 1, ecache_state = 0;
  // nodal variant (basis == PYR_DG_NODAL): per-degree table (V, V^T, V^{-T}, triangle nodal
  // mass, GLL -> GL interpolation), element nodes of the triangle faces (4 x nT), and the
  // matching trace point of every trace point (K x ntr; itself on a boundary)
  int basis = 0;
  int ntr = 0;
  double* ntab = nullptr;
  int32_t* ntri = nullptr;
  int32_t* nmap = nullptr;
  // pyr_dg_stage_state: a second state buffer that a copy stream fills while the handle's
  // stream computes; the next pyr_dg_step waits for the copy (ev_copied), swaps it in as the
  // state and records ev_free on the handle's stream (work enqueued before that point still
  // reads the old buffer, which becomes q_next: the following copy waits for ev_free)
  void* q_next = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied = nullptr, ev_free = nullptr;
  bool staged = false, ev_free_recorded = false;
  double staged_t = 0.0;
  // per-kernel event timing of pyr_dg_step (pyr_dg_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kind;  // per recorded pair: 0 trace, 1 rhs
  size_t events_used = 0;
};

namespace pyrdg {

// Set the thread-local message returned by pyr_dg_last_error and return code.
int fail(int code, const char* fmt, ...);

// Makes a device current for the duration of a call, restoring the caller's.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    int cur = 0;
    err = cudaGetDevice(&cur);
    if (err == cudaSuccess && cur != dev) {
      err = cudaSetDevice(dev);
      if (err == cudaSuccess) prev = cur;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Enqueue nsteps LSRK4 steps of the handle's state (the body of pyr_dg_step); with
// dt_elem set on the handle each element uses its own step. Host-side bookkeeping of
// the time is left to the caller.
int enqueue_steps(pyr_dg* h, int nsteps, double dt);

}  // namespace pyrdg

#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t _e = (expr);                                                                    \
    if (_e != cudaSuccess)                                                                      \
      return pyrdg::fail(PYR_DG_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(_e));      \
  } while (0)
