// C ABI of libpyrdg.so (declared in include/pyrdg.h): handle lifetime, setup
// (host builder + device geometry), and the per-call launch sequences.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pyrdg.h"
#include "builder.h"
#include "exact64.h"
#include "handle.h"
#include "launch.h"

namespace pyrdg {
const Launchers* launchers_n1(int);
const Launchers* launchers_n2(int);
const Launchers* launchers_n3(int);
const Launchers* launchers_n4(int);
const Launchers* launchers_n5(int);
const Launchers* launchers_n6(int);
const Launchers* launchers_n7(int);

const Launchers* get_launchers(int N, int precision) {
  switch (N) {
    case 1: return launchers_n1(precision);
    case 2: return launchers_n2(precision);
    case 3: return launchers_n3(precision);
    case 4: return launchers_n4(precision);
    case 5: return launchers_n5(precision);
    case 6: return launchers_n6(precision);
    case 7: return launchers_n7(precision);
    default: return nullptr;
  }
}
}  // namespace pyrdg

// Carpenter & Kennedy (1994) 5-stage 2N-storage RK4 (cited in Sec. 4.1).
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

static thread_local std::string g_err;

namespace pyrdg {
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
}  // namespace pyrdg

using pyrdg::DeviceGuard;
using pyrdg::fail;

namespace {
// Device address of pyr_dg_rhs_noalloc's static scratch on the current device (defined at
// the end of this file); cached per device.
cudaError_t noalloc_scratch_address(int device, void** out);
}  // namespace

namespace {
// sum of M_ii (a_i - b_i)^2 and M_ii b_i^2 over a state (M_ii = 1 / invM), per block in double
template <typename T>
__global__ void __launch_bounds__(256)
    l2_diff_kernel(int64_t total, int nf, int Np, const T* __restrict__ a, const T* __restrict__ b,
                   const T* __restrict__ invM, double* __restrict__ partial) {
  __shared__ double red[2][8];
  double d2 = 0.0, n2 = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = x / ((int64_t)nf * Np);
    const int n = (int)(x % Np);
    const double m = 1.0 / (double)invM[e * Np + n];
    const double bv = (double)b[x], dv = (double)a[x] - bv;
    d2 += m * dv * dv;
    n2 += m * bv * bv;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, off);
    n2 += __shfl_down_sync(0xffffffffu, n2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = d2;
    red[1][threadIdx.x >> 5] = n2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// out[e][f][i] = sum_n Mt[n Np + i] in[e][f][n] for every element and field: a per-element
// change of basis of the nodal variant (Mt = V^T: coefficients to nodal values; Mt = V^{-T}:
// the reverse).
__global__ void __launch_bounds__(256)
    nodal_apply_kernel(int64_t K, int Np, const double* __restrict__ Mt, const double* __restrict__ in,
                       double* __restrict__ out) {
  const int64_t total = K * 4 * Np;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % Np);
    const double* v = in + (g - i);
    double acc = 0.0;
    for (int n = 0; n < Np; ++n) acc += Mt[(size_t)n * Np + i] * v[n];
    out[g] = acc;
  }
}

void nodal_apply(const pyr_dg* h, const double* Mt, const void* in, void* out) {
  const int64_t total = h->K * 4 * h->Np;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  nodal_apply_kernel<<<blocks, 256, 0, h->stream>>>(h->K, h->Np, Mt, (const double*)in, (double*)out);
}

// Offsets of V^T and V^{-T} in the nodal table (NodalDims layout: V, V^T, V^{-T}, ...).
inline const double* nodal_VT(const pyr_dg* h) { return h->ntab + (size_t)h->Np * h->Np; }
inline const double* nodal_VinvT(const pyr_dg* h) { return h->ntab + 2 * (size_t)h->Np * h->Np; }

// Record an event pair slot around the next launch when profiling (kind 0 trace, 1 rhs).
cudaError_t prof_begin(pyr_dg* h, int kind, size_t* slot) {
  if (!h->profiling) return cudaSuccess;
  if (h->events_used + 2 > h->events.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      h->events.push_back(ev);
    }
  }
  *slot = h->events_used;
  h->events_used += 2;
  h->event_kind.push_back(kind);
  return cudaEventRecord(h->events[*slot], h->stream);
}

cudaError_t prof_end(pyr_dg* h, size_t slot) {
  if (!h->profiling) return cudaSuccess;
  return cudaEventRecord(h->events[slot + 1], h->stream);
}

void free_all(pyr_dg* h) {
  for (cudaEvent_t ev : h->events) cudaEventDestroy(ev);
  h->events.clear();
  if (h->tctr_op) cudaFree(h->tctr_op);
  h->tctr_op = nullptr;
  if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
  if (h->q_next) cudaFree(h->q_next);
  if (h->ev_copied) cudaEventDestroy(h->ev_copied);
  if (h->ev_free) cudaEventDestroy(h->ev_free);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  h->q_next = nullptr;
  h->ev_copied = h->ev_free = nullptr;
  h->copy_stream = nullptr;
  void* ptrs[] = {h->q,    h->res,  h->tr,   h->geo,  h->gface,   h->invM,  h->tab,
                  h->tabd, h->gtab, h->ev,   h->partial, h->mapP, h->tr2,   h->dt_elem,
                  h->ecache, h->ntab, h->ntri, h->nmap};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}
}  // namespace

namespace pyrdg {
int enqueue_steps(pyr_dg* h, int nsteps, double dt) {
  if (h->equation == PYR_DG_ADVECTION && h->use_stage32 && nsteps > 0) {
    // FP32 advection: one launch per stage; traces ping-pong between tr and tr2
    void* buf[2] = {h->tr, h->tr2};
    size_t slot = 0;
    if (!h->tr_valid) {
      CUDA_TRY(prof_begin(h, 0, &slot));
      h->L->trace1(h->K, h->q, h->tab, buf[h->tr_cur], h->stream);
      CUDA_TRY(prof_end(h, slot));
    }
    for (int n = 0; n < nsteps; ++n) {
      for (int s = 0; s < 5; ++s) {
        CUDA_TRY(prof_begin(h, 1, &slot));
        h->L->adv32(h->K, h->q, h->res, buf[h->tr_cur], buf[1 - h->tr_cur], h->mapP, h->geo, h->gface, h->invM,
                    h->beta, h->tau, kRkA[s], kRkB[s], dt, h->stage_epb, h->stage_blocks, h->stream);
        CUDA_TRY(prof_end(h, slot));
        h->tr_cur = 1 - h->tr_cur;
      }
    }
    CUDA_TRY(cudaGetLastError());
    h->tr_valid = true;
    return PYR_DG_OK;
  }
  if (h->equation == PYR_DG_ADVECTION) {
    for (int n = 0; n < nsteps; ++n) {
      for (int s = 0; s < 5; ++s) {
        size_t slot = 0;
        CUDA_TRY(prof_begin(h, 0, &slot));
        h->L->trace1(h->K, h->q, h->tab, h->tr, h->stream);
        CUDA_TRY(prof_end(h, slot));
        CUDA_TRY(prof_begin(h, 1, &slot));
        h->L->rhs1(h->K, h->q, h->q, h->res, h->tr, h->mapP, h->geo, h->gface, h->invM, h->tab, h->beta, h->tau,
                   kRkA[s], kRkB[s], dt, 1, h->stream);
        CUDA_TRY(prof_end(h, slot));
      }
    }
    CUDA_TRY(cudaGetLastError());
    return PYR_DG_OK;
  }
  if (h->use_stage32 && nsteps > 0) {
    // FP32: one launch per stage; traces ping-pong between tr and tr2
    void* buf[2] = {h->tr, h->tr2};
    size_t slot = 0;
    if (!h->tr_valid) {
      CUDA_TRY(prof_begin(h, 0, &slot));
      h->L->trace(h->K, h->q, h->tab, buf[h->tr_cur], h->stream);
      CUDA_TRY(prof_end(h, slot));
    }
    for (int n = 0; n < nsteps; ++n) {
      for (int s = 0; s < 5; ++s) {
        CUDA_TRY(prof_begin(h, 1, &slot));
        const int wtr = h->use_tctr ? 0 : 1;  // the stage kernel writes the new traces itself
        if (h->use_tc)
          h->L->stage32tc(h->K, h->q, h->res, buf[h->tr_cur], buf[1 - h->tr_cur], h->mapP, h->geo, h->gface,
                          h->invM, h->bc, h->tau, kRkA[s], kRkB[s], dt, h->dt_elem, wtr, h->stage_blocks, h->stream);
        else
          h->L->stage32(h->K, h->q, h->res, buf[h->tr_cur], buf[1 - h->tr_cur], h->mapP, h->geo, h->gface,
                        h->invM, h->bc, h->tau, kRkA[s], kRkB[s], dt, h->dt_elem, wtr, h->stage_epb, h->stage_blocks,
                        h->stream);
        CUDA_TRY(prof_end(h, slot));
        if (h->use_tctr) {  // else: the new state's traces on the tensor cores
          CUDA_TRY(prof_begin(h, 0, &slot));
          h->L->trace32tc(h->K, h->q, buf[1 - h->tr_cur], (const float*)h->tctr_op, h->tctr_blocks, h->stream);
          CUDA_TRY(prof_end(h, slot));
        }
        h->tr_cur = 1 - h->tr_cur;
      }
    }
    CUDA_TRY(cudaGetLastError());
    h->tr_valid = true;
    return PYR_DG_OK;
  }
  if (h->basis == PYR_DG_NODAL) {
    // nodal variant: trace points of the nodal state (copies and the base interpolation),
    // then the stage kernel, per stage
    for (int n = 0; n < nsteps; ++n) {
      for (int s = 0; s < 5; ++s) {
        size_t slot = 0;
        CUDA_TRY(prof_begin(h, 0, &slot));
        h->L->nodal_trace(h->K, h->q, h->ntab, h->ntri, h->tr, h->stream);
        CUDA_TRY(prof_end(h, slot));
        CUDA_TRY(prof_begin(h, 1, &slot));
        h->L->nodal_rhs(h->K, h->q, h->q, h->res, h->tr, h->nmap, h->geo, h->gface, h->invM, h->tab, h->ntab,
                        h->ntri, h->bc, h->tau, kRkA[s], kRkB[s], dt, 1, h->stream);
        CUDA_TRY(prof_end(h, slot));
      }
    }
    CUDA_TRY(cudaGetLastError());
    return PYR_DG_OK;
  }
  // FP64: the trace kernel and the fused stage kernel per stage (a fused form that also
  // interpolates the new state runs slower: its shared memory caps the resident CTAs)
  for (int n = 0; n < nsteps; ++n) {
    for (int s = 0; s < 5; ++s) {
      size_t slot = 0;
      CUDA_TRY(prof_begin(h, 0, &slot));
      if (h->use_tctr)
        h->L->trace64tc(h->K, h->q, h->tr, h->tctr_op, h->tctr_blocks, h->stream);
      else
        h->L->trace(h->K, h->q, h->tab, h->tr, h->stream);
      CUDA_TRY(prof_end(h, slot));
      CUDA_TRY(prof_begin(h, 1, &slot));
      h->L->rhs_update(h->K, h->q, h->res, h->tr, h->mapP, h->geo, h->gface, h->invM, h->tab, h->bc, h->tau, kRkA[s],
                       kRkB[s], dt, h->dt_elem, h->stream);
      CUDA_TRY(prof_end(h, slot));
    }
  }
  CUDA_TRY(cudaGetLastError());
  return PYR_DG_OK;
}
}  // namespace pyrdg

namespace {
// Round a float to TF32 (10 explicit mantissa bits), to nearest with ties away from zero.
float tf32_round(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

// Operand of the tensor-core trace kernels: the dense trace map Phi_f (mode n at face point g)
// in FP64, obtained by applying the FP64 trace kernel to the Np unit states (pseudo-element n
// holds mode n in every field). FP32 handles: split into TF32 hi and lo parts and laid out in
// NKC pieces of KC mode columns, each NP x KC (rows = face points) in the K-major no-swizzle
// operand layout. FP64 handles: each face point's row cut into 8 exact balanced BF16 digits
// against the row's largest exponent, slice by slice 128 x KP in the operand layout (core
// matrices of 8 rows x 8 BF16), then the 128 row exponents.
int build_trace_operator(pyr_dg* h) {
  const pyrdg::Launchers* L64 = pyrdg::get_launchers(h->N, 0);
  if (!L64) return fail(PYR_DG_ERR_UNSUPPORTED_N, "no FP64 launchers for N = %d", h->N);
  CUDA_TRY(L64->prepare());
  const int Np = h->Np, Nfc = h->Nfc;
  const size_t nq = (size_t)Np * 4 * Np, ntr = (size_t)Np * Nfc * 4;
  std::vector<double> unit(nq, 0.0), tr(ntr);
  for (int n = 0; n < Np; ++n)
    for (int f = 0; f < 4; ++f) unit[((size_t)n * 4 + f) * Np + n] = 1.0;
  double *dq = nullptr, *dtr = nullptr;
  CUDA_TRY(cudaMalloc(&dq, nq * 8));
  if (cudaMalloc(&dtr, ntr * 8) != cudaSuccess) {
    cudaFree(dq);
    return fail(PYR_DG_ERR_NO_MEMORY, "tensor-core traces: scratch allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(dq, unit.data(), nq * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    L64->trace(Np, dq, h->tabd, dtr, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(tr.data(), dtr, ntr * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(dq);
  cudaFree(dtr);
  if (e != cudaSuccess) return fail(PYR_DG_ERR_CUDA, "tensor-core traces: trace map: %s", cudaGetErrorString(e));
  if (!h->use_stage32) {  // FP64
    const int KP = h->L->tctr64_kp;
    std::vector<unsigned char> op(h->L->tctr64_op_bytes, 0);
    uint16_t* A = reinterpret_cast<uint16_t*>(op.data());
    int32_t* Fx = reinterpret_cast<int32_t*>(op.data() + (size_t)8 * 128 * KP * 2);
    for (int g = 0; g < Nfc; ++g) {
      int F = 0;
      for (int n = 0; n < Np; ++n) F = std::max(F, pyrdg::ex64_exp(tr[((size_t)n * Nfc + g) * 4]));
      Fx[g] = F;
      for (int n = 0; n < Np; ++n) {
        int32_t a[8];
        pyrdg::ex64_slices(tr[((size_t)n * Nfc + g) * 4], F, a);
        for (int j = 0; j < 8; ++j) {
          const float v = (float)a[j];  // at most 8 significant bits: exact in BF16
          uint32_t b;
          std::memcpy(&b, &v, 4);
          A[(size_t)j * 128 * KP + (size_t)(g >> 3) * (8 * KP) + (n >> 3) * 64 + (g & 7) * 8 + (n & 7)] =
              (uint16_t)(b >> 16);
        }
      }
    }
    CUDA_TRY(cudaMalloc(&h->tctr_op, op.size()));
    CUDA_TRY(cudaMemcpy(h->tctr_op, op.data(), op.size(), cudaMemcpyHostToDevice));
    return PYR_DG_OK;
  }
  const int KC = h->L->tctr_kc, NKC = h->L->tctr_nkc, NP = h->L->tctr_np;
  std::vector<float> op(h->L->tctr_op_floats, 0.f);
  for (int kc = 0; kc < NKC; ++kc) {
    float* hi = op.data() + (size_t)kc * 2 * NP * KC;
    float* lo = hi + (size_t)NP * KC;
    for (int g = 0; g < Nfc; ++g)
      for (int k = 0; k < KC; ++k) {
        const int n = kc * KC + k;
        if (n >= Np) continue;
        const double v = tr[((size_t)n * Nfc + g) * 4];  // field 0 of pseudo-element n
        const float vh = tf32_round((float)v);
        const size_t o = (size_t)(g >> 3) * (8 * KC) + (k >> 2) * 32 + (g & 7) * 4 + (k & 3);
        hi[o] = vh;
        lo[o] = tf32_round((float)(v - (double)vh));
      }
  }
  CUDA_TRY(cudaMalloc(&h->tctr_op, op.size() * sizeof(float)));
  CUDA_TRY(cudaMemcpy(h->tctr_op, op.data(), op.size() * sizeof(float), cudaMemcpyHostToDevice));
  return PYR_DG_OK;
}
}  // namespace

namespace {
int enable_tensor_traces(pyr_dg* h) {
  if (!h->tctr_op) {
    const int rc = build_trace_operator(h);
    if (rc != PYR_DG_OK) return rc;
  }
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (!h->use_stage32) {  // FP64: tiles of 8 elements, one CTA per SM
    h->tctr_blocks = (int)std::min<int64_t>((h->K + 7) / 8, (int64_t)nsm);
    h->use_tctr = true;
    return PYR_DG_OK;
  }
  const int64_t tiles = (h->K + 31) / 32;
  h->tctr_blocks = (int)std::min<int64_t>(tiles, (int64_t)nsm * h->L->blocks_per_sm_trace32tc());
  h->use_tctr = true;
  return PYR_DG_OK;
}
}  // namespace

extern "C" {

void pyr_dg_default_opts(pyr_dg_opts* o) {
  if (!o) return;
  o->precision = PYR_DG_F64;
  o->bc = PYR_DG_BC_WALL;
  o->tau = 1.0;
  o->stream = nullptr;
  o->device = -1;
  o->equation = PYR_DG_WAVE;
  o->beta[0] = 1.0;
  o->beta[1] = 0.0;
  o->beta[2] = 0.0;
  o->periodic = 0;
  o->box_lo = 0.0;
  o->box_hi = 1.0;
  o->basis = PYR_DG_MODAL;
}

const char* pyr_dg_last_error(void) { return g_err.c_str(); }

int pyr_dg_host_gauss_jacobi(int n, double alpha, double beta, double* x, double* w) {
  if (!x || !w) return fail(PYR_DG_ERR_BAD_ARG, "null output pointer");
  if (pyrdg::gauss_jacobi(n, alpha, beta, x, w) != 0)
    return fail(PYR_DG_ERR_BAD_ARG, "gauss_jacobi: need 1 <= n <= 64 and alpha, beta > -1");
  return PYR_DG_OK;
}

int pyr_dg_host_nodal_points(int N, double* abc) {
  if (!abc) return fail(PYR_DG_ERR_BAD_ARG, "null output pointer");
  if (N < PYR_DG_MIN_N || N > PYR_DG_MAX_N) return fail(PYR_DG_ERR_UNSUPPORTED_N, "N = %d unsupported", N);
  pyrdg::NodalTables nt;
  if (pyrdg::build_nodal(N, nt) != 0) return fail(PYR_DG_ERR_UNSUPPORTED_N, "nodal set build failed for N = %d", N);
  std::memcpy(abc, nt.nodes.data(), nt.nodes.size() * sizeof(double));
  return PYR_DG_OK;
}

int pyr_dg_host_connectivity(const double* vertices, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                             int64_t* mapP, int64_t* nboundary) {
  if (!vertices || !EToV || !mapP || Nv < 1 || K < 1) return fail(PYR_DG_ERR_BAD_ARG, "bad connectivity arguments");
  if (N < PYR_DG_MIN_N || N > PYR_DG_MAX_N) return fail(PYR_DG_ERR_UNSUPPORTED_N, "N = %d unsupported", N);
  std::vector<int64_t> m;
  std::string err;
  const int rc = pyrdg::build_connectivity(vertices, Nv, EToV, K, N, m, nboundary, err);
  if (rc != 0) return fail(PYR_DG_ERR_BAD_MESH, "%s", err.c_str());
  std::memcpy(mapP, m.data(), m.size() * sizeof(int64_t));
  return PYR_DG_OK;
}

int pyr_dg_host_connectivity_periodic(const double* vertices, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                                      double box_lo, double box_hi, int64_t* mapP, int64_t* nboundary) {
  if (!vertices || !EToV || !mapP || Nv < 1 || K < 1 || !(box_hi > box_lo))
    return fail(PYR_DG_ERR_BAD_ARG, "bad connectivity arguments");
  if (N < PYR_DG_MIN_N || N > PYR_DG_MAX_N) return fail(PYR_DG_ERR_UNSUPPORTED_N, "N = %d unsupported", N);
  std::vector<int64_t> m;
  std::string err;
  const double box[2] = {box_lo, box_hi};
  const int rc = pyrdg::build_connectivity(vertices, Nv, EToV, K, N, m, nboundary, err, box);
  if (rc != 0) return fail(PYR_DG_ERR_BAD_MESH, "%s", err.c_str());
  std::memcpy(mapP, m.data(), m.size() * sizeof(int64_t));
  return PYR_DG_OK;
}

int pyr_dg_setup(const double* vertices, int64_t Nv, const int32_t* EToV, int64_t K, int N, const pyr_dg_opts* opts,
                 pyr_dg** out) {
  g_err.clear();
  if (!out) return fail(PYR_DG_ERR_BAD_ARG, "out is null");
  *out = nullptr;
  if (!vertices || !EToV) return fail(PYR_DG_ERR_BAD_ARG, "vertices or EToV is null");
  if (Nv < 5 || K < 1) return fail(PYR_DG_ERR_BAD_ARG, "need Nv >= 5 and K >= 1 (got %lld, %lld)", (long long)Nv,
                                   (long long)K);
  if (K > 0x7fffffffLL) return fail(PYR_DG_ERR_BAD_ARG, "K = %lld exceeds the grid limit", (long long)K);
  if (N < PYR_DG_MIN_N || N > PYR_DG_MAX_N)
    return fail(PYR_DG_ERR_UNSUPPORTED_N, "N = %d outside [%d, %d]", N, PYR_DG_MIN_N, PYR_DG_MAX_N);
  pyr_dg_opts o;
  pyr_dg_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != PYR_DG_F64 && o.precision != PYR_DG_F32) return fail(PYR_DG_ERR_BAD_ARG, "unknown precision");
  if (o.bc != PYR_DG_BC_WALL && o.bc != PYR_DG_BC_FREE) return fail(PYR_DG_ERR_BAD_ARG, "unknown bc");
  if (!(o.tau >= 0.0) || !std::isfinite(o.tau)) return fail(PYR_DG_ERR_BAD_ARG, "tau must be finite and >= 0");
  if (o.equation != PYR_DG_WAVE && o.equation != PYR_DG_ADVECTION) return fail(PYR_DG_ERR_BAD_ARG, "unknown equation");
  if (o.periodic && !(o.box_hi > o.box_lo)) return fail(PYR_DG_ERR_BAD_ARG, "periodic box needs box_hi > box_lo");
  if (o.equation == PYR_DG_ADVECTION && !o.periodic)
    return fail(PYR_DG_ERR_BAD_ARG, "advection is implemented on periodic boxes only (set periodic = 1)");
  if (o.equation == PYR_DG_ADVECTION &&
      !(std::isfinite(o.beta[0]) && std::isfinite(o.beta[1]) && std::isfinite(o.beta[2])))
    return fail(PYR_DG_ERR_BAD_ARG, "beta must be finite");
  if (o.basis != PYR_DG_MODAL && o.basis != PYR_DG_NODAL) return fail(PYR_DG_ERR_BAD_ARG, "unknown basis");
  if (o.basis == PYR_DG_NODAL && (o.precision != PYR_DG_F64 || o.equation != PYR_DG_WAVE))
    return fail(PYR_DG_ERR_BAD_ARG, "the nodal basis is implemented for the wave equation in double precision");
  const int n1 = N + 1, n2 = n1 * n1, Nfc = 5 * n2, Np = pyrdg::num_modes(N);
  if (K * (int64_t)Nfc > 0x7fffffffLL) return fail(PYR_DG_ERR_BAD_ARG, "K * Nfc exceeds int32 face indexing");

  // ---- host builder
  pyrdg::RefTables T;
  if (pyrdg::build_tables(N, T) != 0) return fail(PYR_DG_ERR_UNSUPPORTED_N, "table build failed for N = %d", N);
  std::vector<int64_t> map64;
  std::string err;
  int64_t nbnd = 0;
  const double box[2] = {o.box_lo, o.box_hi};
  if (pyrdg::build_connectivity(vertices, Nv, EToV, K, N, map64, &nbnd, err, o.periodic ? box : nullptr) != 0)
    return fail(PYR_DG_ERR_BAD_MESH, "%s", err.c_str());
  if (o.equation == PYR_DG_ADVECTION && nbnd > 0)
    return fail(PYR_DG_ERR_BAD_MESH, "advection needs every face matched, %lld faces are unmatched on the periodic box",
                (long long)nbnd);
  std::vector<double> ev((size_t)K * 15);
  const pyrdg::GeoLayout G(N);
  double max_aov = 0.0;
  for (int64_t e = 0; e < K; ++e) {
    double* v = &ev[(size_t)e * 15];
    for (int m = 0; m < 15; ++m) v[m] = vertices[(int64_t)EToV[e * 5 + m / 3] * 3 + m % 3];
    // J is bilinear in (a, b) (Lemma 1): positive everywhere iff positive at the 4 corners
    for (int c = 0; c < 4; ++c) {
      const double J = pyrdg::jacobian_ab(v, (c & 1) ? 1.0 : -1.0, (c & 2) ? 1.0 : -1.0);
      if (!(J > 0.0))
        return fail(PYR_DG_ERR_BAD_MESH, "element %lld has J = %g <= 0 at a base corner (vertex order or inverted)",
                    (long long)e, J);
    }
    const double aov = pyrdg::area_over_volume(v, &T.geo[G.XG], &T.geo[G.WG], n1);
    if (aov > max_aov) max_aov = aov;
  }
  std::vector<int32_t> map32((size_t)K * Nfc);
  for (size_t g = 0; g < map32.size(); ++g) map32[g] = (int32_t)map64[g];

  // ---- nodal variant: tables and the trace-point matching (base Gauss-Legendre points from the
  // face cubature matching; triangle-face nodes from the matched faces' orientation)
  pyrdg::NodalTables NT;
  std::vector<int32_t> nmap;
  const pyrdg::Launchers* Lsel = pyrdg::get_launchers(N, o.precision);
  const int ntr = o.basis == PYR_DG_NODAL ? Lsel->nodal_ntr : 0;
  if (o.basis == PYR_DG_NODAL) {
    if (pyrdg::build_nodal(N, NT) != 0) return fail(PYR_DG_ERR_UNSUPPORTED_N, "nodal set build failed for N = %d", N);
    const int nT = NT.nT;
    std::vector<int> lay(n1 + 1, 0);  // first local node of each layer on a triangle face
    for (int m = 0; m < n1; ++m) lay[m + 1] = lay[m] + (n1 - m);
    nmap.resize((size_t)K * ntr);
    for (int64_t e = 0; e < K; ++e) {
      for (int g = 0; g < n2; ++g) {
        const int64_t gq = map64[(size_t)(e * Nfc + g)];
        const int64_t en = gq / Nfc, gn = gq % Nfc;
        if (gn >= n2) return fail(PYR_DG_ERR_BAD_MESH, "element %lld: base face matched to a triangle", (long long)e);
        nmap[(size_t)(e * ntr + g)] = (int32_t)(en * ntr + gn);
      }
      for (int f = 1; f <= 4; ++f) {
        const int64_t gq = map64[(size_t)(e * Nfc + f * n2)];  // the face's point (edge 0, height 0)
        const int64_t en = gq / Nfc;
        const int fn = (int)((gq % Nfc) / n2), idxn = (int)((gq % Nfc) % n2);
        const bool self = gq == e * Nfc + f * n2;
        if (!self && fn == 0) return fail(PYR_DG_ERR_BAD_MESH, "element %lld: triangle matched to a base", (long long)e);
        const bool rev = (idxn % n1) != 0;  // edge reversal (the apex is shared)
        for (int m = 0; m < n1; ++m)
          for (int t = 0; t < n1 - m; ++t) {
            const int j = lay[m] + t;
            const int64_t own = e * ntr + n2 + (int64_t)(f - 1) * nT + j;
            const int jn = lay[m] + (rev ? n1 - m - 1 - t : t);
            nmap[(size_t)own] = self ? (int32_t)own : (int32_t)(en * ntr + n2 + (int64_t)(fn - 1) * nT + jn);
          }
      }
    }
  }

  pyr_dg* h = new (std::nothrow) pyr_dg();
  if (!h) return fail(PYR_DG_ERR_NO_MEMORY, "host allocation failed");
  h->N = N;
  h->Np = Np;
  h->Nfc = Nfc;
  h->K = K;
  h->precision = o.precision;
  h->bc = o.bc;
  h->tau = o.tau;
  h->equation = o.equation;
  h->nf = o.equation == PYR_DG_ADVECTION ? 1 : 4;
  for (int m = 0; m < 3; ++m) h->beta[m] = o.beta[m];
  h->box_lo = o.box_lo;
  h->box_hi = o.box_hi;
  h->tsize = o.precision == PYR_DG_F64 ? 8 : 4;
  h->stream = (cudaStream_t)o.stream;
  h->max_aov = max_aov;
  h->L = Lsel;
  h->basis = o.basis;
  h->ntr = ntr;
  if (o.device >= 0) {
    h->device = o.device;
  } else if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(PYR_DG_ERR_CUDA, "no CUDA device available");
  }
  DeviceGuard guard(h->device);
  if (guard.err != cudaSuccess) {
    delete h;
    return fail(PYR_DG_ERR_CUDA, "cannot select device %d: %s", h->device, cudaGetErrorString(guard.err));
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  h->err_blocks = (int)std::min<int64_t>(K, (int64_t)(nsm > 0 ? nsm : 1) * 4);

  const size_t ts = h->tsize;
  // FP32 handles take the single-launch stage kernels (wave or advection)
  h->use_stage32 = h->L->stage32 != nullptr;
  const size_t stateB = (size_t)K * h->nf * Np * ts;
  const pyrdg::TabLayout TL(N);
  struct Alloc {
    void** p;
    size_t bytes;
  } allocs[] = {
      {&h->q, stateB},
      {&h->res, stateB},
      {&h->tr, (size_t)K * Nfc * 4 * ts},
      {&h->geo, (size_t)K * n2 * 9 * ts},
      {&h->gface, (size_t)K * (16 + 4 * n2) * ts},
      {&h->invM, (size_t)K * Np * ts},
      {&h->tab, (size_t)TL.size * ts},
      {(void**)&h->tabd, (size_t)TL.size * 8},
      {(void**)&h->gtab, (size_t)G.size * 8},
      {(void**)&h->ev, (size_t)K * 15 * 8},
      {(void**)&h->partial, (size_t)h->err_blocks * 2 * 8},
      {(void**)&h->mapP, (size_t)K * Nfc * 4},
      {&h->tr2, h->use_stage32 ? (size_t)K * Nfc * 4 * ts : 0},
      {(void**)&h->ntab, o.basis == PYR_DG_NODAL ? (size_t)h->L->nodal_ntab * 8 : 0},
      {(void**)&h->ntri, o.basis == PYR_DG_NODAL ? (size_t)4 * NT.nT * 4 : 0},
      {(void**)&h->nmap, o.basis == PYR_DG_NODAL ? (size_t)K * ntr * 4 : 0},
  };
  for (auto& a : allocs) {
    if (a.bytes == 0) continue;
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      free_all(h);
      delete h;
      return fail(e == cudaErrorMemoryAllocation ? PYR_DG_ERR_NO_MEMORY : PYR_DG_ERR_CUDA,
                  "cudaMalloc(%zu bytes): %s", a.bytes, cudaGetErrorString(e));
    }
  }
  std::vector<float> tabf;
  const void* tabsrc = T.tab.data();
  if (ts == 4) {
    tabf.assign(T.tab.begin(), T.tab.end());
    tabsrc = tabf.data();
  }
  cudaError_t e = cudaSuccess;
  cudaStream_t s = h->stream;
  if (e == cudaSuccess) e = h->L->prepare();
  if (e == cudaSuccess && h->use_stage32) {
    e = h->L->upload_c32(T.tab.data());
    const bool adv = h->equation == PYR_DG_ADVECTION;
    h->stage_epb = adv ? h->L->epb_adv32 : h->L->epb32;
    const int bps = adv ? h->L->blocks_per_sm_adv32(h->stage_epb) : h->L->blocks_per_sm32(h->stage_epb);
    const int64_t groups = (K + h->stage_epb - 1) / h->stage_epb;
    h->stage_blocks = (int)std::min<int64_t>(groups, (int64_t)(nsm > 0 ? nsm : 1) * bps);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->tab, tabsrc, (size_t)TL.size * ts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->tabd, T.tab.data(), (size_t)TL.size * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->gtab, T.geo.data(), (size_t)G.size * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->ev, ev.data(), ev.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->mapP, map32.data(), map32.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h->basis == PYR_DG_NODAL) {
    // table layout of NodalDims: V, V^T, V^{-T}, triangle nodal mass, GLL -> GL interpolation
    std::vector<double> nt;
    nt.reserve((size_t)h->L->nodal_ntab);
    nt.insert(nt.end(), NT.V.begin(), NT.V.end());
    nt.insert(nt.end(), NT.VT.begin(), NT.VT.end());
    nt.insert(nt.end(), NT.VinvT.begin(), NT.VinvT.end());
    nt.insert(nt.end(), NT.Mtri.begin(), NT.Mtri.end());
    nt.insert(nt.end(), NT.I1.begin(), NT.I1.end());
    if (nt.size() != (size_t)h->L->nodal_ntab) {
      e = cudaErrorInvalidValue;
    } else {
      std::vector<int32_t> tri(NT.tri_node.begin(), NT.tri_node.end());
      e = cudaMemcpyAsync(h->ntab, nt.data(), nt.size() * 8, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->ntri, tri.data(), tri.size() * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->nmap, nmap.data(), nmap.size() * 4, cudaMemcpyHostToDevice, s);
      // the host vectors must outlive the copies: the stream is synchronised below
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->q, 0, stateB, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->res, 0, stateB, s);
  if (e == cudaSuccess) {
    h->L->geom(K, h->ev, h->gtab, h->geo, h->gface, h->invM, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return fail(PYR_DG_ERR_CUDA, "setup: %s", cudaGetErrorString(e));
  }
  // pyr_dg_rhs_noalloc's static scratch: fetch its address here, where allocating is allowed
  // (with lazy module loading the lookup is what places the array on the device). A failure
  // is left for pyr_dg_rhs_noalloc to retry and report.
  if (h->equation == PYR_DG_WAVE) {
    void* p = nullptr;
    if (noalloc_scratch_address(h->device, &p) != cudaSuccess) cudaGetLastError();
  }
  // FP32 wave handles: the new state's face traces on the tensor cores where that is faster,
  // at the degrees the launchers mark and on meshes of at least 40,000 pyramids (measured: from
  // about 8 tiles of 32 elements per SM up the second launch per stage pays for itself)
  if (h->equation == PYR_DG_WAVE && h->basis == PYR_DG_MODAL && h->K >= 40000 &&
      (h->use_stage32 ? h->L->tctr_default != 0 : (h->L->tctr64_default != 0 && h->L->trace64tc != nullptr))) {
    const int rc = enable_tensor_traces(h);
    if (rc != PYR_DG_OK) {
      free_all(h);
      delete h;
      return rc;
    }
  }
  *out = h;
  return PYR_DG_OK;
}

int pyr_dg_info(const pyr_dg* h, int64_t* K, int* N, int* Np, int* Nfc, int* precision) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  if (K) *K = h->K;
  if (N) *N = h->N;
  if (Np) *Np = h->Np;
  if (Nfc) *Nfc = h->Nfc;
  if (precision) *precision = h->precision;
  return PYR_DG_OK;
}

int pyr_dg_num_fields(const pyr_dg* h, int* nf) {
  if (!h || !nf) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  *nf = h->nf;
  return PYR_DG_OK;
}

int pyr_dg_project(pyr_dg* h, double t0) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  if (!std::isfinite(t0)) return fail(PYR_DG_ERR_BAD_ARG, "t0 must be finite");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  if (h->equation == PYR_DG_ADVECTION) {
    h->L->project1(h->K, h->ev, h->gtab, h->tabd, h->beta, h->box_lo, h->box_hi - h->box_lo, t0, h->q, h->stream);
  } else if (h->basis == PYR_DG_NODAL) {  // coefficients into the residual buffer, then nodal values
    h->L->project(h->K, h->ev, h->gtab, h->tabd, h->bc, t0, h->res, h->stream);
    nodal_apply(h, nodal_VT(h), h->res, h->q);
  } else {
    h->L->project(h->K, h->ev, h->gtab, h->tabd, h->bc, t0, h->q, h->stream);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(h->res, 0, (size_t)h->K * h->nf * h->Np * h->tsize, h->stream));
  h->t = t0;
  h->tr_valid = false;
  h->staged = false;  // a staged state not yet consumed is dropped
  return PYR_DG_OK;
}

int pyr_dg_set_state(pyr_dg* h, const void* q, int where, double t) {
  if (!h || !q) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (where != PYR_DG_HOST && where != PYR_DG_DEVICE) return fail(PYR_DG_ERR_BAD_ARG, "bad `where`");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  const size_t bytes = (size_t)h->K * h->nf * h->Np * h->tsize;
  CUDA_TRY(cudaMemcpyAsync(h->q, q, bytes, where == PYR_DG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           h->stream));
  CUDA_TRY(cudaMemsetAsync(h->res, 0, bytes, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->t = t;
  h->tr_valid = false;
  h->staged = false;  // a staged state not yet consumed is dropped
  return PYR_DG_OK;
}

int pyr_dg_stage_state(pyr_dg* h, const void* q_host, double t) {
  if (!h || !q_host) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (!std::isfinite(t)) return fail(PYR_DG_ERR_BAD_ARG, "t must be finite");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  const size_t bytes = (size_t)h->K * h->nf * h->Np * h->tsize;
  if (!h->copy_stream) {
    CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&h->ev_free, cudaEventDisableTiming));
  }
  if (!h->q_next && cudaMalloc(&h->q_next, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->q_next = nullptr;
    return fail(PYR_DG_ERR_NO_MEMORY, "cannot allocate the staged state (%zu bytes)", bytes);
  }
  // the buffer's previous contents may still be read by work enqueued before the last swap
  if (h->ev_free_recorded) CUDA_TRY(cudaStreamWaitEvent(h->copy_stream, h->ev_free, 0));
  CUDA_TRY(cudaMemcpyAsync(h->q_next, q_host, bytes, cudaMemcpyHostToDevice, h->copy_stream));
  CUDA_TRY(cudaEventRecord(h->ev_copied, h->copy_stream));
  h->staged = true;
  h->staged_t = t;
  return PYR_DG_OK;
}

int pyr_dg_get_state(pyr_dg* h, void* q, int where) {
  if (!h || !q) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (where != PYR_DG_HOST && where != PYR_DG_DEVICE) return fail(PYR_DG_ERR_BAD_ARG, "bad `where`");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  const size_t bytes = (size_t)h->K * h->nf * h->Np * h->tsize;
  CUDA_TRY(cudaMemcpyAsync(q, h->q, bytes, where == PYR_DG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return PYR_DG_OK;
}

int pyr_dg_rhs(pyr_dg* h, const void* q_dev, void* rhs_dev) {
  if (!h || !q_dev || !rhs_dev) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (q_dev == rhs_dev) return fail(PYR_DG_ERR_BAD_ARG, "rhs must not alias q");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  if (h->equation == PYR_DG_ADVECTION) {
    h->L->trace1(h->K, q_dev, h->tab, h->tr, h->stream);
    h->L->rhs1(h->K, q_dev, rhs_dev, nullptr, h->tr, h->mapP, h->geo, h->gface, h->invM, h->tab, h->beta, h->tau, 0.0,
               0.0, 0.0, 0, h->stream);
  } else if (h->basis == PYR_DG_NODAL) {
    h->L->nodal_trace(h->K, q_dev, h->ntab, h->ntri, h->tr, h->stream);
    h->L->nodal_rhs(h->K, q_dev, rhs_dev, nullptr, h->tr, h->nmap, h->geo, h->gface, h->invM, h->tab, h->ntab,
                    h->ntri, h->bc, h->tau, 0.0, 0.0, 0.0, 0, h->stream);
  } else {
    h->L->trace(h->K, q_dev, h->tab, h->tr, h->stream);
    h->L->rhs_out(h->K, q_dev, rhs_dev, h->tr, h->mapP, h->geo, h->gface, h->invM, h->tab, h->bc, h->tau,
                  h->stream);
  }
  CUDA_TRY(cudaGetLastError());
  h->tr_valid = false;  // the trace buffer was used as scratch
  return PYR_DG_OK;
}

int pyr_dg_step(pyr_dg* h, int nsteps, double dt) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(PYR_DG_ERR_BAD_ARG, "need nsteps >= 0, dt > 0");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  if (h->staged) {  // the staged state becomes the state once its copy has landed
    CUDA_TRY(cudaStreamWaitEvent(h->stream, h->ev_copied, 0));
    std::swap(h->q, h->q_next);
    CUDA_TRY(cudaEventRecord(h->ev_free, h->stream));
    h->ev_free_recorded = true;
    CUDA_TRY(cudaMemsetAsync(h->res, 0, (size_t)h->K * h->nf * h->Np * h->tsize, h->stream));
    h->t = h->staged_t;
    h->tr_valid = false;
    h->staged = false;
  }
  const int rc = pyrdg::enqueue_steps(h, nsteps, dt);
  if (rc != PYR_DG_OK) return rc;
  h->t += nsteps * dt;
  return PYR_DG_OK;
}

namespace {
// Sum the error kernels' per-block pairs (synchronises the stream).
int read_partial(pyr_dg* h, double* s0, double* s1) {
  std::vector<double> part((size_t)h->err_blocks * 2);
  CUDA_TRY(cudaMemcpyAsync(part.data(), h->partial, part.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  double a = 0.0, b = 0.0;
  for (int i = 0; i < h->err_blocks; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  *s0 = a;
  *s1 = b;
  return PYR_DG_OK;
}

// Second pyr_dg_error of a wave handle (a single call does not pay for the store): store the
// error rule's projection of the exact fields' spatial factors, the mass diagonal and four
// mesh sums, when that takes at most a quarter of the free device memory; otherwise the
// error kernel evaluates the exact fields at its points at every call.
int build_error_cache(pyr_dg* h) {
  h->ecache_state = -1;
  if (h->ecache_mode == 0) return PYR_DG_OK;
  const size_t Np = (size_t)h->Np;
  const size_t nproj = (size_t)h->K * 5 * Np, npart = (size_t)h->err_blocks * 4;
  const size_t bytes = (nproj + npart) * sizeof(double);
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (bytes > free_b / 4) return PYR_DG_OK;
  if (cudaMalloc((void**)&h->ecache, bytes) != cudaSuccess) {
    cudaGetLastError();  // an allocation failure leaves the context usable: compute on the fly
    h->ecache = nullptr;
    return PYR_DG_OK;
  }
  double* shat = h->ecache;
  double* Md = shat + (size_t)h->K * 4 * Np;
  double* part = h->ecache + nproj;
  h->L->exact_proj(h->K, h->ev, h->gtab, h->bc, shat, Md, part, h->err_blocks, h->stream);
  CUDA_TRY(cudaGetLastError());
  std::vector<double> hp(npart);
  CUDA_TRY(cudaMemcpyAsync(hp.data(), part, npart * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < 4; ++c) {
    double a = 0.0;
    for (int b = 0; b < h->err_blocks; ++b) a += hp[4 * (size_t)b + c];
    h->ecache_sum[c] = a;
  }
  h->ecache_state = 1;
  return PYR_DG_OK;
}
}  // namespace

int pyr_dg_l2_diff(pyr_dg* h, const void* qa, const void* qb, double* d2, double* n2) {
  if (!h || !qa || !qb) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (h->basis != PYR_DG_MODAL) return fail(PYR_DG_ERR_BAD_ARG, "pyr_dg_l2_diff needs a modal-basis handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  const int64_t total = h->K * h->nf * h->Np;
  if (h->tsize == 8)
    l2_diff_kernel<double><<<h->err_blocks, 256, 0, h->stream>>>(total, h->nf, h->Np, (const double*)qa,
                                                                  (const double*)qb, (const double*)h->invM,
                                                                  h->partial);
  else
    l2_diff_kernel<float><<<h->err_blocks, 256, 0, h->stream>>>(total, h->nf, h->Np, (const float*)qa,
                                                                 (const float*)qb, (const float*)h->invM,
                                                                 h->partial);
  CUDA_TRY(cudaGetLastError());
  double s0 = 0.0, s1 = 0.0;
  const int rc = read_partial(h, &s0, &s1);
  if (rc != PYR_DG_OK) return rc;
  if (d2) *d2 = s0;
  if (n2) *n2 = s1;
  return PYR_DG_OK;
}

int pyr_dg_set_error_cache(pyr_dg* h, int enable) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  if (h->ecache) {
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    CUDA_TRY(cudaFree(h->ecache));
    h->ecache = nullptr;
  }
  h->ecache_mode = enable ? 1 : 0;
  h->ecache_state = 0;
  return PYR_DG_OK;
}

int pyr_dg_error(pyr_dg* h, double* l2_abs, double* l2_rel) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  double e2 = 0.0, n2 = 0.0;
  if (h->equation == PYR_DG_ADVECTION) {
    h->L->error1(h->K, h->q, h->ev, h->gtab, h->beta, h->box_lo, h->box_hi - h->box_lo, h->t, h->partial,
                 h->err_blocks, h->stream);
    CUDA_TRY(cudaGetLastError());
    const int rc = read_partial(h, &e2, &n2);
    if (rc != PYR_DG_OK) return rc;
  } else {
    // the error kernels read semi-nodal coefficients: a nodal state is converted into the trace
    // buffer (K x Nfc x 4 >= K x 4 x Np doubles), which holds no state between stages in FP64
    const void* qm = h->q;
    if (h->basis == PYR_DG_NODAL) {
      nodal_apply(h, nodal_VinvT(h), h->q, h->tr);
      CUDA_TRY(cudaGetLastError());
      qm = h->tr;
    }
    if (h->ecache_state == 2) {
      const int rc = build_error_cache(h);
      if (rc != PYR_DG_OK) return rc;
    } else if (h->ecache_state == 0) {
      h->ecache_state = 2;
    }
    if (h->ecache_state == 1 && h->ecache) {
      // time factors of the standing wave: p ~ cos(sqrt3 pi sc t), u ~ sin(sqrt3 pi sc t)/sqrt3
      const double sc = h->bc == 0 ? 1.0 : 0.5;
      const double arg = 3.14159265358979323846 * (1.7320508075688772935 * sc * h->t);
      const double tp = std::cos(arg), tu = std::sin(arg) * 0.57735026918962576451;
      const double* shat = h->ecache;
      const double* Md = shat + (size_t)h->K * 4 * h->Np;
      h->L->error_proj(h->K, qm, shat, Md, tp, tu, h->partial, h->err_blocks, h->stream);
      CUDA_TRY(cudaGetLastError());
      double zero = 0.0;
      const int rc = read_partial(h, &e2, &zero);
      if (rc != PYR_DG_OK) return rc;
      // |U_h - U_ex|^2 = sum M (u - T s)^2 + T^2 |PS - S|^2, per field (orthogonality of P)
      e2 += tp * tp * h->ecache_sum[0] + tu * tu * h->ecache_sum[1];
      n2 = tp * tp * h->ecache_sum[2] + tu * tu * h->ecache_sum[3];
    } else {
      h->L->error(h->K, qm, h->ev, h->gtab, h->bc, h->t, h->partial, h->err_blocks, h->stream);
      CUDA_TRY(cudaGetLastError());
      const int rc = read_partial(h, &e2, &n2);
      if (rc != PYR_DG_OK) return rc;
    }
  }
  if (l2_abs) *l2_abs = std::sqrt(e2);
  if (l2_rel) *l2_rel = n2 > 0 ? std::sqrt(e2 / n2) : std::sqrt(e2);
  return PYR_DG_OK;
}

int pyr_dg_dt_cfl(pyr_dg* h, double cfl, double* dt) {
  if (!h || !dt) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (!(cfl > 0.0)) return fail(PYR_DG_ERR_BAD_ARG, "cfl must be > 0");
  const double CN = 2.0 * (h->N + 1) * (h->N + 3) / 3.0;
  double speed = 1.0;  // wave speed c = 1; advection: |beta|
  if (h->equation == PYR_DG_ADVECTION)
    speed = std::sqrt(h->beta[0] * h->beta[0] + h->beta[1] * h->beta[1] + h->beta[2] * h->beta[2]);
  if (!(speed > 0.0)) return fail(PYR_DG_ERR_BAD_ARG, "advection speed is zero");
  *dt = cfl / (CN * h->max_aov * speed);
  return PYR_DG_OK;
}

int pyr_dg_time(const pyr_dg* h, double* t) {
  if (!h || !t) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  *t = h->t;
  return PYR_DG_OK;
}

int pyr_dg_sync(pyr_dg* h) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (h->copy_stream) CUDA_TRY(cudaStreamSynchronize(h->copy_stream));  // staged copies too
  if (h->use_tc || h->use_tctr) {
    const int n = h->L->tc32_timeouts();
    if (n < 0) return fail(PYR_DG_ERR_CUDA, "cannot read the tensor-core wait counter");
    if (n > 0) return fail(PYR_DG_ERR_TIMEOUT, "%d tensor-core completion wait(s) gave up", n);
  }
  return PYR_DG_OK;
}

int pyr_dg_set_tensor_mixing(pyr_dg* h, int enable) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  if (!enable) {
    if (h->use_tc) {
      h->use_tc = false;
      int nsm = 1;
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
      h->stage_epb = h->L->epb32;
      const int64_t groups = (h->K + h->stage_epb - 1) / h->stage_epb;
      h->stage_blocks = (int)std::min<int64_t>(groups, (int64_t)nsm * h->L->blocks_per_sm32(h->stage_epb));
    }
    return PYR_DG_OK;
  }
  if (!h->use_stage32 || h->equation != PYR_DG_WAVE || !h->L->stage32tc)
    return fail(PYR_DG_ERR_BAD_ARG, "tensor-core mixing needs an FP32 wave handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  const int bps = h->L->blocks_per_sm32tc();
  if (bps <= 0)
    return fail(PYR_DG_ERR_CUDA, "occupancy of the tensor-core stage kernel: %s",
                cudaGetErrorString((cudaError_t)(-bps)));
  h->use_tc = true;
  h->stage_epb = 1;
  h->stage_blocks = (int)std::min<int64_t>(h->K, (int64_t)nsm * bps);
  return PYR_DG_OK;
}


int pyr_dg_set_tensor_traces(pyr_dg* h, int enable) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  if (!enable) {
    h->use_tctr = false;
    return PYR_DG_OK;
  }
  if (h->equation != PYR_DG_WAVE || h->basis != PYR_DG_MODAL ||
      !(h->use_stage32 ? h->L->trace32tc != nullptr : h->L->trace64tc != nullptr))
    return fail(PYR_DG_ERR_BAD_ARG,
                "tensor-core traces need a modal wave handle (FP32, or FP64 with N = 2..4)");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  return enable_tensor_traces(h);
}

int pyr_dg_get_tensor_traces(const pyr_dg* h, int* enabled) {
  if (!h || !enabled) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  *enabled = h->use_tctr ? 1 : 0;
  return PYR_DG_OK;
}

int pyr_dg_profile(pyr_dg* h, int enable) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->profiling = enable != 0;
  h->events_used = 0;
  h->event_kind.clear();
  return PYR_DG_OK;
}

int pyr_dg_profile_read(pyr_dg* h, double* trace_ms, int64_t* trace_launches, double* rhs_ms,
                        int64_t* rhs_launches) {
  if (!h) return fail(PYR_DG_ERR_BAD_ARG, "null handle");
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  double ms[2] = {0.0, 0.0};
  int64_t cnt[2] = {0, 0};
  for (size_t p = 0; p < h->event_kind.size(); ++p) {
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, h->events[2 * p], h->events[2 * p + 1]));
    ms[h->event_kind[p]] += t;
    cnt[h->event_kind[p]] += 1;
  }
  if (trace_ms) *trace_ms = ms[0];
  if (trace_launches) *trace_launches = cnt[0];
  if (rhs_ms) *rhs_ms = ms[1];
  if (rhs_launches) *rhs_launches = cnt[1];
  return PYR_DG_OK;
}

void pyr_dg_destroy(pyr_dg* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"

// ------------------------------------------------------------------------
// pyr_dg_rhs_noalloc: the trace scratch of pyr_dg_rhs in a static device array.
namespace {
constexpr int kMaxNoallocDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[PYR_DG_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxNoallocDevices] = {};

// Host code sees only a stand-in for the array: its device address is fetched once per
// device, with that device current (the callers hold a DeviceGuard for it).
cudaError_t noalloc_scratch_address(int device, void** out) {
  *out = nullptr;
  if (device < 0 || device >= kMaxNoallocDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return cudaSuccess;
}
}  // namespace

extern "C" int pyr_dg_rhs_noalloc(pyr_dg* h, const void* q_dev, void* rhs_dev) {
  if (!h || !q_dev || !rhs_dev) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (q_dev == rhs_dev) return fail(PYR_DG_ERR_BAD_ARG, "rhs must not alias q");
  if (h->equation != PYR_DG_WAVE || h->basis != PYR_DG_MODAL)
    return fail(PYR_DG_ERR_BAD_ARG, "pyr_dg_rhs_noalloc supports modal-basis wave handles only");
  const size_t need = (size_t)h->K * h->Nfc * 4 * h->tsize;
  if (need > (size_t)PYR_DG_NOALLOC_SCRATCH_BYTES)
    return fail(PYR_DG_ERR_BAD_ARG,
                "pyr_dg_rhs_noalloc: this mesh needs %zu bytes of face-trace scratch (K=%lld, Nfc=%d, 4 fields, "
                "%zu-byte elements) but the static scratch holds %d bytes; use pyr_dg_rhs",
                need, (long long)h->K, h->Nfc, h->tsize, (int)PYR_DG_NOALLOC_SCRATCH_BYTES);
  if (h->device < 0 || h->device >= kMaxNoallocDevices)
    return fail(PYR_DG_ERR_BAD_ARG, "pyr_dg_rhs_noalloc supports device ordinals below %d", kMaxNoallocDevices);
  DeviceGuard g(h->device);
  CUDA_TRY(g.err);
  void* scratch = nullptr;
  {
    // cached by pyr_dg_setup; looked up here only if that failed
    const cudaError_t e = noalloc_scratch_address(h->device, &scratch);
    if (e != cudaSuccess)
      return fail(PYR_DG_ERR_CUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", h->device,
                  cudaGetErrorString(e));
  }
  h->L->trace(h->K, q_dev, h->tab, scratch, h->stream);
  h->L->rhs_out(h->K, q_dev, rhs_dev, scratch, h->mapP, h->geo, h->gface, h->invM, h->tab, h->bc, h->tau,
                h->stream);
  CUDA_TRY(cudaGetLastError());
  return PYR_DG_OK;
}
