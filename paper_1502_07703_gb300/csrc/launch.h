// Type-erased launchers for one (degree, precision) pair.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pyrdg {

struct Launchers {
  int nt;  // threads per CTA of the stage kernels
  size_t smem_trace, smem_rhs, smem_proj, smem_err;
  // Raise the dynamic shared-memory limit of every kernel (once per device).
  cudaError_t (*prepare)();
  void (*geom)(int64_t K, const double* ev, const double* gtab, void* geo, void* gface, void* invM, cudaStream_t s);
  void (*trace)(int64_t K, const void* q, const void* tab, void* tr, cudaStream_t s);
  // Fused stage (rhs, M^{-1}, LSRK update) reading the traces of q from tr.
  void (*rhs_update)(int64_t K, void* q, void* res, const void* tr, const int32_t* mapP, const void* geo,
                     const void* gface, const void* invM, const void* tab, int bc, double tau, double rka, double rkb,
                     double dt, const void* dt_elem, cudaStream_t s);
  void (*rhs_out)(int64_t K, const void* q, void* rhs, const void* tr, const int32_t* mapP, const void* geo,
                  const void* gface, const void* invM, const void* tab, int bc, double tau, cudaStream_t s);
  void (*project)(int64_t K, const double* ev, const double* gtab, const double* tabd, int bc, double t, void* q,
                  cudaStream_t s);
  void (*error)(int64_t K, const void* q, const double* ev, const double* gtab, int bc, double t, double* partial,
                int nblocks, cudaStream_t s);
  // Error norm from coefficients (the wave's exact fields are S(x) times a time factor):
  // exact_proj fills shat (K x 4 x Np: coefficients of the error rule's projection of S) and
  // Mdiag (K x Np: M_ii) and writes per-block sums of |PS_p - S_p|^2, sum_m |PS_m - S_m|^2,
  // |S_p|^2 and sum_m |S_m|^2 (4 per block); error_proj sums M_ii (u_i - T s_i)^2 with
  // T = tp (p) or tu (velocities), tp = cos(sqrt3 pi sc t), tu = sin(sqrt3 pi sc t)/sqrt3.
  void (*exact_proj)(int64_t K, const double* ev, const double* gtab, int bc, double* shat, double* Mdiag,
                     double* partial, int nblocks, cudaStream_t s);
  void (*error_proj)(int64_t K, const void* q, const double* shat, const double* Mdiag, double tp, double tu,
                     double* partial, int nblocks, cudaStream_t s);
  // Single-launch FP32 stage (null for double): reads traces of q from tr_cur, writes
  // the updated state, residual and (if write_traces) the new traces into tr_nxt.
  // epb: elements per CTA, one that blocks_per_sm32 reports as built.
  void (*stage32)(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                  const void* geo, const void* gface, const void* invM, int bc, double tau, double rka, double rkb,
                  double dt, const void* dt_elem, int write_traces, int epb, int nblocks, cudaStream_t s);
  // Fill the FP32 stage kernel's constant tables on the current device from the
  // double reference tables (TabLayout); null for double.
  cudaError_t (*upload_c32)(const double* tab);
  // Resident CTAs per SM of the FP32 stage kernel with epb elements per CTA (for its
  // persistent grid); 0 when that epb is not built for this degree.
  int (*blocks_per_sm32)(int epb);
  int epb32;  // default elements per CTA of the FP32 stage kernel
  // Single-launch FP32 advection stage (null for double): reads the traces of q from
  // tr_cur and writes the updated state, residual and the new traces into tr_nxt.
  void (*adv32)(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                const void* geo, const void* gface, const void* invM, const double* beta, double alpha, double rka,
                double rkb, double dt, int epb, int nblocks, cudaStream_t s);
  int (*blocks_per_sm_adv32)(int epb);
  int epb_adv32;  // default elements per CTA of the FP32 advection stage kernel
  size_t smem_stage32;
  // Scalar advection (one field): trace, fused stage / rhs, projection and error norm.
  void (*trace1)(int64_t K, const void* q, const void* tab, void* tr, cudaStream_t s);
  void (*rhs1)(int64_t K, const void* qin, void* qout, void* res, const void* tr, const int32_t* mapP,
               const void* geo, const void* gface, const void* invM, const void* tab, const double* beta,
               double alpha, double rka, double rkb, double dt, int update, cudaStream_t s);
  void (*project1)(int64_t K, const double* ev, const double* gtab, const double* tabd, const double* beta,
                   double lo, double L, double t, void* q, cudaStream_t s);
  void (*error1)(int64_t K, const void* q, const double* ev, const double* gtab, const double* beta, double lo,
                 double L, double t, double* partial, int nblocks, cudaStream_t s);
  // Nodal variant (Sec. 4.4.1; double only, null for float): the trace points of a nodal
  // state (base Gauss-Legendre points, triangle-face nodes) and the stage / rhs from them.
  // ntab: NodalDims<N> table; tri_node: 4 x nT element nodes of the triangle faces; nmap:
  // K x NTR matching trace point (itself on a boundary).
  void (*nodal_trace)(int64_t K, const void* q, const double* ntab, const int32_t* tri_node, void* tr,
                      cudaStream_t s);
  void (*nodal_rhs)(int64_t K, const void* qin, void* qout, void* res, const void* tr, const int32_t* nmap,
                    const void* geo, const void* gface, const void* invM, const void* tab, const double* ntab,
                    const int32_t* tri_node, int bc, double tau, double rka, double rkb, double dt, int update,
                    cudaStream_t s);
  // FP32 stage kernel with the level mixing on the tensor cores (tcgen05, TF32 3-term split),
  // one element per CTA; null for double. Arguments as stage32's.
  void (*stage32tc)(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                    const void* geo, const void* gface, const void* invM, int bc, double tau, double rka, double rkb,
                    double dt, const void* dt_elem, int write_traces, int nblocks, cudaStream_t s);
  int (*blocks_per_sm32tc)();
  // Read and clear the count of its completion waits that gave up (0 in normal operation).
  int (*tc32_timeouts)();
  // FP32 face traces on the tensor cores (element-batched: T = U Phi_f^T over tiles of 32
  // elements x 4 fields); null for double. op: the trace map's TF32 hi and lo parts, tctr_nkc
  // pieces of tctr_kc mode columns, each hi then lo, NP x tctr_kc in the K-major no-swizzle
  // operand layout (core matrices of 8 rows x 4 columns), op_floats floats in all.
  void (*trace32tc)(int64_t K, const void* q, void* tr, const float* op, int nblocks, cudaStream_t s);
  int (*blocks_per_sm_trace32tc)();
  int tctr_kc, tctr_nkc, tctr_np;
  int tctr_default;  // FP32 wave handles start with these traces (measured faster at this degree)
  size_t tctr_op_floats;
  // FP64 face traces on the tensor cores with FP64 accuracy (null for float and where Nfc > 128
  // or Np > 102). op: the trace map's 8 exact BF16 slices, each 128 x tctr64_kp (face points x
  // padded modes) in the K-major no-swizzle operand layout (core matrices of 8 rows x 8
  // columns), then 128 int32 row exponents; tctr64_op_bytes in all. One CTA per SM.
  void (*trace64tc)(int64_t K, const void* q, void* tr, const void* op, int nblocks, cudaStream_t s);
  int tctr64_kp;
  size_t tctr64_op_bytes;
  int tctr64_default;  // FP64 wave handles start with these traces
  int nodal_ntr;      // trace points per element of the nodal variant
  int nodal_ntab;     // doubles in its table
};

// precision: 0 = double, 1 = float. Returns null for an unsupported degree.
const Launchers* get_launchers(int N, int precision);

}  // namespace pyrdg
