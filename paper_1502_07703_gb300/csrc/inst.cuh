// Instantiation of the stage kernels for one degree; included by inst_n<N>.cu.
#pragma once
#include "dg_kernels.cuh"
#include "stage32.cuh"
#include "trace32tc.cuh"
#include "trace64tc.cuh"
#include "adv32.cuh"
#include "adv_kernels.cuh"
#include "launch.h"
#include "nodal.cuh"

namespace pyrdg {

template <int N, typename T>
struct Impl {
  using d = Dims<N>;
  static constexpr int NT = KCfg<N>::NT;
  static constexpr size_t kMaxSmem = 227 * 1024;
  static_assert(TraceSmem<N, T>::bytes <= kMaxSmem, "trace kernel shared memory");
  static_assert(RhsSmem<N, T>::bytes <= kMaxSmem, "rhs kernel shared memory");
  static_assert(ProjSmem<N>::bytes + 15 * 8 <= kMaxSmem, "projection kernel shared memory");
  static_assert(ErrSmem<N>::bytes + 8 * (15 + 2 * 16) <= kMaxSmem, "error kernel shared memory");
  static_assert(ProjQSmem<N>::bytes + 8 * (15 + 4 * 16) <= kMaxSmem, "error-rule projection shared memory");
  static_assert(4 * Dims<N>::n2 <= 4 * Dims<N>::n1 * Dims<N>::P3 * Dims<N>::P3, "projection B/J scratch");
  static_assert(S32<N, 1>::bytes <= kMaxSmem, "FP32 stage kernel shared memory");
  static_assert(Rhs1Smem<N, T>::bytes <= kMaxSmem && Proj1Smem<N>::bytes <= kMaxSmem, "advection shared memory");

  static cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(trace_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TraceSmem<N, T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rhs_kernel<N, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RhsSmem<N, T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rhs_kernel<N, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RhsSmem<N, T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(project_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ProjSmem<N>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trace1_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Trace1Smem<N, T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rhs1_kernel<N, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Rhs1Smem<N, T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rhs1_kernel<N, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Rhs1Smem<N, T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(project1_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Proj1Smem<N>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(exact_proj_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ProjQSmem<N>::bytes);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 8 && T64<N>::OK) {
      e = cudaFuncSetAttribute(trace64tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)T64<N>::launch_bytes);
      if (e != cudaSuccess) return e;
    }
    if constexpr (sizeof(T) == 8) {
      static_assert(NodalSmem<N>::bytes <= kMaxSmem, "nodal stage kernel shared memory");
      e = cudaFuncSetAttribute(nodal_rhs_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)NodalSmem<N>::bytes);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(nodal_rhs_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)NodalSmem<N>::bytes);
      if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(error_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ErrSmem<N>::bytes);
  }
  static AdvParams adv(const double* beta, double alpha, double lo, double L) {
    AdvParams P;
    P.beta[0] = beta[0];
    P.beta[1] = beta[1];
    P.beta[2] = beta[2];
    P.alpha = alpha;
    P.lo = lo;
    P.L = L;
    return P;
  }
  static void trace1(int64_t K, const void* q, const void* tab, void* tr, cudaStream_t s) {
    trace1_kernel<N, T><<<(unsigned)K, NT, Trace1Smem<N, T>::bytes, s>>>(K, (const T*)q, (const T*)tab, (T*)tr);
  }
  static void rhs1(int64_t K, const void* qin, void* qout, void* res, const void* tr, const int32_t* mapP,
                   const void* geo, const void* gface, const void* invM, const void* tab, const double* beta,
                   double alpha, double rka, double rkb, double dt, int update, cudaStream_t s) {
    if (update)
      rhs1_kernel<N, T, true><<<(unsigned)K, NT, Rhs1Smem<N, T>::bytes, s>>>(
          K, (const T*)qin, (T*)qout, (T*)res, (const T*)tr, mapP, (const T*)geo, (const T*)gface, (const T*)invM,
          (const T*)tab, (T)beta[0], (T)beta[1], (T)beta[2], (T)alpha, (T)rka, (T)rkb, (T)dt);
    else
      rhs1_kernel<N, T, false><<<(unsigned)K, NT, Rhs1Smem<N, T>::bytes, s>>>(
          K, (const T*)qin, (T*)qout, nullptr, (const T*)tr, mapP, (const T*)geo, (const T*)gface,
          (const T*)invM, (const T*)tab, (T)beta[0], (T)beta[1], (T)beta[2], (T)alpha, (T)0, (T)0, (T)0);
  }
  static void project1(int64_t K, const double* ev, const double* gtab, const double* tabd, const double* beta,
                       double lo, double L, double t, void* q, cudaStream_t s) {
    project1_kernel<N, T><<<(unsigned)K, NT, Proj1Smem<N>::bytes, s>>>(K, ev, gtab, tabd, adv(beta, 0.0, lo, L), t,
                                                                      (T*)q);
  }
  static void error1(int64_t K, const void* q, const double* ev, const double* gtab, const double* beta, double lo,
                     double L, double t, double* partial, int nblocks, cudaStream_t s) {
    error1_kernel<N, T><<<nblocks, 256, 0, s>>>(K, (const T*)q, ev, gtab, adv(beta, 0.0, lo, L), t, partial);
  }
  static void geom(int64_t K, const double* ev, const double* gtab, void* geo, void* gface, void* invM,
                   cudaStream_t s) {
    geom_kernel<N, T><<<(unsigned)K, 128, 0, s>>>(K, ev, gtab, (T*)geo, (T*)gface, (T*)invM);
  }
  static void trace(int64_t K, const void* q, const void* tab, void* tr, cudaStream_t s) {
    trace_kernel<N, T><<<(unsigned)K, NT, TraceSmem<N, T>::bytes, s>>>(K, (const T*)q, (const T*)tab, (T*)tr);
  }
  static void rhs_update(int64_t K, void* q, void* res, const void* tr, const int32_t* mapP, const void* geo,
                         const void* gface, const void* invM, const void* tab, int bc, double tau, double rka,
                         double rkb, double dt, const void* dt_elem, cudaStream_t s) {
    rhs_kernel<N, T, true><<<(unsigned)K, NT, RhsSmem<N, T>::bytes, s>>>(
        K, (const T*)q, (T*)q, (T*)res, (const T*)tr, mapP, (const T*)geo, (const T*)gface, (const T*)invM,
        (const T*)tab, bc, (T)tau, (T)rka, (T)rkb, (T)dt, (const T*)dt_elem);
  }
  static void rhs_out(int64_t K, const void* q, void* rhs, const void* tr, const int32_t* mapP, const void* geo,
                      const void* gface, const void* invM, const void* tab, int bc, double tau, cudaStream_t s) {
    rhs_kernel<N, T, false><<<(unsigned)K, NT, RhsSmem<N, T>::bytes, s>>>(
        K, (const T*)q, (T*)rhs, nullptr, (const T*)tr, mapP, (const T*)geo, (const T*)gface, (const T*)invM,
        (const T*)tab, bc, (T)tau, (T)0, (T)0, (T)0, nullptr);
  }
  static void project(int64_t K, const double* ev, const double* gtab, const double* tabd, int bc, double t, void* q,
                      cudaStream_t s) {
    project_kernel<N, T><<<(unsigned)K, NT, ProjSmem<N>::bytes, s>>>(K, ev, gtab, tabd, bc, t, (T*)q);
  }
  static void error(int64_t K, const void* q, const double* ev, const double* gtab, int bc, double t,
                    double* partial, int nblocks, cudaStream_t s) {
    error_kernel<N, T><<<nblocks, ErrCfg<N>::NT, ErrSmem<N>::bytes, s>>>(K, (const T*)q, ev, gtab, bc, t, partial);
  }
  static void exact_proj(int64_t K, const double* ev, const double* gtab, int bc, double* shat, double* Mdiag,
                         double* partial, int nblocks, cudaStream_t s) {
    exact_proj_kernel<N><<<nblocks, ErrCfg<N>::NT, ProjQSmem<N>::bytes, s>>>(K, ev, gtab, bc, shat, Mdiag, partial);
  }
  static void error_proj(int64_t K, const void* q, const double* shat, const double* Mdiag, double tp, double tu,
                         double* partial, int nblocks, cudaStream_t s) {
    error_proj_kernel<N, T><<<nblocks, 256, 0, s>>>(K, (const T*)q, shat, Mdiag, tp, tu, partial);
  }
  static void nodal_trace(int64_t K, const void* q, const double* ntab, const int32_t* tri_node, void* tr,
                          cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
      const int64_t total = K * NodalDims<N>::NTR;
      const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
      nodal_trace_kernel<N><<<blocks, 256, 0, s>>>(K, (const double*)q, ntab, tri_node, (double*)tr);
    }
  }
  static void nodal_rhs(int64_t K, const void* qin, void* qout, void* res, const void* tr, const int32_t* nmap,
                        const void* geo, const void* gface, const void* invM, const void* tab, const double* ntab,
                        const int32_t* tri_node, int bc, double tau, double rka, double rkb, double dt, int update,
                        cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
      if (update)
        nodal_rhs_kernel<N, true><<<(unsigned)K, NT, NodalSmem<N>::bytes, s>>>(
            K, (const double*)qin, (double*)qout, (double*)res, (const double*)tr, nmap, (const double*)geo,
            (const double*)gface, (const double*)invM, (const double*)tab, ntab, tri_node, bc, tau, rka, rkb, dt);
      else
        nodal_rhs_kernel<N, false><<<(unsigned)K, NT, NodalSmem<N>::bytes, s>>>(
            K, (const double*)qin, (double*)qout, nullptr, (const double*)tr, nmap, (const double*)geo,
            (const double*)gface, (const double*)invM, (const double*)tab, ntab, tri_node, bc, tau, 0.0, 0.0, 0.0);
    }
  }
  template <int E>
  static void stage32_e(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                        const void* geo, const void* gface, const void* invM, int bc, double tau, double rka,
                        double rkb, double dt, const void* dt_elem, int write_traces, int nblocks, cudaStream_t s) {
    if constexpr (epb_supported(N, E)) {
      static_assert(S32<N, E>::bytes <= kMaxSmem, "FP32 stage kernel shared memory");
      stage32_kernel<N, E><<<nblocks, S32<N, E>::NT, S32<N, E>::bytes, s>>>(
          K, (float*)q, (float*)res, (const float*)tr_cur, (float*)tr_nxt, mapP, (const float*)geo,
          (const float*)gface, (const float*)invM, bc, (float)tau, (float)rka, (float)rkb, (float)dt,
          (const float*)dt_elem, write_traces);
    }
  }
  static constexpr bool kTC = sizeof(T) == 4;  // tensor-core mixing (FP32 handles)
  static void stage32tc(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                        const void* geo, const void* gface, const void* invM, int bc, double tau, double rka,
                        double rkb, double dt, const void* dt_elem, int write_traces, int nblocks, cudaStream_t s) {
    if constexpr (kTC) {
      static_assert(S32<N, 1, true>::bytes <= kMaxSmem, "FP32 tensor-core stage kernel shared memory");
      stage32_kernel<N, 1, true><<<nblocks, S32<N, 1, true>::NT, S32<N, 1, true>::bytes, s>>>(
          K, (float*)q, (float*)res, (const float*)tr_cur, (float*)tr_nxt, mapP, (const float*)geo,
          (const float*)gface, (const float*)invM, bc, (float)tau, (float)rka, (float)rkb, (float)dt,
          (const float*)dt_elem, write_traces);
    }
  }
  // Resident CTAs per SM of the tensor-core variant from its registers and shared memory, or
  // minus a CUDA error. The occupancy calculator reports one CTA per SM for kernels that use
  // tcgen05 (it does not know how much tensor memory they allocate); this kernel allocates 32
  // of the 512 TMEM columns per CTA, so registers and shared memory are the real limits.
  static int blocks_per_sm32tc() {
    if constexpr (kTC) {
      cudaFuncAttributes a;
      cudaError_t e = cudaFuncGetAttributes(&a, stage32_kernel<N, 1, true>);
      int dev = 0, regs = 0, smem = 0, resv = 0;
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
      if (e != cudaSuccess) return -(int)e;
      const int by_regs = regs / (((a.numRegs + 7) / 8 * 8) * 128);
      const int by_smem = smem / ((int)S32<N, 1, true>::bytes + resv);
      const int n = std::min(std::min(by_regs, by_smem), 16);
      return n > 0 ? n : 1;
    }
    return 0;
  }
  // Face traces of an FP32 state on the tensor cores (element-batched tcgen05 product with the
  // trace map's TF32 hi/lo parts in op, laid out as T32<N> describes).
  static void trace32tc(int64_t K, const void* q, void* tr, const float* op, int nblocks, cudaStream_t s) {
    if constexpr (kTC)
      trace32tc_kernel<N><<<nblocks, T32<N>::NT, T32<N>::launch_bytes, s>>>(K, (const float*)q, (float*)tr, op);
  }
  // Resident CTAs per SM of the tensor-core trace kernel: shared memory and tensor memory (the
  // occupancy calculator does not know the latter).
  static int blocks_per_sm_trace32tc() {
    if constexpr (kTC) {
      cudaFuncAttributes a;
      int n = T32<N>::CTAS;
      if (cudaFuncGetAttributes(&a, trace32tc_kernel<N>) == cudaSuccess && a.numRegs > 0)
        n = std::min(n, 65536 / (((a.numRegs + 7) / 8 * 8) * T32<N>::NT));
      return n > 0 ? n : 1;
    }
    return 0;
  }
  // FP64 face traces on the tensor cores with FP64 accuracy (exact BF16 slices, T64<N>); one
  // CTA per SM, over tiles of 8 elements.
  static void trace64tc(int64_t K, const void* q, void* tr, const void* op, int nblocks, cudaStream_t s) {
    if constexpr (sizeof(T) == 8 && T64<N>::OK)
      trace64tc_kernel<N><<<nblocks, T64<N>::NT, T64<N>::launch_bytes, s>>>(
          K, (const double*)q, (double*)tr, (const unsigned char*)op);
  }
  static int tc32_timeouts() {
    int n = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&n, g_tc32_timeouts, sizeof(int)) != cudaSuccess) return -1;
    if (n != 0 && cudaMemcpyToSymbol(g_tc32_timeouts, &zero, sizeof(int)) != cudaSuccess) return -1;
    return n;
  }
  // epb must be one blocks_per_sm32 reports as built (nonzero)
  static void stage32(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                      const void* geo, const void* gface, const void* invM, int bc, double tau, double rka, double rkb,
                      double dt, const void* dt_elem, int write_traces, int epb, int nblocks, cudaStream_t s) {
#define PYRDG_STAGE32_ARGS K, q, res, tr_cur, tr_nxt, mapP, geo, gface, invM, bc, tau, rka, rkb, dt, dt_elem, write_traces, nblocks, s
    switch (epb) {
      case 2: stage32_e<2>(PYRDG_STAGE32_ARGS); break;
      case 4: stage32_e<4>(PYRDG_STAGE32_ARGS); break;
      case 8: stage32_e<8>(PYRDG_STAGE32_ARGS); break;
      default: stage32_e<1>(PYRDG_STAGE32_ARGS); break;
    }
#undef PYRDG_STAGE32_ARGS
  }
  template <int E>
  static void adv32_e(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                      const void* geo, const void* gface, const void* invM, const double* beta, double alpha,
                      double rka, double rkb, double dt, int nblocks, cudaStream_t s) {
    if constexpr (epb1_supported(N, E)) {
      static_assert(A32<N, E>::bytes <= kMaxSmem, "FP32 advection kernel shared memory");
      adv32_kernel<N, E><<<nblocks, A32<N, E>::NT, A32<N, E>::bytes, s>>>(
          K, (float*)q, (float*)res, (const float*)tr_cur, (float*)tr_nxt, mapP, (const float*)geo,
          (const float*)gface, (const float*)invM, (float)beta[0], (float)beta[1], (float)beta[2], (float)alpha,
          (float)rka, (float)rkb, (float)dt);
    }
  }
  // epb must be one blocks_per_sm_adv32 reports as built (nonzero)
  static void adv32(int64_t K, void* q, void* res, const void* tr_cur, void* tr_nxt, const int32_t* mapP,
                    const void* geo, const void* gface, const void* invM, const double* beta, double alpha,
                    double rka, double rkb, double dt, int epb, int nblocks, cudaStream_t s) {
#define PYRDG_ADV32_ARGS K, q, res, tr_cur, tr_nxt, mapP, geo, gface, invM, beta, alpha, rka, rkb, dt, nblocks, s
    switch (epb) {
      case 2: adv32_e<2>(PYRDG_ADV32_ARGS); break;
      case 4: adv32_e<4>(PYRDG_ADV32_ARGS); break;
      case 8: adv32_e<8>(PYRDG_ADV32_ARGS); break;
      default: adv32_e<1>(PYRDG_ADV32_ARGS); break;
    }
#undef PYRDG_ADV32_ARGS
  }
  template <int E>
  static cudaError_t smem_adv32() {
    if constexpr (epb1_supported(N, E))
      return cudaFuncSetAttribute(adv32_kernel<N, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)A32<N, E>::bytes);
    return cudaSuccess;
  }
  template <int E>
  static int bps_adv32() {
    if constexpr (epb1_supported(N, E)) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adv32_kernel<N, E>, A32<N, E>::NT,
                                                        A32<N, E>::bytes) != cudaSuccess)
        return 1;
      return n > 0 ? n : 1;
    }
    return 0;
  }
  // Resident CTAs per SM of the advection stage kernel with epb elements per CTA; 0 if not built.
  static int blocks_per_sm_adv32(int epb) {
    switch (epb) {
      case 1: return bps_adv32<1>();
      case 2: return bps_adv32<2>();
      case 4: return bps_adv32<4>();
      case 8: return bps_adv32<8>();
      default: return 0;
    }
  }
  template <int E>
  static cudaError_t smem32() {
    if constexpr (epb_supported(N, E))
      return cudaFuncSetAttribute(stage32_kernel<N, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)S32<N, E>::bytes);
    return cudaSuccess;
  }
  template <int E>
  static int bps32() {
    if constexpr (epb_supported(N, E)) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage32_kernel<N, E>, S32<N, E>::NT,
                                                        S32<N, E>::bytes) != cudaSuccess)
        return 1;
      return n > 0 ? n : 1;
    }
    return 0;
  }
  static cudaError_t upload_c32(const double* tab) {
    cudaError_t e = upload_c32_tables<N>(tab);
    if (e == cudaSuccess) e = smem32<1>();
    if (e == cudaSuccess) e = smem32<2>();
    if (e == cudaSuccess) e = smem32<4>();
    if (e == cudaSuccess) e = smem32<8>();
    if (e == cudaSuccess) e = smem_adv32<1>();
    if (e == cudaSuccess) e = smem_adv32<2>();
    if (e == cudaSuccess) e = smem_adv32<4>();
    if (e == cudaSuccess) e = smem_adv32<8>();
    if constexpr (kTC) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stage32_kernel<N, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)S32<N, 1, true>::bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trace32tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)T32<N>::launch_bytes);
    }
    return e;
  }
  // Resident CTAs per SM of the stage kernel with epb elements per CTA; 0 if not built.
  static int blocks_per_sm32(int epb) {
    switch (epb) {
      case 1: return bps32<1>();
      case 2: return bps32<2>();
      case 4: return bps32<4>();
      case 8: return bps32<8>();
      default: return 0;
    }
  }
  static Launchers make() {
    Launchers l;
    l.nt = NT;
    l.smem_trace = TraceSmem<N, T>::bytes;
    l.smem_rhs = RhsSmem<N, T>::bytes;
    l.smem_proj = ProjSmem<N>::bytes;
    l.smem_err = ErrSmem<N>::bytes;
    l.prepare = &prepare;
    l.geom = &geom;
    l.trace = &trace;
    l.rhs_update = &rhs_update;
    l.rhs_out = &rhs_out;
    l.project = &project;
    l.error = &error;
    l.exact_proj = &exact_proj;
    l.error_proj = &error_proj;
    l.trace1 = &trace1;
    l.rhs1 = &rhs1;
    l.project1 = &project1;
    l.error1 = &error1;
    l.stage32tc = kTC ? &stage32tc : nullptr;
    l.blocks_per_sm32tc = kTC ? &blocks_per_sm32tc : nullptr;
    l.tc32_timeouts = (kTC || T64<N>::OK) ? &tc32_timeouts : nullptr;
    l.trace32tc = kTC ? &trace32tc : nullptr;
    l.blocks_per_sm_trace32tc = kTC ? &blocks_per_sm_trace32tc : nullptr;
    l.tctr_kc = T32<N>::BK;
    l.tctr_nkc = T32<N>::NBP;
    l.tctr_np = T32<N>::NP;
    l.tctr_op_floats = T32<N>::op_floats;
    // measured (stage without its trace passes + this kernel, against the stage kernel's own
    // traces) on 48,000 to 196,608 pyramids: faster at N = 2 to 7, slower at N = 1
    l.tctr_default = kTC && N >= 2;
    const bool k64 = sizeof(T) == 8 && T64<N>::OK;
    l.trace64tc = k64 ? &trace64tc : nullptr;
    l.tctr64_kp = T64<N>::KP;
    l.tctr64_op_bytes = T64<N>::op_bytes;
    // measured (the trace kernel per stage, against the FP64 trace kernel) on 196,608 pyramids
    l.tctr64_default = k64 && N >= 3;  // a tie at N = 2 (0.50 ms either way)
    l.nodal_ntr = NodalDims<N>::NTR;
    l.nodal_ntab = NodalDims<N>::size;
    l.nodal_trace = sizeof(T) == 8 ? &nodal_trace : nullptr;
    l.nodal_rhs = sizeof(T) == 8 ? &nodal_rhs : nullptr;
    if (sizeof(T) == 4) {
      l.stage32 = &stage32;
      l.upload_c32 = &upload_c32;
      l.blocks_per_sm32 = &blocks_per_sm32;
      // measured best on 196,608 pyramids: groups of 8 at N = 1, 2 at N = 2, 3, else 1
      l.epb32 = N == 1 ? 8 : N <= 3 ? 2 : 1;
      l.adv32 = &adv32;
      l.blocks_per_sm_adv32 = &blocks_per_sm_adv32;
      // one field leaves more of the CTA idle per element than the wave system
      l.epb_adv32 = N <= 2 ? 8 : N <= 4 ? 4 : 2;
      l.smem_stage32 = S32<N, 1>::bytes;
    } else {
      l.stage32 = nullptr;
      l.upload_c32 = nullptr;
      l.blocks_per_sm32 = nullptr;
      l.epb32 = 1;
      l.adv32 = nullptr;
      l.blocks_per_sm_adv32 = nullptr;
      l.epb_adv32 = 1;
      l.smem_stage32 = 0;
    }
    return l;
  }
};

}  // namespace pyrdg

#define PYRDG_INSTANTIATE(NN)                                          \
  namespace pyrdg {                                                    \
  const Launchers* launchers_n##NN(int precision) {                    \
    static const Launchers l64 = Impl<NN, double>::make();             \
    static const Launchers l32 = Impl<NN, float>::make();              \
    return precision == 0 ? &l64 : &l32;                               \
  }                                                                    \
  }
