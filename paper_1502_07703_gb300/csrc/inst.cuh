// Instantiation of the stage kernels for one degree; included by inst_n<N>.cu.
#pragma once
#include "dg_kernels.cuh"
#include "launch.h"

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
  static_assert(4 * Dims<N>::n2 <= 4 * Dims<N>::n1 * Dims<N>::P3 * Dims<N>::P3, "projection B/J scratch");

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
    return cudaFuncSetAttribute(error_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ErrSmem<N>::bytes);
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
                         double rkb, double dt, cudaStream_t s) {
    rhs_kernel<N, T, true><<<(unsigned)K, NT, RhsSmem<N, T>::bytes, s>>>(
        K, (const T*)q, (T*)q, (T*)res, (const T*)tr, mapP, (const T*)geo, (const T*)gface, (const T*)invM,
        (const T*)tab, bc, (T)tau, (T)rka, (T)rkb, (T)dt);
  }
  static void rhs_out(int64_t K, const void* q, void* rhs, const void* tr, const int32_t* mapP, const void* geo,
                      const void* gface, const void* invM, const void* tab, int bc, double tau, cudaStream_t s) {
    rhs_kernel<N, T, false><<<(unsigned)K, NT, RhsSmem<N, T>::bytes, s>>>(
        K, (const T*)q, (T*)rhs, nullptr, (const T*)tr, mapP, (const T*)geo, (const T*)gface, (const T*)invM,
        (const T*)tab, bc, (T)tau, (T)0, (T)0, (T)0);
  }
  static void project(int64_t K, const double* ev, const double* gtab, const double* tabd, int bc, double t, void* q,
                      cudaStream_t s) {
    project_kernel<N, T><<<(unsigned)K, NT, ProjSmem<N>::bytes, s>>>(K, ev, gtab, tabd, bc, t, (T*)q);
  }
  static void error(int64_t K, const void* q, const double* ev, const double* gtab, int bc, double t,
                    double* partial, int nblocks, cudaStream_t s) {
    error_kernel<N, T><<<nblocks, ErrCfg<N>::NT, ErrSmem<N>::bytes, s>>>(K, (const T*)q, ev, gtab, bc, t, partial);
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
