// pyr_dg_fma_peak: measured FMA throughput of the current GPU, the ALU
// ceiling against which the double-precision stage kernels are measured.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/pyrdg.h"

namespace {

template <typename T, int CH>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == (T)12345.678) out[threadIdx.x] = s;  // never true; keeps the chains live
}

template <typename T>
int measure(double* tflops) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  if (cudaMalloc(&out, 256 * sizeof(T)) != cudaSuccess) return -1;
  constexpr int CH = 8, THREADS = 256;
  const int iters = sizeof(T) == 8 ? 2000 : 40000;
  const dim3 grid(nsm * 4);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T, CH><<<grid, THREADS>>>(out, 16, (T)0.999, (T)0.001);
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    fma_chains<T, CH><<<grid, THREADS>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return -1;
  *tflops = 2.0 * CH * (double)iters * grid.x * THREADS / (best * 1e-3) / 1e12;
  return 0;
}

}  // namespace

extern "C" int pyr_dg_fma_peak(int precision, double* tflops) {
  if (!tflops || (precision != PYR_DG_F64 && precision != PYR_DG_F32)) return PYR_DG_ERR_BAD_ARG;
  const int rc = precision == PYR_DG_F64 ? measure<double>(tflops) : measure<float>(tflops);
  return rc == 0 ? PYR_DG_OK : PYR_DG_ERR_CUDA;
}
