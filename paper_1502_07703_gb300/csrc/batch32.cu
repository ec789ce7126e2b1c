// Single-launch FP32 stage for a batch of meshes of several degrees: one persistent kernel
// per RK stage runs every degree group of the batch. CTAs [blk0_g, blk0_g + nblk_g) belong to
// group g and run the FP32 stage body of its degree (stage32_run, the code of the per-degree
// kernel) over that group's elements; the split of the CTAs between the groups is set by the
// batch's autotuner from the groups' measured costs. Each degree runs with its default
// elements per CTA (8 at N = 1, 2 at N = 2, 3, else 1).
#include <cuda_runtime.h>

#include <algorithm>

#include "multi.h"
#include "stage32.cuh"

namespace pyrdg {

namespace {

template <int N>
__host__ __device__ constexpr int multi_epb() {
  return N == 1 ? 8 : N <= 3 ? 2 : 1;
}

template <int N>
__device__ __forceinline__ void run_group(const MultiGroup& G, int par, float rka, float rkb, int64_t blk) {
  stage32_run<N, multi_epb<N>()>(G.K, G.q, G.res, G.tr[par], G.tr[1 - par], G.mapP, G.geo, G.gface, G.invM, G.bc,
                                 G.tau, rka, rkb, 0.f, G.dt_elem, 1, blk, G.nblk);
}

// Register budget of the largest degrees' bodies (5 resident CTAs of 128 threads).
__global__ void __launch_bounds__(128, 5)
    stage32_multi_kernel(const __grid_constant__ MultiArgs a, int par, float rka, float rkb) {
  int g = 0;
  while (g + 1 < a.ngroups && (int)blockIdx.x >= a.g[g + 1].blk0) ++g;
  const MultiGroup& G = a.g[g];
  const int64_t blk = (int64_t)blockIdx.x - G.blk0;
  switch (G.N) {  // uniform per CTA
    case 1: run_group<1>(G, par, rka, rkb, blk); break;
    case 2: run_group<2>(G, par, rka, rkb, blk); break;
    case 3: run_group<3>(G, par, rka, rkb, blk); break;
    case 4: run_group<4>(G, par, rka, rkb, blk); break;
    case 5: run_group<5>(G, par, rka, rkb, blk); break;
    case 6: run_group<6>(G, par, rka, rkb, blk); break;
    default: run_group<7>(G, par, rka, rkb, blk); break;
  }
}

template <int N>
size_t smem_of() {
  return S32<N, multi_epb<N>()>::bytes;
}

}  // namespace

int multi_epb_of(int N) {
  switch (N) {
    case 1: return multi_epb<1>();
    case 2: return multi_epb<2>();
    case 3: return multi_epb<3>();
    default: return 1;
  }
}

size_t multi_smem(int N) {
  switch (N) {
    case 1: return smem_of<1>();
    case 2: return smem_of<2>();
    case 3: return smem_of<3>();
    case 4: return smem_of<4>();
    case 5: return smem_of<5>();
    case 6: return smem_of<6>();
    case 7: return smem_of<7>();
    default: return 0;
  }
}

cudaError_t multi_prepare(int N, const double* tab, size_t smem) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (N) {
    case 1: e = upload_c32_tables<1>(tab); break;
    case 2: e = upload_c32_tables<2>(tab); break;
    case 3: e = upload_c32_tables<3>(tab); break;
    case 4: e = upload_c32_tables<4>(tab); break;
    case 5: e = upload_c32_tables<5>(tab); break;
    case 6: e = upload_c32_tables<6>(tab); break;
    case 7: e = upload_c32_tables<7>(tab); break;
    default: break;
  }
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(stage32_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int multi_blocks_per_sm(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage32_multi_kernel, 128, smem) != cudaSuccess) return 0;
  return n;
}

void multi_launch(const MultiArgs& a, int nblocks, size_t smem, int par, double rka, double rkb, cudaStream_t s) {
  stage32_multi_kernel<<<nblocks, 128, smem, s>>>(a, par, (float)rka, (float)rkb);
}

}  // namespace pyrdg
