// Host interface of the batch's single-launch FP32 stage kernel (batch32.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pyrdg {

constexpr int kMaxMultiGroups = 8;

// One degree group of a batch as the single-launch kernel sees it: its union mesh's arrays,
// the two halves of its face-trace ping-pong pair, and its CTAs [blk0, blk0 + nblk).
struct MultiGroup {
  int N;
  int bc;
  float tau;
  int blk0, nblk;
  int64_t K;
  float* q;
  float* res;
  float* tr[2];
  const int32_t* mapP;
  const float* geo;
  const float* gface;
  const float* invM;
  const float* dt_elem;
};

struct MultiArgs {
  int ngroups;
  MultiGroup g[kMaxMultiGroups];
};

// Elements per CTA the kernel runs degree N with.
int multi_epb_of(int N);
// Dynamic shared memory of degree N's body; the launch takes the largest of its groups'.
size_t multi_smem(int N);
// Upload degree N's constant tables into this kernel's unit and allow `smem` bytes of dynamic
// shared memory (on the current device).
cudaError_t multi_prepare(int N, const double* tab, size_t smem);
// Resident CTAs per SM at that dynamic shared memory (0 on error).
int multi_blocks_per_sm(size_t smem);
// One RK stage of every group: CTAs [g.blk0, g.blk0 + g.nblk) run group g; the groups read
// their traces from tr[par] and write the new state's traces into tr[1 - par].
void multi_launch(const MultiArgs& a, int nblocks, size_t smem, int par, double rka, double rkb, cudaStream_t s);

}  // namespace pyrdg
