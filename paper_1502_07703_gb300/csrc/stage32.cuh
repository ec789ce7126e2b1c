// Single-precision LSRK stage kernel: one launch per RK stage.
//
// Same arithmetic as rhs_kernel (sum-factorised volume term with the c direction
// as level mixing, flux, lift, diagonal M^{-1}, LSRK update), organised for the
// FP32 pipe, which retires 61x more FMAs per cycle than the FP64 pipe and so
// exposes every extra instruction and every exposed load latency:
//  - reference tables live in constant memory and every loop over them is fully
//    unrolled, so table operands are immediate constant-bank operands of FFMA;
//  - each thread owns a column of one pass and keeps its data in registers;
//    the work items of each pass are spread over all four warps;
//  - a CTA works on EPB elements at a time (more at low degree, where one element
//    leaves most threads idle in every pass); item counts are compile-time constants;
//  - CTAs are persistent (grid-stride over element groups); while one group is
//    computed, the next group's contiguous inputs (state, residual, geometry,
//    M^{-1}) arrive in a second shared-memory buffer by cp.async;
//  - the kernel also interpolates the updated state to the face points (the
//    trace step of Alg. 3) into the other half of a ping-pong trace buffer, so
//    a stage is a single launch and the state is read once.
#pragma once

#include "dg_kernels.cuh"
#include "tc32.cuh"

namespace pyrdg {

// Constant-memory table layout of the FP32 stage kernels (wave and advection) for degree N.
template <int N>
struct C32 {
  using d = Dims<N>;
  static constexpr int LX = 0;                      // [tri(k)+i][p'] l_i^k at GL points, -1, +1 (nrow x P3)
  static constexpr int DL = LX + d::nrow * d::P3;   // [tri(k)+i][p]  l_i^k' at GL points (nrow x n1)
  static constexpr int MH = DL + d::nrow * d::n1;   // [k'][k] level mixing of the r, s derivatives
  static constexpr int MG = MH + d::n2;             // [k'][k] level mixing of the c derivative
  static constexpr int GB = MG + d::n2;             // [k] G_k(-1)
  static constexpr int GF = GB + d::n1;             // [k][m] G_k at GJ(1,0) point m
  static constexpr int WB = GF + d::n2;             // [p + n1 q] base-face weights
  static constexpr int WFT = WB + d::n2;            // [e + n1 m] triangle-face weights
  static constexpr int CB = WFT + d::n2;            // [tri(k)+j][c] G_k(-1) l_j^k(b_c): base trace
  static constexpr int size = CB + d::nrow * d::n1;
};

// One copy per translation unit and degree; filled by upload_c32_tables<N>() from the double
// tables, rounded to float.
template <int N>
static __constant__ float c32[C32<N>::size];

// Fill this translation unit's constant table of degree N from the double tables (TabLayout).
// Internal linkage like the table itself: an instantiation shared between units (the default
// for function templates) could upload into another unit's copy.
template <int N>
static cudaError_t upload_c32_tables(const double* tab) {
  using C = C32<N>;
  using d = Dims<N>;
  constexpr TabLayout L(N);
  float h[C::size];
  for (int x = 0; x < d::nrow * d::P3; ++x) h[C::LX + x] = (float)tab[L.LX + x];
  for (int x = 0; x < d::nrow * d::n1; ++x) h[C::DL + x] = (float)tab[L.DL + x];
  for (int x = 0; x < d::n2; ++x) {
    h[C::MH + x] = (float)tab[L.MH + x];
    h[C::MG + x] = (float)tab[L.MG + x];
    h[C::GF + x] = (float)tab[L.GF + x];
    h[C::WB + x] = (float)tab[L.WB + x];
    h[C::WFT + x] = (float)tab[L.WFT + x];
  }
  for (int k = 0; k <= N; ++k) h[C::GB + k] = (float)tab[L.GB + k];
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= k; ++j)
      for (int c = 0; c <= N; ++c)
        h[C::CB + (tri_num(k) + j) * d::n1 + c] = (float)(tab[L.GB + k] * tab[L.LX + (tri_num(k) + j) * d::P3 + c]);
  return cudaMemcpyToSymbol(c32<N>, h, sizeof(float) * C::size);
}

// Ask L2 to fetch the 128-byte lines of [p, p + bytes) (one line per participating thread).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, int tid, int nthr) {
  const char* c = reinterpret_cast<const char*>(p);
  const size_t first = reinterpret_cast<size_t>(c) & ~size_t(127);
  const size_t last = (reinterpret_cast<size_t>(c) + bytes - 1) & ~size_t(127);
  for (size_t a = first + (size_t)tid * 128; a <= last; a += (size_t)nthr * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Asynchronous global -> shared copies (cp.async): 16 bytes (both addresses 16-byte
// aligned) or 4 bytes; a commit closes the group, wait_all waits for this thread's groups.
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g));
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Elements per CTA the FP32 stage kernel is built for at degree N: both halves of the
// level mixing must fit the CTA's 128 threads, and EPB is one of 1, 2, 4, 8.
constexpr bool epb_supported(int N, int EPB) {
  return (EPB == 1 || EPB == 2 || EPB == 4 || EPB == 8) &&
         2 * ((EPB * (N + 1) * (N + 1) + 31) / 32) * 32 <= 128;
}

// Shared-memory layout and work decomposition for degree N with EPB elements per CTA.
template <int N, int EPB, bool TC = false>
struct S32 {
  using d = Dims<N>;
  static constexpr int NT = 128;
  static constexpr int G = (d::n1 + 1) / 2;        // level groups {g, N-g}
  static constexpr int YS = (d::P3 + 3) / 4 * 4;   // padded row stride of Y and Z
  static constexpr int nY = d::P3 * YS;            // Y block per (field, level)
  static constexpr int r32(int x) { return (x + 31) / 32 * 32; }
  // items of one level group, padded to whole warps so that a warp runs one group
  static constexpr int GA = r32(EPB * 4 * d::n1);  // a pass: (element, field, a point)
  // b^T and trace a pass: (element, field, point); at N >= 6 with one element per CTA the
  // unpadded count (two warps per group) runs faster than whole warps per group
  static constexpr int GT = (EPB == 1 && N >= 6) ? 4 * d::P3 : r32(EPB * 4 * d::P3);
  static constexpr int WV = (EPB * d::n2 + 31) / 32;  // warps per mixing half
  static constexpr int MIXT = 2 * WV * 32;
  // shared-memory layout (floats)
  static constexpr size_t al4(size_t x) { return (x + 3) / 4 * 4; }  // 16-byte alignment
  static constexpr size_t lx = 0;                                // LX copy (nrow x P3)
  static constexpr size_t dl = lx + d::nrow * d::P3;             // DL copy (nrow x n1)
  static constexpr size_t dec = dl + d::nrow * d::n1;            // Np mode decodings k | j << 8 | i << 16
  // inputs of one element: state (4 Np; the new state replaces it), residual (4 Np),
  // geometry (9 n2), face geometry (NGF), M^{-1} (Np); each part on a 16-byte boundary.
  // EPB elements form a group; two group buffers (the next group's arrive by cp.async).
  static constexpr size_t bu = 0, bres = al4(4 * d::Np), bgeo = bres + al4(4 * d::Np),
                          bgf = bgeo + al4(d::NGEO * d::n2), binv = bgf + al4(d::NGF), bsz = binv + al4(d::Np);
  static constexpr size_t buf = al4(dec + d::Np);                // 2 x EPB x bsz
  static constexpr size_t Fs = buf + 2 * EPB * bsz;              // EPB x 4 Nfc  [f][g]
  static constexpr size_t ZA = 4 * d::nrow * YS > 8 * d::nrow * d::n1 ? 4 * d::nrow * YS : 8 * d::nrow * d::n1;
  static constexpr size_t A = Fs + EPB * 4 * d::Nfc;             // EPB x ZA: A, dA as [row][p][f], later Z, At
  static constexpr size_t Y = A + EPB * ZA;                      // EPB x 4 n1 nY  [f][k][p'][q']
  static constexpr size_t total0 = Y + EPB * 4 * d::n1 * nY;
  // Tensor-core level mixing (TC, one element per CTA): the mixing inputs of every (a, b)
  // point form one row of an M = 128 TF32 operand tile, row = thread: velocity-half rows
  // hold [Zc | X] in columns [0, 2 n1), pressure-half rows [U0 | Ua0 | Ub0] in [2 n1, 5 n1),
  // other entries zero. B holds the mixing matrices (velocity outputs Y_p in columns
  // [0, n1), then G, alpha, beta of the pressure half in [n1, 4 n1)). The tile aliases the
  // A/dA and Y regions when they are large enough (their contents are dead or rewritten while
  // it is in use), else it follows them; B (hi and lo parts) and the mbarrier come last.
  static constexpr int KT = (5 * d::n1 + 7) / 8 * 8;      // K of the MMA (multiple of 8 for kind::tf32)
  static constexpr int NPT = (4 * d::n1 + 15) / 16 * 16;  // N of the MMA (multiple of 16 at M = 128)
  static constexpr bool TC_ALIAS = 128 * KT <= EPB * ZA + EPB * 4 * d::n1 * nY;
  static constexpr size_t tcA = TC_ALIAS ? A : total0;
  static constexpr size_t tcBh = TC_ALIAS ? total0 : total0 + 128 * KT;
  static constexpr size_t tcBl = tcBh + NPT * KT;
  static constexpr size_t tcbar = tcBl + NPT * KT;        // mbarrier (2 words), TMEM address, timeout flag
  static constexpr size_t total = TC ? tcbar + 4 : total0;
  static_assert(!TC || EPB == 1, "tensor-core mixing: one element per CTA");
  static_assert(!TC || 4 * d::n1 <= 32, "tensor-core mixing: at most 32 accumulator columns");
  static_assert(4 * d::nrow * d::P3 <= ZA, "trace a pass (At) aliases the A/dA region");
  static_assert(MIXT <= NT, "mixing slots");
  // resident CTAs per SM the register budget is tuned for (at N = 6, 5 CTAs with 96
  // registers run faster than 4 with 127; N = 7 is held to 4 by shared memory); the
  // tensor-core variant is held to fewer by its shared memory, so it may use more registers
  static constexpr int MIN_BLOCKS_CC = N <= 5 ? 8 : 5;
  static constexpr int SMEM_BLOCKS = (int)((227 * 1024) / (total * sizeof(float)));
  static constexpr int MIN_BLOCKS = TC && SMEM_BLOCKS < MIN_BLOCKS_CC ? (SMEM_BLOCKS > 0 ? SMEM_BLOCKS : 1)
                                                                      : MIN_BLOCKS_CC;
  // L2 prefetch of the next element's own and neighbour traces and connectivity: used at
  // N >= 6, where each element's flux gathers are longest
  static constexpr bool PREFETCH = N >= 6 && EPB == 1;
  static constexpr size_t bytes = total * sizeof(float);
};

// Inputs of the velocity half's level mixing at the (a_p, b_q) point: per level k,
// X[k] = sum_m (g1_m (u_m)_a + g2_m (u_m)_b) and Zc[k] = sum_m g3_m u_m from the a-pass
// output (A, dA as [row][p][field]) and the b-direction tables; g: the point's 9 factors.
template <int N>
__device__ __forceinline__ void mix_velocity_inputs(const float* s_A, const float* s_dA, const float* s_lx,
                                                    const float* s_dl, const float* g, int p, int qq, float* X,
                                                    float* Zc) {
  using d = Dims<N>;
  constexpr int n1 = d::n1, P3 = d::P3;
#pragma unroll
  for (int k = 0; k <= N; ++k) {
    float lq[n1], dlq[n1];
#pragma unroll
    for (int j = 0; j <= k; ++j) {
      if (k < N) lq[j] = s_lx[(tri_num(k) + j) * P3 + qq];
      dlq[j] = s_dl[(tri_num(k) + j) * n1 + qq];
    }
    // the three velocity fields of A, dA at (row, p) in one float4 each
    float v[3] = {0.f, 0.f, 0.f}, va[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j <= k; ++j) {
      const int o = ((tri_num(k) + j) * n1 + p) * 4;
      const float4 a4 = *reinterpret_cast<const float4*>(s_A + o);
      const float a3[3] = {a4.y, a4.z, a4.w};
#pragma unroll
      for (int m = 0; m < 3; ++m) vb[m] = fmaf(a3[m], dlq[j], vb[m]);
      if (k < N) {
        const float4 d4 = *reinterpret_cast<const float4*>(s_dA + o);
        const float d3[3] = {d4.y, d4.z, d4.w};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          v[m] = fmaf(a3[m], lq[j], v[m]);
          va[m] = fmaf(d3[m], lq[j], va[m]);
        }
      }
    }
    if (k == N) {  // l_j^N(b_q) = delta_jq
      const int o = ((tri_num(k) + qq) * n1 + p) * 4;
      const float4 a4 = *reinterpret_cast<const float4*>(s_A + o);
      const float4 d4 = *reinterpret_cast<const float4*>(s_dA + o);
      v[0] = a4.y, v[1] = a4.z, v[2] = a4.w;
      va[0] = d4.y, va[1] = d4.z, va[2] = d4.w;
    }
    float xs = 0.f, zs = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      xs = fmaf(g[m], va[m], fmaf(g[3 + m], vb[m], xs));
      zs = fmaf(g[6 + m], v[m], zs);
    }
    X[k] = xs;
    Zc[k] = zs;
  }
}

// Inputs of the pressure half's level mixing at (a_p, b_q): per level k the value U0, the
// a-derivative Ua0 and the b-derivative Ub0 of p.
template <int N>
__device__ __forceinline__ void mix_pressure_inputs(const float* s_A, const float* s_dA, const float* s_lx,
                                                    const float* s_dl, int p, int qq, float* U0, float* Ua0,
                                                    float* Ub0) {
  using d = Dims<N>;
  constexpr int n1 = d::n1, P3 = d::P3;
#pragma unroll
  for (int k = 0; k <= N; ++k) {
    float u = 0.f, ua = 0.f, ub = 0.f;
#pragma unroll
    for (int j = 0; j <= k; ++j) {
      const int o = ((tri_num(k) + j) * n1 + p) * 4;
      const float a = s_A[o];
      ub = fmaf(a, s_dl[(tri_num(k) + j) * n1 + qq], ub);
      if (k < N) {
        const float lq = s_lx[(tri_num(k) + j) * P3 + qq];
        u = fmaf(a, lq, u);
        ua = fmaf(s_dA[o], lq, ua);
      }
    }
    if (k == N) {  // l_j^N(b_q) = delta_jq
      const int o = ((tri_num(k) + qq) * n1 + p) * 4;
      u = s_A[o];
      ua = s_dA[o];
    }
    U0[k] = u;
    Ua0[k] = ua;
    Ub0[k] = ub;
  }
}

// Polls of the tensor-core completion wait before the stage kernel gives up and counts a
// timeout (each poll may suspend for a bounded time): far beyond an MMA's microseconds.
constexpr int kTcWaitPolls = 1 << 20;
// Timeouts of the tensor-core mixing's waits since the host last read and cleared them.
static __device__ int g_tc32_timeouts;

// One RK stage of a mesh by CTA blk of nblk persistent CTAs (grid-stride over element groups):
// the body of stage32_kernel, also run per degree group by the batch's single-launch kernel.
template <int N, int EPB, bool TC = false>
__device__ __forceinline__ void stage32_run(int64_t K, float* __restrict__ q, float* __restrict__ res,
                                            const float* __restrict__ tr_cur, float* __restrict__ tr_nxt,
                                            const int32_t* __restrict__ mapP, const float* __restrict__ geo,
                                            const float* __restrict__ gface, const float* __restrict__ invM, int bc,
                                            float tau, float rka, float rkb, float dt,
                                            const float* __restrict__ dt_elem, int write_traces, int64_t blk,
                                            int64_t nblk) {
  using d = Dims<N>;
  using S = S32<N, EPB, TC>;
  using C = C32<N>;
  constexpr int n1 = d::n1, n2 = d::n2, P3 = d::P3, nrow = d::nrow, Np = d::Np, Nfc = d::Nfc;
  constexpr int YS = S::YS, nY = S::nY, ZA = (int)S::ZA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* s_lx = sm + S::lx;
  float* s_dl = sm + S::dl;
  float* s_Fs0 = sm + S::Fs;
  float* s_A0 = sm + S::A;
  float* s_Y0 = sm + S::Y;
  int* s_dec = reinterpret_cast<int*>(sm + S::dec);
  const int tid = threadIdx.x;
  for (int n = tid; n < Np; n += S::NT) {
    int k, j, i;
    decode_mode(n, k, j, i);
    s_dec[n] = k | j << 8 | i << 16;
  }
  for (int x = tid; x < nrow * P3; x += S::NT) s_lx[x] = c32<N>[C::LX + x];
  for (int x = tid; x < nrow * n1; x += S::NT) s_dl[x] = c32<N>[C::DL + x];
  // Y entries that no pass writes (face rows x face columns) stay zero
  for (int x = tid; x < EPB * 4 * n1 * nY; x += S::NT) s_Y0[x] = 0.f;
  // tensor-core mixing: B tiles (TF32 hi and lo parts of the mixing matrices), the mbarrier
  // the MMAs complete on, and 32 TMEM columns for the accumulators
  uint32_t tmem = 0, mbar = 0;
  bool tc_ok = true;
  uint32_t* tc_flag = nullptr;  // set to 1 once a completion wait gave up
  if constexpr (TC) {
    constexpr int KT = S::KT;
    float* Bh = sm + S::tcBh;
    float* Bl = sm + S::tcBl;
    for (int x = tid; x < S::NPT * KT; x += S::NT) {
      const int n = x / KT, k = x - n * KT;
      float v = 0.f;
      const int kp = n % n1, kk = k % n1;  // output level k', input level k
      if (n < n1 && k < n1) v = c32<N>[C::MG + kp * n1 + kk];                          // Y_p <- Zc (c derivative)
      else if (n < n1 && k < 2 * n1) v = c32<N>[C::MH + kp * n1 + kk];                 // Y_p <- X (r, s derivatives)
      else if (n >= n1 && n < 2 * n1 && k >= 2 * n1 && k < 3 * n1) v = c32<N>[C::MG + kp * n1 + kk];  // G <- U
      else if (n >= 2 * n1 && n < 3 * n1 && k >= 3 * n1 && k < 4 * n1) v = c32<N>[C::MH + kp * n1 + kk];  // alpha <- U_a
      else if (n >= 3 * n1 && n < 4 * n1 && k >= 4 * n1 && k < 5 * n1) v = c32<N>[C::MH + kp * n1 + kk];  // beta <- U_b
      float hi, lo;
      tf32_split(v, hi, lo);
      Bh[tc_offset<KT>(n, k)] = hi;
      Bl[tc_offset<KT>(n, k)] = lo;
    }
    uint32_t* bar = reinterpret_cast<uint32_t*>(sm + S::tcbar);
    mbar = smem_addr(bar);
    tc_flag = bar + 3;
    if (tid == 0) {
      tc_mbar_init(mbar, 1);
      *tc_flag = 0u;
    }
    if (tid < 32) tc_alloc(bar + 2, 32);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = bar[2];
  }

  // Element ei of the group starting at e0. Every pass works on all EPB elements, so its
  // item counts are compile-time constants; past the end of the mesh (the last group)
  // an element slot holds a copy of element K-1 and only its stores are skipped.
  auto elem = [&](int64_t e0, int ei) -> int64_t { return e0 + ei < K ? e0 + ei : K - 1; };
  // asynchronous copy of the group starting at e0 into group buffer bb
  auto issue = [&](int64_t e0, float* bb) {
    for (int x = tid; x < EPB * Np; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / Np, xx = x - ei * Np;
      const int64_t ee = elem(e0, ei);
      cp_async16(bb + ei * S::bsz + S::bu + 4 * xx, q + ee * 4 * Np + 4 * xx);
      cp_async16(bb + ei * S::bsz + S::bres + 4 * xx, res + ee * 4 * Np + 4 * xx);
    }
    for (int x = tid; x < EPB * d::NGEO * n2; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (d::NGEO * n2), xx = x - ei * (d::NGEO * n2);
      cp_async4(bb + ei * S::bsz + S::bgeo + xx, geo + elem(e0, ei) * d::NGEO * n2 + xx);
    }
    for (int x = tid; x < EPB * (d::NGF / 4); x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (d::NGF / 4), xx = x - ei * (d::NGF / 4);
      cp_async16(bb + ei * S::bsz + S::bgf + 4 * xx, gface + elem(e0, ei) * d::NGF + 4 * xx);
    }
    for (int x = tid; x < EPB * Np; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / Np, xx = x - ei * Np;
      cp_async4(bb + ei * S::bsz + S::binv + xx, invM + elem(e0, ei) * Np + xx);
    }
    cp_async_commit();
  };
  const int64_t gstride = nblk * EPB;
  if (blk * EPB < K) issue(blk * EPB, sm + S::buf);
  int it = 0;
  for (int64_t e0 = blk * EPB; e0 < K; e0 += gstride, ++it) {
    const int ne = EPB == 1 ? 1 : (int)min((int64_t)EPB, K - e0);  // elements of the group in the mesh
    float* bcur = sm + S::buf + (it & 1) * EPB * S::bsz;
    cp_async_wait_all();  // this thread's copies of the group have landed
    __syncthreads();      // ... everyone's; and the other buffer's last reader is done
    const int64_t en = e0 + gstride;
    if (en < K) issue(en, sm + S::buf + ((it + 1) & 1) * EPB * S::bsz);
    if (S::PREFETCH && en < K) {  // the next element's traces and connectivity: into L2
      prefetch_l2(tr_cur + en * Nfc * 4, sizeof(float) * 4 * Nfc, tid, S::NT);
      prefetch_l2(mapP + en * Nfc, sizeof(int32_t) * Nfc, tid, S::NT);
    }

    // ---- surface flux at every face point (a4), weighted by w sJ
    for (int x = tid; x < EPB * Nfc; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / Nfc, g = x - ei * Nfc;
      const float* s_gf = bcur + ei * S::bsz + S::bgf;
      const int face = g / n2, idx = g - face * n2;
      const int64_t gl = elem(e0, ei) * Nfc + g;
      const int64_t gn = mapP[gl];
      const float4 a4 = reinterpret_cast<const float4*>(tr_cur)[gl];
      const float4 b4 = reinterpret_cast<const float4*>(tr_cur)[gn];
      const float um[4] = {a4.x, a4.y, a4.z, a4.w};
      const float up[4] = {b4.x, b4.y, b4.z, b4.w};
      const float* nv = face == 0 ? s_gf + 16 + 4 * idx : s_gf + 4 * (face - 1);
      const float w = face == 0 ? c32<N>[C::WB + idx] : c32<N>[C::WFT + idx];
      float F[4];
      face_flux<float>(um, up, gn == gl, bc, tau, nv, w * nv[3], F);
      float* s_Fs = s_Fs0 + ei * 4 * Nfc;
#pragma unroll
      for (int f = 0; f < 4; ++f) s_Fs[f * Nfc + g] = F[f];
    }
    // ---- a pass per (level group, element, field, a point p): A = l^k(a_p) u, dA = l^k'(a_p) u.
    // Each group's items fill whole warps; group g takes levels g and N-g.
    for (int x = tid; x < S::G * S::GA; x += S::NT) {
      const int grp = x / S::GA, r = x - grp * S::GA;
      if (r >= EPB * 4 * n1) continue;
      const int ei = EPB == 1 ? 0 : r / (4 * n1), l = r - ei * 4 * n1;
      const int f = l / n1, p = l - f * n1;
      const float* uf = bcur + ei * S::bsz + S::bu + f * Np;
      float* s_A = s_A0 + ei * ZA;
      float* s_dA = s_A + 4 * nrow * n1;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        if (k != grp && k != N - grp) continue;
        float lxc[n1], dlc[n1];
#pragma unroll
        for (int i = 0; i <= k; ++i) {
          if (k < N) lxc[i] = s_lx[(tri_num(k) + i) * P3 + p];
          dlc[i] = s_dl[(tri_num(k) + i) * n1 + p];
        }
#pragma unroll
        for (int j = 0; j <= k; ++j) {
          float a = 0.f, da = 0.f;
#pragma unroll
          for (int i = 0; i <= k; ++i) {
            const float c = uf[lvl_off(k) + j * (k + 1) + i];
            if (k < N) a = fmaf(c, lxc[i], a);
            da = fmaf(c, dlc[i], da);
          }
          // the level-N nodes are the volume-rule points: l_i^N(a_p) = delta_ip
          if (k == N) a = uf[lvl_off(k) + j * (k + 1) + p];
          const int o = ((tri_num(k) + j) * n1 + p) * 4 + f;
          s_A[o] = a;
          s_dA[o] = da;
        }
      }
    }
    if (S::PREFETCH && en < K) {  // neighbour traces of the next element (its mapP is in L2 by now)
      for (int g = tid; g < Nfc; g += S::NT) {
        const float* pn = tr_cur + (int64_t)mapP[en * Nfc + g] * 4;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pn));
      }
    }
    __syncthreads();

    // ---- level mixing (c direction of Alg. 1) per (element, a, b point), base lift;
    // triangle-face c^T. Two warp-aligned halves: the velocity half forms div(u) and
    // feeds the p equation, the pressure half forms grad(p) and feeds the velocity equations.
    if constexpr (TC) {
      // Tensor-core form (one element per CTA): every thread's mixing inputs become row tid of
      // the TF32 operand tile (zeros outside its half and for idle threads), and one chain of
      // M = 128, N = NPT, K = KT MMAs forms all outputs at once:
      // D = A_hi B_hi + A_hi B_lo + A_lo B_hi (the 3-term split, about FP32 accuracy), in two
      // phases through the one tile: hi parts first, then lo parts once the first MMAs are done.
      constexpr int KT = S::KT;
      const int half = tid / (S::WV * 32);
      const int y = tid - half * S::WV * 32;
      const bool act = tid < S::MIXT && y < n2;
      const int pq = act ? y : 0, p = pq % n1, qq = pq / n1;
      const float* g = bcur + S::bgeo + pq * d::NGEO;
      float kv[5 * n1];
#pragma unroll
      for (int c = 0; c < 5 * n1; ++c) kv[c] = 0.f;
      if (act) {
        if (half == 0)
          mix_velocity_inputs<N>(s_A0, s_A0 + 4 * nrow * n1, s_lx, s_dl, g, p, qq, kv + n1, kv);
        else
          mix_pressure_inputs<N>(s_A0, s_A0 + 4 * nrow * n1, s_lx, s_dl, p, qq, kv + 2 * n1, kv + 3 * n1,
                                 kv + 4 * n1);
      }
      if (S::TC_ALIAS) __syncthreads();  // the tile overwrites A/dA, which the inputs came from
      float* tA = sm + S::tcA;
      const uint32_t a0 = smem_addr(tA), bh0 = smem_addr(sm + S::tcBh), bl0 = smem_addr(sm + S::tcBl);
      constexpr uint32_t idesc = tc_idesc_tf32(128, S::NPT);
#pragma unroll
      for (int c4 = 0; c4 < KT / 4; ++c4) {  // phase 1: hi parts; kv keeps the lo parts
        float h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = 4 * c4 + i;
          float lo = 0.f;
          h[i] = 0.f;
          if (c < 5 * n1) {
            tf32_split(kv[c], h[i], lo);
            kv[c] = lo;
          }
        }
        *reinterpret_cast<float4*>(tA + tc_offset<KT>(tid, 4 * c4)) = make_float4(h[0], h[1], h[2], h[3]);
      }
      tc_fence_smem();
      __syncthreads();
      if (tid == 0 && tc_ok) {
        tc_fence_after();
#pragma unroll
        for (int st = 0; st < KT / 8; ++st)
          tc_mma_tf32(tmem, tc_smem_desc(a0 + 256 * st, 128, 32 * KT), tc_smem_desc(bh0 + 256 * st, 128, 32 * KT),
                      idesc, st > 0);
#pragma unroll
        for (int st = 0; st < KT / 8; ++st)
          tc_mma_tf32(tmem, tc_smem_desc(a0 + 256 * st, 128, 32 * KT), tc_smem_desc(bl0 + 256 * st, 128, 32 * KT),
                      idesc, true);
        tc_commit(mbar);
      }
      // the issuing thread waits for completion and the CTA barrier releases the rest; once a
      // wait has given up (results flagged invalid) no further MMA is issued or waited for, so a
      // stuck tensor core costs one bounded wait, not one per element
      if (tid == 0 && tc_ok && !tc_mbar_wait(mbar, 0, kTcWaitPolls)) tc_flag[0] = 1u;
      __syncthreads();
      tc_ok = tc_flag[0] == 0u;
      tc_fence_after();
#pragma unroll
      for (int c4 = 0; c4 < KT / 4; ++c4) {  // phase 2: lo parts
        float l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) l[i] = 4 * c4 + i < 5 * n1 ? kv[4 * c4 + i] : 0.f;
        *reinterpret_cast<float4*>(tA + tc_offset<KT>(tid, 4 * c4)) = make_float4(l[0], l[1], l[2], l[3]);
      }
      tc_fence_smem();
      __syncthreads();
      if (tid == 0 && tc_ok) {
        tc_fence_after();
#pragma unroll
        for (int st = 0; st < KT / 8; ++st)
          tc_mma_tf32(tmem, tc_smem_desc(a0 + 256 * st, 128, 32 * KT), tc_smem_desc(bh0 + 256 * st, 128, 32 * KT),
                      idesc, true);
        tc_commit(mbar);
      }
      if (tid == 0 && tc_ok && !tc_mbar_wait(mbar, 1, kTcWaitPolls)) tc_flag[0] = 1u;
      __syncthreads();
      tc_ok = tc_flag[0] == 0u;
      tc_fence_after();
      // accumulators: warp w reads TMEM lanes 32 w .. 32 w + 31, i.e. its own threads' rows
      float acc[24];
      const int warp = tid >> 5;
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
      if (warp < S::WV) {
        tc_ld8(tl, acc);
      } else if (warp < 2 * S::WV) {
        tc_ld16(tl + n1, acc);
        tc_ld8(tl + n1 + 16, acc + 16);
      }
      tc_wait_ld();
      tc_fence_before();  // these loads precede the next element's MMAs (issued after barriers)
      if (act) {
        if (half == 0) {
          const float Fb = s_Fs0[pq];
#pragma unroll
          for (int kp = 0; kp <= N; ++kp) s_Y0[kp * nY + p * YS + qq] = fmaf(c32<N>[C::GB + kp], Fb, acc[kp]);
        } else {
          float Fb[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) Fb[m] = s_Fs0[(m + 1) * Nfc + pq];
#pragma unroll
          for (int kp = 0; kp <= N; ++kp) {
            const float ga = acc[kp], al = acc[n1 + kp], be = acc[2 * n1 + kp];
            const float gb = c32<N>[C::GB + kp];
            const int yo = kp * nY + p * YS + qq;
#pragma unroll
            for (int m = 0; m < 3; ++m)
              s_Y0[(m + 1) * n1 * nY + yo] = fmaf(gb, Fb[m], fmaf(g[m], al, fmaf(g[3 + m], be, g[6 + m] * ga)));
          }
        }
      }
      if (S::TC_ALIAS) {  // face rows x face columns of Y, which no pass writes: the tile overwrote them
        for (int x = tid; x < 16 * n1; x += S::NT) {
          const int f = x / (4 * n1), k = (x / 4) % n1, ij = x % 4;
          s_Y0[(f * n1 + k) * nY + (n1 + ij / 2) * YS + n1 + ij % 2] = 0.f;
        }
      }
    } else {
      if (tid < S::MIXT) {
        const int half = tid / (S::WV * 32);
        const int y = tid - half * S::WV * 32;
        if (y < EPB * n2) {
          const int ei = EPB == 1 ? 0 : y / n2, pq = y - ei * n2;
          const int p = pq % n1, qq = pq / n1;
          const float* g = bcur + ei * S::bsz + S::bgeo + pq * d::NGEO;
          const float* s_A = s_A0 + ei * ZA;
          const float* s_dA = s_A + 4 * nrow * n1;
          const float* s_Fs = s_Fs0 + ei * 4 * Nfc;
          float* s_Y = s_Y0 + ei * 4 * n1 * nY;
          if (half == 0) {
            float X[n1], Zc[n1];
            mix_velocity_inputs<N>(s_A, s_dA, s_lx, s_dl, g, p, qq, X, Zc);
            const float Fb = s_Fs[pq];
#pragma unroll
            for (int kp = 0; kp <= N; ++kp) {
              float dv = 0.f;
#pragma unroll
              for (int k = 0; k <= N; ++k) {  // MG lower Hessenberg, MH tridiagonal
                if (k > kp + 1) continue;
                dv = fmaf(c32<N>[C::MG + kp * n1 + k], Zc[k], dv);
                if (k >= kp - 1) dv = fmaf(c32<N>[C::MH + kp * n1 + k], X[k], dv);
              }
              s_Y[kp * nY + p * YS + qq] = fmaf(c32<N>[C::GB + kp], Fb, dv);
            }
          } else {
            float U0[n1], Ua0[n1], Ub0[n1];
            mix_pressure_inputs<N>(s_A, s_dA, s_lx, s_dl, p, qq, U0, Ua0, Ub0);
            float Fb[3];
#pragma unroll
            for (int m = 0; m < 3; ++m) Fb[m] = s_Fs[(m + 1) * Nfc + pq];
#pragma unroll
            for (int kp = 0; kp <= N; ++kp) {
              float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
              for (int k = 0; k <= N; ++k) {  // MG lower Hessenberg, MH tridiagonal
                if (k > kp + 1) continue;
                ga = fmaf(c32<N>[C::MG + kp * n1 + k], U0[k], ga);
                if (k < kp - 1) continue;
                al = fmaf(c32<N>[C::MH + kp * n1 + k], Ua0[k], al);
                be = fmaf(c32<N>[C::MH + kp * n1 + k], Ub0[k], be);
              }
              const float gb = c32<N>[C::GB + kp];
              const int yo = kp * nY + p * YS + qq;
#pragma unroll
              for (int m = 0; m < 3; ++m)
                s_Y[(m + 1) * n1 * nY + yo] = fmaf(gb, Fb[m], fmaf(g[m], al, fmaf(g[3 + m], be, g[6 + m] * ga)));
            }
          }
        }
      }
    }
    for (int x = (tid + S::NT - S::MIXT) % S::NT; x < EPB * 16 * n1; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (16 * n1), y = x - ei * 16 * n1;
      const int ee = y % n1;
      const int slot = (y / n1) % 4;
      const int f = y / (4 * n1);
      const int face = slot == 0 ? 1 : slot == 1 ? 3 : slot == 2 ? 4 : 2;
      const float* fs = s_Fs0 + ei * 4 * Nfc + f * Nfc + face * n2 + ee;
      float Fm[n1];
#pragma unroll
      for (int m = 0; m <= N; ++m) Fm[m] = fs[m * n1];
      float* Yf = s_Y0 + ei * 4 * n1 * nY + f * n1 * nY;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m <= N; ++m) acc = fmaf(c32<N>[C::GF + k * n1 + m], Fm[m], acc);
        if (slot < 2)
          Yf[k * nY + ee * YS + n1 + slot] = acc;  // b = -1, +1 columns
        else
          Yf[k * nY + (n1 + slot - 2) * YS + ee] = acc;  // a = -1, +1 rows
      }
    }
    __syncthreads();

    // ---- b^T pass per (field, row p' of Y): Z[f][row(k,j)][p'] = sum_q' l_j^k(x_q') Y[f][k][p'][q']
    for (int x = tid; x < S::G * S::GT; x += S::NT) {
      const int grp = x / S::GT, r = x - grp * S::GT;
      if (r >= EPB * 4 * P3) continue;
      const int ei = EPB == 1 ? 0 : r / (4 * P3), y = r - ei * 4 * P3;
      const int f = y / P3, pp = y - f * P3;
      const float* s_Y = s_Y0 + ei * 4 * n1 * nY;
      float* s_Z = s_A0 + ei * ZA;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        if (k != grp && k != N - grp) continue;
        const float* Yr = s_Y + (f * n1 + k) * nY + pp * YS;
        float yv[P3];
#pragma unroll
        for (int c = 0; c < P3; ++c) yv[c] = Yr[c];
#pragma unroll
        for (int j = 0; j <= k; ++j) {
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < P3; ++c) {
            if (k == N && c < n1) {  // l_j^N(x_c) = delta_jc on the volume points
              if (c == j) acc = yv[c];
              continue;
            }
            acc = fmaf(c32<N>[C::LX + (tri_num(k) + j) * P3 + c], yv[c], acc);
          }
          s_Z[(f * nrow + tri_num(k) + j) * YS + pp] = acc;
        }
      }
    }
    __syncthreads();

    // ---- a^T pass, M^{-1} (a6), LSRK update (a7); the new state goes back to shared memory
    const float dte0 = dt_elem ? 0.f : dt;
    for (int x = tid; x < EPB * 4 * Np; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (4 * Np), xx = x - ei * 4 * Np;
      const int f = xx / Np, n = xx - f * Np;
      const int kji = s_dec[n];
      const int k = kji & 0xff, j = (kji >> 8) & 0xff, i = kji >> 16;
      const float* Zr = s_A0 + ei * ZA + (f * nrow + tri_num(k) + j) * YS;
      const float* lr = s_lx + (tri_num(k) + i) * P3;
      float acc = 0.f;
      if (k == N) {  // l_i^N(x_c) = delta_ic on the volume points; the face columns remain
        acc = fmaf(lr[n1 + 1], Zr[n1 + 1], fmaf(lr[n1], Zr[n1], Zr[i]));
      } else {
#pragma unroll
        for (int c = 0; c < P3; ++c) acc = fmaf(lr[c], Zr[c], acc);
      }
      float* be = bcur + ei * S::bsz;
      const float rhs = -be[S::binv + n] * acc;
      const int64_t ee = elem(e0, ei);
      const int64_t gi = ee * 4 * Np + xx;
      const float dte = dt_elem ? dt_elem[ee] : dte0;  // per-element step when meshes are batched
      const float rnew = fmaf(rka, be[S::bres + xx], dte * rhs);
      const float unew = fmaf(rkb, rnew, be[S::bu + xx]);
      be[S::bu + xx] = unew;
      if (ei < ne) {
        res[gi] = rnew;
        q[gi] = unew;
      }
    }
    if (!write_traces) continue;
    __syncthreads();

    // ---- traces of the updated state (Alg. 3's interpolation to face points) into tr_nxt.
    // First the a direction at every a point and a = -1, +1, by level groups:
    // At[f][row(k,j)][pp] = sum_i u[f][k,j,i] l_i^k(a_pp)   (aliases the dead A/dA/Z region)
    for (int x = tid; x < S::G * S::GT; x += S::NT) {
      const int grp = x / S::GT, r = x - grp * S::GT;
      if (r >= EPB * 4 * P3) continue;
      const int ei = EPB == 1 ? 0 : r / (4 * P3), y = r - ei * 4 * P3;
      const int f = y / P3, pp = y - f * P3;
      const float* uf = bcur + ei * S::bsz + S::bu + f * Np;
      float* s_At = s_A0 + ei * ZA;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        if (k != grp && k != N - grp) continue;
        if (k == N && pp < n1) continue;  // At[f][N,j][pp] = u[f][N,j,pp]: read from u below
        float lxc[n1];
#pragma unroll
        for (int i = 0; i <= k; ++i) lxc[i] = s_lx[(tri_num(k) + i) * P3 + pp];
#pragma unroll
        for (int j = 0; j <= k; ++j) {
          float a = 0.f;
#pragma unroll
          for (int i = 0; i <= k; ++i) a = fmaf(uf[lvl_off(k) + j * (k + 1) + i], lxc[i], a);
          s_At[(f * nrow + tri_num(k) + j) * P3 + pp] = a;
        }
      }
    }
    __syncthreads();
    // then the face points: 16 n1 items per element for the four triangular faces (a level
    // sum, then the c direction), 4 n1 for the base (one a point, all b points)
    for (int x = tid; x < EPB * 20 * n1; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (20 * n1), xx = x - ei * 20 * n1;
      if (ei >= ne) continue;
      const float* s_At = s_A0 + ei * ZA;
      const float* s_u = bcur + ei * S::bsz + S::bu;
      float* dst = tr_nxt + (e0 + ei) * Nfc * 4;
      if (xx < 16 * n1) {
        const int f = xx & 3, y = xx >> 2;
        const int t = y % n1, kind = y / n1;  // kind: 0 b=-1, 1 b=+1, 2 a=-1, 3 a=+1
        // faces b = -1, +1 at (a_t, c_m): weights l_j^k(-1 or +1), A column t;
        // faces a = -1, +1 at (b_t, c_m): weights l_j^k(b_t), A column a = -1 or +1
        const int wcol = kind < 2 ? n1 + (kind & 1) : t;
        const int acol = kind < 2 ? t : n1 + (kind & 1);
        const float* Ar = s_At + f * nrow * P3 + acol;
        const float* wr = s_lx + wcol;
        // level N at a volume column t: At is the state itself
        const float* ArN = kind < 2 ? s_u + f * Np + lvl_off(N) + t : Ar + tri_num(N) * P3;
        const int sN = kind < 2 ? n1 : P3;
        float Sk[n1];
#pragma unroll
        for (int k = 0; k <= N; ++k) {
          float sacc = 0.f;
#pragma unroll
          for (int j = 0; j <= k; ++j) {
            const int rr = tri_num(k) + j;
            sacc = fmaf(wr[rr * P3], k == N ? ArN[j * sN] : Ar[rr * P3], sacc);
          }
          Sk[k] = sacc;
        }
        const int face = kind == 0 ? 1 : kind == 1 ? 3 : kind == 2 ? 4 : 2;
#pragma unroll
        for (int m = 0; m <= N; ++m) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k <= N; ++k) acc = fmaf(c32<N>[C::GF + k * n1 + m], Sk[k], acc);
          dst[4 * (face * n2 + t + n1 * m) + f] = acc;
        }
      } else {  // base (c = -1) at (a_t, b_c) for every c
        const int y = xx - 16 * n1;
        const int f = y & 3, t = y >> 2;
        const float* Ar = s_At + f * nrow * P3 + t;
        float at[nrow];
#pragma unroll
        for (int rr = 0; rr < tri_num(N); ++rr) at[rr] = Ar[rr * P3];
#pragma unroll
        for (int c = 0; c <= N; ++c) {
          float acc = 0.f;
#pragma unroll
          for (int rr = 0; rr < tri_num(N); ++rr) acc = fmaf(c32<N>[C::CB + rr * n1 + c], at[rr], acc);
          // level N: l_j^N(b_c) = delta_jc and At[N][t < n1] is u
          acc = fmaf(c32<N>[C::GB + N], s_u[f * Np + lvl_off(N) + c * n1 + t], acc);
          dst[4 * (t + n1 * c) + f] = acc;
        }
      }
    }
  }
  if constexpr (TC) {
    // a wait that gave up leaves its MMAs possibly in flight: wait for the last phase once more
    // (returns at once when every phase completed or none was issued), then free the TMEM
    if (!tc_ok && tid == 0) {
      atomicAdd(&g_tc32_timeouts, 1);
      tc_mbar_wait(mbar, 1, kTcWaitPolls);
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) tc_dealloc(tmem, 32);
  }
}

template <int N, int EPB, bool TC = false>
__global__ void __launch_bounds__(128, S32<N, EPB, TC>::MIN_BLOCKS)
    stage32_kernel(int64_t K, float* __restrict__ q, float* __restrict__ res, const float* __restrict__ tr_cur,
                   float* __restrict__ tr_nxt, const int32_t* __restrict__ mapP, const float* __restrict__ geo,
                   const float* __restrict__ gface, const float* __restrict__ invM, int bc, float tau, float rka,
                   float rkb, float dt, const float* __restrict__ dt_elem, int write_traces) {
  stage32_run<N, EPB, TC>(K, q, res, tr_cur, tr_nxt, mapP, geo, gface, invM, bc, tau, rka, rkb, dt, dt_elem,
                          write_traces, blockIdx.x, gridDim.x);
}

}  // namespace pyrdg
