// Face traces of an FP32 state on the tensor cores, batched over elements (the interpolation
// to the face points of Alg. 3). The trace map is a fixed dense Nfc x Np matrix Phi_f (mode n
// at face point g), the same for every element and field, so the traces of a tile of 32
// elements are one product T = U Phi_f^T with M = 128 rows: row 4 e + f of U holds field f of
// element e, which is the state's own row-major layout (K x 4 x Np). K runs over the Np modes
// (zero-padded), N over the Nfc face points (padded to whole MMA columns).
//  - tcgen05.mma kind::tf32 with the 3-term split A_hi B_hi + A_hi B_lo + A_lo B_hi (about FP32
//    accuracy) and FP32 accumulation in TMEM: 128 lanes (the tile's rows) x the padded N columns;
//  - Phi_f's hi and lo parts are built on the host from the FP64 trace map and stored in the
//    operand layout (K-major, no swizzle), cut along K into NKC pieces that fit shared memory;
//    with one piece it stays resident for the CTA's lifetime, else each piece is brought in per
//    tile (from L2);
//  - persistent CTAs of 128 threads; a tile's state arrives by cp.async (the next tile's while
//    the current one is multiplied, where two buffers fit), then each thread converts its own row
//    into the TF32 hi and lo operand tiles;
//  - thread t reads TMEM lane t (its row: element t / 4, field t % 4) and stores that field of its
//    element's face points into the trace layout (K x Nfc x 4), four threads filling each 16-byte
//    point.
// The completion waits are bounded like the tensor-core stage kernel's; a wait that gives up is
// counted in g_tc32_timeouts and leaves the rest of the CTA's tiles unwritten.
#pragma once

#include "stage32.cuh"

namespace pyrdg {

template <int N>
struct T32 {
  using d = Dims<N>;
  static constexpr int NT = 128;
  static constexpr int EPT = 32;                        // elements per tile (x 4 fields = M)
  static constexpr int KP = (d::Np + 7) / 8 * 8;        // modes, padded to the TF32 K step
  static constexpr int NP = (d::Nfc + 15) / 16 * 16;    // face points, padded (MMA N step)
  static constexpr int KC = N <= 4 ? KP : N <= 6 ? 48 : 32;  // K columns per operand piece
  static constexpr int NKC = (KP + KC - 1) / KC;        // pieces
  static constexpr int NCH = (NP + 255) / 256;          // MMA column chunks (N <= 256 each)
  static constexpr int CN = (NP / NCH + 15) / 16 * 16;  // columns per chunk
  static_assert(CN * NCH == NP, "column chunks must tile the padded face points");
  static constexpr int TCOLS = NP <= 32 ? 32 : NP <= 64 ? 64 : NP <= 128 ? 128 : NP <= 256 ? 256 : 512;
  static constexpr int RB = N <= 5 ? 2 : 1;             // state buffers (2: next tile prefetched)
  // shared-memory layout (floats)
  static constexpr size_t rawsz = (size_t)EPT * 4 * d::Np;
  static constexpr size_t raw = 0;
  static constexpr size_t ahi = (raw + RB * rawsz + 31) / 32 * 32;
  static constexpr size_t alo = ahi + 128 * KC;
  static constexpr size_t bhi = alo + 128 * KC;
  static constexpr size_t blo = bhi + (size_t)NP * KC;
  static constexpr size_t bar = blo + (size_t)NP * KC;  // mbarrier (2 words), TMEM address, flag
  static constexpr size_t bytes = (bar + 4) * sizeof(float);
  static_assert(bytes <= 227 * 1024, "tensor-core trace kernel shared memory");
  // resident CTAs per SM (shared memory, at most 16 of 128 threads); their TMEM must fit the
  // SM's 512 columns, or an allocation would wait for another CTA to finish
  static constexpr int CTAS = (int)((228 * 1024) / (bytes + 1024)) < 16 ? (int)((228 * 1024) / (bytes + 1024)) : 16;
  static_assert(CTAS >= 1 && TCOLS * CTAS <= 512, "tensor memory per SM");
  // the operator buffer: per piece, hi then lo, each NP x KC in the operand layout
  static constexpr size_t op_floats = (size_t)NKC * 2 * NP * KC;
};

template <int N>
__global__ void __launch_bounds__(128, 1)
    trace32tc_kernel(int64_t K, const float* __restrict__ q, float* __restrict__ tr, const float* __restrict__ op) {
  using T = T32<N>;
  using d = Dims<N>;
  constexpr int Np = d::Np, Nfc = d::Nfc, KC = T::KC, NKC = T::NKC, NP = T::NP, EPT = T::EPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* Ahi = sm + T::ahi;
  float* Alo = sm + T::alo;
  float* Bhi = sm + T::bhi;
  uint32_t* bar = reinterpret_cast<uint32_t*>(sm + T::bar);
  const uint32_t mbar = smem_addr(bar);
  uint32_t* flag = bar + 3;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc_mbar_init(mbar, 1);
    *flag = 0u;
  }
  if (tid < 32) tc_alloc(bar + 2, T::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bar[2];
  const int64_t ntiles = (K + EPT - 1) / EPT;

  // operator piece kc into Bhi/Blo (contiguous hi then lo, 16-byte copies)
  auto load_op = [&](int kc) {
    const float* src = op + (size_t)kc * 2 * NP * KC;
    for (int x = tid; x < 2 * NP * KC / 4; x += T::NT) cp_async16(Bhi + 4 * x, src + 4 * x);
  };
  // state of the tile starting at element e0 (its elements in the mesh) into buffer b
  auto load_tile = [&](int64_t e0, int b) {
    const int ne = (int)min((int64_t)EPT, K - e0);
    float* dst = sm + T::raw + b * T::rawsz;
    const float* src = q + e0 * 4 * Np;
    for (int x = tid; x < ne * Np; x += T::NT) cp_async16(dst + 4 * x, src + 4 * x);  // 4 Np floats per element
  };
  if constexpr (NKC == 1) load_op(0);
  if (blockIdx.x < ntiles) load_tile((int64_t)blockIdx.x * EPT, 0);
  cp_async_commit();

  bool ok = true;
  uint32_t phase = 0;  // completions waited for so far
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
    const int64_t e0 = tile * EPT;
    const int ne = (int)min((int64_t)EPT, K - e0);
    const float* rawc = sm + T::raw + (T::RB == 2 ? (it & 1) : 0) * T::rawsz;
    const int64_t tnext = tile + gridDim.x;
    for (int kc = 0; kc < NKC && ok; ++kc) {
      if constexpr (NKC > 1) {
        load_op(kc);
        cp_async_commit();
      }
      cp_async_wait_all();  // this thread's copies of the tile (and the piece) have landed
      __syncthreads();      // ... everyone's; the previous MMAs and TMEM reads are complete
      if (kc == 0 && T::RB == 2 && tnext < ntiles) {  // the next tile into the other buffer
        load_tile(tnext * EPT, (it + 1) & 1);
        cp_async_commit();
      }
      // row tid of the operand tiles: field tid % 4 of element tid / 4, modes [kc KC, kc KC + KC)
      {
        const int r = tid;
        const bool live = (r >> 2) < ne;
        const float* src = rawc + r * Np;
#pragma unroll 4
        for (int c4 = 0; c4 < KC / 4; ++c4) {
          float h[4], l[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int n = kc * KC + 4 * c4 + i;
            const float x = (live && n < Np) ? src[n] : 0.f;
            tf32_split(x, h[i], l[i]);
          }
          const int o = tc_offset<KC>(r, 4 * c4);
          *reinterpret_cast<float4*>(Ahi + o) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(Alo + o) = make_float4(l[0], l[1], l[2], l[3]);
        }
      }
      tc_fence_smem();
      __syncthreads();
      if (T::RB == 1 && kc == NKC - 1 && tnext < ntiles) {  // the state buffer is free: next tile
        load_tile(tnext * EPT, 0);
        cp_async_commit();
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_hi = smem_addr(Ahi), a_lo = smem_addr(Alo), b_hi = smem_addr(Bhi),
                       b_lo = b_hi + NP * KC * 4;
        constexpr uint32_t idesc = tc_idesc_tf32(128, T::CN);
#pragma unroll
        for (int ch = 0; ch < T::NCH; ++ch) {
          const uint32_t boff = (uint32_t)ch * T::CN * KC * 4;  // CN rows of B
#pragma unroll
          for (int st = 0; st < KC / 8; ++st) {
            const uint64_t ah = tc_smem_desc(a_hi + 256 * st, 128, 32 * KC);
            const uint64_t al = tc_smem_desc(a_lo + 256 * st, 128, 32 * KC);
            const uint64_t bh = tc_smem_desc(b_hi + boff + 256 * st, 128, 32 * KC);
            const uint64_t bl = tc_smem_desc(b_lo + boff + 256 * st, 128, 32 * KC);
            const uint32_t dcol = tmem + ch * T::CN;
            tc_mma_tf32(dcol, ah, bh, idesc, kc > 0 || st > 0);
            tc_mma_tf32(dcol, ah, bl, idesc, true);
            tc_mma_tf32(dcol, al, bh, idesc, true);
          }
        }
        tc_commit(mbar);
        if (!tc_mbar_wait(mbar, phase & 1, kTcWaitPolls)) *flag = 1u;
      }
      ++phase;
      __syncthreads();
      ok = *flag == 0u;
      tc_fence_after();
    }
    if (!ok) break;
    // thread tid: TMEM lane tid = field f of element el; its face points to the trace layout
    const int el = tid >> 2, f = tid & 3;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    float* dst = tr + ((e0 + el) * Nfc) * 4 + f;
#pragma unroll 1
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float v[16];
      tc_ld16(tl + c0, v);
      tc_wait_ld();
      if (el < ne) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < Nfc) dst[(c0 + i) * 4] = v[i];
      }
    }
    tc_fence_before();  // these reads precede the next tile's MMAs (issued after a barrier)
  }
  // a wait that gave up may leave MMAs in flight: wait for the last commit once more, then free
  if (!ok && tid == 0) {
    atomicAdd(&g_tc32_timeouts, 1);
    tc_mbar_wait(mbar, (phase - 1) & 1, kTcWaitPolls);
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (tid < 32) tc_dealloc(tmem, T::TCOLS);
}

}  // namespace pyrdg
