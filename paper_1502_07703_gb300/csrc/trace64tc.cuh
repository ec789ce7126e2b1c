// Face traces of an FP64 state on the tensor cores with FP64 accuracy (the interpolation to the
// face points of Alg. 3), batched over elements. The trace map is a fixed dense Nfc x Np matrix
// Phi_f, so the traces of a tile are T^T = Phi_f U^T. Both operands are cut into eight exact
// balanced BF16 digits against a per-row exponent (exact64.h): Phi_f's rows (face points) once
// on the host, the state's rows (element-field pairs) per tile here. The level sums
// G_s = sum_{i+j=s} a_i b_j^T, s = 0..7, are integers below 2^22, exact in FP32 accumulators, and
// the epilogue recombines them (integer operations and one integer-to-FP64 conversion) into an
// FP64 value of sum_s G_s 2^(-7s) times the two rows' scales (ex64_combine_fast: within 2^-55
// of the scales' product plus half an ulp).
//  - tcgen05.mma kind::f16 (BF16 operands, FP32 accumulation in TMEM), M = 128 face points
//    (Nfc <= 128 for N <= 4), K = the Np modes padded to 16, 32 state rows per tile (8 elements
//    x 4 fields, the state's own row order). The accumulator of a tile is 8 levels x 32 columns;
//    operator slice i times the state slices j = 0..7-i, stacked along N, is one MMA of N =
//    32 (8 - i) into the adjacent level blocks i..7, so a K step takes 8 MMAs. Two accumulators
//    fill the SM's 512 TMEM columns; one CTA per SM.
//  - the operator's 8 slices stay in shared memory for the CTA's lifetime (8 x 128 x KP BF16);
//    the state is sliced into two alternating slots (8 x 32 x KP BF16), both in the K-major
//    no-swizzle operand layout (core matrices of 8 rows x 8 BF16).
//  - warp-specialised persistent CTAs: 4 producer warps (from warp EW) load the next tile while
//    they slice the current one (lane l of producer warp w takes state row 8 w + l % 8 and mode
//    groups l / 8 + 4 t of 8 modes, so that each 8-lane phase of a slice store fills one core
//    matrix); the row's exponent is a maximum over the 4 lanes that hold the row; thread 0 of
//    the group issues the MMAs. Warps 0 .. EW-1 drain the accumulators (warp w reads TMEM lane
//    quarter w % 4, i.e. face points 32 (w % 4) + lane, and the CPW = 128 / EW columns from
//    CPW (w / 4), i.e. CPW / 4 elements of the tile) and store the four fields of a face point
//    as 32 contiguous bytes of the trace layout K x Nfc x 4.
// Every wait is bounded like the other tensor-core kernels'; a wait that gives up is counted in
// g_tc32_timeouts, and the CTA stops (its remaining tiles are left unwritten).
#pragma once

#include "exact64.h"
#include "trace32tc.cuh"

namespace pyrdg {

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both K-major, N x M.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] x B[smem]^T with BF16 operands, issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate));
}

// BF16 element index of (row, k) in a K-major no-swizzle tile with KP columns (LBO = 128 bytes
// between core matrices along K, SBO = 16 KP bytes between groups of 8 rows).
template <int KP>
__host__ __device__ constexpr int bf16_offset(int row, int k) {
  return (row >> 3) * (8 * KP) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

template <int N>
struct T64 {
  using d = Dims<N>;
  // one M block of face points and level sums exact in FP32 (Np <= 102)
  static constexpr bool OK = N >= 2 && d::Nfc <= 128 && d::Np <= 102;
  static constexpr int KP = (d::Np + 15) / 16 * 16;  // modes, padded to the BF16 K step
  static constexpr int NG = KP / 8;                   // 8-mode groups per state row
  static constexpr int GPT = (NG + 3) / 4;            // groups per producer thread
  static constexpr int CW = 32;                       // state rows per tile (8 elements x 4 fields)
  static constexpr int EPT = CW / 4;
  static constexpr int EW = 8, PW = 4;  // epilogue warps (EW / 4 per TMEM lane quarter), producer warps
  static_assert(EW % 4 == 0 && (4 * CW / EW) % 8 == 0, "epilogue warps: whole lane quarters, 8-column chunks");
  static constexpr int NT = 32 * (EW + PW);
  static constexpr uint32_t TCOLS = 512;  // two accumulators of 8 levels x 32 columns
  // shared memory (bytes): operator slices, two state slots, 4 exponent rows, mbarriers
  static constexpr size_t asz = (size_t)128 * KP * 2;     // one operator slice
  static constexpr size_t bsz = (size_t)8 * CW * KP * 2;  // one state slot (8 slices x 32 rows)
  static constexpr size_t a0 = 0, b0 = 8 * asz, e0 = b0 + 2 * bsz, bars = e0 + 4 * CW * 4;
  static constexpr size_t bytes = bars + 6 * 8 + 16;
  static_assert(!OK || bytes <= 227 * 1024, "FP64 tensor-core trace kernel shared memory");
  // more than half an SM's shared memory, so that one CTA (which holds all 512 TMEM columns)
  // is resident per SM
  static constexpr size_t launch_bytes = bytes > 120 * 1024 ? bytes : 120 * 1024;
  // the operator buffer: 8 slices (BF16, operand layout) then 128 row exponents (int32)
  static constexpr size_t op_bytes = 8 * asz + 128 * 4;
};

template <int N>
__global__ void __launch_bounds__(T64<N>::NT, 1)
    trace64tc_kernel(int64_t K, const double* __restrict__ q, double* __restrict__ tr,
                     const unsigned char* __restrict__ op) {
  using T = T64<N>;
  using d = Dims<N>;
  constexpr int Np = d::Np, Nfc = d::Nfc, KP = T::KP, NG = T::NG, GPT = T::GPT, CW = T::CW, EPT = T::EPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = smem_raw;
  uint64_t* mb = reinterpret_cast<uint64_t*>(sm + T::bars);  // slot_free[2], acc_full[2], acc_empty[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mb + 6);
  volatile uint32_t* stop = tslot + 1;
  int* Erow = reinterpret_cast<int*>(sm + T::e0);  // [tile % 4][state row]
  const uint32_t slot_free0 = smem_addr(mb), acc_full0 = smem_addr(mb + 2), acc_empty0 = smem_addr(mb + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc_mbar_init(slot_free0 + 8 * i, 1);
      // the MMAs' commit and the issuing thread's own arrival (which releases the tile's row
      // exponents to the epilogue)
      tc_mbar_init(acc_full0 + 8 * i, 2);
      tc_mbar_init(acc_empty0 + 8 * i, 32 * T::EW);
    }
    *stop = 0u;
  }
  if (warp == 0) tc_alloc(tslot, T::TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t ntiles = (K + EPT - 1) / EPT;
  bool ok = true;

  if (warp >= T::EW) {
    // ---- producers: state slices and the MMAs
    constexpr int NPT = 32 * T::PW;
    const int r = tid - 32 * T::EW;
    const int ro = lane & 7, cq = lane >> 3;
    const int row = 8 * (r >> 5) + ro;  // state row: element row / 4 of the tile, field row % 4
    for (int x = r; x < (int)(8 * T::asz / 16); x += NPT) cp_async16(sm + T::a0 + 16 * x, op + 16 * x);
    cp_async_commit();
    cp_async_wait_all();
    // this thread's values of a tile (zeros past the mesh and in the padding modes)
    auto load = [&](int64_t tile, double (&x)[GPT][8]) {
      const int64_t e0 = tile * EPT;
      const bool rl = e0 + (row >> 2) < K;
      const double* rs = q + (e0 * 4 + row) * Np;
#pragma unroll
      for (int t = 0; t < GPT; ++t) {
        const int g = cq + 4 * t;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int n = 8 * g + u;
          x[t][u] = (rl && g < NG && n < Np) ? rs[n] : 0.0;
        }
      }
    };
    double cur[GPT][8], nxt[GPT][8];
    if (blockIdx.x < ntiles) load(blockIdx.x, cur);
    uint32_t last_free = 0;  // the last commit's slot barrier and parity (teardown after a stop)
    int last_use = -1, i = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
      const int slot = i & 1, use = i >> 1, acc = i & 1;
      const int64_t tn = tile + gridDim.x;
      if (tn < ntiles) load(tn, nxt);  // in flight while this tile is sliced
      // the row's exponent: the largest over its Np values (held by lanes ro, ro + 8, ro + 16, ro + 24)
      int E = 0;
#pragma unroll
      for (int t = 0; t < GPT; ++t)
#pragma unroll
        for (int u = 0; u < 8; ++u) E = max(E, ex64_exp(cur[t][u]));
      E = max(E, __shfl_xor_sync(0xffffffffu, E, 8));
      E = max(E, __shfl_xor_sync(0xffffffffu, E, 16));
      // the slot's previous tile has been multiplied
      if (use >= 1 && !tc_mbar_wait(slot_free0 + 8 * slot, (use - 1) & 1, kTcWaitPolls)) *stop = 1u;
      unsigned char* Bs = sm + T::b0 + slot * T::bsz;
#pragma unroll
      for (int t = 0; t < GPT; ++t) {
        const int g = cq + 4 * t;
        if (g >= NG) continue;
        uint32_t pk[8][4];  // slice j, modes 8 g + 2 p, 8 g + 2 p + 1 as two BF16
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const uint64_t bl = ex64_bits(cur[t][2 * p]), bh = ex64_bits(cur[t][2 * p + 1]);
          const uint64_t Xl = ex64_fixed(bl, E) + EX64_BALANCE, Xh = ex64_fixed(bh, E) + EX64_BALANCE;
          const uint32_t sgn = ((uint32_t)(bl >> 63) << 15) | ((uint32_t)(bh >> 63) << 31);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // digit d as the float 2^23 + d, minus 2^23 (top digit, in [0, 128]) or 2^23 + 64
            // (the others, balanced into [-64, 63]): exact, and its upper half is the BF16
            const uint32_t dl = j == 0 ? (uint32_t)(Xl >> 56) : (uint32_t)(Xl >> (56 - 7 * j)) & 127u;
            const uint32_t dh = j == 0 ? (uint32_t)(Xh >> 56) : (uint32_t)(Xh >> (56 - 7 * j)) & 127u;
            const float off = j == 0 ? 8388608.f : 8388672.f;
            const float fl = __uint_as_float(0x4B000000u | dl) - off;
            const float fh = __uint_as_float(0x4B000000u | dh) - off;
            pk[j][p] = __byte_perm(__float_as_uint(fl), __float_as_uint(fh), 0x7632) ^ sgn;
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<uint4*>(Bs + 2 * bf16_offset<KP>(32 * j + row, 8 * g)) =
              make_uint4(pk[j][0], pk[j][1], pk[j][2], pk[j][3]);
      }
      if (cq == 0) Erow[(i & 3) * CW + row] = E;
#pragma unroll
      for (int t = 0; t < GPT; ++t)
#pragma unroll
        for (int u = 0; u < 8; ++u) cur[t][u] = nxt[t][u];
      tc_fence_smem();
      // the producers' slices of this tile; a stop flag raised anywhere ends every producer
      ok = !producers_sync_or<NPT>(*stop != 0u);
      if (r == 0 && ok) {
        // the accumulator's previous tile has been read out
        if (i >= 2 && !tc_mbar_wait(acc_empty0 + 8 * acc, ((i >> 1) - 1) & 1, kTcWaitPolls)) {
          *stop = 1u;
        } else {
          tc_fence_after();
          const uint32_t a_s = smem_addr(sm + T::a0), b_s = smem_addr(Bs);
          const uint32_t dacc = tmem + 256u * acc;
#pragma unroll
          for (int st = 0; st < KP / 16; ++st) {
            const uint64_t bd = tc_smem_desc(b_s + 256 * st, 128, 16 * KP);
#pragma unroll
            for (int is = 0; is < 8; ++is) {
              // operator slice is times state slices 0 .. 7 - is into levels is .. 7
              const uint64_t ad = tc_smem_desc(a_s + (uint32_t)(is * T::asz) + 256 * st, 128, 16 * KP);
              tc_mma_bf16(dacc + 32 * is, ad, bd, tc_idesc_bf16(128, 32 * (8 - is)), st > 0 || is > 0);
            }
          }
          tc_commit(slot_free0 + 8 * slot);
          tc_commit(acc_full0 + 8 * acc);
          tc_mbar_arrive(acc_full0 + 8 * acc);
          last_free = slot_free0 + 8 * slot;
          last_use = use;
        }
      }
    }
    if (r == 0 && last_use >= 0) tc_mbar_wait(last_free, last_use & 1, kTcWaitPolls);  // no MMA left in flight
  } else {
    // ---- epilogue: face point g = TMEM lane, CPW state columns (CPW / 4 elements) per warp
    constexpr int CPW = 4 * CW / T::EW, NCC = CPW / 8;
    const int quarter = warp & 3, part = warp >> 2;
    const int g = 32 * quarter + lane;
    const int F = reinterpret_cast<const int*>(op + 8 * T::asz)[g];
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int64_t e0 = tile * EPT;
      const int ne = (int)min((int64_t)EPT, K - e0);
      const int acc = i & 1;
      if (!tc_mbar_wait(acc_full0 + 8 * acc, (i >> 1) & 1, kTcWaitPolls)) {
        *stop = 1u;
        ok = false;
        break;
      }
      tc_fence_after();
      int Z[CPW];  // scale exponents of this thread's outputs
#pragma unroll
      for (int c = 0; c < CPW; ++c) Z[c] = Erow[(i & 3) * CW + CPW * part + c] + F - 2107;
      const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16) + 256u * acc + CPW * part;
#pragma unroll
      for (int cc = 0; cc < NCC; ++cc) {
        float v[8][8];  // level s, column 8 cc + k
#pragma unroll
        for (int s = 0; s < 8; ++s) tc_ld8(tl + 32 * s + 8 * cc, v[s]);
        tc_wait_ld();
        if (cc == NCC - 1) {  // the accumulator is free for the tile after next
          tc_fence_before();
          tc_mbar_arrive(acc_empty0 + 8 * acc);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = (CPW * part + 8 * cc) / 4 + h;  // element of the tile
          double o[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            int32_t G[8];
#pragma unroll
            for (int s = 0; s < 8; ++s)  // |G_s| < 2^22: the integer sits in the low mantissa bits
              G[s] = (int32_t)__float_as_uint(v[s][4 * h + f] + 12582912.f) - 0x4B400000;
            o[f] = ex64_combine_fast(G, Z[8 * cc + 4 * h + f]);
          }
          if (e < ne && g < Nfc) {
            double2* dst = reinterpret_cast<double2*>(tr + ((e0 + e) * Nfc + g) * 4);
            dst[0] = make_double2(o[0], o[1]);
            dst[1] = make_double2(o[2], o[3]);
          }
        }
      }
    }
  }
  if (!ok && (tid == 0 || tid == 32 * T::EW)) atomicAdd(&g_tc32_timeouts, 1);
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, T::TCOLS);
}

}  // namespace pyrdg
