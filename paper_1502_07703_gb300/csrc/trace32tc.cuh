// Face traces of an FP32 state on the tensor cores, batched over elements (the interpolation
// to the face points of Alg. 3). The trace map is a fixed dense Nfc x Np matrix Phi_f (mode n
// at face point g), the same for every element and field, so the traces of a tile of 32
// elements are one product T = U Phi_f^T with M = 128 rows: row 4 e + f of U holds field f of
// element e, which is the state's own row-major layout (K x 4 x Np). K runs over the Np modes
// (zero-padded), N over the Nfc face points (padded to whole MMA columns).
//  - tcgen05.mma kind::tf32 with the 3-term split A_hi B_hi + A_hi B_lo + A_lo B_hi (about FP32
//    accuracy) and FP32 accumulation in TMEM: 128 lanes (the tile's rows) x the padded N columns;
//  - Phi_f's hi and lo parts are built on the host from the FP64 trace map and stored in the
//    operand layout (K-major, no swizzle). At N <= 5 the whole map stays in shared memory for
//    the CTA's lifetime; above that it is cut along K into pieces of 32 modes brought in per tile
//    (from L2) into two alternating slots. The state side is cut the same way at N >= 5;
//  - warp-specialised persistent CTAs: PW producer warps from warp 4 on convert the state into
//    TF32 hi and lo operand pieces (the operator piece arrives by cp.async, and thread 0 of the
//    group issues the MMAs), warps 0-3 drain the accumulators
//    (thread t reads TMEM lane t, its row, and stores that field of its element's face points
//    into the trace layout K x Nfc x 4). Two operand slots and, where TMEM holds them, two
//    accumulators let the conversion of the next piece and the stores of the previous tile
//    overlap the MMAs; mbarriers hand slots and accumulators between the roles.
// Every wait is bounded like the tensor-core stage kernel's; a wait that gives up is counted in
// g_tc32_timeouts, and the CTA stops (its remaining tiles are left unwritten).
#pragma once

#include "stage32.cuh"

namespace pyrdg {

__device__ __forceinline__ void tc_mbar_arrive(uint32_t mbar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

// Barrier of the producer threads (named barrier 1, nthr of them) that also ORs a flag across
// them, so that every producer takes the same branch after it.
template <int nthr>
__device__ __forceinline__ bool producers_sync_or(bool v) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "n"(nthr)
      : "memory");
  return out != 0;
}

// 4 x 4 transpose within each quad of lanes: lane u of the quad holds a[j] = M[j][u] on entry
// and M[u][j] on exit (two butterfly exchanges of two values each).
__device__ __forceinline__ void quad_transpose(float (&a)[4], int u) {
#pragma unroll
  for (int sb = 1; sb <= 2; sb <<= 1) {
    const bool hi = (u & sb) != 0;
    // the two entries whose index bit sb differs from this lane's go to the partner lane u ^ sb
    const float s0 = hi ? a[0] : a[sb];
    const float s1 = hi ? a[sb == 1 ? 2 : 1] : a[3];
    const float r0 = __shfl_xor_sync(0xffffffffu, s0, sb);
    const float r1 = __shfl_xor_sync(0xffffffffu, s1, sb);
    if (sb == 1) {
      if (hi) {
        a[0] = r0;
        a[2] = r1;
      } else {
        a[1] = r0;
        a[3] = r1;
      }
    } else {
      if (hi) {
        a[0] = r0;
        a[1] = r1;
      } else {
        a[2] = r0;
        a[3] = r1;
      }
    }
  }
}

template <int N>
struct T32 {
  using d = Dims<N>;
  // producer warps (4 .. 4 + PW - 1): more warps cover more of the state loads' latency; 16
  // measured faster from N = 5 up, 8 below (the MMAs per piece are few there)
  static constexpr int PW = N >= 5 ? 16 : 8;
  static constexpr int NT = 128 + 32 * PW;              // warps 0-3 drain the accumulators
  static constexpr int EPT = 32;                        // elements per tile (x 4 fields = M)
  static constexpr int KP = (d::Np + 7) / 8 * 8;        // modes, padded to the TF32 K step
  static constexpr int NP = (d::Nfc + 15) / 16 * 16;    // face points, padded (MMA N step)
  static constexpr bool BRES = N <= 5;                  // operator resident for the CTA's lifetime
  static constexpr int KC = N <= 4 ? KP : 32;           // mode columns per A piece
  static constexpr int NKC = (KP + KC - 1) / KC;        // A pieces per tile
  static constexpr int BK = BRES ? NKC * KC : KC;       // mode columns of the operator in shared memory
  static constexpr int NBP = BRES ? 1 : NKC;            // operator pieces (of BK columns)
  static constexpr int NCH = (NP + 255) / 256;          // MMA column chunks (N <= 256 each)
  static constexpr int CN = (NP / NCH + 15) / 16 * 16;  // columns per chunk
  static_assert(CN * NCH == NP, "column chunks must tile the padded face points");
  static constexpr int NACC = 2 * NP <= 512 ? 2 : 1;    // accumulators in TMEM
  static constexpr int TCOLS = NACC * NP <= 32 ? 32 : NACC * NP <= 64 ? 64 : NACC * NP <= 128 ? 128
                             : NACC * NP <= 256 ? 256 : 512;
  // shared-memory layout (floats): two A slots (hi, lo), the operator slots (hi, lo), mbarriers
  static constexpr size_t asz = (size_t)128 * KC, bsz = (size_t)NP * BK;
  static constexpr int NBS = BRES ? 1 : 2;
  static constexpr size_t a0 = 0;
  static constexpr size_t b0 = a0 + 2 * 2 * asz;
  static constexpr size_t bars = b0 + NBS * 2 * bsz;    // 6 mbarriers, TMEM address, stop flag
  static constexpr size_t bytes = (bars + 16) * sizeof(float);
  static_assert(bytes <= 227 * 1024, "tensor-core trace kernel shared memory");
  // resident CTAs per SM: at most 2048 / NT, and as many as their TMEM columns fit in
  // the SM's 512 (an allocation beyond that would wait for another CTA to exit); the launch
  // asks for enough shared memory that no more than that many fit
  static constexpr int CTAS_TMEM = 512 / TCOLS < 2048 / NT ? 512 / TCOLS : 2048 / NT;
  static constexpr size_t pad_bytes = (228 * 1024) / (CTAS_TMEM + 1) - 1024 + 1024;
  static constexpr size_t launch_bytes = bytes > pad_bytes ? bytes : pad_bytes;
  static constexpr int CTAS_SMEM = (int)((228 * 1024) / (launch_bytes + 1024));
  static constexpr int CTAS = CTAS_SMEM < CTAS_TMEM ? CTAS_SMEM : CTAS_TMEM;
  static_assert(CTAS >= 1 && CTAS * TCOLS <= 512, "tensor memory per SM");
  static_assert(launch_bytes <= 227 * 1024, "padded shared memory");
  // the operator buffer: per piece, hi then lo, each NP x BK in the operand layout
  static constexpr size_t op_floats = (size_t)NBP * 2 * NP * BK;
};

template <int N>
__global__ void __launch_bounds__(T32<N>::NT, 1)
    trace32tc_kernel(int64_t K, const float* __restrict__ q, float* __restrict__ tr, const float* __restrict__ op) {
  using T = T32<N>;
  using d = Dims<N>;
  constexpr int Np = d::Np, Nfc = d::Nfc, KC = T::KC, NKC = T::NKC, NP = T::NP, EPT = T::EPT, NACC = T::NACC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  uint64_t* mb = reinterpret_cast<uint64_t*>(sm + T::bars);  // slot_free[2], acc_full[2], acc_empty[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mb + 6);
  volatile uint32_t* stop = tslot + 1;
  const uint32_t slot_free0 = smem_addr(mb), acc_full0 = smem_addr(mb + 2), acc_empty0 = smem_addr(mb + 4);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc_mbar_init(slot_free0 + 8 * i, 1);
      tc_mbar_init(acc_full0 + 8 * i, 1);
      tc_mbar_init(acc_empty0 + 8 * i, 128);
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

  if (warp >= 4) {
    // ---- producers: operand pieces and the MMAs
    constexpr int NPT = 32 * T::PW;  // producer threads
    const int r = tid - 128;         // producer index
    float* Bs = sm + T::b0;
    if constexpr (T::BRES) {  // the operator, once
      for (int x = r; x < (int)(2 * T::bsz / 4); x += NPT) cp_async16(Bs + 4 * x, op + 4 * x);
      cp_async_commit();
      cp_async_wait_all();
    }
    // operand rows: lane l of producer warp w takes rows RW w + 8 o + (l % 8) (RW = 128 / PW rows
    // per warp) and column groups 4 cb + l / 8 (4 modes each), so that each 8-lane store fills
    // one core matrix
    constexpr int RW = 128 / T::PW, NO = RW / 8, NCB = (KC / 4 + 3) / 4;
    const int lane = r & 31, wq = r >> 5, ro = lane & 7, cq = lane >> 3;
    // this thread's loads of piece kc of the tile starting at element e0 (ne of its elements in
    // the mesh; zeros for the rest and for the padding modes)
    auto load_piece = [&](int64_t e0, int ne, int kc, float (&x)[NO][NCB][4]) {
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const int row = RW * wq + 8 * o + ro;
        const bool rl = (row >> 2) < ne;
        const float* rs = q + e0 * 4 * Np + (int64_t)row * Np;
#pragma unroll
        for (int cb = 0; cb < NCB; ++cb) {
          const int cg = 4 * cb + cq;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int n = kc * KC + 4 * cg + j;
            x[o][cb][j] = (rl && cg < KC / 4 && n < Np) ? rs[n] : 0.f;
          }
        }
      }
    };
    // software pipeline from N = 4 up: the loads of the following piece are in flight while this
    // one waits for its slot, is converted and handed to the MMAs (measured 2-6 % faster there,
    // 2-5 % slower at N = 2, 3, where a tile is one small piece)
    constexpr bool SWP = N >= 4;
    float cur[NO][NCB][4], nxt[NO][NCB][4];
    if (SWP && blockIdx.x < ntiles)
      load_piece((int64_t)blockIdx.x * EPT, (int)min((int64_t)EPT, K - (int64_t)blockIdx.x * EPT), 0, cur);
    int pc = 0, i = 0;
    uint32_t last_free = 0;  // the last commit's slot barrier and parity (teardown after a stop)
    int last_use = -1;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
      const int64_t e0 = tile * EPT;
      const int acc = i % NACC;
      const int64_t tn = tile + gridDim.x;
      if (tn < ntiles)  // the next tile's state into L2
        prefetch_l2(q + tn * EPT * 4 * Np, sizeof(float) * 4 * Np * (size_t)min((int64_t)EPT, K - tn * EPT), r, NPT);
      for (int kc = 0; kc < NKC && ok; ++kc, ++pc) {
        const int slot = pc & 1, use = pc >> 1;
        if constexpr (SWP) {  // the following piece: this tile's next, or the next tile's first
          const int64_t t2 = kc + 1 < NKC ? tile : tn;
          if (t2 < ntiles) load_piece(t2 * EPT, (int)min((int64_t)EPT, K - t2 * EPT), kc + 1 < NKC ? kc + 1 : 0, nxt);
        } else {
          load_piece(e0, (int)min((int64_t)EPT, K - e0), kc, cur);
        }
        // the slot's previous piece has been multiplied
        if (use >= 1 && !tc_mbar_wait(slot_free0 + 8 * slot, (use - 1) & 1, kTcWaitPolls)) *stop = 1u;
        float* Ah = sm + T::a0 + slot * 2 * T::asz;
        float* Al = Ah + T::asz;
        if constexpr (!T::BRES) {
          float* Bh = Bs + slot * 2 * T::bsz;
          const float* ps = op + (size_t)kc * 2 * T::bsz;
          for (int x = r; x < (int)(2 * T::bsz / 4); x += NPT) cp_async16(Bh + 4 * x, ps + 4 * x);
          cp_async_commit();
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          const int row = RW * wq + 8 * o + ro;
#pragma unroll
          for (int cb = 0; cb < NCB; ++cb) {
            const int cg = 4 * cb + cq;
            if (cg >= KC / 4) continue;
            float h[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) tf32_split(cur[o][cb][j], h[j], l[j]);
            const int off = tc_offset<KC>(row, 4 * cg);
            *reinterpret_cast<float4*>(Ah + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(Al + off) = make_float4(l[0], l[1], l[2], l[3]);
          }
        }
        if constexpr (SWP) {
#pragma unroll
          for (int o = 0; o < NO; ++o)
#pragma unroll
            for (int cb = 0; cb < NCB; ++cb)
#pragma unroll
              for (int j = 0; j < 4; ++j) cur[o][cb][j] = nxt[o][cb][j];
        }
        if constexpr (!T::BRES) cp_async_wait_all();
        tc_fence_smem();
        // the producers' writes of this piece; a stop flag raised anywhere ends every producer
        ok = !producers_sync_or<NPT>(*stop != 0u);
        if (r == 0 && ok) {
          // the accumulator's previous tile has been read out
          if (kc == 0 && i >= NACC && !tc_mbar_wait(acc_empty0 + 8 * acc, ((i / NACC) - 1) & 1, kTcWaitPolls)) {
            *stop = 1u;
          } else {
            tc_fence_after();
            const uint32_t a_hi = smem_addr(Ah), a_lo = smem_addr(Al);
            const uint32_t b_hi = smem_addr(Bs + (T::BRES ? 0 : slot) * 2 * T::bsz), b_lo = b_hi + T::bsz * 4;
            // the piece's first K step within the operator's columns (resident: all of them)
            const uint32_t bk0 = T::BRES ? (uint32_t)kc * (KC / 8) * 256 : 0u;
            constexpr uint32_t idesc = tc_idesc_tf32(128, T::CN);
#pragma unroll
            for (int ch = 0; ch < T::NCH; ++ch) {
              const uint32_t boff = (uint32_t)ch * T::CN * T::BK * 4 + bk0;  // CN rows of B
              const uint32_t dcol = tmem + acc * NP + ch * T::CN;
#pragma unroll
              for (int st = 0; st < KC / 8; ++st) {
                const uint64_t ah = tc_smem_desc(a_hi + 256 * st, 128, 32 * KC);
                const uint64_t al = tc_smem_desc(a_lo + 256 * st, 128, 32 * KC);
                const uint64_t bh = tc_smem_desc(b_hi + boff + 256 * st, 128, 32 * T::BK);
                const uint64_t bl = tc_smem_desc(b_lo + boff + 256 * st, 128, 32 * T::BK);
                tc_mma_tf32(dcol, ah, bh, idesc, kc > 0 || st > 0);
                tc_mma_tf32(dcol, ah, bl, idesc, true);
                tc_mma_tf32(dcol, al, bh, idesc, true);
              }
            }
            tc_commit(slot_free0 + 8 * slot);
            if (kc == NKC - 1) tc_commit(acc_full0 + 8 * acc);
            last_free = slot_free0 + 8 * slot;
            last_use = use;
          }
        }
      }
    }
    if (r == 0 && last_use >= 0) tc_mbar_wait(last_free, last_use & 1, kTcWaitPolls);  // no MMA left in flight
  } else {
    // ---- epilogue: thread tid reads TMEM lane tid (field f of element el of the tile)
    const int el = tid >> 2, f = tid & 3;
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int64_t e0 = tile * EPT;
      const int ne = (int)min((int64_t)EPT, K - e0);
      const int acc = i % NACC;
      if (!tc_mbar_wait(acc_full0 + 8 * acc, (i / NACC) & 1, kTcWaitPolls)) {
        *stop = 1u;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16) + acc * NP;
      float* dst = tr + (e0 + el) * Nfc * 4;
#pragma unroll 1
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float v[16];
        tc_ld16(tl + c0, v);
        tc_wait_ld();
        // 4 x 4 transposes within each quad of lanes (the element's four fields): lane f ends
        // with the four fields of points c0 + 4 b + f, one 16-byte store each
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float a[4] = {v[4 * b], v[4 * b + 1], v[4 * b + 2], v[4 * b + 3]};
          quad_transpose(a, f);
          const int g = c0 + 4 * b + f;
          if (el < ne && g < Nfc) *reinterpret_cast<float4*>(dst + 4 * g) = make_float4(a[0], a[1], a[2], a[3]);
        }
      }
      tc_fence_before();
      tc_mbar_arrive(acc_empty0 + 8 * acc);
    }
  }
  if (!ok && (tid == 0 || tid == 128)) atomicAdd(&g_tc32_timeouts, 1);
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, T::TCOLS);
}

}  // namespace pyrdg
