// Single-precision LSRK stage kernel: one launch per RK stage.
//
// Same arithmetic as rhs_kernel (sum-factorised volume term with the c direction
// as level mixing, flux, lift, diagonal M^{-1}, LSRK update), organised for the
// FP32 pipe, which retires 61x more FMAs per cycle than the FP64 pipe and so
// exposes every extra instruction:
//  - reference tables live in constant memory and every loop over them is fully
//    unrolled, so table operands are immediate constant-bank operands of FFMA;
//  - each thread owns a column of one pass and keeps its data in registers;
//  - the kernel also interpolates the updated state to the face points (the
//    trace step of Alg. 3) into the other half of a ping-pong trace buffer, so
//    a stage is a single launch and the state is read once;
//  - CTAs are persistent (grid-stride over elements); tables are staged once.
#pragma once

#include "dg_kernels.cuh"

namespace pyrdg {

// Constant-memory table layout of the FP32 stage kernel for degree N.
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
  static constexpr int CB = WFT + d::n2;            // [tri(k)+j][q] G_k(-1) l_j^k(b_q): base trace
  static constexpr int CFm = CB + d::nrow * d::n1;  // [tri(k)+j][m] G_k(c_m) l_j^k(-1): face b = -1
  static constexpr int CFp = CFm + d::nrow * d::n1; // [tri(k)+j][m] G_k(c_m) l_j^k(+1): face b = +1
  static constexpr int size = CFp + d::nrow * d::n1;
};

// One copy per translation unit (each unit instantiates one degree); filled by
// upload_c32() from the double tables, rounded to float.
static __constant__ float c32[C32<7>::size];

// Ask L2 to fetch the 128-byte lines of [p, p + bytes) (one line per participating thread).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, int tid, int nthr) {
  const char* c = reinterpret_cast<const char*>(p);
  const size_t first = reinterpret_cast<size_t>(c) & ~size_t(127);
  const size_t last = (reinterpret_cast<size_t>(c) + bytes - 1) & ~size_t(127);
  for (size_t a = first + (size_t)tid * 128; a <= last; a += (size_t)nthr * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

template <int N>
struct S32 {
  using d = Dims<N>;
  static constexpr int NT = 128;
  static constexpr int G = (d::n1 + 1) / 2;        // level groups {g, N-g}
  static constexpr int YS = (d::P3 + 3) / 4 * 4;   // padded row stride of Y and Z
  static constexpr int nY = d::P3 * YS;            // Y block per (field, level)
  // shared-memory layout (floats)
  static constexpr size_t al4(size_t x) { return (x + 3) / 4 * 4; }  // 16-byte alignment
  static constexpr size_t lx = 0;                                // LX copy (nrow x P3)
  static constexpr size_t dl = lx + d::nrow * d::P3;             // DL copy (nrow x n1)
  static constexpr size_t u = al4(dl + d::nrow * d::n1);         // state (4 Np), old then new
  static constexpr size_t geo = u + 4 * d::Np;                   // 9 n2
  static constexpr size_t gf = geo + d::NGEO * d::n2;            // NGF
  static constexpr size_t Fs = gf + d::NGF;                      // 4 Nfc  [f][g]
  static constexpr size_t A = Fs + 4 * d::Nfc;                   // [f][row][p]: a pass of u_old
  static constexpr size_t dA = A + 4 * d::nrow * d::n1;          // [f][row][p]: a pass, d/da
  static constexpr size_t ZA = 4 * d::nrow * YS > 8 * d::nrow * d::n1 ? 4 * d::nrow * YS : 8 * d::nrow * d::n1;
  static constexpr size_t Y = A + ZA;                            // 4 n1 nY  [f][k][p'][q']
  static constexpr size_t Af = Y + 4 * d::n1 * nY;               // 4 x 2 x nrow: A at a = -1, +1 of u_new
  static constexpr size_t total = Af + 8 * d::nrow;
  static constexpr size_t Z = A;                                 // 4 nrow YS [f][row][p'] (A, dA dead by then)
  // resident CTAs per SM the register budget is tuned for
  static constexpr int MIN_BLOCKS = N <= 5 ? 8 : 4;
  // L2 prefetch of the next element: pays at N >= 6, where the per-element load latency
  // is exposed longest; at lower N its registers push the kernel into spills
  static constexpr bool PREFETCH = N >= 6;
  static constexpr size_t bytes = total * sizeof(float);
};

template <int N>
__global__ void __launch_bounds__(128, S32<N>::MIN_BLOCKS)
    stage32_kernel(int64_t K, float* __restrict__ q, float* __restrict__ res, const float* __restrict__ tr_cur,
                   float* __restrict__ tr_nxt, const int32_t* __restrict__ mapP, const float* __restrict__ geo,
                   const float* __restrict__ gface, const float* __restrict__ invM, int bc, float tau, float rka,
                   float rkb, float dt, const float* __restrict__ dt_elem, int write_traces) {
  using d = Dims<N>;
  using S = S32<N>;
  using C = C32<N>;
  constexpr int n1 = d::n1, n2 = d::n2, P3 = d::P3, nrow = d::nrow, Np = d::Np, Nfc = d::Nfc;
  constexpr int YS = S::YS, nY = S::nY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* s_lx = sm + S::lx;
  float* s_dl = sm + S::dl;
  float* s_u = sm + S::u;
  float* s_geo = sm + S::geo;
  float* s_gf = sm + S::gf;
  float* s_Fs = sm + S::Fs;
  float* s_A = sm + S::A;
  float* s_dA = sm + S::dA;
  float* s_Y = sm + S::Y;
  float* s_Af = sm + S::Af;
  float* s_Z = sm + S::Z;
  const int tid = threadIdx.x;

  for (int x = tid; x < nrow * P3; x += S::NT) s_lx[x] = c32[C::LX + x];
  for (int x = tid; x < nrow * n1; x += S::NT) s_dl[x] = c32[C::DL + x];
  // Y entries that no pass writes (face rows x face columns) stay zero
  for (int x = tid; x < 4 * n1 * nY; x += S::NT) s_Y[x] = 0.f;

  for (int64_t e = blockIdx.x; e < K; e += gridDim.x) {
    __syncthreads();
    // ---- load the element
    {
      const float4* src = reinterpret_cast<const float4*>(q + e * 4 * Np);
      float4* dst = reinterpret_cast<float4*>(s_u);
      for (int x = tid; x < Np; x += S::NT) dst[x] = src[x];  // 4 Np floats = Np float4
    }
    for (int x = tid; x < d::NGEO * n2; x += S::NT) s_geo[x] = geo[e * d::NGEO * n2 + x];
    for (int x = tid; x < d::NGF; x += S::NT) s_gf[x] = gface[e * d::NGF + x];
    // the next element of this CTA: bring its contiguous inputs into L2 while this one computes
    const int64_t en = e + gridDim.x;
    if (S::PREFETCH && en < K) {
      prefetch_l2(q + en * 4 * Np, sizeof(float) * 4 * Np, tid, S::NT);
      prefetch_l2(res + en * 4 * Np, sizeof(float) * 4 * Np, tid, S::NT);
      prefetch_l2(geo + en * d::NGEO * n2, sizeof(float) * d::NGEO * n2, tid, S::NT);
      prefetch_l2(gface + en * d::NGF, sizeof(float) * d::NGF, tid, S::NT);
      prefetch_l2(invM + en * Np, sizeof(float) * Np, tid, S::NT);
      prefetch_l2(tr_cur + en * Nfc * 4, sizeof(float) * 4 * Nfc, tid, S::NT);
      prefetch_l2(mapP + en * Nfc, sizeof(int32_t) * Nfc, tid, S::NT);
    }
    __syncthreads();

    // ---- surface flux at every face point (a4), weighted by w sJ
    for (int g = tid; g < Nfc; g += S::NT) {
      const int face = g / n2, idx = g - face * n2;
      const int64_t gl = e * Nfc + g;
      const int64_t gn = mapP[gl];
      const float4 a4 = reinterpret_cast<const float4*>(tr_cur)[gl];
      const float4 b4 = reinterpret_cast<const float4*>(tr_cur)[gn];
      const float um[4] = {a4.x, a4.y, a4.z, a4.w};
      const float up[4] = {b4.x, b4.y, b4.z, b4.w};
      const float* nv = face == 0 ? s_gf + 16 + 4 * idx : s_gf + 4 * (face - 1);
      const float w = face == 0 ? c32[C::WB + idx] : c32[C::WFT + idx];
      float F[4];
      face_flux<float>(um, up, gn == gl, bc, tau, nv, w * nv[3], F);
#pragma unroll
      for (int f = 0; f < 4; ++f) s_Fs[f * Nfc + g] = F[f];
    }
    // ---- a pass per (level group, field, a point p): A = l^k(a_p) u, dA = l^k'(a_p) u.
    // Warp g takes levels g and N-g, whose (k+1)^2 costs pair up.
    if ((tid & 31) < 4 * n1 && (tid >> 5) < S::G) {
      const int grp = tid >> 5, lane = tid & 31;
      const int f = lane / n1, p = lane - f * n1;
      const float* uf = s_u + f * Np;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        if (k != grp && k != N - grp) continue;
        float lxc[n1], dlc[n1];
#pragma unroll
        for (int i = 0; i <= k; ++i) {
          lxc[i] = s_lx[(tri_num(k) + i) * P3 + p];
          dlc[i] = s_dl[(tri_num(k) + i) * n1 + p];
        }
#pragma unroll
        for (int j = 0; j <= k; ++j) {
          float a = 0.f, da = 0.f;
#pragma unroll
          for (int i = 0; i <= k; ++i) {
            const float c = uf[lvl_off(k) + j * (k + 1) + i];
            a = fmaf(c, lxc[i], a);
            da = fmaf(c, dlc[i], da);
          }
          const int o = (f * nrow + tri_num(k) + j) * n1 + p;
          s_A[o] = a;
          s_dA[o] = da;
        }
      }
    }
    if (S::PREFETCH && e + gridDim.x < K) {  // neighbour traces of the next element (its mapP is in L2 by now)
      const int64_t en = e + gridDim.x;
      for (int g = tid; g < Nfc; g += S::NT) {
        const float* pn = tr_cur + (int64_t)mapP[en * Nfc + g] * 4;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pn));
      }
    }
    __syncthreads();

    // ---- level mixing (c direction of Alg. 1) per (a,b) point, base lift; triangle-face c^T
    for (int x = tid; x < n2 + 16 * n1; x += S::NT) {
      if (x < n2) {
        // b pass at this (a_p, b_q) point for all fields and levels, in registers
        const int pq = x, p = pq % n1, qq = pq / n1;
        const float* g = s_geo + pq * d::NGEO;
        float lq[nrow], dlq[nrow];
#pragma unroll
        for (int r = 0; r < nrow; ++r) {
          lq[r] = s_lx[r * P3 + qq];
          dlq[r] = s_dl[r * n1 + qq];
        }
        float U0[n1], Ua0[n1], Ub0[n1], X[n1], Zc[n1];
#pragma unroll
        for (int k = 0; k <= N; ++k) {
          float u = 0.f, ua = 0.f, ub = 0.f;
#pragma unroll
          for (int j = 0; j <= k; ++j) {
            const int o = (tri_num(k) + j) * n1 + p;
            const float a = s_A[o], da = s_dA[o];
            u = fmaf(a, lq[tri_num(k) + j], u);
            ub = fmaf(a, dlq[tri_num(k) + j], ub);
            ua = fmaf(da, lq[tri_num(k) + j], ua);
          }
          U0[k] = u;
          Ua0[k] = ua;
          Ub0[k] = ub;
          float xs = 0.f, zs = 0.f;
#pragma unroll
          for (int m = 0; m < 3; ++m) {  // velocity fields: only the div combination is kept
            float v = 0.f, va = 0.f, vb = 0.f;
#pragma unroll
            for (int j = 0; j <= k; ++j) {
              const int o = ((m + 1) * nrow + tri_num(k) + j) * n1 + p;
              const float a = s_A[o], da = s_dA[o];
              v = fmaf(a, lq[tri_num(k) + j], v);
              vb = fmaf(a, dlq[tri_num(k) + j], vb);
              va = fmaf(da, lq[tri_num(k) + j], va);
            }
            xs = fmaf(g[m], va, fmaf(g[3 + m], vb, xs));
            zs = fmaf(g[6 + m], v, zs);
          }
          X[k] = xs;
          Zc[k] = zs;
        }
        float Fb[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) Fb[f] = s_Fs[f * Nfc + pq];
#pragma unroll
        for (int kp = 0; kp <= N; ++kp) {
          float al = 0.f, be = 0.f, ga = 0.f, dv = 0.f;
#pragma unroll
          for (int k = 0; k <= N; ++k) {
            const float mh = c32[C::MH + kp * n1 + k], mg = c32[C::MG + kp * n1 + k];
            al = fmaf(mh, Ua0[k], al);
            be = fmaf(mh, Ub0[k], be);
            ga = fmaf(mg, U0[k], ga);
            dv = fmaf(mh, X[k], fmaf(mg, Zc[k], dv));
          }
          const float gb = c32[C::GB + kp];
          const int yo = kp * nY + p * YS + qq;
          s_Y[0 * n1 * nY + yo] = fmaf(gb, Fb[0], dv);
#pragma unroll
          for (int m = 0; m < 3; ++m)
            s_Y[(m + 1) * n1 * nY + yo] = fmaf(gb, Fb[m + 1], fmaf(g[m], al, fmaf(g[3 + m], be, g[6 + m] * ga)));
        }
      } else {
        const int y = x - n2;
        const int ee = y % n1;
        const int slot = (y / n1) % 4;
        const int f = y / (4 * n1);
        const int face = slot == 0 ? 1 : slot == 1 ? 3 : slot == 2 ? 4 : 2;
        const float* fs = s_Fs + f * Nfc + face * n2 + ee;
        float Fm[n1];
#pragma unroll
        for (int m = 0; m <= N; ++m) Fm[m] = fs[m * n1];
        float* Yf = s_Y + f * n1 * nY;
#pragma unroll
        for (int k = 0; k <= N; ++k) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m <= N; ++m) acc = fmaf(c32[C::GF + k * n1 + m], Fm[m], acc);
          if (slot < 2)
            Yf[k * nY + ee * YS + n1 + slot] = acc;  // b = -1, +1 columns
          else
            Yf[k * nY + (n1 + slot - 2) * YS + ee] = acc;  // a = -1, +1 rows
        }
      }
    }
    __syncthreads();

    // ---- b^T pass per (field, row p' of Y): Z[f][row(k,j)][p'] = sum_q' l_j^k(x_q') Y[f][k][p'][q']
    for (int x = tid; x < S::G * 4 * P3; x += S::NT) {
      const int grp = x / (4 * P3), y = x - grp * 4 * P3;
      const int f = y / P3, pp = y - f * P3;
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
          for (int c = 0; c < P3; ++c) acc = fmaf(c32[C::LX + (tri_num(k) + j) * P3 + c], yv[c], acc);
          s_Z[(f * nrow + tri_num(k) + j) * YS + pp] = acc;
        }
      }
    }
    __syncthreads();

    // ---- a^T pass, M^{-1} (a6), LSRK update (a7); the new state goes back to shared memory
    for (int x = tid; x < 4 * Np; x += S::NT) {
      const int f = x / Np, n = x - f * Np;
      int k, j, i;
      decode_mode(n, k, j, i);
      const float* Zr = s_Z + (f * nrow + tri_num(k) + j) * YS;
      const float* lr = s_lx + (tri_num(k) + i) * P3;
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < P3; ++c) acc = fmaf(lr[c], Zr[c], acc);
      const float rhs = -invM[e * Np + n] * acc;
      const int64_t gi = e * 4 * Np + x;
      const float dte = dt_elem ? dt_elem[e] : dt;  // per-element step when meshes are batched
      const float rnew = fmaf(rka, res[gi], dte * rhs);
      res[gi] = rnew;
      const float unew = fmaf(rkb, rnew, s_u[x]);
      q[gi] = unew;
      s_u[x] = unew;
    }
    if (!write_traces) continue;
    __syncthreads();

    // ---- traces of the updated state (Alg. 3's interpolation to face points) into tr_nxt
    if (tid < 4 * P3) {
      const int f = tid / P3, pp = tid - f * P3;
      const float* uf = s_u + f * Np;
      float A[nrow];
#pragma unroll
      for (int k = 0; k <= N; ++k) {
#pragma unroll
        for (int j = 0; j <= k; ++j) {
          float a = 0.f;
#pragma unroll
          for (int i = 0; i <= k; ++i)
            a = fmaf(uf[lvl_off(k) + j * (k + 1) + i], s_lx[(tri_num(k) + i) * P3 + pp], a);
          A[tri_num(k) + j] = a;
        }
      }
      float* dst = tr_nxt + e * Nfc * 4 + f;
      if (pp <= N) {
#pragma unroll
        for (int c = 0; c <= N; ++c) {
          float tb = 0.f, tm = 0.f, tp = 0.f;
#pragma unroll
          for (int r = 0; r < nrow; ++r) {
            tb = fmaf(c32[C::CB + r * n1 + c], A[r], tb);
            tm = fmaf(c32[C::CFm + r * n1 + c], A[r], tm);
            tp = fmaf(c32[C::CFp + r * n1 + c], A[r], tp);
          }
          dst[4 * (pp + n1 * c)] = tb;               // base point (a_pp, b_c)
          dst[4 * (1 * n2 + pp + n1 * c)] = tm;      // face b = -1 at (a_pp, c_c)
          dst[4 * (3 * n2 + pp + n1 * c)] = tp;      // face b = +1
        }
      } else {
#pragma unroll
        for (int r = 0; r < nrow; ++r) s_Af[(f * 2 + (pp - n1)) * nrow + r] = A[r];
      }
    }
    __syncthreads();
    if (tid < 8 * n1) {  // faces a = -1 (face 4) and a = +1 (face 2) at (b_e, c_m)
      const int ee = tid % n1, side = (tid / n1) % 2, f = tid / (2 * n1);
      const float* Af = s_Af + (f * 2 + side) * nrow;
      float t[nrow];
#pragma unroll
      for (int r = 0; r < nrow; ++r) t[r] = Af[r] * s_lx[r * P3 + ee];
      float* dst = tr_nxt + e * Nfc * 4 + f;
      const int face = side == 0 ? 4 : 2;
#pragma unroll
      for (int m = 0; m <= N; ++m) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k <= N; ++k) {
          float s = 0.f;
#pragma unroll
          for (int j = 0; j <= k; ++j) s += t[tri_num(k) + j];
          acc = fmaf(c32[C::GF + k * n1 + m], s, acc);
        }
        dst[4 * (face * n2 + ee + n1 * m)] = acc;
      }
    }
  }
}

}  // namespace pyrdg
