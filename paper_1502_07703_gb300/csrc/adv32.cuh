// Single-precision LSRK stage kernel for scalar advection u_t + div(beta u) = 0
// (Sec. 4.1): one launch per RK stage, one field.
//
// Same arithmetic as rhs1_kernel (sum-factorised volume term J beta.grad(u) =
// u_r (beta.g1) + u_s (beta.g2) + u_c (beta.g3) with the c direction as banded level
// mixing, the upwind-weighted alpha-flux, lift, diagonal M^{-1}, LSRK update),
// organised like stage32_kernel: constant-bank tables, fully unrolled per-level loops,
// persistent CTAs with cp.async double buffering, EPB elements per CTA, and the traces
// of the updated state written into the other half of a ping-pong trace buffer.
#pragma once

#include "stage32.cuh"

namespace pyrdg {

// Elements per CTA the advection kernel is built for at degree N: the (element, a, b)
// points of the mixing pass must fit the CTA's 128 threads.
constexpr bool epb1_supported(int N, int EPB) {
  return (EPB == 1 || EPB == 2 || EPB == 4 || EPB == 8) && EPB * (N + 1) * (N + 1) <= 128;
}

template <int N, int EPB>
struct A32 {
  using d = Dims<N>;
  static constexpr int NT = 128;
  static constexpr int G = (d::n1 + 1) / 2;        // level groups {g, N-g}
  static constexpr int YS = (d::P3 + 3) / 4 * 4;   // padded row stride of Y and Z
  static constexpr int nY = d::P3 * YS;            // Y block per level
  static constexpr int r32(int x) { return (x + 31) / 32 * 32; }
  static constexpr int GA = r32(EPB * d::n1);      // a pass items per level group: (element, a point)
  static constexpr int GT = r32(EPB * d::P3);      // b^T and trace a pass: (element, point)
  static constexpr int MIXT = r32(EPB * d::n2);    // mixing: (element, a, b point)
  static constexpr size_t al4(size_t x) { return (x + 3) / 4 * 4; }
  static constexpr size_t lx = 0;                                // LX copy (nrow x P3)
  static constexpr size_t dl = lx + d::nrow * d::P3;             // DL copy (nrow x n1)
  static constexpr size_t dec = dl + d::nrow * d::n1;            // Np mode decodings
  // inputs of one element: state (Np; the new state replaces it), residual (Np),
  // geometry (9 n2), face geometry (NGF), M^{-1} (Np); two group buffers of EPB elements
  static constexpr size_t bu = 0, bres = al4(d::Np), bgeo = bres + al4(d::Np), bgf = bgeo + al4(d::NGEO * d::n2),
                          binv = bgf + al4(d::NGF), bsz = binv + al4(d::Np);
  static constexpr size_t buf = al4(dec + d::Np);
  static constexpr size_t Fs = buf + 2 * EPB * bsz;              // EPB x Nfc
  static constexpr size_t ZA0 = d::nrow * YS > 2 * d::nrow * d::n1 ? d::nrow * YS : 2 * d::nrow * d::n1;
  static constexpr size_t ZA = ZA0 > d::nrow * d::P3 ? ZA0 : d::nrow * d::P3;
  static constexpr size_t A = Fs + EPB * d::Nfc;                 // EPB x ZA: A, dA [row][p], later Z, At
  static constexpr size_t Y = A + EPB * ZA;                      // EPB x n1 nY  [k][p'][q']
  static constexpr size_t total = Y + EPB * d::n1 * nY;
  static_assert(MIXT <= NT, "mixing slots");
  static constexpr int MIN_BLOCKS = N <= 5 ? 8 : 4;
  static constexpr size_t bytes = total * sizeof(float);
};

template <int N, int EPB>
__global__ void __launch_bounds__(128, A32<N, EPB>::MIN_BLOCKS)
    adv32_kernel(int64_t K, float* __restrict__ q, float* __restrict__ res, const float* __restrict__ tr_cur,
                 float* __restrict__ tr_nxt, const int32_t* __restrict__ mapP, const float* __restrict__ geo,
                 const float* __restrict__ gface, const float* __restrict__ invM, float bx, float by, float bz,
                 float alpha, float rka, float rkb, float dt) {
  using d = Dims<N>;
  using S = A32<N, EPB>;
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
  for (int x = tid; x < EPB * n1 * nY; x += S::NT) s_Y0[x] = 0.f;

  // Element ei of the group starting at e0; past the end of the mesh a slot holds a
  // copy of element K-1 and only its stores are skipped.
  auto elem = [&](int64_t e0, int ei) -> int64_t { return e0 + ei < K ? e0 + ei : K - 1; };
  // asynchronous copy of the group starting at e0 into group buffer bb (Np is not a
  // multiple of 4, so state, residual and M^{-1} go by 4-byte copies)
  auto issue = [&](int64_t e0, float* bb) {
    for (int x = tid; x < EPB * Np; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / Np, xx = x - ei * Np;
      const int64_t ee = elem(e0, ei);
      cp_async4(bb + ei * S::bsz + S::bu + xx, q + ee * Np + xx);
      cp_async4(bb + ei * S::bsz + S::bres + xx, res + ee * Np + xx);
      cp_async4(bb + ei * S::bsz + S::binv + xx, invM + ee * Np + xx);
    }
    for (int x = tid; x < EPB * d::NGEO * n2; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (d::NGEO * n2), xx = x - ei * (d::NGEO * n2);
      cp_async4(bb + ei * S::bsz + S::bgeo + xx, geo + elem(e0, ei) * d::NGEO * n2 + xx);
    }
    for (int x = tid; x < EPB * (d::NGF / 4); x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (d::NGF / 4), xx = x - ei * (d::NGF / 4);
      cp_async16(bb + ei * S::bsz + S::bgf + 4 * xx, gface + elem(e0, ei) * d::NGF + 4 * xx);
    }
    cp_async_commit();
  };
  const int64_t gstride = (int64_t)gridDim.x * EPB;
  if ((int64_t)blockIdx.x * EPB < K) issue((int64_t)blockIdx.x * EPB, sm + S::buf);
  int it = 0;
  for (int64_t e0 = (int64_t)blockIdx.x * EPB; e0 < K; e0 += gstride, ++it) {
    const int ne = EPB == 1 ? 1 : (int)min((int64_t)EPB, K - e0);  // elements of the group in the mesh
    float* bcur = sm + S::buf + (it & 1) * EPB * S::bsz;
    cp_async_wait_all();  // this thread's copies of the group have landed
    __syncthreads();      // ... everyone's; and the other buffer's last reader is done
    const int64_t en = e0 + gstride;
    if (en < K) issue(en, sm + S::buf + ((it + 1) & 1) * EPB * S::bsz);

    // ---- upwind-weighted flux at every face point, times w sJ:
    // ((beta.n - alpha |beta.n|)/2) (u+ - u-)
    for (int x = tid; x < EPB * Nfc; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / Nfc, g = x - ei * Nfc;
      const float* s_gf = bcur + ei * S::bsz + S::bgf;
      const int face = g / n2, idx = g - face * n2;
      const int64_t gl = elem(e0, ei) * Nfc + g;
      const float um = tr_cur[gl], up = tr_cur[mapP[gl]];
      const float* nv = face == 0 ? s_gf + 16 + 4 * idx : s_gf + 4 * (face - 1);
      const float w = face == 0 ? c32<N>[C::WB + idx] : c32<N>[C::WFT + idx];
      const float bn = bx * nv[0] + by * nv[1] + bz * nv[2];
      s_Fs0[ei * Nfc + g] = w * nv[3] * 0.5f * (bn - alpha * fabsf(bn)) * (up - um);
    }
    // ---- a pass per (level group, element, a point p): A = l^k(a_p) u, dA = l^k'(a_p) u
    for (int x = tid; x < S::G * S::GA; x += S::NT) {
      const int grp = x / S::GA, r = x - grp * S::GA;
      if (r >= EPB * n1) continue;
      const int ei = EPB == 1 ? 0 : r / n1, p = r - ei * n1;
      const float* uf = bcur + ei * S::bsz + S::bu;
      float* s_A = s_A0 + ei * ZA;
      float* s_dA = s_A + nrow * n1;
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
          if (k == N) a = uf[lvl_off(k) + j * (k + 1) + p];  // l_i^N(a_p) = delta_ip
          s_A[(tri_num(k) + j) * n1 + p] = a;
          s_dA[(tri_num(k) + j) * n1 + p] = da;
        }
      }
    }
    __syncthreads();

    // ---- b pass and level mixing (c direction) per (element, a, b point), chain rule with
    // beta, base lift; then the triangle-face c^T
    if (tid < S::MIXT) {
      const int y = tid;
      if (y < EPB * n2) {
        const int ei = EPB == 1 ? 0 : y / n2, pq = y - ei * n2;
        const int p = pq % n1, qq = pq / n1;
        const float* g = bcur + ei * S::bsz + S::bgeo + pq * d::NGEO;
        const float* s_A = s_A0 + ei * ZA;
        const float* s_dA = s_A + nrow * n1;
        float U0[n1], Ua0[n1], Ub0[n1];
#pragma unroll
        for (int k = 0; k <= N; ++k) {
          float u = 0.f, ua = 0.f, ub = 0.f;
#pragma unroll
          for (int j = 0; j <= k; ++j) {
            const int o = (tri_num(k) + j) * n1 + p;
            const float a = s_A[o];
            ub = fmaf(a, s_dl[(tri_num(k) + j) * n1 + qq], ub);
            if (k < N) {
              const float lq = s_lx[(tri_num(k) + j) * P3 + qq];
              u = fmaf(a, lq, u);
              ua = fmaf(s_dA[o], lq, ua);
            }
          }
          if (k == N) {  // l_j^N(b_q) = delta_jq
            const int o = (tri_num(k) + qq) * n1 + p;
            u = s_A[o];
            ua = s_dA[o];
          }
          U0[k] = u;
          Ua0[k] = ua;
          Ub0[k] = ub;
        }
        const float b1 = fmaf(bx, g[0], fmaf(by, g[1], bz * g[2]));
        const float b2 = fmaf(bx, g[3], fmaf(by, g[4], bz * g[5]));
        const float b3 = fmaf(bx, g[6], fmaf(by, g[7], bz * g[8]));
        const float Fb = s_Fs0[ei * Nfc + pq];
        float* s_Y = s_Y0 + ei * n1 * nY;
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
          s_Y[kp * nY + p * YS + qq] = fmaf(c32<N>[C::GB + kp], Fb, fmaf(b1, al, fmaf(b2, be, b3 * ga)));
        }
      }
    }
    for (int x = (tid + S::NT - S::MIXT) % S::NT; x < EPB * 4 * n1; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (4 * n1), y = x - ei * 4 * n1;
      const int ee = y % n1, slot = y / n1;
      const int face = slot == 0 ? 1 : slot == 1 ? 3 : slot == 2 ? 4 : 2;
      const float* fs = s_Fs0 + ei * Nfc + face * n2 + ee;
      float Fm[n1];
#pragma unroll
      for (int m = 0; m <= N; ++m) Fm[m] = fs[m * n1];
      float* Yf = s_Y0 + ei * n1 * nY;
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

    // ---- b^T pass per (element, row p' of Y): Z[row(k,j)][p'] = sum_q' l_j^k(x_q') Y[k][p'][q']
    for (int x = tid; x < S::G * S::GT; x += S::NT) {
      const int grp = x / S::GT, r = x - grp * S::GT;
      if (r >= EPB * P3) continue;
      const int ei = EPB == 1 ? 0 : r / P3, pp = r - ei * P3;
      const float* s_Y = s_Y0 + ei * n1 * nY;
      float* s_Z = s_A0 + ei * ZA;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        if (k != grp && k != N - grp) continue;
        const float* Yr = s_Y + k * nY + pp * YS;
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
          s_Z[(tri_num(k) + j) * YS + pp] = acc;
        }
      }
    }
    __syncthreads();

    // ---- a^T pass, M^{-1}, LSRK update; the new state goes back to shared memory
    for (int x = tid; x < EPB * Np; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / Np, n = x - ei * Np;
      const int kji = s_dec[n];
      const int k = kji & 0xff, j = (kji >> 8) & 0xff, i = kji >> 16;
      const float* Zr = s_A0 + ei * ZA + (tri_num(k) + j) * YS;
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
      const float rnew = fmaf(rka, be[S::bres + n], dt * rhs);
      const float unew = fmaf(rkb, rnew, be[S::bu + n]);
      be[S::bu + n] = unew;
      if (ei < ne) {
        const int64_t gi = (e0 + ei) * Np + n;
        res[gi] = rnew;
        q[gi] = unew;
      }
    }
    __syncthreads();

    // ---- traces of the updated state (Alg. 3) into tr_nxt: the a direction at every a
    // point and a = -1, +1 by level groups (level N at the volume columns is u itself) ...
    for (int x = tid; x < S::G * S::GT; x += S::NT) {
      const int grp = x / S::GT, r = x - grp * S::GT;
      if (r >= EPB * P3) continue;
      const int ei = EPB == 1 ? 0 : r / P3, pp = r - ei * P3;
      const float* uf = bcur + ei * S::bsz + S::bu;
      float* s_At = s_A0 + ei * ZA;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        if (k != grp && k != N - grp) continue;
        if (k == N && pp < n1) continue;
        float lxc[n1];
#pragma unroll
        for (int i = 0; i <= k; ++i) lxc[i] = s_lx[(tri_num(k) + i) * P3 + pp];
#pragma unroll
        for (int j = 0; j <= k; ++j) {
          float a = 0.f;
#pragma unroll
          for (int i = 0; i <= k; ++i) a = fmaf(uf[lvl_off(k) + j * (k + 1) + i], lxc[i], a);
          s_At[(tri_num(k) + j) * P3 + pp] = a;
        }
      }
    }
    __syncthreads();
    // ... then the face points: 4 n1 items per element for the triangular faces (a level
    // sum, then the c direction), n1 for the base (one a point, all b points)
    for (int x = tid; x < EPB * 5 * n1; x += S::NT) {
      const int ei = EPB == 1 ? 0 : x / (5 * n1), xx = x - ei * 5 * n1;
      if (ei >= ne) continue;
      const float* s_At = s_A0 + ei * ZA;
      const float* s_u = bcur + ei * S::bsz + S::bu;
      float* dst = tr_nxt + (e0 + ei) * Nfc;
      if (xx < 4 * n1) {
        const int t = xx % n1, kind = xx / n1;  // kind: 0 b=-1, 1 b=+1, 2 a=-1, 3 a=+1
        const int wcol = kind < 2 ? n1 + (kind & 1) : t;
        const int acol = kind < 2 ? t : n1 + (kind & 1);
        const float* Ar = s_At + acol;
        const float* wr = s_lx + wcol;
        const float* ArN = kind < 2 ? s_u + lvl_off(N) + t : Ar + tri_num(N) * P3;
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
          dst[face * n2 + t + n1 * m] = acc;
        }
      } else {  // base (c = -1) at (a_t, b_c) for every c
        const int t = xx - 4 * n1;
        const float* Ar = s_At + t;
        float at[nrow];
#pragma unroll
        for (int rr = 0; rr < tri_num(N); ++rr) at[rr] = Ar[rr * P3];
#pragma unroll
        for (int c = 0; c <= N; ++c) {
          float acc = 0.f;
#pragma unroll
          for (int rr = 0; rr < tri_num(N); ++rr) acc = fmaf(c32<N>[C::CB + rr * n1 + c], at[rr], acc);
          acc = fmaf(c32<N>[C::GB + N], s_u[lvl_off(N) + c * n1 + t], acc);
          dst[t + n1 * c] = acc;
        }
      }
    }
  }
}

}  // namespace pyrdg
