// CUDA kernels of one LSRK stage of the pyramid DG acoustic-wave method
// (Sec. 4.2 Alg. 1-3 with the semi-nodal basis of Lemma 3), templated on the
// degree N and the scalar type T (double or float).
//
// Sum factorisation. phi_ijk(a,b,c) = l_i^k(a) l_j^k(b) G_k(c) and the volume
// rule is a tensor grid (a_p, b_q, c_r), so every interpolation and every
// projection factors into three one-dimensional passes (a, then b, then c, or
// the reverse). Face points reuse the same passes: the base face is c = -1 on
// the (a_p, b_q) grid, the triangle faces sit at a = +-1 or b = +-1, which are
// the two extra entries (-1, +1) appended to the a and b point sets.
//
// One CTA processes one element; all intermediates live in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace pyrdg {

template <int N>
struct KCfg {
  using d = Dims<N>;
  static constexpr int NT = d::Nc <= 128 ? 128 : (d::Nc <= 256 ? 256 : 512);
  static constexpr int NT_ERR = 256;
};

__device__ __forceinline__ void decode_mode(int n, int& k, int& j, int& i) {
  k = 0;
  while (lvl_off(k + 1) <= n) ++k;
  const int rem = n - lvl_off(k);
  j = rem / (k + 1);
  i = rem - j * (k + 1);
}

__device__ __forceinline__ void decode_row(int row, int& k, int& j) {
  k = 0;
  while (tri_num(k + 1) <= row) ++k;
  j = row - tri_num(k);
}

template <typename T>
__device__ __forceinline__ size_t align_up(size_t x) {
  return (x + 15) & ~size_t(15);
}

// Bilinear base map B(a,b) of v1..v4 and its a, b derivatives (double).
__device__ __forceinline__ void d_bilinear(const double* v, double a, double b, double* B, double* Ba, double* Bb) {
  const double w1 = 0.25 * (1 - a) * (1 - b), w2 = 0.25 * (1 + a) * (1 - b);
  const double w3 = 0.25 * (1 + a) * (1 + b), w4 = 0.25 * (1 - a) * (1 + b);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double v1 = v[m], v2 = v[3 + m], v3 = v[6 + m], v4 = v[9 + m];
    B[m] = w1 * v1 + w2 * v2 + w3 * v3 + w4 * v4;
    Ba[m] = 0.25 * ((1 - b) * (v2 - v1) + (1 + b) * (v3 - v4));
    Bb[m] = 0.25 * ((1 - a) * (v4 - v1) + (1 + a) * (v3 - v2));
  }
}

__device__ __forceinline__ void d_cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// J(a,b) = det[B_a, B_b, D], D = (v5 - B)/2 (Lemma 1: bilinear in a, b).
__device__ __forceinline__ double d_jacobian(const double* v, double a, double b) {
  double B[3], Ba[3], Bb[3], D[3], g1[3];
  d_bilinear(v, a, b, B, Ba, Bb);
#pragma unroll
  for (int m = 0; m < 3; ++m) D[m] = 0.5 * (v[12 + m] - B[m]);
  d_cross(Bb, D, g1);
  return Ba[0] * g1[0] + Ba[1] * g1[1] + Ba[2] * g1[2];
}

// Exact standing waves (wall on [0,1]^3, free surface on [-1,1]^3). The spatial
// factors are cos/sin(pi s x) with s = 1 (wall) or 1/2 (free), evaluated with
// sincospi; ct, st = cos, sin(sqrt(3) pi s t) come from the caller once per launch.
// The exact fields from the sines and cosines s[m], c[m] of pi sc x_m.
__device__ __forceinline__ void d_exact_sc(const double* s, const double* c, double ct, double st, double* out) {
  const double inv_s3 = 0.57735026918962576451;
  const double cyz = c[1] * c[2];
  out[0] = c[0] * cyz * ct;
  out[1] = s[0] * cyz * (st * inv_s3);
  out[2] = c[0] * s[1] * c[2] * (st * inv_s3);
  out[3] = c[0] * c[1] * s[2] * (st * inv_s3);
}

__device__ __forceinline__ void d_exact(int bc, double x, double y, double z, double ct, double st, double* out) {
  const double sc = bc == 0 ? 1.0 : 0.5;
  double s[3], c[3];
  sincospi(sc * x, &s[0], &c[0]);
  sincospi(sc * y, &s[1], &c[1]);
  sincospi(sc * z, &s[2], &c[2]);
  d_exact_sc(s, c, ct, st, out);
}

// sin(alpha + eps), cos(alpha + eps) from sin, cos of alpha and a small eps, |eps| <= 0.1,
// by the angle-addition formulas with the Taylor series of sin(eps) and cos(eps) to
// eps^9 and eps^8 (the first omitted terms are below 3e-17 for |eps| <= 0.1).
__device__ __forceinline__ void d_sincos_shift(double sa, double ca, double eps, double* s, double* c) {
  const double e2 = eps * eps;
  const double ce = 1.0 + e2 * (-1.0 / 2 + e2 * (1.0 / 24 + e2 * (-1.0 / 720 + e2 * (1.0 / 40320))));
  const double se = eps * (1.0 + e2 * (-1.0 / 6 + e2 * (1.0 / 120 + e2 * (-1.0 / 5040 + e2 * (1.0 / 362880)))));
  *s = sa * ce + ca * se;
  *c = ca * ce - sa * se;
}

__device__ __forceinline__ void d_time_factors(int bc, double t, double* ct, double* st) {
  const double sc = bc == 0 ? 1.0 : 0.5;
  sincospi(1.7320508075688772935 * sc * t, st, ct);
}

// ============================================================ geometry (a1)
// Per element, in double: at the (a_p, b_q) grid the nine factors
// w_p w_q (g1, g2, g3), g1 = B_b x D, g2 = D x B_a, g3 = B_a x B_b, so that
// J grad(u) = u_r g1 + u_s g2 + u_c g3 with u_r = 2/(1-c) u_a, u_s = 2/(1-c) u_b
// (all c-independent); base-face unit normal and surface Jacobian from
// n sJ = -g3; triangle faces: constant n sJ from the face's edge and apex;
// mass diagonal inverse 1/(J(a_i^k, b_j^k) w_i^k w_j^k C_k) (Lemma 3).
template <int N, typename T>
__global__ void geom_kernel(int64_t K, const double* __restrict__ ev, const double* __restrict__ gtab,
                            T* __restrict__ geo, T* __restrict__ gface, T* __restrict__ invM) {
  using d = Dims<N>;
  constexpr GeoLayout G(N);
  const int64_t e = blockIdx.x;
  __shared__ double v[15];
  if (threadIdx.x < 15) v[threadIdx.x] = ev[e * 15 + threadIdx.x];
  __syncthreads();
  for (int pq = threadIdx.x; pq < d::n2; pq += blockDim.x) {
    const int p = pq % d::n1, q = pq / d::n1;
    const double a = gtab[G.XG + p], b = gtab[G.XG + q];
    double B[3], Ba[3], Bb[3], D[3], g1[3], g2[3], g3[3];
    d_bilinear(v, a, b, B, Ba, Bb);
    for (int m = 0; m < 3; ++m) D[m] = 0.5 * (v[12 + m] - B[m]);
    d_cross(Bb, D, g1);
    d_cross(D, Ba, g2);
    d_cross(Ba, Bb, g3);
    const double w = gtab[G.WG + p] * gtab[G.WG + q];
    T* out = geo + (e * d::n2 + pq) * d::NGEO;
    for (int m = 0; m < 3; ++m) {
      out[m] = (T)(w * g1[m]);
      out[3 + m] = (T)(w * g2[m]);
      out[6 + m] = (T)(w * g3[m]);
    }
    const double sJ = sqrt(g3[0] * g3[0] + g3[1] * g3[1] + g3[2] * g3[2]);
    T* gf = gface + e * d::NGF + 16 + 4 * pq;
    for (int m = 0; m < 3; ++m) gf[m] = (T)(-g3[m] / sJ);
    gf[3] = (T)sJ;
  }
  if (threadIdx.x < 4) {
    // faces b=-1, a=+1, b=+1, a=-1: outward n sJ = (x1 - x0) x (x2 - x0) / 4
    const int f = threadIdx.x;
    // b=-1: (v2-v1)x(v5-v1); a=+1: (v3-v2)x(v5-v2); b=+1: (v3-v5)x(v4-v5); a=-1: (v5-v1)x(v4-v1)
    const int i0[4] = {0, 1, 4, 0}, i1[4] = {1, 2, 2, 4}, i2[4] = {4, 4, 3, 3};
    double e1[3], e2[3], ns[3];
    for (int m = 0; m < 3; ++m) {
      e1[m] = v[i1[f] * 3 + m] - v[i0[f] * 3 + m];
      e2[m] = v[i2[f] * 3 + m] - v[i0[f] * 3 + m];
    }
    d_cross(e1, e2, ns);
    const double sJ = 0.25 * sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    T* gf = gface + e * d::NGF + 4 * f;
    for (int m = 0; m < 3; ++m) gf[m] = (T)(0.25 * ns[m] / sJ);
    gf[3] = (T)sJ;
  }
  for (int n = threadIdx.x; n < d::Np; n += blockDim.x) {
    int k, j, i;
    decode_mode(n, k, j, i);
    const double J = d_jacobian(v, gtab[G.XL + tri_num(k) + i], gtab[G.XL + tri_num(k) + j]);
    invM[e * d::Np + n] = (T)(gtab[G.IMR + n] / J);
  }
}

// ============================================================ trace (a2)
// u^f = V^f u at all 5(N+1)^2 face points for the four fields; the output
// tr[(e*Nfc + g)*4 + field] feeds the neighbours' flux in the next kernel.
template <int N, typename T>
struct TraceSmem {
  using d = Dims<N>;
  static constexpr int nB = d::n2 + 4 * d::n1;  // base grid + 4 face rows per level
  static constexpr size_t tab = 0;
  static constexpr size_t u = tab + TabLayout(N).size;
  static constexpr size_t A = u + 4 * d::Np;
  static constexpr size_t B = A + 4 * d::nrow * d::P3;
  static constexpr size_t total = B + 4 * d::n1 * nB;
  static constexpr size_t bytes = total * sizeof(T);
};

// The passes of the trace interpolation for one element: s_u holds its 4 Np
// coefficients, s_A (4 nrow P3) and s_B (4 n1 (n2 + 4 n1)) are scratch, and the
// 4 Nfc trace values go to tr_e[g*4 + f].
template <int N, typename T>
__device__ __forceinline__ void trace_passes(const T* s_tab, const T* s_u, T* s_A, T* s_B, T* __restrict__ tr_e,
                                             int tid, int nthr) {
  using d = Dims<N>;
  using S = TraceSmem<N, T>;
  constexpr TabLayout L(N);
  // a pass: A[f][row(k,j)][p'] = sum_i l_i^k(x_p') u[f][k][j][i], p' over GL points and -1, +1.
  // Work items run level-major so that a warp's lanes share the trip count k+1.
  // The level-N nodes are the volume-rule points (l_i^N(x_p) = delta_ip), so level N at
  // the volume columns is a copy; those items come last, apart from the summing ones.
  constexpr int nLow = 4 * d::P3 * tri_num(N);       // levels below N, all columns
  constexpr int nSum = nLow + 4 * (N + 1) * 2;       // + level N at a = -1, +1
  for (int x = tid; x < 4 * d::nrow * d::P3; x += nthr) {
    int k, f, j, pp;
    if (x < nLow) {
      k = 0;
      while (x >= 4 * d::P3 * tri_num(k + 1)) ++k;
      const int rem = x - 4 * d::P3 * tri_num(k);
      f = rem / ((k + 1) * d::P3);
      j = (rem / d::P3) % (k + 1);
      pp = rem % d::P3;
    } else if (x < nSum) {
      const int rem = x - nLow;
      k = N;
      f = rem / (2 * (N + 1));
      j = (rem / 2) % (N + 1);
      pp = d::n1 + rem % 2;
    } else {
      const int rem = x - nSum;
      k = N;
      f = rem / ((N + 1) * d::n1);
      j = (rem / d::n1) % (N + 1);
      pp = rem % d::n1;
    }
    const T* uc = s_u + f * d::Np + lvl_off(k) + j * (k + 1);
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + pp;
    T acc = 0;
    if (x >= nSum)
      acc = uc[pp];
    else
      for (int i = 0; i <= k; ++i) acc += uc[i] * lx[i * d::P3];
    s_A[(f * d::nrow + tri_num(k) + j) * d::P3 + pp] = acc;
  }
  __syncthreads();
  // b pass per level k: base grid (p,q) and the four triangle-face rows
  // Level-major (equal trip counts within a warp). At level N, l_j^N is the identity on
  // the b points: only the b = -1, +1 rows sum; the base grid and the a = -1, +1 rows are
  // copies, taken last.
  constexpr int bLow = 4 * N * S::nB;                // levels below N
  constexpr int bSum = bLow + 4 * 2 * d::n1;         // + level N, faces b = -1, +1
  for (int x = tid; x < 4 * d::n1 * S::nB; x += nthr) {
    int s, f, k;
    if (x < bLow) {
      s = x % S::nB;
      const int t = x / S::nB;
      f = t % 4;
      k = t / 4;
    } else if (x < bSum) {
      const int rem = x - bLow;
      k = N;
      f = rem / (2 * d::n1);
      s = d::n2 + rem % (2 * d::n1);
    } else {
      const int rem = x - bSum;
      k = N;
      f = rem / (d::n2 + 2 * d::n1);
      s = rem % (d::n2 + 2 * d::n1);
      if (s >= d::n2) s += 2 * d::n1;  // skip the b = -1, +1 rows
    }
    int pa, qb;  // A column (a point) and l^k_j evaluation column (b point)
    if (s < d::n2) {
      pa = s % d::n1;
      qb = s / d::n1;
    } else {
      const int slot = (s - d::n2) / d::n1, ee = (s - d::n2) % d::n1;
      // slot 0: b=-1 (face 1), 1: b=+1 (face 3), 2: a=-1 (face 4), 3: a=+1 (face 2)
      if (slot < 2) {
        pa = ee;
        qb = d::n1 + slot;
      } else {
        pa = d::n1 + (slot - 2);
        qb = ee;
      }
    }
    const T* Ar = s_A + (f * d::nrow + tri_num(k)) * d::P3 + pa;
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + qb;
    T acc = 0;
    if (x >= bSum)  // l_j^N(b_q) = delta_jq
      acc = Ar[qb * d::P3];
    else
      for (int j = 0; j <= k; ++j) acc += Ar[j * d::P3] * lx[j * d::P3];
    s_B[(f * d::n1 + k) * S::nB + s] = acc;
  }
  __syncthreads();
  // c pass: sum over levels with G_k(-1) (base) or G_k(c_m) (triangles)
  // One code path for both kinds of face (only the weight row and the column differ), so
  // that a warp holding base and triangle points runs the sums once.
  for (int g = tid; g < d::Nfc; g += nthr) {
    const int face = g / d::n2, idx = g % d::n2;
    const T* cw;  // weights of levels k = 0..N at stride cs
    int cs, col;  // s_B column
    if (face == 0) {
      cw = s_tab + L.GB;
      cs = 1;
      col = idx;
    } else {
      const int ee = idx % d::n1, m = idx / d::n1;
      const int slot = face == 1 ? 0 : face == 3 ? 1 : face == 4 ? 2 : 3;
      cw = s_tab + L.GF + m;
      cs = d::n1;
      col = d::n2 + slot * d::n1 + ee;
    }
    T out[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k <= N; ++k) acc += cw[k * cs] * s_B[(f * d::n1 + k) * S::nB + col];
      out[f] = acc;
    }
    T* dst = tr_e + g * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) dst[f] = out[f];
  }
}

template <int N, typename T>
__global__ void __launch_bounds__(KCfg<N>::NT) trace_kernel(int64_t K, const T* __restrict__ q,
                                                            const T* __restrict__ tab, T* __restrict__ tr) {
  using d = Dims<N>;
  using S = TraceSmem<N, T>;
  constexpr TabLayout L(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* s_tab = sm + S::tab;
  T* s_u = sm + S::u;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  // the passes read LX, GB and GF only (GF follows GB in the table)
  static_assert(L.LX == 0 && L.GF == L.GB + d::n1, "trace table ranges");
  for (int x = tid; x < d::nrow * d::P3; x += blockDim.x) s_tab[x] = tab[x];
  for (int x = L.GB + tid; x < L.GF + d::n2; x += blockDim.x) s_tab[x] = tab[x];
  for (int x = tid; x < 4 * d::Np; x += blockDim.x) s_u[x] = q[e * 4 * d::Np + x];
  __syncthreads();
  trace_passes<N, T>(s_tab, s_u, sm + S::A, sm + S::B, tr + e * d::Nfc * 4, tid, blockDim.x);
}

// ===================================================== rhs / update (a3-a7)
template <int N, typename T>
struct RhsSmem {
  using d = Dims<N>;
  static constexpr int nY = d::P3 * d::P3;
  static constexpr size_t tab = 0;
  static constexpr size_t u = tab + TabLayout(N).size;
  static constexpr size_t geo = u + 4 * d::Np;
  static constexpr size_t gf = geo + d::NGEO * d::n2;
  static constexpr size_t Fs = gf + d::NGF;
  static constexpr size_t A = Fs + 4 * d::Nfc;
  static constexpr size_t dA = A + 4 * d::nrow * d::n1;
  static constexpr size_t U = dA + 4 * d::nrow * d::n1;
  static constexpr size_t Ua = U + 4 * d::n1 * d::n2;
  static constexpr size_t Ub = Ua + 4 * d::n1 * d::n2;
  static constexpr size_t Y = Ub + 4 * d::n1 * d::n2;
  static constexpr size_t total = Y + 4 * d::n1 * nY;
  // A/dA are dead after the b pass: the div combination X, Z and later the
  // b^T output reuse their space.
  static constexpr size_t X = A;
  static constexpr size_t Zc = X + d::n1 * d::n2;
  static constexpr size_t Zb = A;
  static_assert(2 * d::n1 * d::n2 <= 8 * d::nrow * d::n1, "X/Z overflow the A region");
  static_assert(4 * d::nrow * d::P3 <= 8 * d::nrow * d::n1, "b^T output overflows the A region");
  static constexpr size_t bytes = total * sizeof(T);
};

// Surface flux of Sec. 4.3 at one face point, scaled by weight * sJ:
// F_p = 1/2 (n.[[u]] - tau [[p]]), F_u = 1/2 n ([[p]] - tau n.[[u]]).
template <typename T>
__device__ __forceinline__ void face_flux(const T* um, const T* up_in, bool boundary, int bc, T tau, const T* n,
                                          T ws, T* F) {
  T up[4];
  if (!boundary) {
    up[0] = up_in[0];
    up[1] = up_in[1];
    up[2] = up_in[2];
    up[3] = up_in[3];
  } else if (bc == 0) {  // wall: mirror the normal velocity
    const T un = n[0] * um[1] + n[1] * um[2] + n[2] * um[3];
    up[0] = um[0];
    up[1] = um[1] - 2 * un * n[0];
    up[2] = um[2] - 2 * un * n[1];
    up[3] = um[3] - 2 * un * n[2];
  } else {  // free surface p = 0
    up[0] = -um[0];
    up[1] = um[1];
    up[2] = um[2];
    up[3] = um[3];
  }
  const T dp = up[0] - um[0];
  const T nd = n[0] * (up[1] - um[1]) + n[1] * (up[2] - um[2]) + n[2] * (up[3] - um[3]);
  const T hp = T(0.5) * ws * (nd - tau * dp);
  const T hu = T(0.5) * ws * (dp - tau * nd);
  F[0] = hp;
  F[1] = hu * n[0];
  F[2] = hu * n[1];
  F[3] = hu * n[2];
}

// Transposed passes shared by the rhs and projection kernels: from point
// data Fv[f][r*n2 + pq] (already weighted) and face data Fs[f][g] (already
// weighted; may be null) to the projections sum_q phi_n(x_q) F_q into out.
template <int N, typename T>
__device__ __forceinline__ void project_passes(const T* s_tab, const T* Fv, const T* Fs, T* Y, T* Z, int tid,
                                               int nthr) {
  using d = Dims<N>;
  constexpr TabLayout L(N);
  constexpr int nY = d::P3 * d::P3;
  constexpr int nS = d::n2 + 4 * d::n1;
  // c^T pass: Y[f][k][p'][q']
  for (int x = tid; x < 4 * d::n1 * nS; x += nthr) {
    const int s = x % nS;
    const int t = x / nS;
    const int k = t % d::n1, f = t / d::n1;
    T* Yk = Y + (f * d::n1 + k) * nY;
    if (s < d::n2) {
      const int p = s % d::n1, q = s / d::n1;
      const T* fv = Fv + f * d::Nc + s;
      const T* gc = s_tab + L.GC + k * d::n1;
      T acc = 0;
      for (int r = 0; r < d::n1; ++r) acc += gc[r] * fv[r * d::n2];
      if (Fs) acc += s_tab[L.GB + k] * Fs[f * d::Nfc + s];
      Yk[p * d::P3 + q] = acc;
    } else if (Fs) {
      const int slot = (s - d::n2) / d::n1, ee = (s - d::n2) % d::n1;
      const int face = slot == 0 ? 1 : slot == 1 ? 3 : slot == 2 ? 4 : 2;
      const T* fs = Fs + f * d::Nfc + face * d::n2 + ee;
      const T* gfk = s_tab + L.GF + k * d::n1;
      T acc = 0;
      for (int m = 0; m < d::n1; ++m) acc += gfk[m] * fs[m * d::n1];
      if (slot < 2)
        Yk[ee * d::P3 + d::n1 + slot] = acc;  // b = -1, +1 columns
      else
        Yk[(d::n1 + slot - 2) * d::P3 + ee] = acc;  // a = -1, +1 rows
    }
  }
  __syncthreads();
  // b^T pass: Z[f][row(k,j)][p'] = sum_q' l_j^k(x_q') Y[f][k][p'][q']
  const int nq_main = Fs ? d::P3 : d::n1;
  const int np_out = Fs ? d::P3 : d::n1;
  for (int x = tid; x < 4 * d::nrow * np_out; x += nthr) {
    const int pp = x % np_out;
    const int t = x / np_out;
    const int row = t % d::nrow, f = t / d::nrow;
    int k, j;
    decode_row(row, k, j);
    const T* Yr = Y + ((f * d::n1 + k) * d::P3 + pp) * d::P3;
    const T* lx = s_tab + L.LX + (tri_num(k) + j) * d::P3;
    const int nq = pp < d::n1 ? nq_main : d::n1;
    T acc = 0;
    for (int q = 0; q < nq; ++q) acc += lx[q] * Yr[q];
    Z[(f * d::nrow + row) * d::P3 + pp] = acc;
  }
  __syncthreads();
}

// Volume passes of the rhs (a3 with the base-face lift of a5): from the coefficients s_u and
// the weighted face fluxes s_Fs (written before the call; the first barrier below orders
// them) to s_Zb, the b^T output the a^T pass reads. Shared by the modal stage kernel and the
// nodal one; TRI_LIFT = false leaves the triangle-face rows and columns of Y zero (the nodal
// kernel lifts its triangle faces with face mass matrices instead).
template <int N, typename T, bool TRI_LIFT>
__device__ __forceinline__ void volume_passes(const T* s_tab, const T* s_u, const T* s_geo, const T* s_Fs, T* s_A,
                                              T* s_dA, T* s_U, T* s_Ua, T* s_Ub, T* s_Y, T* s_X, T* s_Zc, T* s_Zb,
                                              int tid, int nthr) {
  using d = Dims<N>;
  constexpr TabLayout L(N);
  constexpr int nY = d::P3 * d::P3;
  // a pass, level-major: A = l^k(a_p) u, dA = l^k'(a_p) u. Levels run in the order
  // 1..N-1, 0, N: the warp that straddles into level N's short form then also holds
  // the cheapest level.
  constexpr int aLow = 4 * d::n1 * (tri_num(N) - 1);  // items of levels 1..N-1
  for (int x = tid; x < 4 * d::nrow * d::n1; x += nthr) {
    int k, rem;
    if (x < aLow) {
      const int y = x + 4 * d::n1;
      k = 1;
      while (y >= 4 * d::n1 * tri_num(k + 1)) ++k;
      rem = y - 4 * d::n1 * tri_num(k);
    } else if (x < aLow + 4 * d::n1) {
      k = 0;
      rem = x - aLow;
    } else {
      k = N;
      rem = x - 4 * d::n1 * tri_num(N);
    }
    const int f = rem / ((k + 1) * d::n1);
    const int j = (rem / d::n1) % (k + 1);
    const int p = rem % d::n1;
    const T* uc = s_u + f * d::Np + lvl_off(k) + j * (k + 1);
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + p;
    const T* dl = s_tab + L.DL + tri_num(k) * d::n1 + p;
    T a = 0, da = 0;
    if (k == N) {  // the level-N nodes are the volume-rule points: l_i^N(a_p) = delta_ip
      a = uc[p];
      for (int i = 0; i <= k; ++i) da += uc[i] * dl[i * d::n1];
    } else {
      for (int i = 0; i <= k; ++i) {
        a += uc[i] * lx[i * d::P3];
        da += uc[i] * dl[i * d::n1];
      }
    }
    const int o = (f * d::nrow + tri_num(k) + j) * d::n1 + p;
    s_A[o] = a;
    s_dA[o] = da;
  }
  __syncthreads();
  // b pass, level-major: U_k, (d_a U)_k, (d_b U)_k on the (a_p, b_q) grid
  for (int x = tid; x < 4 * d::n1 * d::n2; x += nthr) {
    const int pq = x % d::n2;
    const int t = x / d::n2;
    const int f = t % 4, k = t / 4;
    const int p = pq % d::n1, q = pq / d::n1;
    const T* Ar = s_A + (f * d::nrow + tri_num(k)) * d::n1 + p;
    const T* dAr = s_dA + (f * d::nrow + tri_num(k)) * d::n1 + p;
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + q;
    const T* dl = s_tab + L.DL + tri_num(k) * d::n1 + q;
    T u = 0, ua = 0, ub = 0;
    if (k == N) {  // l_j^N(b_q) = delta_jq
      u = Ar[q * d::n1];
      ua = dAr[q * d::n1];
      for (int j = 0; j <= k; ++j) ub += Ar[j * d::n1] * dl[j * d::n1];
    } else {
      for (int j = 0; j <= k; ++j) {
        const T av = Ar[j * d::n1], lv = lx[j * d::P3];
        u += av * lv;
        ub += av * dl[j * d::n1];
        ua += dAr[j * d::n1] * lv;
      }
    }
    const int o = (f * d::n1 + k) * d::n2 + pq;
    s_U[o] = u;
    s_Ua[o] = ua;
    s_Ub[o] = ub;
  }
  __syncthreads();
  // div(u) needs only sum_m J d(u_m)/dx_m = sum_m (u_r^m g1_m + u_s^m g2_m + u_c^m g3_m); the
  // factors do not depend on c, so combine the fields per level before the c direction.
  for (int x = tid; x < d::n1 * d::n2; x += nthr) {
    const int pq = x % d::n2, k = x / d::n2;
    const T* g = s_geo + pq * d::NGEO;
    T xs = 0, zs = 0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int o = ((m + 1) * d::n1 + k) * d::n2 + pq;
      xs = fma(g[m], s_Ua[o], fma(g[3 + m], s_Ub[o], xs));  // two FMAs, no separate multiply and add
      zs = fma(g[6 + m], s_U[o], zs);
    }
    s_X[x] = xs;
    s_Zc[x] = zs;
  }
  __syncthreads();
  // c direction of the volume term (Alg. 1) as level mixing: the projection onto level k'
  // of the weighted derivatives, sum_r WC G_k'(c_r) (...)(c_r), is MH / MG applied to the
  // level values at each (a_p, b_q). Base-face lift (c = -1) joins here; the triangle
  // faces fill the extra rows/columns of Y.
  for (int x = tid; x < d::n1 * d::n2 + 4 * d::n1 * 4 * d::n1; x += nthr) {
    if (x < d::n1 * d::n2) {
      const int pq = x % d::n2, kp = x / d::n2;
      const int p = pq % d::n1, q = pq / d::n1;
      const T* mh = s_tab + L.MH + kp * d::n1;
      const T* mg = s_tab + L.MG + kp * d::n1;
      T al = 0, be = 0, ga = 0, dv = 0;
      // MG is lower Hessenberg (k <= k'+1), MH tridiagonal (|k - k'| <= 1)
      const int k1 = kp < N ? kp + 1 : N;
      for (int k = 0; k <= k1; ++k) {
        const int o = k * d::n2 + pq;  // field 0 (p)
        ga += mg[k] * s_U[o];
        dv += mg[k] * s_Zc[o];
      }
      for (int k = kp > 0 ? kp - 1 : 0; k <= k1; ++k) {
        const int o = k * d::n2 + pq;
        al += mh[k] * s_Ua[o];
        be += mh[k] * s_Ub[o];
        dv += mh[k] * s_X[o];
      }
      const T* g = s_geo + pq * d::NGEO;
      const T gb = s_tab[L.GB + kp];
      const int yo = kp * nY + p * d::P3 + q;
      s_Y[0 * d::n1 * nY + yo] = dv + gb * s_Fs[0 * d::Nfc + pq];
#pragma unroll
      for (int m = 0; m < 3; ++m)
        s_Y[(m + 1) * d::n1 * nY + yo] =
            g[m] * al + g[3 + m] * be + g[6 + m] * ga + gb * s_Fs[(m + 1) * d::Nfc + pq];
    } else {
      const int y = x - d::n1 * d::n2;
      const int ee = y % d::n1;
      const int slot = (y / d::n1) % 4;
      const int f = (y / (4 * d::n1)) % 4;
      const int k = y / (16 * d::n1);
      const int face = slot == 0 ? 1 : slot == 1 ? 3 : slot == 2 ? 4 : 2;
      const T* fs = s_Fs + f * d::Nfc + face * d::n2 + ee;
      const T* gfk = s_tab + L.GF + k * d::n1;
      T acc = 0;
      if (TRI_LIFT) {
#pragma unroll
        for (int m = 0; m <= N; ++m) acc += gfk[m] * fs[m * d::n1];
      }
      T* Yk = s_Y + (f * d::n1 + k) * nY;
      if (slot < 2)
        Yk[ee * d::P3 + d::n1 + slot] = acc;  // b = -1, +1 columns
      else
        Yk[(d::n1 + slot - 2) * d::P3 + ee] = acc;  // a = -1, +1 rows
    }
  }
  __syncthreads();
  // b^T pass: Z[f][row(k,j)][p'] = sum_q' l_j^k(x_q') Y[f][k][p'][q']; the items with
  // p' on the (a) grid sum N+3 terms, the two face rows N+1 terms; they are kept apart.
  constexpr int nMain = 4 * d::nrow * d::n1;
  for (int x = tid; x < 4 * d::nrow * d::P3; x += nthr) {
    int row, f, pp, nq;
    if (x < nMain) {
      pp = x % d::n1;
      f = (x / d::n1) % 4;
      row = x / (4 * d::n1);
      nq = d::P3;
    } else {
      const int y = x - nMain;
      pp = d::n1 + y % 2;
      f = (y / 2) % 4;
      row = y / 8;
      nq = d::n1;
    }
    int k, j;
    decode_row(row, k, j);
    const T* Yr = s_Y + ((f * d::n1 + k) * d::P3 + pp) * d::P3;
    const T* lx = s_tab + L.LX + (tri_num(k) + j) * d::P3;
    T acc = 0;
    if (k == N) {  // l_j^N(x_q) = delta_jq on the volume points; the face columns remain
      acc = Yr[j];
      for (int q = d::n1; q < nq; ++q) acc += lx[q] * Yr[q];
    } else {
      for (int q = 0; q < nq; ++q) acc += lx[q] * Yr[q];
    }
    s_Zb[(f * d::nrow + row) * d::P3 + pp] = acc;
  }
  __syncthreads();
}

template <int N, typename T, bool UPDATE>
__global__ void __launch_bounds__(KCfg<N>::NT)
    rhs_kernel(int64_t K, const T* qin, T* qout, T* __restrict__ res,  // qin == qout when updating in place
               const T* __restrict__ tr, const int32_t* __restrict__ mapP, const T* __restrict__ geo,
               const T* __restrict__ gface, const T* __restrict__ invM, const T* __restrict__ tab, int bc, T tau,
               T rka, T rkb, T dt, const T* __restrict__ dt_elem) {
  using d = Dims<N>;
  using S = RhsSmem<N, T>;
  constexpr TabLayout L(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* s_tab = sm + S::tab;
  T* s_u = sm + S::u;
  T* s_geo = sm + S::geo;
  T* s_gf = sm + S::gf;
  T* s_Fs = sm + S::Fs;
  T* s_A = sm + S::A;
  T* s_dA = sm + S::dA;
  T* s_U = sm + S::U;
  T* s_Ua = sm + S::Ua;
  T* s_Ub = sm + S::Ub;
  T* s_Y = sm + S::Y;
  T* s_X = sm + S::X;
  T* s_Zc = sm + S::Zc;
  T* s_Zb = sm + S::Zb;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;

  for (int x = tid; x < L.size; x += nthr) s_tab[x] = tab[x];
  for (int x = tid; x < 4 * d::Np; x += nthr) s_u[x] = qin[e * 4 * d::Np + x];
  for (int x = tid; x < d::NGEO * d::n2; x += nthr) s_geo[x] = geo[e * d::NGEO * d::n2 + x];
  for (int x = tid; x < d::NGF; x += nthr) s_gf[x] = gface[e * d::NGF + x];
  __syncthreads();

  // surface flux at every face point (a4), weighted by w sJ
  for (int g = tid; g < d::Nfc; g += nthr) {
    const int face = g / d::n2, idx = g % d::n2;
    const int64_t gl = e * d::Nfc + g;
    const int64_t gn = mapP[gl];
    T um[4], up[4], F[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      um[f] = tr[gl * 4 + f];
      up[f] = tr[gn * 4 + f];
    }
    const T* nv = face == 0 ? s_gf + 16 + 4 * idx : s_gf + 4 * (face - 1);
    const T w = face == 0 ? s_tab[L.WB + idx] : s_tab[L.WFT + idx];
    face_flux<T>(um, up, gn == gl, bc, tau, nv, w * nv[3], F);
#pragma unroll
    for (int f = 0; f < 4; ++f) s_Fs[f * d::Nfc + g] = F[f];
  }
  volume_passes<N, T, true>(s_tab, s_u, s_geo, s_Fs, s_A, s_dA, s_U, s_Ua, s_Ub, s_Y, s_X, s_Zc, s_Zb, tid, nthr);
  // a^T pass, M^{-1} (a6), LSRK stage (a7). Items run level-major (k, f, j, i) so that
  // a warp's lanes share a level: level N takes the short form below.
  for (int y = tid; y < 4 * d::Np; y += nthr) {
    int k = 0;
    while (y >= 4 * lvl_off(k + 1)) ++k;
    const int rem = y - 4 * lvl_off(k);
    const int f = rem / ((k + 1) * (k + 1));
    const int n = lvl_off(k) + rem % ((k + 1) * (k + 1));
    const int j = (n - lvl_off(k)) / (k + 1), i = (n - lvl_off(k)) % (k + 1);
    const int x = f * d::Np + n;
    const T* lx = s_tab + L.LX + (tri_num(k) + i) * d::P3;
    const T* Zr = s_Zb + (f * d::nrow + tri_num(k) + j) * d::P3;
    T acc = 0;
    if (k == N) {  // l_i^N(x_p') = delta_ip' on the volume points; the face columns remain
      acc = Zr[i] + lx[d::n1] * Zr[d::n1] + lx[d::n1 + 1] * Zr[d::n1 + 1];
    } else {
#pragma unroll
      for (int pp = 0; pp < d::P3; ++pp) acc += lx[pp] * Zr[pp];
    }
    const T rhs = -invM[e * d::Np + n] * acc;
    const int64_t gi = e * 4 * d::Np + x;
    if (UPDATE) {
      const T dte = dt_elem ? dt_elem[e] : dt;  // per-element step when meshes are batched
      const T rnew = rka * res[gi] + dte * rhs;
      res[gi] = rnew;
      qout[gi] = s_u[x] + rkb * rnew;
    } else {
      qout[gi] = rhs;
    }
  }
}

// ============================================================ projection
// L2 projection of the exact standing wave at time t (double arithmetic):
// coefficient = M^{-1} sum_q w_q J_q phi_n(x_q) U_exact(x_q).
template <int N>
struct ProjSmem {
  using d = Dims<N>;
  static constexpr size_t tab = 0;
  static constexpr size_t Fv = tab + TabLayout(N).size;
  static constexpr size_t Y = Fv + 4 * d::Nc;
  static constexpr size_t Z = Y + 4 * d::n1 * d::P3 * d::P3;
  static constexpr size_t total = Z + 4 * d::nrow * d::P3;
  static constexpr size_t bytes = total * sizeof(double);
};

template <int N, typename T>
__global__ void __launch_bounds__(KCfg<N>::NT)
    project_kernel(int64_t K, const double* __restrict__ ev, const double* __restrict__ gtab,
                   const double* __restrict__ tabd, int bc, double t, T* __restrict__ qout) {
  using d = Dims<N>;
  using S = ProjSmem<N>;
  constexpr TabLayout L(N);
  constexpr GeoLayout G(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* s_tab = sm + S::tab;
  double* s_Fv = sm + S::Fv;
  double* s_Y = sm + S::Y;
  double* s_Z = sm + S::Z;
  __shared__ double v[15];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int x = tid; x < L.size; x += nthr) s_tab[x] = tabd[x];
  if (tid < 15) v[tid] = ev[e * 15 + tid];
  __syncthreads();
  double ct, st;
  d_time_factors(bc, t, &ct, &st);
  // B(a,b) and w_p w_q J(a,b) once per (a,b) point, parked in the Y region until the c^T pass
  double* s_XB = s_Y;
  for (int pq = tid; pq < d::n2; pq += nthr) {
    const int p = pq % d::n1, q = pq / d::n1;
    const double a = gtab[G.XG + p], b = gtab[G.XG + q];
    double B[3], Ba[3], Bb[3];
    d_bilinear(v, a, b, B, Ba, Bb);
    s_XB[4 * pq + 0] = B[0];
    s_XB[4 * pq + 1] = B[1];
    s_XB[4 * pq + 2] = B[2];
    s_XB[4 * pq + 3] = gtab[G.WG + p] * gtab[G.WG + q] * d_jacobian(v, a, b);
  }
  __syncthreads();
  for (int x = tid; x < d::Nc; x += nthr) {
    const int pq = x % d::n2, r = x / d::n2;
    const double c = gtab[G.XC + r];
    const double* xb = s_XB + 4 * pq;
    double X[3], U[4];
    for (int m = 0; m < 3; ++m) X[m] = 0.5 * (1 - c) * xb[m] + 0.5 * (1 + c) * v[12 + m];
    const double w = xb[3] * gtab[G.WC4 + r];
    d_exact(bc, X[0], X[1], X[2], ct, st, U);
    for (int f = 0; f < 4; ++f) s_Fv[f * d::Nc + x] = w * U[f];
  }
  __syncthreads();
  project_passes<N, double>(s_tab, s_Fv, nullptr, s_Y, s_Z, tid, nthr);
  for (int x = tid; x < 4 * d::Np; x += nthr) {
    const int f = x / d::Np, n = x % d::Np;
    int k, j, i;
    decode_mode(n, k, j, i);
    const double* lx = s_tab + L.LX + (tri_num(k) + i) * d::P3;
    const double* Zr = s_Z + (f * d::nrow + tri_num(k) + j) * d::P3;
    double acc = 0;
    for (int pp = 0; pp < d::n1; ++pp) acc += lx[pp] * Zr[pp];
    const double J = d_jacobian(v, gtab[G.XL + tri_num(k) + i], gtab[G.XL + tri_num(k) + j]);
    qout[e * 4 * d::Np + x] = (T)(acc * gtab[G.IMR + n] / J);
  }
}

// ============================================================ error norm (a8)
// sum over elements and (N+3)^3 points of w J |U_h - U_exact|^2 and w J |U_exact|^2,
// in double; grid-stride over elements, one partial pair per block. The base map
// B(a,b) and J(a,b) do not depend on c, so they are computed once per (a,b) point.
template <int N>
struct ErrCfg {
  static constexpr int Q = N + 3;
  static constexpr int pts = Q * Q * Q;
  static constexpr int iters = (pts + 511) / 512;
  static constexpr int NT = (((pts + iters - 1) / iters) + 31) / 32 * 32;
};

template <int N>
struct ErrSmem {
  using d = Dims<N>;
  static constexpr int Q = d::Q;
  static constexpr size_t u = 0;
  static constexpr size_t A = u + 4 * d::Np;
  static constexpr size_t B = A + 4 * d::nrow * Q;
  static constexpr size_t LQ = B + 4 * d::n1 * Q * Q;
  static constexpr size_t GQ = LQ + d::nrow * Q;
  static constexpr size_t XB = GQ + d::n1 * Q;  // per (a,b) point: B(a,b) and w_p w_q J(a,b)
  // per (a,b) point and coordinate m: sin, cos of pi sc alpha_m and pi sc beta_m, where
  // x_m(c) = alpha_m + beta_m c along the c line through (a, b)
  static constexpr size_t TS = XB + 4 * Q * Q;
  static constexpr size_t total = TS + 9 * Q * Q;
  static constexpr size_t bytes = total * sizeof(double);
};

template <int N, typename T>
__global__ void __launch_bounds__(ErrCfg<N>::NT)
    error_kernel(int64_t K, const T* __restrict__ q, const double* __restrict__ ev, const double* __restrict__ gtab,
                 int bc, double t, double* __restrict__ partial) {
  using d = Dims<N>;
  using S = ErrSmem<N>;
  constexpr GeoLayout G(N);
  constexpr int Q = d::Q;
  constexpr int NW = ErrCfg<N>::NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* s_u = sm + S::u;
  double* s_A = sm + S::A;
  double* s_B = sm + S::B;
  double* s_LQ = sm + S::LQ;
  double* s_GQ = sm + S::GQ;
  double* s_XB = sm + S::XB;
  double* s_TS = sm + S::TS;
  __shared__ double v[15];
  __shared__ double red[2][NW];
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int x = tid; x < d::nrow * Q; x += nthr) s_LQ[x] = gtab[G.LQ + x];
  for (int x = tid; x < d::n1 * Q; x += nthr) s_GQ[x] = gtab[G.GQ + x];
  double e2 = 0.0, n2 = 0.0;
  double ct, st;
  d_time_factors(bc, t, &ct, &st);
  const double sc = bc == 0 ? 1.0 : 0.5;  // the exact fields are trigonometric in pi sc x
  for (int64_t e = blockIdx.x; e < K; e += gridDim.x) {
    __syncthreads();
    for (int x = tid; x < 4 * d::Np; x += nthr) s_u[x] = (double)q[e * 4 * d::Np + x];
    if (tid < 15) v[tid] = ev[e * 15 + tid];
    __syncthreads();
    for (int x = tid; x < Q * Q; x += nthr) {
      const int p = x % Q, qq = x / Q;
      double B[3], Ba[3], Bb[3], D[3], g1[3];
      d_bilinear(v, gtab[G.XQ + p], gtab[G.XQ + qq], B, Ba, Bb);
      for (int m = 0; m < 3; ++m) D[m] = 0.5 * (v[12 + m] - B[m]);
      d_cross(Bb, D, g1);
      s_XB[4 * x + 0] = B[0];
      s_XB[4 * x + 1] = B[1];
      s_XB[4 * x + 2] = B[2];
      s_XB[4 * x + 3] = gtab[G.WQ + p] * gtab[G.WQ + qq] * (Ba[0] * g1[0] + Ba[1] * g1[1] + Ba[2] * g1[2]);
      for (int m = 0; m < 3; ++m) {
        const double alpha = 0.5 * (B[m] + v[12 + m]);
        sincospi(sc * alpha, &s_TS[9 * x + m], &s_TS[9 * x + 3 + m]);
        s_TS[9 * x + 6 + m] = 3.14159265358979323846 * sc * D[m];  // pi sc beta_m (beta = (v5 - B)/2 = D)
      }
    }
    for (int x = tid; x < 4 * d::nrow * Q; x += nthr) {  // a pass, level-major
      int k = 0;
      while (x >= 4 * Q * tri_num(k + 1)) ++k;
      const int rem = x - 4 * Q * tri_num(k);
      const int f = rem / ((k + 1) * Q);
      const int j = (rem / Q) % (k + 1);
      const int p = rem % Q;
      const double* uc = s_u + f * d::Np + lvl_off(k) + j * (k + 1);
      const double* lq = s_LQ + tri_num(k) * Q + p;
      double acc = 0;
      for (int i = 0; i <= k; ++i) acc += uc[i] * lq[i * Q];
      s_A[(f * d::nrow + tri_num(k) + j) * Q + p] = acc;
    }
    __syncthreads();
    for (int x = tid; x < 4 * d::n1 * Q * Q; x += nthr) {  // b pass, level-major
      const int pq = x % (Q * Q);
      const int tt = x / (Q * Q);
      const int f = tt % 4, k = tt / 4;
      const int p = pq % Q, qq = pq / Q;
      const double* Ar = s_A + (f * d::nrow + tri_num(k)) * Q + p;
      const double* lq = s_LQ + tri_num(k) * Q + qq;
      double acc = 0;
      for (int j = 0; j <= k; ++j) acc += Ar[j * Q] * lq[j * Q];
      s_B[(f * d::n1 + k) * Q * Q + pq] = acc;
    }
    __syncthreads();
    for (int x = tid; x < Q * Q * Q; x += nthr) {  // c pass and the error integrand
      const int pq = x % (Q * Q), r = x / (Q * Q);
      const double c = gtab[G.XQC + r];
      const double* xb = s_XB + 4 * pq;
      const double* ts = s_TS + 9 * pq;
      double sn[3], cs[3], Ue[4];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        // pi sc x_m = pi sc alpha_m + eps with eps = pi sc beta_m c: on fine meshes eps is small
        // and one angle addition replaces the sincospi of every point
        const double eps = ts[6 + m] * c;
        if (fabs(eps) <= 0.1)
          d_sincos_shift(ts[m], ts[3 + m], eps, &sn[m], &cs[m]);
        else
          sincospi(sc * (0.5 * (1 - c) * xb[m] + 0.5 * (1 + c) * v[12 + m]), &sn[m], &cs[m]);
      }
      d_exact_sc(sn, cs, ct, st, Ue);
      const double w = xb[3] * gtab[G.WQC + r];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        double uh = 0;
#pragma unroll
        for (int k = 0; k <= N; ++k) uh += s_GQ[k * Q + r] * s_B[(f * d::n1 + k) * Q * Q + pq];
        const double df = uh - Ue[f];
        e2 += w * df * df;
        n2 += w * Ue[f] * Ue[f];
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e2 += __shfl_down_sync(0xffffffffu, e2, off);
    n2 += __shfl_down_sync(0xffffffffu, n2, off);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = e2;
    red[1][tid >> 5] = n2;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NW; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}


// ============================================================ error norm from coefficients (a8)
// The exact standing wave is S_p(x) tp(t) for p and S_m(x) tu(t) for the velocities, with
// S_p = cos cos cos and S_u, S_v, S_w one sine each (of pi sc x, pi sc y, pi sc z), and
// tp = cos(sqrt3 pi sc t), tu = sin(sqrt3 pi sc t)/sqrt3. Write <.,.>_Q for the error rule's
// inner product ((N+3)-point rules) and P for the <.,.>_Q-orthogonal projection onto one
// element's polynomial space. The rule integrates the mass matrix exactly, so under it M is
// the diagonal of Lemma 3. With U_h in that space, U_h - P U_ex is orthogonal to
// P U_ex - U_ex, hence per field
//   |U_h - U_ex|_Q^2 = sum_i M_ii (u_i - T s_i)^2 + T^2 |P S - S|_Q^2,
// s = coefficients of P S, T = tp or tu. The second term and |S|_Q^2 do not depend on t.
// exact_proj_kernel computes, once per handle: s (shat[e][f][n]), M_ii (Mdiag[e][n]) and,
// per block, the sums of |P S_p - S_p|^2, |P S_m - S_m|^2 over m, |S_p|^2 and |S_m|^2 over m
// (partial[4 b + 0..3]). error_proj_kernel then sums M_ii (u_i - T s_i)^2 at any t.
template <int N>
struct ProjQSmem {
  using d = Dims<N>;
  static constexpr int Q = d::Q;
  static constexpr size_t u = 0;                      // 4 Np: coefficients s
  static constexpr size_t F = u + 4 * d::Np;          // 4 Q^3: w S at the points
  static constexpr size_t S = F + 4 * Q * Q * Q;      // 4 Q^3: S at the points
  static constexpr size_t C = S + 4 * Q * Q * Q;      // 4 n1 Q^2: c^T sums, then the forward b pass
  static constexpr size_t Bt = C + 4 * d::n1 * Q * Q; // 4 nrow Q: b^T sums, then the forward a pass
  static constexpr size_t XB = Bt + 4 * d::nrow * Q;  // 4 Q^2: B(a,b) and w_p w_q J(a,b)
  static constexpr size_t LQ = XB + 4 * Q * Q;
  static constexpr size_t GQ = LQ + d::nrow * Q;
  static constexpr size_t total = GQ + d::n1 * Q;
  static constexpr size_t bytes = total * sizeof(double);
};

template <int N>
__global__ void __launch_bounds__(ErrCfg<N>::NT)
    exact_proj_kernel(int64_t K, const double* __restrict__ ev, const double* __restrict__ gtab, int bc,
                      double* __restrict__ shat, double* __restrict__ Mdiag, double* __restrict__ partial) {
  using d = Dims<N>;
  using SM = ProjQSmem<N>;
  constexpr GeoLayout G(N);
  constexpr int Q = d::Q, Q2 = Q * Q, Q3 = Q * Q * Q;
  constexpr int NW = ErrCfg<N>::NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* s_u = sm + SM::u;
  double* s_F = sm + SM::F;
  double* s_S = sm + SM::S;
  double* s_C = sm + SM::C;
  double* s_Bt = sm + SM::Bt;
  double* s_XB = sm + SM::XB;
  double* s_LQ = sm + SM::LQ;
  double* s_GQ = sm + SM::GQ;
  __shared__ double v[15];
  __shared__ double red[4][NW];
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int x = tid; x < d::nrow * Q; x += nthr) s_LQ[x] = gtab[G.LQ + x];
  for (int x = tid; x < d::n1 * Q; x += nthr) s_GQ[x] = gtab[G.GQ + x];
  const double sc = bc == 0 ? 1.0 : 0.5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // |PS_p - S_p|^2, sum_m |PS_m - S_m|^2, |S_p|^2, sum_m |S_m|^2
  for (int64_t e = blockIdx.x; e < K; e += gridDim.x) {
    __syncthreads();
    if (tid < 15) v[tid] = ev[e * 15 + tid];
    __syncthreads();
    for (int x = tid; x < Q2; x += nthr) {
      const int p = x % Q, qq = x / Q;
      double B[3], Ba[3], Bb[3], D[3], g1[3];
      d_bilinear(v, gtab[G.XQ + p], gtab[G.XQ + qq], B, Ba, Bb);
      for (int m = 0; m < 3; ++m) D[m] = 0.5 * (v[12 + m] - B[m]);
      d_cross(Bb, D, g1);
      s_XB[4 * x + 0] = B[0];
      s_XB[4 * x + 1] = B[1];
      s_XB[4 * x + 2] = B[2];
      s_XB[4 * x + 3] = gtab[G.WQ + p] * gtab[G.WQ + qq] * (Ba[0] * g1[0] + Ba[1] * g1[1] + Ba[2] * g1[2]);
    }
    __syncthreads();
    for (int x = tid; x < Q3; x += nthr) {  // S and w S at every point
      const int pq = x % Q2, r = x / Q2;
      const double c = gtab[G.XQC + r];
      const double* xb = s_XB + 4 * pq;
      double sn[3], cs[3];
#pragma unroll
      for (int m = 0; m < 3; ++m)  // x_m = B_m (1-c)/2 + v5_m (1+c)/2 on the c line through (a, b)
        sincospi(sc * (0.5 * (1 - c) * xb[m] + 0.5 * (1 + c) * v[12 + m]), &sn[m], &cs[m]);
      const double Sf[4] = {cs[0] * cs[1] * cs[2], sn[0] * cs[1] * cs[2], cs[0] * sn[1] * cs[2],
                            cs[0] * cs[1] * sn[2]};
      const double w = xb[3] * gtab[G.WQC + r];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        s_S[f * Q3 + x] = Sf[f];
        s_F[f * Q3 + x] = w * Sf[f];
      }
      acc[2] += w * Sf[0] * Sf[0];
      acc[3] += w * (Sf[1] * Sf[1] + Sf[2] * Sf[2] + Sf[3] * Sf[3]);
    }
    __syncthreads();
    // <phi_n, S>_Q by transposed passes: c^T, then b^T, then a^T
    for (int x = tid; x < 4 * d::n1 * Q2; x += nthr) {
      const int pq = x % Q2, t = x / Q2;
      const int k = t % d::n1, f = t / d::n1;
      double a = 0;
      for (int r = 0; r < Q; ++r) a += s_GQ[k * Q + r] * s_F[f * Q3 + r * Q2 + pq];
      s_C[(f * d::n1 + k) * Q2 + pq] = a;
    }
    __syncthreads();
    for (int x = tid; x < 4 * d::nrow * Q; x += nthr) {
      const int p = x % Q, t = x / Q;
      const int row = t % d::nrow, f = t / d::nrow;
      int k, j;
      decode_row(row, k, j);
      double a = 0;
      for (int q2 = 0; q2 < Q; ++q2)
        a += s_LQ[(tri_num(k) + j) * Q + q2] * s_C[(f * d::n1 + k) * Q2 + p + Q * q2];
      s_Bt[(f * d::nrow + row) * Q + p] = a;
    }
    __syncthreads();
    for (int x = tid; x < 4 * d::Np; x += nthr) {  // s = M^{-1} <phi, S>_Q, M_ii = J w_i w_j C_k
      const int f = x / d::Np, n = x % d::Np;
      int k, j, i;
      decode_mode(n, k, j, i);
      double a = 0;
      for (int p = 0; p < Q; ++p) a += s_LQ[(tri_num(k) + i) * Q + p] * s_Bt[(f * d::nrow + tri_num(k) + j) * Q + p];
      const double J = d_jacobian(v, gtab[G.XL + tri_num(k) + i], gtab[G.XL + tri_num(k) + j]);
      const double M = J / gtab[G.IMR + n];
      const double sv = a / M;
      s_u[x] = sv;
      shat[e * 4 * d::Np + x] = sv;
      if (f == 0) Mdiag[e * d::Np + n] = M;
    }
    __syncthreads();
    // P S at the points (a, b, c passes), and |P S - S|_Q^2
    for (int x = tid; x < 4 * d::nrow * Q; x += nthr) {
      const int p = x % Q, t = x / Q;
      const int row = t % d::nrow, f = t / d::nrow;
      int k, j;
      decode_row(row, k, j);
      const double* uc = s_u + f * d::Np + lvl_off(k) + j * (k + 1);
      double a = 0;
      for (int i = 0; i <= k; ++i) a += uc[i] * s_LQ[(tri_num(k) + i) * Q + p];
      s_Bt[(f * d::nrow + row) * Q + p] = a;
    }
    __syncthreads();
    for (int x = tid; x < 4 * d::n1 * Q2; x += nthr) {
      const int pq = x % Q2, t = x / Q2;
      const int k = t % d::n1, f = t / d::n1;
      const int p = pq % Q, qq = pq / Q;
      double a = 0;
      for (int j = 0; j <= k; ++j) a += s_Bt[(f * d::nrow + tri_num(k) + j) * Q + p] * s_LQ[(tri_num(k) + j) * Q + qq];
      s_C[(f * d::n1 + k) * Q2 + pq] = a;
    }
    __syncthreads();
    for (int x = tid; x < Q3; x += nthr) {
      const int pq = x % Q2, r = x / Q2;
      const double w = s_XB[4 * pq + 3] * gtab[G.WQC + r];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        double ps = 0;
        for (int k = 0; k <= N; ++k) ps += s_GQ[k * Q + r] * s_C[(f * d::n1 + k) * Q2 + pq];
        const double df = ps - s_S[f * Q3 + x];
        acc[f == 0 ? 0 : 1] += w * df * df;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], off);
  if ((tid & 31) == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][tid >> 5] = acc[c];
  __syncthreads();
  if (tid < 4) {
    double a = 0.0;
    for (int w = 0; w < NW; ++w) a += red[tid][w];
    partial[4 * blockIdx.x + tid] = a;
  }
}

// sum over all elements, fields and modes of M_ii (u_i - T s_i)^2 (T = tp for p, tu for the
// velocities); partial[2 b] gets the block's sum, partial[2 b + 1] zero.
template <int N, typename T>
__global__ void __launch_bounds__(256)
    error_proj_kernel(int64_t K, const T* __restrict__ q, const double* __restrict__ shat,
                      const double* __restrict__ Mdiag, double tp, double tu, double* __restrict__ partial) {
  constexpr int Np = Dims<N>::Np;
  __shared__ double red[8];
  double acc = 0.0;
  const int64_t total = K * 4 * Np;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = x / (4 * Np);
    const int r = (int)(x - e * 4 * Np);
    const int f = r / Np, n = r - f * Np;
    const double df = fma(-(f == 0 ? tp : tu), shat[x], (double)q[x]);
    acc += Mdiag[e * Np + n] * df * df;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = 0.0;
  }
}

}  // namespace pyrdg
