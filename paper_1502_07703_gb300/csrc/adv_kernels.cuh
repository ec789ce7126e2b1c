// Scalar advection u_t + div(beta u) = 0 (Sec. 4.1) with the semi-nodal basis:
// the same sum-factorised passes as the acoustic kernels, for one field.
//   M du/dt = -( S^beta u + L^f F ),  F = ((beta_n - alpha |beta_n|)/2) (u+ - u-),
// the upwind-weighted alpha-flux (alpha = 1 upwind, 0 central), written with the
// jump u+ - u- under which the scheme is energy stable. Volume term: J beta.grad(u)
// = u_r (beta.g1) + u_s (beta.g2) + u_c (beta.g3), with the c direction collapsed
// into the level mixing MH, MG as in rhs_kernel. One CTA per element.
#pragma once

#include "dg_kernels.cuh"

namespace pyrdg {

struct AdvParams {
  double beta[3];
  double alpha;
  double lo, L;  // periodic box [lo, lo + L]^3 of the exact solution
};

// Exact solution u0(x - beta t), u0 = sin(k(x-lo)) cos(k(y-lo)) sin(k(z-lo)), k = 2 pi / L.
__device__ __forceinline__ double d_exact_adv(const AdvParams& P, double x, double y, double z, double t) {
  const double s = 2.0 / P.L;  // sin(k x) = sinpi(s x)
  return sinpi(s * (x - P.beta[0] * t - P.lo)) * cospi(s * (y - P.beta[1] * t - P.lo)) *
         sinpi(s * (z - P.beta[2] * t - P.lo));
}

template <int N, typename T>
struct Trace1Smem {
  using d = Dims<N>;
  static constexpr int nB = d::n2 + 4 * d::n1;
  static constexpr size_t tab = 0;
  static constexpr size_t u = tab + TabLayout(N).size;
  static constexpr size_t A = u + d::Np;
  static constexpr size_t B = A + d::nrow * d::P3;
  static constexpr size_t total = B + d::n1 * nB;
  static constexpr size_t bytes = total * sizeof(T);
};

// u^f at all 5(N+1)^2 face points: tr[e*Nfc + g].
template <int N, typename T>
__global__ void __launch_bounds__(KCfg<N>::NT) trace1_kernel(int64_t K, const T* __restrict__ q,
                                                             const T* __restrict__ tab, T* __restrict__ tr) {
  using d = Dims<N>;
  using S = Trace1Smem<N, T>;
  constexpr TabLayout L(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* s_tab = sm + S::tab;
  T* s_u = sm + S::u;
  T* s_A = sm + S::A;
  T* s_B = sm + S::B;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int x = tid; x < L.size; x += nthr) s_tab[x] = tab[x];
  for (int x = tid; x < d::Np; x += nthr) s_u[x] = q[e * d::Np + x];
  __syncthreads();
  // a pass; at level N the volume columns are copies (l_i^N(x_p) = delta_ip), taken last
  constexpr int nLow = tri_num(N) * d::P3, nSum = nLow + (N + 1) * 2;
  for (int x = tid; x < d::nrow * d::P3; x += nthr) {
    int pp, row;
    if (x < nLow) {
      pp = x % d::P3;
      row = x / d::P3;
    } else if (x < nSum) {
      pp = d::n1 + (x - nLow) % 2;
      row = tri_num(N) + (x - nLow) / 2;
    } else {
      pp = (x - nSum) % d::n1;
      row = tri_num(N) + (x - nSum) / d::n1;
    }
    int k, j;
    decode_row(row, k, j);
    const T* uc = s_u + lvl_off(k) + j * (k + 1);
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + pp;
    T acc = 0;
    if (x >= nSum)
      acc = uc[pp];
    else
      for (int i = 0; i <= k; ++i) acc += uc[i] * lx[i * d::P3];
    s_A[row * d::P3 + pp] = acc;
  }
  __syncthreads();
  for (int x = tid; x < d::n1 * S::nB; x += nthr) {
    const int s = x % S::nB, k = x / S::nB;
    int pa, qb;
    if (s < d::n2) {
      pa = s % d::n1;
      qb = s / d::n1;
    } else {
      const int slot = (s - d::n2) / d::n1, ee = (s - d::n2) % d::n1;
      if (slot < 2) {
        pa = ee;
        qb = d::n1 + slot;
      } else {
        pa = d::n1 + (slot - 2);
        qb = ee;
      }
    }
    const T* Ar = s_A + tri_num(k) * d::P3 + pa;
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + qb;
    T acc = 0;
    if (k == N && qb < d::n1)  // l_j^N(b_q) = delta_jq
      acc = Ar[qb * d::P3];
    else
      for (int j = 0; j <= k; ++j) acc += Ar[j * d::P3] * lx[j * d::P3];
    s_B[k * S::nB + s] = acc;
  }
  __syncthreads();
  for (int g = tid; g < d::Nfc; g += nthr) {
    const int face = g / d::n2, idx = g % d::n2;
    T acc = 0;
    if (face == 0) {
      for (int k = 0; k <= N; ++k) acc += s_tab[L.GB + k] * s_B[k * S::nB + idx];
    } else {
      const int ee = idx % d::n1, m = idx / d::n1;
      const int slot = face == 1 ? 0 : face == 3 ? 1 : face == 4 ? 2 : 3;
      const int s = d::n2 + slot * d::n1 + ee;
      for (int k = 0; k <= N; ++k) acc += s_tab[L.GF + k * d::n1 + m] * s_B[k * S::nB + s];
    }
    tr[e * d::Nfc + g] = acc;
  }
}

template <int N, typename T>
struct Rhs1Smem {
  using d = Dims<N>;
  static constexpr int nY = d::P3 * d::P3;
  static constexpr size_t tab = 0;
  static constexpr size_t u = tab + TabLayout(N).size;
  static constexpr size_t geo = u + d::Np;
  static constexpr size_t gf = geo + d::NGEO * d::n2;
  static constexpr size_t Fs = gf + d::NGF;
  static constexpr size_t A = Fs + d::Nfc;
  static constexpr size_t dA = A + d::nrow * d::n1;
  static constexpr size_t U = dA + d::nrow * d::n1;
  static constexpr size_t Ua = U + d::n1 * d::n2;
  static constexpr size_t Ub = Ua + d::n1 * d::n2;
  static constexpr size_t Y = Ub + d::n1 * d::n2;
  static constexpr size_t Zb = Y + d::n1 * nY;
  static constexpr size_t total = Zb + d::nrow * d::P3;
  static constexpr size_t bytes = total * sizeof(T);
};

template <int N, typename T, bool UPDATE>
__global__ void __launch_bounds__(KCfg<N>::NT)
    rhs1_kernel(int64_t K, const T* qin, T* qout, T* __restrict__ res, const T* __restrict__ tr,
                const int32_t* __restrict__ mapP, const T* __restrict__ geo, const T* __restrict__ gface,
                const T* __restrict__ invM, const T* __restrict__ tab, T bx, T by, T bz, T alpha, T rka, T rkb,
                T dt) {
  using d = Dims<N>;
  using S = Rhs1Smem<N, T>;
  constexpr TabLayout L(N);
  constexpr int nY = S::nY;
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
  T* s_Zb = sm + S::Zb;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int x = tid; x < L.size; x += nthr) s_tab[x] = tab[x];
  for (int x = tid; x < d::Np; x += nthr) s_u[x] = qin[e * d::Np + x];
  for (int x = tid; x < d::NGEO * d::n2; x += nthr) s_geo[x] = geo[e * d::NGEO * d::n2 + x];
  for (int x = tid; x < d::NGF; x += nthr) s_gf[x] = gface[e * d::NGF + x];
  // Y entries no pass writes (face rows x face columns) are read as zeros
  for (int x = tid; x < d::n1 * nY; x += nthr) s_Y[x] = 0;
  __syncthreads();
  // flux at the face points, weighted by w sJ
  for (int g = tid; g < d::Nfc; g += nthr) {
    const int face = g / d::n2, idx = g % d::n2;
    const int64_t gl = e * d::Nfc + g;
    const T um = tr[gl], up = tr[mapP[gl]];
    const T* nv = face == 0 ? s_gf + 16 + 4 * idx : s_gf + 4 * (face - 1);
    const T w = face == 0 ? s_tab[L.WB + idx] : s_tab[L.WFT + idx];
    const T bn = bx * nv[0] + by * nv[1] + bz * nv[2];
    s_Fs[g] = w * nv[3] * T(0.5) * (bn - alpha * fabs(bn)) * (up - um);
  }
  for (int x = tid; x < d::nrow * d::n1; x += nthr) {  // a pass
    const int p = x % d::n1, row = x / d::n1;
    int k, j;
    decode_row(row, k, j);
    const T* uc = s_u + lvl_off(k) + j * (k + 1);
    const T* lx = s_tab + L.LX + tri_num(k) * d::P3 + p;
    const T* dl = s_tab + L.DL + tri_num(k) * d::n1 + p;
    T a = 0, da = 0;
    if (k == N) {  // l_i^N(a_p) = delta_ip
      a = uc[p];
      for (int i = 0; i <= k; ++i) da += uc[i] * dl[i * d::n1];
    } else {
      for (int i = 0; i <= k; ++i) {
        a += uc[i] * lx[i * d::P3];
        da += uc[i] * dl[i * d::n1];
      }
    }
    s_A[x] = a;
    s_dA[x] = da;
  }
  __syncthreads();
  for (int x = tid; x < d::n1 * d::n2; x += nthr) {  // b pass
    const int pq = x % d::n2, k = x / d::n2;
    const int p = pq % d::n1, q = pq / d::n1;
    const T* Ar = s_A + tri_num(k) * d::n1 + p;
    const T* dAr = s_dA + tri_num(k) * d::n1 + p;
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
    s_U[x] = u;
    s_Ua[x] = ua;
    s_Ub[x] = ub;
  }
  __syncthreads();
  // level mixing of the c direction, chain rule with beta, base-face lift; triangle-face c^T
  for (int x = tid; x < d::n1 * d::n2 + 4 * d::n1 * d::n1; x += nthr) {
    if (x < d::n1 * d::n2) {
      const int pq = x % d::n2, kp = x / d::n2;
      const int p = pq % d::n1, q = pq / d::n1;
      const T* mh = s_tab + L.MH + kp * d::n1;
      const T* mg = s_tab + L.MG + kp * d::n1;
      T al = 0, be = 0, ga = 0;
      // MG is lower Hessenberg (k <= k'+1), MH tridiagonal (|k - k'| <= 1)
      const int k1 = kp < N ? kp + 1 : N;
      for (int k = 0; k <= k1; ++k) ga += mg[k] * s_U[k * d::n2 + pq];
      for (int k = kp > 0 ? kp - 1 : 0; k <= k1; ++k) {
        al += mh[k] * s_Ua[k * d::n2 + pq];
        be += mh[k] * s_Ub[k * d::n2 + pq];
      }
      const T* g = s_geo + pq * d::NGEO;
      const T b1 = bx * g[0] + by * g[1] + bz * g[2];
      const T b2 = bx * g[3] + by * g[4] + bz * g[5];
      const T b3 = bx * g[6] + by * g[7] + bz * g[8];
      s_Y[kp * nY + p * d::P3 + q] = b1 * al + b2 * be + b3 * ga + s_tab[L.GB + kp] * s_Fs[pq];
    } else {
      const int y = x - d::n1 * d::n2;
      const int ee = y % d::n1, slot = (y / d::n1) % 4, k = y / (4 * d::n1);
      const int face = slot == 0 ? 1 : slot == 1 ? 3 : slot == 2 ? 4 : 2;
      const T* fs = s_Fs + face * d::n2 + ee;
      T acc = 0;
      for (int m = 0; m <= N; ++m) acc += s_tab[L.GF + k * d::n1 + m] * fs[m * d::n1];
      T* Yk = s_Y + k * nY;
      if (slot < 2)
        Yk[ee * d::P3 + d::n1 + slot] = acc;
      else
        Yk[(d::n1 + slot - 2) * d::P3 + ee] = acc;
    }
  }
  __syncthreads();
  for (int x = tid; x < d::nrow * d::P3; x += nthr) {  // b^T pass
    const int pp = x % d::P3, row = x / d::P3;
    int k, j;
    decode_row(row, k, j);
    const T* Yr = s_Y + (k * d::P3 + pp) * d::P3;
    const T* lx = s_tab + L.LX + (tri_num(k) + j) * d::P3;
    T acc = 0;
    if (k == N) {  // l_j^N(x_c) = delta_jc on the volume points; the face columns remain
      acc = Yr[j];
      for (int c = d::n1; c < d::P3; ++c) acc += lx[c] * Yr[c];
    } else {
      for (int c = 0; c < d::P3; ++c) acc += lx[c] * Yr[c];
    }
    s_Zb[row * d::P3 + pp] = acc;
  }
  __syncthreads();
  for (int n = tid; n < d::Np; n += nthr) {  // a^T pass, M^{-1}, LSRK stage
    int k, j, i;
    decode_mode(n, k, j, i);
    const T* lx = s_tab + L.LX + (tri_num(k) + i) * d::P3;
    const T* Zr = s_Zb + (tri_num(k) + j) * d::P3;
    T acc = 0;
    if (k == N) {  // l_i^N(x_c) = delta_ic on the volume points; the face columns remain
      acc = Zr[i] + lx[d::n1] * Zr[d::n1] + lx[d::n1 + 1] * Zr[d::n1 + 1];
    } else {
      for (int c = 0; c < d::P3; ++c) acc += lx[c] * Zr[c];
    }
    const T rhs = -invM[e * d::Np + n] * acc;
    const int64_t gi = e * d::Np + n;
    if (UPDATE) {
      const T rnew = rka * res[gi] + dt * rhs;
      res[gi] = rnew;
      qout[gi] = s_u[n] + rkb * rnew;
    } else {
      qout[gi] = rhs;
    }
  }
}

// L2 projection of the exact advected field at time t (double arithmetic).
template <int N, typename T>
__global__ void __launch_bounds__(KCfg<N>::NT)
    project1_kernel(int64_t K, const double* __restrict__ ev, const double* __restrict__ gtab,
                    const double* __restrict__ tabd, AdvParams P, double t, T* __restrict__ qout) {
  using d = Dims<N>;
  constexpr TabLayout L(N);
  constexpr GeoLayout G(N);
  constexpr int nY = d::P3 * d::P3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* s_tab = sm;
  double* s_Fv = s_tab + L.size;      // Nc
  double* s_Y = s_Fv + d::Nc;         // n1 nY
  double* s_Z = s_Y + d::n1 * nY;     // nrow P3
  __shared__ double v[15];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int x = tid; x < L.size; x += nthr) s_tab[x] = tabd[x];
  if (tid < 15) v[tid] = ev[e * 15 + tid];
  __syncthreads();
  for (int x = tid; x < d::Nc; x += nthr) {
    const int pq = x % d::n2, r = x / d::n2;
    const int p = pq % d::n1, q = pq / d::n1;
    const double a = gtab[G.XG + p], b = gtab[G.XG + q], c = gtab[G.XC + r];
    double B[3], Ba[3], Bb[3];
    d_bilinear(v, a, b, B, Ba, Bb);
    const double X0 = 0.5 * (1 - c) * B[0] + 0.5 * (1 + c) * v[12];
    const double X1 = 0.5 * (1 - c) * B[1] + 0.5 * (1 + c) * v[13];
    const double X2 = 0.5 * (1 - c) * B[2] + 0.5 * (1 + c) * v[14];
    const double w = gtab[G.WG + p] * gtab[G.WG + q] * gtab[G.WC4 + r] * d_jacobian(v, a, b);
    s_Fv[x] = w * d_exact_adv(P, X0, X1, X2, t);
  }
  __syncthreads();
  for (int x = tid; x < d::n1 * d::n2; x += nthr) {  // c^T
    const int pq = x % d::n2, k = x / d::n2;
    const int p = pq % d::n1, q = pq / d::n1;
    double acc = 0;
    for (int r = 0; r < d::n1; ++r) acc += s_tab[L.GC + k * d::n1 + r] * s_Fv[r * d::n2 + pq];
    s_Y[k * nY + p * d::P3 + q] = acc;
  }
  __syncthreads();
  for (int x = tid; x < d::nrow * d::n1; x += nthr) {  // b^T
    const int pp = x % d::n1, row = x / d::n1;
    int k, j;
    decode_row(row, k, j);
    double acc = 0;
    for (int q = 0; q < d::n1; ++q) acc += s_tab[L.LX + (tri_num(k) + j) * d::P3 + q] * s_Y[k * nY + pp * d::P3 + q];
    s_Z[row * d::P3 + pp] = acc;
  }
  __syncthreads();
  for (int n = tid; n < d::Np; n += nthr) {  // a^T and M^{-1}
    int k, j, i;
    decode_mode(n, k, j, i);
    double acc = 0;
    for (int p = 0; p < d::n1; ++p)
      acc += s_tab[L.LX + (tri_num(k) + i) * d::P3 + p] * s_Z[(tri_num(k) + j) * d::P3 + p];
    const double J = d_jacobian(v, gtab[G.XL + tri_num(k) + i], gtab[G.XL + tri_num(k) + j]);
    qout[e * d::Np + n] = (T)(acc * gtab[G.IMR + n] / J);
  }
}

template <int N>
struct Proj1Smem {
  using d = Dims<N>;
  static constexpr size_t total = TabLayout(N).size + d::Nc + d::n1 * d::P3 * d::P3 + d::nrow * d::P3;
  static constexpr size_t bytes = total * sizeof(double);
};

// L2 error against the exact advected field, (N+3)-point rules in double.
template <int N, typename T>
__global__ void __launch_bounds__(256)
    error1_kernel(int64_t K, const T* __restrict__ q, const double* __restrict__ ev, const double* __restrict__ gtab,
                  AdvParams P, double t, double* __restrict__ partial) {
  using d = Dims<N>;
  constexpr GeoLayout G(N);
  constexpr int Q = d::Q;
  __shared__ double s_u[d::Np];
  __shared__ double s_A[d::nrow * Q];
  __shared__ double s_B[d::n1 * Q * Q];
  __shared__ double v[15];
  __shared__ double red[2][8];
  const int tid = threadIdx.x, nthr = blockDim.x;
  double e2 = 0.0, n2 = 0.0;
  for (int64_t e = blockIdx.x; e < K; e += gridDim.x) {
    __syncthreads();
    for (int x = tid; x < d::Np; x += nthr) s_u[x] = (double)q[e * d::Np + x];
    if (tid < 15) v[tid] = ev[e * 15 + tid];
    __syncthreads();
    for (int x = tid; x < d::nrow * Q; x += nthr) {
      const int p = x % Q, row = x / Q;
      int k, j;
      decode_row(row, k, j);
      double acc = 0;
      for (int i = 0; i <= k; ++i) acc += s_u[lvl_off(k) + j * (k + 1) + i] * gtab[G.LQ + (tri_num(k) + i) * Q + p];
      s_A[x] = acc;
    }
    __syncthreads();
    for (int x = tid; x < d::n1 * Q * Q; x += nthr) {
      const int pq = x % (Q * Q), k = x / (Q * Q);
      const int p = pq % Q, qq = pq / Q;
      double acc = 0;
      for (int j = 0; j <= k; ++j) acc += s_A[(tri_num(k) + j) * Q + p] * gtab[G.LQ + (tri_num(k) + j) * Q + qq];
      s_B[x] = acc;
    }
    __syncthreads();
    for (int x = tid; x < Q * Q * Q; x += nthr) {
      const int pq = x % (Q * Q), r = x / (Q * Q);
      const int p = pq % Q, qq = pq / Q;
      const double a = gtab[G.XQ + p], b = gtab[G.XQ + qq], c = gtab[G.XQC + r];
      double B[3], Ba[3], Bb[3];
      d_bilinear(v, a, b, B, Ba, Bb);
      const double w = gtab[G.WQ + p] * gtab[G.WQ + qq] * gtab[G.WQC + r] * d_jacobian(v, a, b);
      const double ue = d_exact_adv(P, 0.5 * (1 - c) * B[0] + 0.5 * (1 + c) * v[12],
                                    0.5 * (1 - c) * B[1] + 0.5 * (1 + c) * v[13],
                                    0.5 * (1 - c) * B[2] + 0.5 * (1 + c) * v[14], t);
      double uh = 0;
      for (int k = 0; k <= N; ++k) uh += gtab[G.GQ + k * Q + r] * s_B[k * Q * Q + pq];
      e2 += w * (uh - ue) * (uh - ue);
      n2 += w * ue * ue;
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
    for (int w = 0; w < nthr / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

}  // namespace pyrdg
