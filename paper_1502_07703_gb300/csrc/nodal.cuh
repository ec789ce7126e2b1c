// Nodal variant of the FP64 stage (Sec. 4.4.1): the state holds the values of each field at
// Np nodes of a layered nodal set (layer m = 0..N at the m-th GLL point in c, carrying the
// (N+1-m)^2 GLL grid in (a, b)); the Lagrange basis at those nodes spans the same space as the
// semi-nodal basis phi of Lemma 3, so the discrete solution is the modal one, written in
// another basis. With V[i][n] = phi_n(node i), ell = V^{-T} phi, so the nodal mass matrix is
// V^{-T} M V^{-1} and its inverse V M^{-1} V^T, M the diagonal of Lemma 3. One stage:
//   - traces without interpolation on the triangle faces: their nodal values are state
//     entries; the base face's GLL nodal values are interpolated to its Gauss-Legendre
//     points, where the non-planar base needs the quadrature of the modal path;
//   - coefficients c = V^{-1} u, then the modal volume passes (sum-factorised, with the
//     base-face lift);
//   - triangle faces: flux at the face nodes and the nodal face mass matrix (a scaling of
//     the reference triangle's: the faces are affine), which integrates the flux exactly
//     because it is a degree-N polynomial there; lifted by V^T;
//   - du/dt = -V M^{-1} (volume + V^T surface), then the LSRK update of the nodal values.
#pragma once

#include "dg_kernels.cuh"

namespace pyrdg {

template <int N>
struct NodalDims {
  using d = Dims<N>;
  static constexpr int nT = d::n1 * (d::n1 + 1) / 2;  // nodes per triangle face
  static constexpr int NTR = d::n2 + 4 * nT;          // trace points per element: base GL points, triangle nodes
  // per-degree double table (ntab): V, V^T, V^{-T}, triangle nodal mass, GLL -> GL interpolation
  static constexpr int V = 0, VT = d::Np * d::Np, VinvT = 2 * d::Np * d::Np, Mtri = 3 * d::Np * d::Np,
                       I1 = Mtri + nT * nT, size = I1 + d::n2;
};

template <int N>
struct NodalSmem {
  using d = Dims<N>;
  using R = RhsSmem<N, double>;
  using D = NodalDims<N>;
  static constexpr size_t un = R::total;                 // nodal state (4 Np)
  static constexpr size_t sl = un + 4 * d::Np;           // triangle-face integrals against ell (4 Np)
  static constexpr size_t Ft = sl + 4 * d::Np;           // triangle-face fluxes at the nodes (4 faces x 4 x nT)
  static constexpr size_t mt = Ft + 16 * D::nT;          // triangle nodal mass (nT x nT)
  static constexpr size_t total = mt + D::nT * D::nT;
  static constexpr size_t bytes = total * sizeof(double);
};

// Trace points of the nodal state: per element the base face at its (N+1)^2 Gauss-Legendre
// points (the GLL base nodes interpolated, tensor form), then the 4 x nT triangle-face nodes
// (copies); tr[(e NTR + x) 4 + f].
template <int N>
__global__ void __launch_bounds__(256)
    nodal_trace_kernel(int64_t K, const double* __restrict__ q, const double* __restrict__ ntab,
                       const int32_t* __restrict__ tri_node, double* __restrict__ tr) {
  using d = Dims<N>;
  using D = NodalDims<N>;
  const int64_t total = K * D::NTR;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / D::NTR;
    const int x = (int)(g - e * D::NTR);
    const double* u = q + e * 4 * d::Np;
    double out[4];
    if (x < d::n2) {  // layer 0 is the base: node q' n1 + p'
      const int p = x % d::n1, qq = x / d::n1;
      const double* Ip = ntab + D::I1 + p * d::n1;
      const double* Iq = ntab + D::I1 + qq * d::n1;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        double acc = 0.0;
        for (int q2 = 0; q2 < d::n1; ++q2) {
          double s = 0.0;
          for (int p2 = 0; p2 < d::n1; ++p2) s += Ip[p2] * u[f * d::Np + q2 * d::n1 + p2];
          acc += Iq[q2] * s;
        }
        out[f] = acc;
      }
    } else {
      const int node = tri_node[x - d::n2];
#pragma unroll
      for (int f = 0; f < 4; ++f) out[f] = u[f * d::Np + node];
    }
    double* dst = tr + g * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) dst[f] = out[f];
  }
}

template <int N, bool UPDATE>
__global__ void __launch_bounds__(KCfg<N>::NT)
    nodal_rhs_kernel(int64_t K, const double* qin, double* qout, double* __restrict__ res,  // qin == qout when updating
                     const double* __restrict__ tr, const int32_t* __restrict__ nmap, const double* __restrict__ geo,
                     const double* __restrict__ gface, const double* __restrict__ invM,
                     const double* __restrict__ tab, const double* __restrict__ ntab,
                     const int32_t* __restrict__ tri_node, int bc, double tau, double rka, double rkb, double dt) {
  using d = Dims<N>;
  using S = RhsSmem<N, double>;
  using NS = NodalSmem<N>;
  using D = NodalDims<N>;
  constexpr TabLayout L(N);
  constexpr int Np = d::Np, nT = D::nT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* s_tab = sm + S::tab;
  double* s_u = sm + S::u;
  double* s_geo = sm + S::geo;
  double* s_gf = sm + S::gf;
  double* s_Fs = sm + S::Fs;
  double* s_Zb = sm + S::Zb;
  double* s_un = sm + NS::un;
  double* s_sl = sm + NS::sl;
  double* s_Ft = sm + NS::Ft;
  double* s_mt = sm + NS::mt;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;

  for (int x = tid; x < L.size; x += nthr) s_tab[x] = tab[x];
  for (int x = tid; x < 4 * Np; x += nthr) {
    s_un[x] = qin[e * 4 * Np + x];
    s_sl[x] = 0.0;
  }
  for (int x = tid; x < d::NGEO * d::n2; x += nthr) s_geo[x] = geo[e * d::NGEO * d::n2 + x];
  for (int x = tid; x < d::NGF; x += nthr) s_gf[x] = gface[e * d::NGF + x];
  for (int x = tid; x < nT * nT; x += nthr) s_mt[x] = ntab[D::Mtri + x];
  __syncthreads();

  // coefficients of the semi-nodal basis: c = V^{-1} u
  for (int x = tid; x < 4 * Np; x += nthr) {
    const int f = x / Np, n = x - f * Np;
    const double* uf = s_un + f * Np;
    double acc = 0.0;
    for (int i = 0; i < Np; ++i) acc += ntab[D::VinvT + i * Np + n] * uf[i];
    s_u[x] = acc;
  }
  // flux (a4): base at its Gauss-Legendre points weighted by w sJ (lifted by the volume
  // passes); triangle faces at their nodes, unweighted (the face mass matrix follows)
  for (int x = tid; x < D::NTR; x += nthr) {
    const int64_t gl = e * D::NTR + x;
    const int64_t gn = nmap[gl];
    double um[4], up[4], F[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      um[f] = tr[gl * 4 + f];
      up[f] = tr[gn * 4 + f];
    }
    if (x < d::n2) {
      const double* nv = s_gf + 16 + 4 * x;
      face_flux<double>(um, up, gn == gl, bc, tau, nv, s_tab[L.WB + x] * nv[3], F);
#pragma unroll
      for (int f = 0; f < 4; ++f) s_Fs[f * d::Nfc + x] = F[f];
    } else {
      const int y = x - d::n2, face = y / nT, j = y - face * nT;
      face_flux<double>(um, up, gn == gl, bc, tau, s_gf + 4 * face, 1.0, F);
#pragma unroll
      for (int f = 0; f < 4; ++f) s_Ft[(face * 4 + f) * nT + j] = F[f];
    }
  }
  __syncthreads();
  // triangle faces: integrals against the Lagrange basis, sJ Mtri F, accumulated per node
  // (one face at a time: edge and apex nodes belong to two or four faces)
  for (int face = 0; face < 4; ++face) {
    const double sJ = s_gf[4 * face + 3];
    for (int x = tid; x < 4 * nT; x += nthr) {
      const int f = x / nT, i = x - f * nT;
      const double* Ff = s_Ft + (face * 4 + f) * nT;
      double acc = 0.0;
      for (int j = 0; j < nT; ++j) acc += s_mt[i * nT + j] * Ff[j];
      s_sl[f * Np + tri_node[face * nT + i]] += sJ * acc;
    }
    __syncthreads();
  }
  volume_passes<N, double, false>(s_tab, s_u, s_geo, s_Fs, sm + S::A, sm + S::dA, sm + S::U, sm + S::Ua, sm + S::Ub,
                                  sm + S::Y, sm + S::X, sm + S::Zc, s_Zb, tid, nthr);
  // a^T pass, the triangle lift V^T s and M^{-1}: rhs in the semi-nodal basis, into s_u
  for (int x = tid; x < 4 * Np; x += nthr) {
    const int f = x / Np, n = x - f * Np;
    int k, j, i;
    decode_mode(n, k, j, i);
    const double* lx = s_tab + L.LX + (tri_num(k) + i) * d::P3;
    const double* Zr = s_Zb + (f * d::nrow + tri_num(k) + j) * d::P3;
    double acc = 0.0;
    for (int pp = 0; pp < d::P3; ++pp) acc += lx[pp] * Zr[pp];
    const double* sf = s_sl + f * Np;
    for (int ii = 0; ii < Np; ++ii) acc += ntab[D::V + ii * Np + n] * sf[ii];
    s_u[x] = -invM[e * Np + n] * acc;
  }
  __syncthreads();
  // nodal rhs V (M^{-1} r), LSRK stage (a7)
  for (int x = tid; x < 4 * Np; x += nthr) {
    const int f = x / Np, i = x - f * Np;
    const double* rf = s_u + f * Np;
    double rhs = 0.0;
    for (int n = 0; n < Np; ++n) rhs += ntab[D::VT + n * Np + i] * rf[n];
    const int64_t gi = e * 4 * Np + x;
    if (UPDATE) {
      const double rnew = rka * res[gi] + dt * rhs;
      res[gi] = rnew;
      qout[gi] = s_un[x] + rkb * rnew;
    } else {
      qout[gi] = rhs;
    }
  }
}

}  // namespace pyrdg
