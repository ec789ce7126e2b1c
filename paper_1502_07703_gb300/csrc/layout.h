// Compile-time sizes and reference-table layouts for degree N, shared by the
// host builder and the CUDA kernels.
//
// Semi-nodal basis (Lemma 3): level k = 0..N carries (k+1)^2 functions
// l_i^k(a) l_j^k(b) G_k(c), G_k(c) = ((1-c)/2)^k P_{N-k}^{(2k+3,0)}(c).
// Coefficient n of a field is (k, j, i) with n = lvl(k) + j(k+1) + i.
// A "row" is a pair (k, j) (or (k, i)); row index tri(k) + j, nrow rows.
//
// Point sets in one direction (a or b): the N+1 Gauss-Legendre points of the
// volume rule, extended by the two face coordinates -1 and +1 (P3 = N+3
// entries). The c direction uses the N+1 Gauss-Jacobi (2,0) points of the
// volume rule, c = -1 for the base face and N+1 Gauss-Jacobi (1,0) points
// for the triangle faces.
#pragma once

#if defined(__CUDACC__)
#define PYR_HD __host__ __device__
#else
#define PYR_HD
#endif

namespace pyrdg {

PYR_HD constexpr int tri_num(int k) { return k * (k + 1) / 2; }
PYR_HD constexpr int lvl_off(int k) { return k * (k + 1) * (2 * k + 1) / 6; }
PYR_HD constexpr int num_modes(int N) { return (N + 1) * (N + 2) * (2 * N + 3) / 6; }

template <int N_>
struct Dims {
  static constexpr int N = N_;
  static constexpr int n1 = N + 1;           // points per direction, volume rule
  static constexpr int P3 = N + 3;           // n1 volume points + faces at -1, +1
  static constexpr int n2 = n1 * n1;         // points on one face / (a,b) grid
  static constexpr int Nc = n1 * n2;         // volume cubature points
  static constexpr int nrow = n1 * (n1 + 1) / 2;
  static constexpr int Np = num_modes(N);
  static constexpr int Nfc = 5 * n2;         // face cubature points per element
  static constexpr int Q = N + 3;            // error-rule points per direction
  static constexpr int NGEO = 9;             // geometric factors per (a,b) point
  static constexpr int NGF = 16 + 4 * n2;    // face geometry per element
};

// Precision-typed operator tables (one contiguous array per degree).
struct TabLayout {
  int LX, DL, GC, DGC, HC, GB, GF, WC, WB, WFT, MH, MG, size;
  PYR_HD constexpr TabLayout(int N)
      : LX(0),
        DL(LX + tri_num(N + 1) * (N + 3)),
        GC(DL + tri_num(N + 1) * (N + 1)),
        DGC(GC + (N + 1) * (N + 1)),
        HC(DGC + (N + 1) * (N + 1)),
        GB(HC + (N + 1) * (N + 1)),
        GF(GB + (N + 1)),
        WC(GF + (N + 1) * (N + 1)),
        WB(WC + (N + 1)),
        WFT(WB + (N + 1) * (N + 1)),
        MH(WFT + (N + 1) * (N + 1)),
        MG(MH + (N + 1) * (N + 1)),
        size(MG + (N + 1) * (N + 1)) {}
};
// LX[(tri(k)+i)*P3 + p]  = l_i^k(x_p), x_p: GL points p<=N, then -1, +1
// DL[(tri(k)+i)*n1 + p]  = l_i^k'(x_p), p <= N
// GC/DGC/HC[k*n1 + r]    = G_k, G_k', H_k = 2/(1-c) G_k at GJ(2,0) point r
// GB[k]                  = G_k(-1)
// GF[k*n1 + m]           = G_k at GJ(1,0) point m
// WC[r]                  = GJ(2,0) weight / 4  (Duffy factor ((1-c)/2)^2)
// WB[p + n1 q]           = w_p w_q (base face)
// WFT[e + n1 m]          = w_e * GJ(1,0) weight / 2 (triangle faces)
// MH[k'*n1 + k]          = sum_r WC[r] G_{k'}(c_r) H_k(c_r)    (the c direction of the
// MG[k'*n1 + k]          = sum_r WC[r] G_{k'}(c_r) G_k'(c_r)   volume term as level mixing)

// Double tables for geometry, mass diagonal, projection and error rule.
struct GeoLayout {
  int XG, WG, XC, WC4, XF, WF2, XL, IMR, XQ, WQ, XQC, WQC, LQ, GQ, size;
  PYR_HD constexpr GeoLayout(int N)
      : XG(0),
        WG(XG + (N + 1)),
        XC(WG + (N + 1)),
        WC4(XC + (N + 1)),
        XF(WC4 + (N + 1)),
        WF2(XF + (N + 1)),
        XL(WF2 + (N + 1)),
        IMR(XL + tri_num(N + 1)),
        XQ(IMR + num_modes(N)),
        WQ(XQ + (N + 3)),
        XQC(WQ + (N + 3)),
        WQC(XQC + (N + 3)),
        LQ(WQC + (N + 3)),
        GQ(LQ + tri_num(N + 1) * (N + 3)),
        size(GQ + (N + 1) * (N + 3)) {}
};
// XG, WG: GL(N+1); XC, WC4: GJ(2,0)(N+1) nodes and weights/4;
// XF, WF2: GJ(1,0)(N+1) nodes and weights/2; XL[tri(k)+i] = level-k GL node i;
// IMR[n] = 1 / (w_i^k w_j^k C_k); error rule Q = N+3: XQ/WQ GL, XQC/WQC
// GJ(2,0) (weights/4), LQ[(tri(k)+i)*Q + p] = l_i^k(XQ_p), GQ[k*Q + r] = G_k(XQC_r).

}  // namespace pyrdg
