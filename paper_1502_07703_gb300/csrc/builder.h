// Host FP64 builder interface (Gauss rules, reference tables, connectivity).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "layout.h"

namespace pyrdg {

struct RefTables {
  int N = 0;
  std::vector<double> tab;  // TabLayout(N)
  std::vector<double> geo;  // GeoLayout(N)
  std::vector<double> Ck;   // c-direction normalisation, C_k = 2/(2k+3)
};

// Nodal variant (Sec. 4.4.1): Lagrange basis at a layered nodal set. Layer m = 0..N sits
// at c = the m-th of the N+1 Gauss-Lobatto-Legendre (GLL) points and carries the tensor
// grid of the N+1-m GLL points in (a, b) (the apex layer: one node). Nodes are ordered
// by layer, then b index q, then a index p. The base face carries the (N+1)^2 GLL grid,
// each triangle face (N+1)(N+2)/2 nodes: per layer the GLL points of its edge.
struct NodalTables {
  int N = 0, Np = 0, nT = 0;
  std::vector<double> nodes;  // Np x 3: (a, b, c) of node i
  std::vector<double> V;      // V[i * Np + n] = phi_n(node i) (semi-nodal basis, Lemma 3)
  std::vector<double> VT;     // VT[n * Np + i] = V[i][n]
  std::vector<double> VinvT;  // VinvT[i * Np + n] = (V^{-1})[n][i]
  std::vector<double> Mtri;   // nT x nT nodal mass matrix of a triangle face, reference measure
  std::vector<double> I1;     // I1[q * n1 + p] = GLL Lagrange basis p at Gauss-Legendre point q
  std::vector<int> tri_node;  // 4 x nT: element node of local node j of faces 1..4 (b=-1, a=+1, b=+1, a=-1)
  double cond_inf = 0.0;      // |V|_inf |V^{-1}|_inf
};
// Returns 0, or -1 for N outside 1..7, -2 if V is numerically singular.
int build_nodal(int N, NodalTables& nt);
int gll_points(int n, double* x);  // n Gauss-Lobatto-Legendre points, ascending (n = 1: {0})

double jacobi_p(int n, double al, double be, double x);
double jacobi_dp(int n, double al, double be, double x);
int gauss_jacobi(int n, double al, double be, double* x, double* w);
int build_tables(int N, RefTables& t);
double jacobian_ab(const double* v15, double a, double b);
double area_over_volume(const double* v15, const double* xg, const double* wg, int n1);
// Returns 0, or -2 (bad mesh) with a message in err.
// period_box: null, or {lo, hi} to make the box [lo, hi]^3 periodic (faces on
// opposite boundary planes are matched as neighbours).
int build_connectivity(const double* V, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                       std::vector<int64_t>& mapP, int64_t* nbnd, std::string& err,
                       const double* period_box = nullptr);

}  // namespace pyrdg
