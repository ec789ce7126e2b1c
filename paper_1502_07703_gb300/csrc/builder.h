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
