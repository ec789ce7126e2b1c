/* Host build of the exact FP64 slicing and recombination used by the FP64 tensor-core trace
 * kernel, for the CPU tests: slices, the exact integer slice-product sums G_s of a dot product
 * and their recombination. */
#include <stdint.h>

#include "exact64.h"

void shim_slices(const double* x, int n, int E, int32_t* a) {
  for (int i = 0; i < n; ++i) ex64_slices(x[i], E, a + 8 * i);
}

double shim_combine(const int32_t* G, int Z) { return ex64_combine(G, Z); }

double shim_combine_fast(const int32_t* G, int Z) { return ex64_combine_fast(G, Z); }

/* sum_n x_n y_n through the slices: E, F are the largest biased exponents of x and y; G (8
 * int64) receives the exact level sums; returns the recombined result (ex64_combine_fast if
 * fast, else ex64_combine). */
double shim_dot(const double* x, const double* y, int K, int64_t* G, int* EF, int fast) {
  int E = 0, F = 0;
  for (int n = 0; n < K; ++n) {
    if (ex64_exp(x[n]) > E) E = ex64_exp(x[n]);
    if (ex64_exp(y[n]) > F) F = ex64_exp(y[n]);
  }
  for (int s = 0; s < 8; ++s) G[s] = 0;
  for (int n = 0; n < K; ++n) {
    int32_t a[8], b[8];
    ex64_slices(x[n], E, a);
    ex64_slices(y[n], F, b);
    for (int i = 0; i < 8; ++i)
      for (int j = 0; i + j < 8; ++j) G[i + j] += (int64_t)a[i] * b[j];
  }
  int32_t G32[8];
  for (int s = 0; s < 8; ++s) G32[s] = (int32_t)G[s];
  EF[0] = E;
  EF[1] = F;
  return fast ? ex64_combine_fast(G32, E + F - 2107) : ex64_combine(G32, E + F - 2107);
}
