// Host FP64 builder: Gauss rules, semi-nodal reference tables, vertex-map
// geometry checks and face connectivity. Everything here runs once per setup.
#include "builder.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace pyrdg {

// ---------------------------------------------------------------- polynomials
// Jacobi P_n^{(al,be)} with P_n(1) = binom(n+al, n), three-term recurrence.
double jacobi_p(int n, double al, double be, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0;
  double p = 0.5 * (al - be + (al + be + 2.0) * x);
  for (int m = 2; m <= n; ++m) {
    const double s = 2.0 * m + al + be;
    const double c1 = 2.0 * m * (m + al + be) * (s - 2.0);
    const double c2 = (s - 1.0) * (al * al - be * be);
    const double c3 = (s - 2.0) * (s - 1.0) * s;
    const double c4 = 2.0 * (m + al - 1.0) * (m + be - 1.0) * s;
    const double pn = ((c2 + c3 * x) * p - c4 * pm) / c1;
    pm = p;
    p = pn;
  }
  return p;
}

double jacobi_dp(int n, double al, double be, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + al + be + 1.0) * jacobi_p(n - 1, al + 1.0, be + 1.0, x);
}

// Gauss-Jacobi nodes by Newton iteration with deflation from Chebyshev
// starting guesses (Karniadakis & Sherwin's zero finder), then the weights
// w_i = 2^{al+be+1} G(n+al+1) G(n+be+1) / (G(n+al+be+1) n!) / ((1-x^2) P_n'(x)^2).
int gauss_jacobi(int n, double al, double be, double* x, double* w) {
  if (n < 1 || n > 64 || !(al > -1.0) || !(be > -1.0)) return -1;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += 1.0 / (r - x[i]);
      const double p = jacobi_p(n, al, be, r);
      const double dp = jacobi_dp(n, al, be, r);
      const double delta = -p / (dp - s * p);
      r += delta;
      if (std::fabs(delta) < 1e-16) break;
    }
    x[k] = r;
  }
  for (int k = 0; k < n; ++k) {  // polish without deflation
    double r = x[k];
    for (int it = 0; it < 3; ++it) r -= jacobi_p(n, al, be, r) / jacobi_dp(n, al, be, r);
    x[k] = r;
  }
  std::sort(x, x + n);
  const double lc = (al + be + 1.0) * std::log(2.0) + std::lgamma(n + al + 1.0) + std::lgamma(n + be + 1.0) -
                    std::lgamma(n + al + be + 1.0) - std::lgamma(n + 1.0);
  const double C = std::exp(lc);
  for (int k = 0; k < n; ++k) {
    const double dp = jacobi_dp(n, al, be, x[k]);
    w[k] = C / ((1.0 - x[k] * x[k]) * dp * dp);
  }
  return 0;
}

// Lagrange basis on `nodes` (size n) and its derivative at x.
static void lagrange(const double* nodes, int n, double x, double* L, double* dL) {
  for (int i = 0; i < n; ++i) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) v *= (x - nodes[m]) / (nodes[i] - nodes[m]);
    L[i] = v;
    double d = 0.0;
    for (int l = 0; l < n; ++l) {
      if (l == i) continue;
      double t = 1.0 / (nodes[i] - nodes[l]);
      for (int m = 0; m < n; ++m)
        if (m != i && m != l) t *= (x - nodes[m]) / (nodes[i] - nodes[m]);
      d += t;
    }
    dL[i] = d;
  }
}

// G_k(c) = ((1-c)/2)^k P_{N-k}^{(2k+3,0)}(c), its derivative, and
// H_k(c) = ((1-c)/2)^{k-1} P_{N-k}^{(2k+3,0)}(c) = 2/(1-c) G_k(c) (0 for k = 0).
static void cfun(int N, int k, double c, double* G, double* dG, double* H) {
  const double h = 0.5 * (1.0 - c);
  const double P = jacobi_p(N - k, 2.0 * k + 3.0, 0.0, c);
  const double dP = jacobi_dp(N - k, 2.0 * k + 3.0, 0.0, c);
  const double hk = std::pow(h, k);
  const double hk1 = k >= 1 ? std::pow(h, k - 1) : 0.0;
  if (G) *G = hk * P;
  if (dG) *dG = -0.5 * k * hk1 * P + hk * dP;
  if (H) *H = hk1 * P;
}

int build_tables(int N, RefTables& t) {
  if (N < 1 || N > 7) return -1;
  const int n1 = N + 1, P3 = N + 3, Q = N + 3, nrow = tri_num(n1), Np = num_modes(N);
  const TabLayout L(N);
  const GeoLayout G(N);
  t.N = N;
  t.tab.assign(L.size, 0.0);
  t.geo.assign(G.size, 0.0);
  std::vector<double> xg(n1), wg(n1), xc(n1), wc(n1), xf(n1), wf(n1);
  gauss_jacobi(n1, 0.0, 0.0, xg.data(), wg.data());
  gauss_jacobi(n1, 2.0, 0.0, xc.data(), wc.data());
  gauss_jacobi(n1, 1.0, 0.0, xf.data(), wf.data());
  std::vector<double> xe(P3);
  for (int p = 0; p < n1; ++p) xe[p] = xg[p];
  xe[n1] = -1.0;
  xe[n1 + 1] = 1.0;

  // C_k = int ((1-c)/2)^{2k+2} (P_{N-k}^{(2k+3,0)})^2 dc by an exact Gauss-Legendre rule
  std::vector<double> xh(N + 3), wh(N + 3), Ck(n1);
  gauss_jacobi(N + 3, 0.0, 0.0, xh.data(), wh.data());
  for (int k = 0; k <= N; ++k) {
    double s = 0.0;
    for (int q = 0; q < N + 3; ++q) {
      const double P = jacobi_p(N - k, 2.0 * k + 3.0, 0.0, xh[q]);
      s += wh[q] * std::pow(0.5 * (1.0 - xh[q]), 2 * k + 2) * P * P;
    }
    Ck[k] = s;
  }
  t.Ck = Ck;

  std::vector<double> Lv(n1), dLv(n1);
  std::vector<double> xq(Q), wq(Q), xqc(Q), wqc(Q);
  gauss_jacobi(Q, 0.0, 0.0, xq.data(), wq.data());
  gauss_jacobi(Q, 2.0, 0.0, xqc.data(), wqc.data());
  for (int k = 0; k <= N; ++k) {
    std::vector<double> xk(k + 1), wk(k + 1);
    gauss_jacobi(k + 1, 0.0, 0.0, xk.data(), wk.data());
    for (int i = 0; i <= k; ++i) t.geo[G.XL + tri_num(k) + i] = xk[i];
    for (int p = 0; p < P3; ++p) {
      lagrange(xk.data(), k + 1, xe[p], Lv.data(), dLv.data());
      for (int i = 0; i <= k; ++i) {
        t.tab[L.LX + (tri_num(k) + i) * P3 + p] = Lv[i];
        if (p < n1) t.tab[L.DL + (tri_num(k) + i) * n1 + p] = dLv[i];
      }
    }
    for (int p = 0; p < Q; ++p) {
      lagrange(xk.data(), k + 1, xq[p], Lv.data(), dLv.data());
      for (int i = 0; i <= k; ++i) t.geo[G.LQ + (tri_num(k) + i) * Q + p] = Lv[i];
    }
    for (int r = 0; r < n1; ++r) {
      cfun(N, k, xc[r], &t.tab[L.GC + k * n1 + r], &t.tab[L.DGC + k * n1 + r], &t.tab[L.HC + k * n1 + r]);
      cfun(N, k, xf[r], &t.tab[L.GF + k * n1 + r], nullptr, nullptr);
    }
    cfun(N, k, -1.0, &t.tab[L.GB + k], nullptr, nullptr);
    for (int r = 0; r < Q; ++r) cfun(N, k, xqc[r], &t.geo[G.GQ + k * Q + r], nullptr, nullptr);
    for (int j = 0; j <= k; ++j)
      for (int i = 0; i <= k; ++i)
        t.geo[G.IMR + lvl_off(k) + j * (k + 1) + i] = 1.0 / (wk[i] * wk[j] * Ck[k]);
  }
  for (int r = 0; r < n1; ++r) t.tab[L.WC + r] = 0.25 * wc[r];
  // The volume geometric factors do not depend on c, so the c-interpolation of
  // derivatives and the c-projection onto level k' collapse into these sums.
  // Both are banded. With G_k = ((1-c)/2)^k P_{N-k}^{(2k+3,0)}, the integrand of
  // MH[k'][k] is (1-c)^{k+k'+1} P_{N-k'} P_{N-k} (up to a constant), symmetric in k, k';
  // for k >= k'+2 it is (1-c)^{2k'+3} times a polynomial of degree N-k'-2, which
  // P_{N-k'}^{(2k'+3,0)} is orthogonal to. So MH is tridiagonal. G_k' carries
  // ((1-c)/2)^{k-1}, so MG[k'][k] vanishes for k >= k'+2 by the same argument (lower
  // Hessenberg). The GJ(2,0) rule is exact on these entries (polynomials of degree
  // 2N-1), so the sums are zero up to rounding; they are stored as exact zeros and
  // the kernels skip them.
  double mmax = 0.0, resid = 0.0;
  for (int kp = 0; kp <= N; ++kp)
    for (int k = 0; k <= N; ++k) {
      double mh = 0.0, mg = 0.0;
      for (int r = 0; r < n1; ++r) {
        const double w = 0.25 * wc[r] * t.tab[L.GC + kp * n1 + r];
        mh += w * t.tab[L.HC + k * n1 + r];
        mg += w * t.tab[L.DGC + k * n1 + r];
      }
      mmax = std::max(mmax, std::max(std::fabs(mh), std::fabs(mg)));
      if (k > kp + 1 || k < kp - 1) {
        resid = std::max(resid, std::fabs(mh));
        mh = 0.0;
      }
      if (k > kp + 1) {
        resid = std::max(resid, std::fabs(mg));
        mg = 0.0;
      }
      t.tab[L.MH + kp * n1 + k] = mh;
      t.tab[L.MG + kp * n1 + k] = mg;
    }
  if (resid > 1e-12 * mmax) return -3;  // the band structure must hold to rounding
  for (int q = 0; q < n1; ++q)
    for (int p = 0; p < n1; ++p) {
      t.tab[L.WB + p + n1 * q] = wg[p] * wg[q];
      t.tab[L.WFT + p + n1 * q] = wg[p] * 0.5 * wf[q];
    }
  for (int p = 0; p < n1; ++p) {
    t.geo[G.XG + p] = xg[p];
    t.geo[G.WG + p] = wg[p];
    t.geo[G.XC + p] = xc[p];
    t.geo[G.WC4 + p] = 0.25 * wc[p];
    t.geo[G.XF + p] = xf[p];
    t.geo[G.WF2 + p] = 0.5 * wf[p];
  }
  for (int p = 0; p < Q; ++p) {
    t.geo[G.XQ + p] = xq[p];
    t.geo[G.WQ + p] = wq[p];
    t.geo[G.XQC + p] = xqc[p];
    t.geo[G.WQC + p] = 0.25 * wqc[p];
  }
  (void)nrow;
  (void)Np;
  return 0;
}

// ------------------------------------------------------------------ geometry
// Vertex map in collapsed coordinates: x(a,b,c) = (1-c)/2 B(a,b) + (1+c)/2 v5,
// B the bilinear map of the base quadrilateral v1..v4 (the Bedrosian map of
// Sec. 2 rewritten in (a,b,c)).
static inline void bilinear(const double* v, double a, double b, double* B, double* Ba, double* Bb) {
  const double w1 = 0.25 * (1 - a) * (1 - b), w2 = 0.25 * (1 + a) * (1 - b);
  const double w3 = 0.25 * (1 + a) * (1 + b), w4 = 0.25 * (1 - a) * (1 + b);
  for (int m = 0; m < 3; ++m) {
    const double v1 = v[0 * 3 + m], v2 = v[1 * 3 + m], v3 = v[2 * 3 + m], v4 = v[3 * 3 + m];
    if (B) B[m] = w1 * v1 + w2 * v2 + w3 * v3 + w4 * v4;
    if (Ba) Ba[m] = 0.25 * ((1 - b) * (v2 - v1) + (1 + b) * (v3 - v4));
    if (Bb) Bb[m] = 0.25 * ((1 - a) * (v4 - v1) + (1 + a) * (v3 - v2));
  }
}

double jacobian_ab(const double* v, double a, double b) {
  double B[3], Ba[3], Bb[3], D[3];
  bilinear(v, a, b, B, Ba, Bb);
  for (int m = 0; m < 3; ++m) D[m] = 0.5 * (v[12 + m] - B[m]);
  // det[Ba, Bb, D] = Ba . (Bb x D)
  const double cx = Bb[1] * D[2] - Bb[2] * D[1];
  const double cy = Bb[2] * D[0] - Bb[0] * D[2];
  const double cz = Bb[0] * D[1] - Bb[1] * D[0];
  return Ba[0] * cx + Ba[1] * cy + Ba[2] * cz;
}

static inline void map_point(const double* v, double a, double b, double c, double* X) {
  double B[3];
  bilinear(v, a, b, B, nullptr, nullptr);
  for (int m = 0; m < 3; ++m) X[m] = 0.5 * (1 - c) * B[m] + 0.5 * (1 + c) * v[12 + m];
}

static inline double norm3(const double* a) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }
static inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// |K| = int J = (8/3) J(0,0) (J bilinear in a,b; int ((1-c)/2)^2 dc = 2/3).
// |dK| = base area by the (N+1)^2 Gauss-Legendre rule + the four triangle areas.
double area_over_volume(const double* v, const double* xg, const double* wg, int n1) {
  const double vol = (8.0 / 3.0) * jacobian_ab(v, 0.0, 0.0);
  double area = 0.0;
  for (int q = 0; q < n1; ++q)
    for (int p = 0; p < n1; ++p) {
      double Ba[3], Bb[3], c[3];
      bilinear(v, xg[p], xg[q], nullptr, Ba, Bb);
      cross3(Ba, Bb, c);
      area += wg[p] * wg[q] * norm3(c);
    }
  static const int tri[4][3] = {{0, 1, 4}, {1, 2, 4}, {3, 2, 4}, {0, 3, 4}};
  for (int f = 0; f < 4; ++f) {
    double e1[3], e2[3], c[3];
    for (int m = 0; m < 3; ++m) {
      e1[m] = v[tri[f][1] * 3 + m] - v[tri[f][0] * 3 + m];
      e2[m] = v[tri[f][2] * 3 + m] - v[tri[f][0] * 3 + m];
    }
    cross3(e1, e2, c);
    area += 0.5 * norm3(c);
  }
  return area / vol;
}

// ----------------------------------------------------------- connectivity
// Local vertex lists of the five faces (0-based v1..v5): base, b=-1, a=+1, b=+1, a=-1.
static const int kFaceVerts[5][4] = {{0, 1, 2, 3}, {0, 1, 4, -1}, {1, 2, 4, -1}, {3, 2, 4, -1}, {0, 3, 4, -1}};

// Cube coordinates of face point idx of face f.
static inline void face_abc(int f, int idx, int n1, const double* xg, const double* xf, double* a, double* b,
                            double* c) {
  const int e = idx % n1, m = idx / n1;
  switch (f) {
    case 0: *a = xg[e]; *b = xg[m]; *c = -1.0; break;
    case 1: *a = xg[e]; *b = -1.0; *c = xf[m]; break;
    case 2: *a = 1.0; *b = xg[e]; *c = xf[m]; break;
    case 3: *a = xg[e]; *b = 1.0; *c = xf[m]; break;
    default: *a = -1.0; *b = xg[e]; *c = xf[m]; break;
  }
}

// The symmetries of a face's point grid: the dihedral group of the square for
// the base, edge reversal for a triangle (the apex stays the collapse point).
static inline int permute(int code, int idx, int n1) {
  const int N = n1 - 1;
  const int p = idx % n1, q = idx / n1;
  int pp = p, qq = q;
  switch (code) {
    case 0: pp = p; qq = q; break;
    case 1: pp = N - p; qq = q; break;
    case 2: pp = p; qq = N - q; break;
    case 3: pp = N - p; qq = N - q; break;
    case 4: pp = q; qq = p; break;
    case 5: pp = N - q; qq = p; break;
    case 6: pp = q; qq = N - p; break;
    default: pp = N - q; qq = N - p; break;
  }
  return pp + n1 * qq;
}

struct FaceKey {
  int64_t v[4];
  int64_t elem;
  int face;
  bool operator<(const FaceKey& o) const {
    for (int i = 0; i < 4; ++i)
      if (v[i] != o.v[i]) return v[i] < o.v[i];
    return elem != o.elem ? elem < o.elem : face < o.face;
  }
  bool same(const FaceKey& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2] && v[3] == o.v[3]; }
};

// Canonical vertex ids for a box [lo, hi]^3 made periodic: a vertex on an upper
// boundary plane is identified with its image on the lower plane (and so on for
// edges and corners); every other vertex is its own representative.
static void periodic_canonical(const double* V, int64_t Nv, double lo, double hi, std::vector<int64_t>& canon) {
  const double L = hi - lo, tol = 1e-9 * L;
  canon.resize((size_t)Nv);
  struct Key {
    int64_t q[3];
    bool operator<(const Key& o) const {
      return q[0] != o.q[0] ? q[0] < o.q[0] : (q[1] != o.q[1] ? q[1] < o.q[1] : q[2] < o.q[2]);
    }
  };
  std::vector<std::pair<Key, int64_t>> keys;
  for (int64_t v = 0; v < Nv; ++v) {
    canon[(size_t)v] = v;
    bool on_bnd = false;
    Key k;
    for (int m = 0; m < 3; ++m) {
      double x = V[v * 3 + m] - lo;
      if (std::fabs(x) < tol || std::fabs(x - L) < tol) on_bnd = true;
      if (std::fabs(x - L) < tol) x = 0.0;
      k.q[m] = (int64_t)std::llround(x / L * 1e8);
    }
    if (on_bnd) keys.push_back({k, v});
  }
  std::sort(keys.begin(), keys.end(), [](const std::pair<Key, int64_t>& a, const std::pair<Key, int64_t>& b) {
    return a.first < b.first || (!(b.first < a.first) && a.second < b.second);
  });
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && !(keys[i].first < keys[j].first) && !(keys[j].first < keys[i].first)) ++j;
    for (size_t t = i; t < j; ++t) canon[(size_t)keys[t].second] = keys[i].second;
    i = j;
  }
}

int build_connectivity(const double* V, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                       std::vector<int64_t>& mapP, int64_t* nbnd, std::string& err, const double* period_box) {
  const int n1 = N + 1, n2 = n1 * n1, Nfc = 5 * n2;
  std::vector<int64_t> canon;
  const bool periodic = period_box != nullptr;
  const double pL = periodic ? period_box[1] - period_box[0] : 1.0;
  if (periodic) periodic_canonical(V, Nv, period_box[0], period_box[1], canon);
  std::vector<double> xg(n1), wg(n1), xf(n1), wf(n1);
  gauss_jacobi(n1, 0.0, 0.0, xg.data(), wg.data());
  gauss_jacobi(n1, 1.0, 0.0, xf.data(), wf.data());
  for (int64_t e = 0; e < K; ++e)
    for (int i = 0; i < 5; ++i)
      if (EToV[e * 5 + i] < 0 || EToV[e * 5 + i] >= Nv) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "EToV[%lld][%d] = %d is outside [0, %lld)", (long long)e, i,
                      EToV[e * 5 + i], (long long)Nv);
        err = buf;
        return -2;
      }
  std::vector<FaceKey> keys((size_t)K * 5);
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 5; ++f) {
      FaceKey& k = keys[(size_t)e * 5 + f];
      const int nv = f == 0 ? 4 : 3;
      for (int i = 0; i < 4; ++i) {
        if (i >= nv) {
          k.v[i] = INT64_MAX;
          continue;
        }
        const int64_t gv = EToV[e * 5 + kFaceVerts[f][i]];
        k.v[i] = periodic ? canon[(size_t)gv] : gv;
      }
      std::sort(k.v, k.v + 4);
      k.elem = e;
      k.face = f;
    }
  std::sort(keys.begin(), keys.end());
  mapP.resize((size_t)K * Nfc);
  for (int64_t g = 0; g < K * Nfc; ++g) mapP[(size_t)g] = g;
  int64_t boundary = 0;
  std::vector<double> X1((size_t)n2 * 3), X2((size_t)n2 * 3);
  double ev1[15], ev2[15];
  // Match the cubature points of faces A and B (coincident modulo the period on a
  // periodic box) under one of the face's point symmetries; on success write both
  // directions of mapP. Returns false if no symmetry makes the points coincide.
  auto try_pair = [&](const FaceKey& A, const FaceKey& B) -> bool {
    for (int m = 0; m < 15; ++m) {
      ev1[m] = V[(int64_t)EToV[A.elem * 5 + m / 3] * 3 + m % 3];
      ev2[m] = V[(int64_t)EToV[B.elem * 5 + m / 3] * 3 + m % 3];
    }
    double scale = 0.0;
    for (int idx = 0; idx < n2; ++idx) {
      double a, b, c;
      face_abc(A.face, idx, n1, xg.data(), xf.data(), &a, &b, &c);
      map_point(ev1, a, b, c, &X1[(size_t)idx * 3]);
      face_abc(B.face, idx, n1, xg.data(), xf.data(), &a, &b, &c);
      map_point(ev2, a, b, c, &X2[(size_t)idx * 3]);
    }
    for (int m = 0; m < 3; ++m) {
      double lo = X1[m], hi = X1[m];
      for (int idx = 1; idx < n2; ++idx) {
        lo = std::min(lo, X1[(size_t)idx * 3 + m]);
        hi = std::max(hi, X1[(size_t)idx * 3 + m]);
      }
      scale = std::max(scale, hi - lo);
    }
    const double tol = 1e-9 * scale;
    const int ncodes = A.face == 0 ? 8 : 2;
    int found = -1;
    for (int code = 0; code < ncodes && found < 0; ++code) {
      bool ok = true;
      for (int idx = 0; idx < n2 && ok; ++idx) {
        const int jdx = permute(code, idx, n1);
        for (int m = 0; m < 3; ++m) {
          double dx = X1[(size_t)idx * 3 + m] - X2[(size_t)jdx * 3 + m];
          if (periodic) dx -= pL * std::nearbyint(dx / pL);  // equal modulo the period
          if (std::fabs(dx) > tol) ok = false;
        }
      }
      if (ok) found = code;
    }
    if (found < 0) return false;
    for (int idx = 0; idx < n2; ++idx) {
      const int jdx = permute(found, idx, n1);
      const int64_t ga = A.elem * Nfc + (int64_t)A.face * n2 + idx;
      const int64_t gb = B.elem * Nfc + (int64_t)B.face * n2 + jdx;
      mapP[(size_t)ga] = gb;
      mapP[(size_t)gb] = ga;
    }
    return true;
  };
  size_t i = 0;
  while (i < keys.size()) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].same(keys[i])) ++j;
    const size_t cnt = j - i;
    if (cnt > 2 && !periodic) {
      err = "a face is shared by more than two elements";
      return -2;
    }
    if (cnt == 1) {
      ++boundary;
      i = j;
      continue;
    }
    if (cnt == 2) {
      if (!try_pair(keys[i], keys[i + 1])) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "face %d of element %lld and face %d of element %lld share vertices but not cubature "
                      "points (non-conforming collapse)",
                      keys[i].face, (long long)keys[i].elem, keys[i + 1].face, (long long)keys[i + 1].elem);
        err = buf;
        return -2;
      }
      i = j;
      continue;
    }
    // Periodic box with two cells along an axis: distinct faces can share all vertices
    // once opposite planes are identified; pair them by their cubature points.
    std::vector<char> used(cnt, 0);
    for (size_t a = 0; a < cnt; ++a) {
      if (used[a]) continue;
      for (size_t b2 = a + 1; b2 < cnt; ++b2) {
        if (used[b2] || keys[i + a].elem == keys[i + b2].elem) continue;
        if (try_pair(keys[i + a], keys[i + b2])) {
          used[a] = used[b2] = 1;
          break;
        }
      }
      if (!used[a]) ++boundary;
    }
    i = j;
  }
  if (nbnd) *nbnd = boundary;
  return 0;
}


// ------------------------------------------------------------ nodal variant
int gll_points(int n, double* x) {
  if (n < 1 || n > 64) return -1;
  if (n == 1) {
    x[0] = 0.0;
    return 0;
  }
  x[0] = -1.0;
  x[n - 1] = 1.0;
  if (n > 2) {  // interior GLL points: the zeros of P'_{n-1}, i.e. of P_{n-2}^{(1,1)}
    std::vector<double> xi(n - 2), wi(n - 2);
    gauss_jacobi(n - 2, 1.0, 1.0, xi.data(), wi.data());
    for (int i = 0; i < n - 2; ++i) x[i + 1] = xi[i];
  }
  return 0;
}

// In-place inverse of the n x n row-major matrix A (Gauss-Jordan, partial pivoting);
// returns false if a pivot vanishes.
static bool invert(std::vector<double>& A, int n) {
  std::vector<double> B((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) B[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * n + c]) > 1e-300)) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)piv * n + k], A[(size_t)c * n + k]);
        std::swap(B[(size_t)piv * n + k], B[(size_t)c * n + k]);
      }
    const double d = 1.0 / A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] *= d;
      B[(size_t)c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
        B[(size_t)r * n + k] -= f * B[(size_t)c * n + k];
      }
    }
  }
  A.swap(B);
  return true;
}

static double inf_norm(const std::vector<double>& A, int n) {
  double m = 0.0;
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += std::fabs(A[(size_t)r * n + c]);
    m = std::max(m, s);
  }
  return m;
}

int build_nodal(int N, NodalTables& nt) {
  if (N < 1 || N > 7) return -1;
  const int n1 = N + 1, Np = num_modes(N), nT = n1 * (n1 + 1) / 2;
  nt.N = N;
  nt.Np = Np;
  nt.nT = nT;
  std::vector<double> cl(n1);
  gll_points(n1, cl.data());
  // nodes: layer m at c = cl[m], the (N+1-m)^2 GLL grid in (a, b); apex layer (0, 0, 1)
  nt.nodes.clear();
  std::vector<int> off(n1 + 1, 0);
  for (int m = 0; m <= N; ++m) {
    const int nm = n1 - m;
    std::vector<double> xs(nm);
    gll_points(nm, xs.data());
    off[m + 1] = off[m] + nm * nm;
    for (int q = 0; q < nm; ++q)
      for (int p = 0; p < nm; ++p) {
        nt.nodes.push_back(xs[p]);
        nt.nodes.push_back(xs[q]);
        nt.nodes.push_back(cl[m]);
      }
  }
  // Vandermonde of the semi-nodal basis phi_(k,j,i) = l_i^k(a) l_j^k(b) G_k(c) at the nodes
  std::vector<std::vector<double>> xk(n1);
  for (int k = 0; k <= N; ++k) {
    std::vector<double> w(k + 1);
    xk[k].resize(k + 1);
    gauss_jacobi(k + 1, 0.0, 0.0, xk[k].data(), w.data());
  }
  nt.V.assign((size_t)Np * Np, 0.0);
  std::vector<double> La(n1), Lb(n1), dL(n1);
  for (int i = 0; i < Np; ++i) {
    const double a = nt.nodes[3 * i], b = nt.nodes[3 * i + 1], c = nt.nodes[3 * i + 2];
    for (int k = 0; k <= N; ++k) {
      double Gk = 0.0;
      cfun(N, k, c, &Gk, nullptr, nullptr);
      lagrange(xk[k].data(), k + 1, a, La.data(), dL.data());
      lagrange(xk[k].data(), k + 1, b, Lb.data(), dL.data());
      for (int j = 0; j <= k; ++j)
        for (int ii = 0; ii <= k; ++ii) nt.V[(size_t)i * Np + lvl_off(k) + j * (k + 1) + ii] = La[ii] * Lb[j] * Gk;
    }
  }
  std::vector<double> Vinv = nt.V;
  if (!invert(Vinv, Np)) return -2;
  nt.cond_inf = inf_norm(nt.V, Np) * inf_norm(Vinv, Np);
  nt.VT.assign((size_t)Np * Np, 0.0);
  nt.VinvT.assign((size_t)Np * Np, 0.0);
  for (int i = 0; i < Np; ++i)
    for (int n = 0; n < Np; ++n) {
      nt.VT[(size_t)n * Np + i] = nt.V[(size_t)i * Np + n];
      nt.VinvT[(size_t)i * Np + n] = Vinv[(size_t)n * Np + i];
    }
  // triangle face: nodes (e, c) per layer (GLL points of the layer's edge), apex last; P_N basis
  // chi_(al,be)(e, c) = P_al(e) ((1-c)/2)^al P_be^{(2al+1,0)}(c), al + be <= N
  std::vector<double> te, tc;
  for (int m = 0; m <= N; ++m) {
    const int nm = n1 - m;
    std::vector<double> xs(nm);
    gll_points(nm, xs.data());
    for (int t = 0; t < nm; ++t) {
      te.push_back(nm == 1 ? 0.0 : xs[t]);
      tc.push_back(cl[m]);
    }
  }
  auto chi = [&](double e, double c, double* out) {
    int col = 0;
    for (int al = 0; al <= N; ++al)
      for (int be = 0; al + be <= N; ++be)
        out[col++] = jacobi_p(al, 0.0, 0.0, e) * std::pow(0.5 * (1.0 - c), al) * jacobi_p(be, 2.0 * al + 1.0, 0.0, c);
  };
  std::vector<double> Vt((size_t)nT * nT);
  for (int j = 0; j < nT; ++j) chi(te[j], tc[j], &Vt[(size_t)j * nT]);
  if (!invert(Vt, nT)) return -2;  // Vt now holds the Lagrange coefficients (columns)
  std::vector<double> xg(n1), wg(n1), xf(n1), wf(n1), row(nT), Lq((size_t)n1 * n1 * nT);
  gauss_jacobi(n1, 0.0, 0.0, xg.data(), wg.data());
  gauss_jacobi(n1, 1.0, 0.0, xf.data(), wf.data());
  std::vector<double> wq((size_t)n1 * n1);
  for (int mq = 0; mq < n1; ++mq)
    for (int eq = 0; eq < n1; ++eq) {
      const int qi = eq + n1 * mq;
      wq[qi] = wg[eq] * 0.5 * wf[mq];  // collapse factor (1-c)/2 in the Gauss-Jacobi (1,0) weights
      chi(xg[eq], xf[mq], row.data());
      for (int j = 0; j < nT; ++j) {
        double v = 0.0;
        for (int r = 0; r < nT; ++r) v += row[r] * Vt[(size_t)r * nT + j];
        Lq[(size_t)qi * nT + j] = v;
      }
    }
  nt.Mtri.assign((size_t)nT * nT, 0.0);
  for (int qi = 0; qi < n1 * n1; ++qi)
    for (int i = 0; i < nT; ++i)
      for (int j = 0; j < nT; ++j)
        nt.Mtri[(size_t)i * nT + j] += wq[qi] * Lq[(size_t)qi * nT + i] * Lq[(size_t)qi * nT + j];
  // GLL -> Gauss-Legendre interpolation on the base edge
  std::vector<double> xl(n1);
  gll_points(n1, xl.data());
  nt.I1.assign((size_t)n1 * n1, 0.0);
  for (int q = 0; q < n1; ++q) {
    lagrange(xl.data(), n1, xg[q], La.data(), dL.data());
    for (int p = 0; p < n1; ++p) nt.I1[(size_t)q * n1 + p] = La[p];
  }
  // element node of each triangle-face node: face 1 b = -1, 2 a = +1, 3 b = +1, 4 a = -1;
  // local node (m, t) with t along the face's edge coordinate (a on faces 1 and 3, b on 2 and 4)
  nt.tri_node.assign((size_t)4 * nT, 0);
  for (int f = 1; f <= 4; ++f) {
    int j = 0;
    for (int m = 0; m <= N; ++m) {
      const int nm = n1 - m;
      for (int t = 0; t < nm; ++t, ++j) {
        int p = 0, q = 0;
        if (nm > 1) {
          if (f == 1) { p = t; q = 0; }
          else if (f == 2) { p = nm - 1; q = t; }
          else if (f == 3) { p = t; q = nm - 1; }
          else { p = 0; q = t; }
        }
        nt.tri_node[(size_t)(f - 1) * nT + j] = off[m] + q * nm + p;
      }
    }
  }
  return 0;
}

}  // namespace pyrdg
