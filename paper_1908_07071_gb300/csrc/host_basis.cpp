// Host-side 1D rules and bases (Sections 2 and 3.1: GLL-nodal Q_p bases and the
// Gauss-Lobatto-refined low-order grid; Section 3.3: the element-structured
// level hierarchy).  Computed in long double, returned as double.
#include <cmath>
#include <vector>

#include "lor_internal.h"

namespace lorh {

// Legendre P_n(x) and its first derivative by the Bonnet recurrence carried
// together with its derivative (P_k' = P_{k-2}' + (2k-1) P_{k-1}).
static void legendre_pd(int n, long double x, long double* P, long double* dP) {
  long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
  if (n == 0) { *P = 1.0L; *dP = 0.0L; return; }
  for (int k = 2; k <= n; ++k) {
    long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    long double d2 = d0 + (2 * k - 1) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

void gll(int p, double* x, double* w) {
  // interior nodes: roots of P_p' on (-1,1), Newton with P_p'' from the
  // Legendre equation (1-x^2) P'' = 2x P' - p(p+1) P.
  std::vector<long double> t(p + 1);
  t[0] = -1.0L; t[p] = 1.0L;
  for (int i = 1; i < p; ++i) {
    long double z = -cosl(3.14159265358979323846264338327950288L * i / p);
    for (int it = 0; it < 200; ++it) {
      long double P, dP;
      legendre_pd(p, z, &P, &dP);
      long double d2 = (2.0L * z * dP - p * (p + 1.0L) * P) / (1.0L - z * z);
      long double dz = dP / d2;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    t[i] = z;
  }
  for (int i = 0; i <= p; ++i) {
    long double P, dP;
    legendre_pd(p, t[i], &P, &dP);
    x[i] = (double)(0.5L * (t[i] + 1.0L));
    w[i] = (double)(1.0L / (p * (p + 1.0L) * P * P));   // 2/(p(p+1)P^2), halved for [0,1]
  }
}

void gauss(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    long double z = -cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (q + 0.5L));
    long double P, dP;
    for (int it = 0; it < 200; ++it) {
      legendre_pd(q, z, &P, &dP);
      long double dz = P / dP;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    legendre_pd(q, z, &P, &dP);
    x[i] = (double)(0.5L * (z + 1.0L));
    w[i] = (double)(1.0L / ((1.0L - z * z) * dP * dP));   // 2/((1-z^2)P'^2), halved
  }
}

// Barycentric Lagrange interpolation and differentiation (Berrut & Trefethen,
// SIAM Review 46(3), 2004): lambda_i = 1/prod_{j!=i}(x_i-x_j).
void lagrange(int m, const double* nodes, int nt, const double* t, double* B, double* D) {
  std::vector<long double> lam(m, 1.0L);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      if (j != i) lam[i] /= ((long double)nodes[i] - nodes[j]);
  for (int a = 0; a < nt; ++a) {
    long double ta = t[a];
    int hit = -1;
    for (int i = 0; i < m; ++i)
      if (fabsl(ta - nodes[i]) < 1e-15L) hit = i;
    if (hit >= 0) {
      // row `hit` of the nodal differentiation matrix
      long double diag = 0.0L;
      for (int i = 0; i < m; ++i) {
        B[a * m + i] = (i == hit) ? 1.0 : 0.0;
        if (i != hit) {
          long double dki = (lam[i] / lam[hit]) / ((long double)nodes[hit] - nodes[i]);
          D[a * m + i] = (double)dki;
          diag -= dki;
        }
      }
      D[a * m + hit] = (double)diag;
      continue;
    }
    long double den = 0.0L;
    for (int i = 0; i < m; ++i) den += lam[i] / (ta - nodes[i]);
    long double sinv = 0.0L;
    for (int j = 0; j < m; ++j) sinv += 1.0L / (ta - nodes[j]);
    for (int i = 0; i < m; ++i) {
      long double li = (lam[i] / (ta - nodes[i])) / den;
      B[a * m + i] = (double)li;
      // l_i'/l_i = sum_{j != i} 1/(t - x_j)
      D[a * m + i] = (double)(li * (sinv - 1.0L / (ta - nodes[i])));
    }
  }
}

std::vector<std::vector<int>> level_selections(int p, int mg_levels) {
  std::vector<std::vector<int>> out;
  std::vector<int> s(p + 1);
  for (int i = 0; i <= p; ++i) s[i] = i;
  out.push_back(s);
  while (out.back().size() > 2) {
    const std::vector<int>& f = out.back();
    std::vector<int> c;
    for (size_t i = 0; i < f.size(); i += 2) c.push_back(f[i]);
    if (c.back() != f.back()) c.push_back(f.back());
    out.push_back(c);
  }
  if (mg_levels >= 2 && mg_levels < (int)out.size()) {
    std::vector<std::vector<int>> cut(out.begin(), out.begin() + (mg_levels - 1));
    cut.push_back(out.back());
    out = cut;
  }
  return out;
}

}  // namespace lorh
