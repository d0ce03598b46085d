// GLL tables of Table 1 for the library (host code).
//
// Points: -1, +1 and the N-1 zeros of L_N', found by Newton's method on
//   L_N'(x) with L_N'' from the Legendre differential equation, starting from
//   the Chebyshev-Gauss-Lobatto points; evaluated in double.
// Weights: w_i = 2 / (N (N+1) L_N(x_i)^2)   (Table 1).
// Differentiation matrix D[i][j] = pi_j'(x_i), by the barycentric formula
//   (Berrut & Trefethen, SIAM Review 46, 2004): with lambda_j = 1 / prod_{m!=j}(x_j - x_m),
//   D[i][j] = (lambda_j / lambda_i) / (x_i - x_j) for i != j, and the diagonal
//   from the rows summing to zero (D 1 = 0), which keeps D exact on constants.
#include "gll.h"

#include <cmath>

namespace ax {

static void legendre(int N, double x, double *L, double *dL) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { *L = 1.0; *dL = 0.0; return; }
  for (int n = 2; n <= N; ++n) {
    const double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
    const double d2 = d0 + (2.0 * n - 1.0) * p1;  // L_n' = L_{n-2}' + (2n-1) L_{n-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *L = p1; *dL = d1;
}

bool gll_tables(int N, double *x, double *w, double *D) {
  if (N < 1 || N > kMaxN) return false;
  const int N1 = N + 1;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 60; ++it) {
      double L, dL;
      legendre(N, z, &L, &dL);
      const double d2L = (2.0 * z * dL - N * (N + 1.0) * L) / (1.0 - z * z);
      const double dz = dL / d2L;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[i] = z;
  }
  // symmetrise (the exact points are symmetric about 0)
  for (int i = 0; i < N1 / 2; ++i) {
    const double a = 0.5 * (x[N - i] - x[i]);
    x[i] = -a;
    x[N - i] = a;
  }
  if (N1 % 2) x[N / 2] = 0.0;
  for (int i = 0; i < N1; ++i) {
    double L, dL;
    legendre(N, x[i], &L, &dL);
    w[i] = 2.0 / (N * (N + 1.0) * L * L);
  }
  double lam[kMaxN1];
  for (int j = 0; j < N1; ++j) {
    double p = 1.0;
    for (int m = 0; m < N1; ++m)
      if (m != j) p *= (x[j] - x[m]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < N1; ++i) {
    double diag = 0.0;
    for (int j = 0; j < N1; ++j) {
      if (j == i) continue;
      const double d = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * N1 + j] = d;
      diag -= d;
    }
    D[i * N1 + i] = diag;
  }
  return true;
}

}  // namespace ax
