// Per-translation-unit constant-memory copies of the GLL tables (Table 1)
// for every supported order, so that contexts of different N can coexist.
// Each .cu file that includes this header gets its own copy (internal
// linkage) and uploads it once per device through upload_tables<T>().
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "gll.h"

namespace ax {

// Offsets of order N1 (2..16) inside the packed tables.
__host__ __device__ constexpr int tab_off_D(int N1) { return (N1 - 1) * N1 * (2 * N1 - 1) / 6 - 1; }  // sum_{m=2}^{N1-1} m^2
__host__ __device__ constexpr int tab_off_v(int N1) { return (N1 - 1) * N1 / 2 - 1; }                 // sum_{m=2}^{N1-1} m
constexpr int kTabD = tab_off_D(kMaxN1 + 1);
constexpr int kTabV = tab_off_v(kMaxN1 + 1);
// Offsets of order N1 inside the paired even-odd tables (floor(N1/2)^2
// entries per order): sum_{m=2}^{N1-1} floor(m/2)^2
__host__ __device__ constexpr int tab_off_P(int N1) {
  int s = 0;
  for (int m = 2; m < N1; ++m) s += (m / 2) * (m / 2);
  return s;
}
constexpr int kTabP = tab_off_P(kMaxN1 + 1);

// Fill packed host tables (double) for all orders 1..kMaxN.
inline bool build_packed_tables(double *D, double *w, double *x) {
  for (int N = 1; N <= kMaxN; ++N) {
    const int N1 = N + 1;
    double xx[kMaxN1], ww[kMaxN1], DD[kMaxN1 * kMaxN1];
    if (!gll_tables(N, xx, ww, DD)) return false;
    for (int q = 0; q < N1 * N1; ++q) D[tab_off_D(N1) + q] = DD[q];
    for (int q = 0; q < N1; ++q) {
      w[tab_off_v(N1) + q] = ww[q];
      x[tab_off_v(N1) + q] = xx[q];
    }
  }
  return true;
}

// Even-odd blocks (see ax_fiber.cuh) of D and of D^T for every order, from
// the packed D tables.  Block of order N1 at tab_off_D(N1), c = N1/2:
//   rows i < c: [ (M[i][m]+M[i][N-m])/2 , (M[i][m]-M[i][N-m])/2 (m < c) | M[i][c] if N1 odd ]
//   row c (N1 odd): M[c][m], m < c.
inline void build_eo_tables(const double *Dp, double *eoD, double *eoDT) {
  for (int N1 = 2; N1 <= kMaxN1; ++N1) {
    const double *D = Dp + tab_off_D(N1);
    const int c = N1 / 2, N = N1 - 1;
    for (int t = 0; t < 2; ++t) {
      double *out = (t == 0 ? eoD : eoDT) + tab_off_D(N1);
      auto M = [&](int a, int b) { return t == 0 ? D[a * N1 + b] : D[b * N1 + a]; };
      for (int q = 0; q < N1 * N1; ++q) out[q] = 0.0;
      for (int i = 0; i < c; ++i) {
        for (int m = 0; m < c; ++m) {
          out[i * N1 + m] = 0.5 * (M(i, m) + M(i, N - m));
          out[i * N1 + c + m] = 0.5 * (M(i, m) - M(i, N - m));
        }
        if (N1 & 1) out[i * N1 + 2 * c] = M(i, c);
      }
      if (N1 & 1)
        for (int m = 0; m < c; ++m) out[c * N1 + m] = M(c, m);
    }
  }
}

// Paired even-odd tables for the packed double-word fiber product
// (dw2.cuh): for every order, entry i * c + m (i, m < c = N1/2) holds the
// pair (A, B) = (eo[i][m], eo[i][c + m]) of the even-odd block, as
// pair[4 * q + 0..1] = (A, B) and pair[4 * q + 2..3] = (A, B) again (the
// caller splits the second copy into low parts).
inline void build_pair_tables(const double *eoD, const double *eoDT, double *pD, double *pDT) {
  for (int N1 = 2; N1 <= kMaxN1; ++N1) {
    const int c = N1 / 2;
    for (int t = 0; t < 2; ++t) {
      const double *eo = (t == 0 ? eoD : eoDT) + tab_off_D(N1);
      double *out = (t == 0 ? pD : pDT) + 4 * tab_off_P(N1);
      for (int i = 0; i < c; ++i)
        for (int m = 0; m < c; ++m) {
          const double A = eo[i * N1 + m], B = eo[i * N1 + c + m];
          double *q = out + 4 * (i * c + m);
          q[0] = A;
          q[1] = B;
          q[2] = A;
          q[3] = B;
        }
    }
  }
}

// Per-device "uploaded" bookkeeping for one translation unit.
struct UploadOnce {
  std::mutex mu;
  unsigned long long done = 0;  // bit per device ordinal (< 64)
};

}  // namespace ax
