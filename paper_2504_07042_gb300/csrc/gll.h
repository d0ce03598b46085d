// GLL constants (Table 1) for the library; see gll.cpp.
#pragma once

namespace ax {

constexpr int kMaxN = 15;
constexpr int kMaxN1 = kMaxN + 1;

// Fill x[N1], w[N1], D[N1*N1] (row-major D[i][j] = pi_j'(x_i)).  false if N is out of range.
bool gll_tables(int N, double *x, double *w, double *D);

}  // namespace ax
