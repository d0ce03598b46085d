// Design instruction counts of the fiber-per-thread AxLocal kernels
// (ax_fiber.cuh), per node, on the binding arithmetic pipe (FP64 pipe for
// native FP64, FP32 pipe for native FP32 and double-word).  Used by
// ax_query for the time-based roofline of Sec. 3.4.
#include "ax_internal.h"

namespace ax {

double pipe_ops_per_node(int N1, int kind, int prec) {
  const bool dwp = (prec == AX_F64DW);
  const bool tc = (prec == AX_TF32 || prec == AX_BF16 || prec == AX_FP16);
  // cost of one scalar op in the arithmetic (dw.cuh): normalised sum, sum
  // without the final Fast2Sum, product, first product of an accumulator,
  // multiply-accumulate, finalisation, a*b + c, sum of two accumulators
  const double add = dwp ? 11.0 : 1.0, lazy = dwp ? 8.0 : 1.0, mul = dwp ? 9.0 : 1.0;
  const double mul0 = dwp ? 4.0 : 1.0, mac = dwp ? 12.0 : 1.0, fin = dwp ? 3.0 : 0.0;
  const double fma = dwp ? 15.0 : 1.0, accsum = dwp ? 8.0 : 1.0;
  const double div = dwp ? 14.0 : 8.0;
  // one even-odd fiber product of length N1 (c = N1/2 output pairs): 2c
  // even/odd sums, N1 accumulators started by a product, the remaining
  // terms as multiply-accumulates, each output pair formed from its two
  // accumulators (N1 = 16: finalised first, then a normalised sum each),
  // the middle output of odd N1 finalised
  const int c = N1 / 2, odd = N1 & 1;
  const double terms = c * (2.0 * c + odd) + odd * c;
  const double pair = N1 < 16 ? 2.0 * accsum : 2.0 * fin + 2.0 * add;
  const double fiber = 2.0 * c * lazy + N1 * mul0 + (terms - N1) * mac + c * pair + odd * fin;
  // six contractions, each node in one fiber of each; on the tensor cores
  // only the operand conversions stay on the FP32 pipe (one per operand for
  // TF32, one per pair for the 16-bit formats)
  double ops = tc ? (prec == AX_TF32 ? 6.0 : 3.0) : 6.0 * fiber / N1;
  const double dot3 = mul0 + 2.0 * mac + fin, det2 = mul0 + mac + fin;
  ops += 3.0 * dot3;                      // (r, s, t) = G (x0, x1, x2)
  ops += dwp ? 17.0 : 2.0;                // Y = Y_t + Y_r + Y_s (two TwoSums and the low parts)
  // trilinear geometry (Algorithm 2 with K = J^T J and det J as polynomials in t):
  // per thread (i,j), from the record's monomial coefficients: J2 (a 3-term
  // dot product plus C, and rs), the axis terms E0/E1 with the K00
  // coefficients (per s) and F0/F1 with the K11 coefficients (per r): 12
  // multiply-adds, 6 dot products, 2 exact doublings; the 9 dot products of
  // the K01, K02, K12, K22 coefficients and, for det J, 6 two-term
  // determinants and 4 dot products; all amortised over the N1 nodes of the
  // thread's fiber.  Where the kernel shares the axis terms (native FP64;
  // double-word up to N1 = 6) the first 2 N1 threads of an element compute
  // them once, counted as the whole warps that run them (an element's share
  // of a warp below 32 threads per element).
  const bool share = (kind == AX_GEOM_TRILINEAR || kind == AX_GEOM_TRILINEAR_PARTIAL) &&
                     (dwp ? N1 <= 6 : prec == AX_FP64);
  const double twice = dwp ? 2.0 : 1.0;
  const double axis_set = 6.0 * fma + 3.0 * dot3 + twice;  // one r- or s-axis set
  const int F = N1 * N1;
  const double axis_lanes = F < 32 ? F : 32.0 * ((2 * N1 + 31) / 32);
  const double axis = share ? axis_lanes * axis_set / F : 2.0 * axis_set;  // per thread
  const double cols = 3.0 * (dot3 + add) + mul;
  const double coeffs = 9.0 * dot3 + add + axis, det_coeffs = 6.0 * det2 + 4.0 * dot3 + add;
  const double quad = 2.0 * fma, lin = fma;
  const double knode = 3.0 * quad + 2.0 * lin, adj = 6.0 * det2, scale = 3.0 * mul;
  switch (kind) {
    case AX_GEOM_STORED: break;
    case AX_GEOM_PARALLELEPIPED: ops += mul + 3.0 * mul; break;
    case AX_GEOM_TRILINEAR:
      ops += knode + quad + adj + mul + div + scale + (cols + coeffs + det_coeffs) / N1;
      break;
    case AX_GEOM_TRILINEAR_PARTIAL: ops += knode + adj + scale + (cols + coeffs) / N1; break;
  }
  return ops;
}

}  // namespace ax
