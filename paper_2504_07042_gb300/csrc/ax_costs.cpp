// Design instruction counts of the fiber-per-thread AxLocal kernels
// (ax_fiber.cuh), per node, on the binding arithmetic pipe (FP64 pipe for
// native FP64, FP32 pipe for native FP32 and double-word).  Used by
// ax_query for the time-based roofline of Sec. 3.4.
#include "ax_internal.h"

namespace ax {

double pipe_ops_per_node(int N1, int kind, int prec) {
  const bool dwp = (prec == AX_F64DW);
  const bool tc = (prec == AX_TF32 || prec == AX_BF16 || prec == AX_FP16);
  // cost of one scalar op in the arithmetic: add, multiply, multiply-accumulate, finalise
  const double add = dwp ? 11.0 : 1.0, mul = dwp ? 9.0 : 1.0, mac = dwp ? 12.0 : 1.0, fin = dwp ? 3.0 : 0.0;
  const double div = dwp ? 14.0 : 8.0;
  const double fma = dwp ? mul + add : 1.0;  // a*b + c: one FFMA/DFMA natively, a product and a sum in double-word
  // one even-odd fiber product of length N1: N1 prep adds, N1^2/2 macs, N1 finalisations, N1 post adds
  const double fiber = N1 * add + 0.5 * N1 * N1 * mac + N1 * fin + N1 * add;
  // six contractions, each node in one fiber of each; on the tensor cores
  // only the operand conversions stay on the FP32 pipe (one per operand for
  // TF32, one per pair for the 16-bit formats)
  double ops = tc ? (prec == AX_TF32 ? 6.0 : 3.0) : 6.0 * fiber / N1;
  ops += 3.0 * (3.0 * mac + fin);        // (r, s, t) = G (x0, x1, x2)
  ops += 2.0 * add;                      // Y accumulation of passes 3 and 4
  // trilinear geometry (Algorithm 2 with K = J^T J and det J as polynomials in t):
  // per thread (i,j), from the record's monomial coefficients: E0/E1/F0/F1
  // (12 multiply-adds), J2 (3 dot products of 3 terms plus C), the 15 dot
  // products of the K coefficients and, for det J, 6 two-term determinants
  // and 4 dot products, amortised over the N1 nodes of its fiber
  const double dot3 = 3.0 * mac + fin, det2 = 2.0 * mac + fin;
  const double cols = 12.0 * (mul + add) + 3.0 * (3.0 * mac + fin + add) + mul;
  const double coeffs = 15.0 * dot3 + 3.0 * add, det_coeffs = 6.0 * det2 + 4.0 * dot3 + add;
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
