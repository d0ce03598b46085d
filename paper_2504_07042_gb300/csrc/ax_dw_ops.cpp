// Design instruction counts of the double-word kernels (see ax_dw.cuh).
#include "ax_internal.h"

namespace ax {

// FP32-pipe instructions per node of this kernel (design count): a
// double-word multiply-accumulate is 12 instructions; contractions 6*N1 of
// them, the geometric product 9, plus finalisation and the geometry by kind.
double dw_ops_per_node(int N1, int kind) {
  const double mac = 12.0;
  double ops = 6.0 * N1 * mac + 9.0 * mac + 6 * 3.0;
  switch (kind) {
    case AX_GEOM_STORED: break;
    case AX_GEOM_PARALLELEPIPED: ops += 7 * 9.0; break;
    case AX_GEOM_TRILINEAR: ops += 6 * 20.0 + 5 * 27.0 + 6 * 27.0 + 3 * 27.0 + 27.0 + 9.0 + 16.0 + 6 * 9.0; break;
    case AX_GEOM_TRILINEAR_PARTIAL: ops += 6 * 20.0 + 5 * 27.0 + 6 * 27.0 + 9.0 + 6 * 9.0; break;
  }
  return ops;
}

}  // namespace ax
