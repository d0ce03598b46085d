// AxLocal with the six sum-factorised contractions of Algorithm 1 on the
// tensor cores (TF32, BF16 or FP16 operands, FP32 accumulation); X, Y, the
// geometry and (r,s,t) = G (x0,x1,x2) stay FP32.  Every order runs on the
// tcgen05 kernels of ax_umma.cuh: the kernel tuned for order 7 (N1 = 8) and
// the order-sized kernel for every other order.  (A warp-level mma.sync
// m16n8k8 form, kept earlier as a second variant for the autotuner, measured
// slower at every order once the order-sized tcgen05 kernel had its searched
// layouts and CTA counts, and was removed.)
#pragma once

#include <cuda_runtime.h>

#include "ax_umma.cuh"

namespace ax {
namespace tcx {

enum Mode { kTF32 = 0, kBF16 = 1, kFP16 = 2 };  // the operand format (umma's OP)

template <int MODE, int N1, int KIND>
cudaError_t launch_tc_kind(const AxArgs &a, const float *Dp) {
  if constexpr (N1 == 8)
    return umma::launch_kind<KIND, MODE>(a, Dp);
  else
    return umma::launch_gen<N1, KIND, MODE>(a, Dp);
}

// AxLocal of order N1 - 1 in operand format MODE; Dp: the order's plain D
template <int MODE, int N1>
cudaError_t launch_tc_n(const AxArgs &a, const float *Dp) {
  switch (a.kind) {
    case AX_GEOM_STORED: return launch_tc_kind<MODE, N1, AX_GEOM_STORED>(a, Dp);
    case AX_GEOM_TRILINEAR: return launch_tc_kind<MODE, N1, AX_GEOM_TRILINEAR>(a, Dp);
    case AX_GEOM_PARALLELEPIPED: return launch_tc_kind<MODE, N1, AX_GEOM_PARALLELEPIPED>(a, Dp);
    case AX_GEOM_TRILINEAR_PARTIAL: return launch_tc_kind<MODE, N1, AX_GEOM_TRILINEAR_PARTIAL>(a, Dp);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tcx
}  // namespace ax
