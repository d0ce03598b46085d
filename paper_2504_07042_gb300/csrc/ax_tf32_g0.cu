// AxLocal kernels with TF32 tensor-core contractions, orders N = 1..5.
#define AX_MODE tcx::kTF32
#define AX_TAG tf32_g0
#define AX_N_LIST(X) X(1) X(2) X(3) X(4) X(5)
#include "inst_tc.inc"
