// AxLocal kernels with TF32 tensor-core contractions, orders N = 6..9.
#define AX_MODE tcx::kTF32
#define AX_TAG tf32_g1
#define AX_N_LIST(X) X(6) X(7) X(8) X(9)
#include "inst_tc.inc"
