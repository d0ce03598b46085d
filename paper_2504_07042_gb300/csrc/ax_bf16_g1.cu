// AxLocal kernels with BF16 tensor-core contractions, orders N = 6..9.
#define AX_MODE tcx::kBF16
#define AX_TAG bf16_g1
#define AX_N_LIST(X) X(6) X(7) X(8) X(9)
#include "inst_tc.inc"
