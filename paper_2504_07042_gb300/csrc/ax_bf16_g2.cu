// AxLocal kernels with BF16 tensor-core contractions, orders N = 10..15.
#define AX_MODE tcx::kBF16
#define AX_TAG bf16_g2
#define AX_N_LIST(X) X(10) X(11) X(12) X(13) X(14) X(15)
#include "inst_tc.inc"
