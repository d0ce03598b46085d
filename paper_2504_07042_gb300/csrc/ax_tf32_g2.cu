// AxLocal kernels with TF32 tensor-core contractions, orders N = 10..15.
#define AX_MODE tcx::kTF32
#define AX_TAG tf32_g2
#define AX_N_LIST(X) X(10) X(11) X(12) X(13) X(14) X(15)
#include "inst_tc.inc"
