// AxLocal kernels with FP16 tensor-core contractions, orders N = 10..15.
#define AX_MODE tcx::kFP16
#define AX_TAG fp16_g2
#define AX_N_LIST(X) X(10) X(11) X(12) X(13) X(14) X(15)
#include "inst_tc.inc"
