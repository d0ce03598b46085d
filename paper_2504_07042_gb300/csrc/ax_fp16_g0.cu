// AxLocal kernels with FP16 tensor-core contractions, orders N = 1..5.
#define AX_MODE tcx::kFP16
#define AX_TAG fp16_g0
#define AX_N_LIST(X) X(1) X(2) X(3) X(4) X(5)
#include "inst_tc.inc"
