// AxLocal kernels, native FP32 arithmetic, orders N = 14.
#define AX_T float
#define AX_TAG fp32_g5
#define AX_N_LIST(X) X(14)
#include "inst_native.inc"
