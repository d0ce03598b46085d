// AxLocal kernels, native FP32 arithmetic, orders N = 6, 7.
#define AX_T float
#define AX_TAG fp32_g1
#define AX_N_LIST(X) X(6) X(7)
#include "inst_native.inc"
