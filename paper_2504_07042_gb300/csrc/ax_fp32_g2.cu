// AxLocal kernels, native FP32 arithmetic, orders N = 8, 9.
#define AX_T float
#define AX_TAG fp32_g2
#define AX_N_LIST(X) X(8) X(9)
#include "inst_native.inc"
