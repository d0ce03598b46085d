// AxLocal kernels, native FP32 arithmetic, orders N = 15.
#define AX_T float
#define AX_TAG fp32_g6
#define AX_N_LIST(X) X(15)
#include "inst_native.inc"
