// AxLocal kernels, native FP64 arithmetic, orders N = 14.
#define AX_T double
#define AX_TAG fp64_g5
#define AX_N_LIST(X) X(14)
#include "inst_native.inc"
