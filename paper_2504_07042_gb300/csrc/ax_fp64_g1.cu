// AxLocal kernels, native FP64 arithmetic, orders N = 6, 7.
#define AX_T double
#define AX_TAG fp64_g1
#define AX_N_LIST(X) X(6) X(7)
#include "inst_native.inc"
