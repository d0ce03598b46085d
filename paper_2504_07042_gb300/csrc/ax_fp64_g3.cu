// AxLocal kernels, native FP64 arithmetic, orders N = 10, 11.
#define AX_T double
#define AX_TAG fp64_g3
#define AX_N_LIST(X) X(10) X(11)
#include "inst_native.inc"
