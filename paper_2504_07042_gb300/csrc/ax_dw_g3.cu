// AxLocal kernels, double-word arithmetic, orders N = 10, 11.
#define AX_TAG dw_g3
#define AX_N_LIST(X) X(10) X(11)
#include "inst_dw.inc"
