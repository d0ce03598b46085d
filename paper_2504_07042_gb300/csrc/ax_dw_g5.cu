// AxLocal kernels, double-word arithmetic, orders N = 14.
#define AX_TAG dw_g5
#define AX_N_LIST(X) X(14)
#include "inst_dw.inc"
