// AxLocal kernels, double-word arithmetic, orders N = 15.
#define AX_TAG dw_g6
#define AX_N_LIST(X) X(15)
#include "inst_dw.inc"
