// AxLocal kernels, double-word arithmetic, orders N = 12, 13.
#define AX_TAG dw_g4
#define AX_N_LIST(X) X(12) X(13)
#include "inst_dw.inc"
