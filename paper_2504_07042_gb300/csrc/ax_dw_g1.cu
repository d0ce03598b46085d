// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 6, 7.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g1
#define AX_N_LIST(X) X(6) X(7)
#include "inst_fiber.inc"
