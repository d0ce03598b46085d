// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 8, 9.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g2
#define AX_N_LIST(X) X(8) X(9)
#include "inst_fiber.inc"
