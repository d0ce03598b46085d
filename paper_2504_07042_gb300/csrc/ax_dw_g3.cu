// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 10, 11.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g3
#define AX_N_LIST(X) X(10) X(11)
#include "inst_fiber.inc"
