// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 14.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g5
#define AX_N_LIST(X) X(14)
#include "inst_fiber.inc"
