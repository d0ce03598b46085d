// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 15.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g6
#define AX_N_LIST(X) X(15)
#include "inst_fiber.inc"
