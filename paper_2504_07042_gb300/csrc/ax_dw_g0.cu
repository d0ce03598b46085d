// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 1, 2, 3, 4, 5.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g0
#define AX_N_LIST(X) X(1) X(2) X(3) X(4) X(5)
#include "inst_fiber.inc"
