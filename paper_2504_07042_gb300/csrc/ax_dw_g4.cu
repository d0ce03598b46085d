// AxLocal kernels (fiber-per-thread), double-word arithmetic, orders N = 12, 13.
#define AX_POLICY fiber::DW
#define AX_CT float2
#define AX_TAG dw_g4
#define AX_N_LIST(X) X(12) X(13)
#include "inst_fiber.inc"
