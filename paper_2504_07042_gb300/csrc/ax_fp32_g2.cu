// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 8, 9.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g2
#define AX_N_LIST(X) X(8) X(9)
#include "inst_fiber.inc"
