// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 6, 7.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g1
#define AX_N_LIST(X) X(6) X(7)
#include "inst_fiber.inc"
