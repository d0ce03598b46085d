// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 10, 11.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g3
#define AX_N_LIST(X) X(10) X(11)
#include "inst_fiber.inc"
