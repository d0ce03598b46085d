// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 15.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g6
#define AX_N_LIST(X) X(15)
#include "inst_fiber.inc"
