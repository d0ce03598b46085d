// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 14.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g5
#define AX_N_LIST(X) X(14)
#include "inst_fiber.inc"
