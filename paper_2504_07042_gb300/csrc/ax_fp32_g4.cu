// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 12, 13.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g4
#define AX_N_LIST(X) X(12) X(13)
#include "inst_fiber.inc"
