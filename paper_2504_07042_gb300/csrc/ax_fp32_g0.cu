// AxLocal kernels (fiber-per-thread), native FP32 arithmetic, orders N = 1, 2, 3, 4, 5.
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_g0
#define AX_N_LIST(X) X(1) X(2) X(3) X(4) X(5)
#include "inst_fiber.inc"
