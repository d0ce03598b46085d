// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 8, 9.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g2
#define AX_N_LIST(X) X(8) X(9)
#include "inst_fiber.inc"
