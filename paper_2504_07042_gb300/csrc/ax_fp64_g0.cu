// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 1, 2, 3, 4, 5.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g0
#define AX_N_LIST(X) X(1) X(2) X(3) X(4) X(5)
#include "inst_fiber.inc"
