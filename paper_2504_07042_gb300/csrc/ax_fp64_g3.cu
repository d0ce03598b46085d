// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 10, 11.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g3
#define AX_N_LIST(X) X(10) X(11)
#include "inst_fiber.inc"
