// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 6, 7.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g1
#define AX_N_LIST(X) X(6) X(7)
#include "inst_fiber.inc"
