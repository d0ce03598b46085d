// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 14.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g5
#define AX_N_LIST(X) X(14)
#include "inst_fiber.inc"
