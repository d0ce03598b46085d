// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 15.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g6
#define AX_N_LIST(X) X(15)
#include "inst_fiber.inc"
