// AxLocal kernels (fiber-per-thread), native FP64 arithmetic, orders N = 12, 13.
#define AX_POLICY fiber::Native<double>
#define AX_CT double
#define AX_TAG fp64_g4
#define AX_N_LIST(X) X(12) X(13)
#include "inst_fiber.inc"
