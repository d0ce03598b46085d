// Host stand-ins for the few CUDA intrinsics that csrc/dw.cuh uses, so that
// its double-word arithmetic can be checked on the CPU.  Each stand-in is the
// correctly rounded IEEE operation the intrinsic names (round to nearest, no
// contraction: the harness is built with -ffp-contract=off and the results go
// through volatile floats).
#pragma once
#include <cmath>
#define __device__
#define __host__
#define __forceinline__ inline
struct float2 {
  float x, y;
};
static inline float2 make_float2(float a, float b) { return float2{a, b}; }
static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __frcp_rn(float a) { volatile float r = 1.0f / a; return r; }
static inline float __double2float_rn(double v) { volatile float r = (float)v; return r; }
