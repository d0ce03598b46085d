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
// bit-level intrinsics used by the FP64-pipe-free conversions
#include <cstdint>
#include <cstring>
static inline int __double2hiint(double v) { uint64_t u; std::memcpy(&u, &v, 8); return (int)(uint32_t)(u >> 32); }
static inline int __double2loint(double v) { uint64_t u; std::memcpy(&u, &v, 8); return (int)(uint32_t)u; }
static inline double __hiloint2double(int hi, int lo) {
  const uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
  double v;
  std::memcpy(&v, &u, 8);
  return v;
}
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline unsigned __funnelshift_l(unsigned lo, unsigned hi, unsigned s) {
  s &= 31;
  return s ? (hi << s) | (lo >> (32 - s)) : hi;
}
static inline float __uint2float_rn(unsigned u) { volatile float r = (float)u; return r; }
