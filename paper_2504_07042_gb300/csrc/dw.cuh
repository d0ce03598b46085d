// Double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 47-48 significant bits.  GB300 runs FP32 FMA at 64x the FP64 rate,
// so FP64-accurate AxLocal is cheaper in this form than in native FP64.
//
// Building blocks (all with round-to-nearest intrinsics, so the compiler can
// neither contract nor reassociate them):
//   TwoSum           Knuth, TAOCP vol. 2 (error-free a + b, 6 flops)
//   Fast2Sum         Dekker 1971 (error-free a + b when |a| >= |b|, 3 flops)
//   TwoProd          error-free a * b with one FMA (2 flops)
//   DW * DW, DW + DW Joldes, Muller, Popescu, "Tight and rigorous error bounds
//                    for basic building blocks of double-word arithmetic",
//                    ACM TOMS 44(2), 2017 (DWTimesDW3, SloppyDWPlusDW)
//   dot accumulator  compensated dot product of Ogita, Rump, Oishi,
//                    "Accurate sum and dot product", SIAM J. Sci. Comput. 26,
//                    2005 (Dot2), extended with the lo-part cross terms
//   DW / DW          the same paper's DW division (DWDivDW2) with a
//                    correctly rounded FP32 reciprocal as the seed.
// Errors are absolute, of order 2^-47 times the magnitudes involved, which is
// what a relative max-norm tolerance needs.
#pragma once

#include <cuda_runtime.h>

namespace ax {
namespace dw {

struct dw {
  float hi, lo;
};

__device__ __forceinline__ dw make(float h, float l) { return dw{h, l}; }
__device__ __forceinline__ dw from_float2(float2 v) { return dw{v.x, v.y}; }

__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dw{s, e};
}

__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dw{s, e};
}

__device__ __forceinline__ dw add(dw x, dw y) {
  const dw s = two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, v));
}

__device__ __forceinline__ dw neg(dw x) { return dw{-x.hi, -x.lo}; }
__device__ __forceinline__ dw sub(dw x, dw y) { return add(x, neg(y)); }

__device__ __forceinline__ dw mul(dw x, dw y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

// Unnormalised dot-product accumulator: value = s + c.
struct acc {
  float s, c;
};

__device__ __forceinline__ acc acc_zero() { return acc{0.0f, 0.0f}; }

// a += x * y  (x, y double-word)
__device__ __forceinline__ void mac(acc &a, dw x, dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float pe = __fmaf_rn(x.hi, y.hi, -p);
  const dw t = two_sum(a.s, p);
  a.s = t.hi;
  float c = __fadd_rn(a.c, __fadd_rn(t.lo, pe));
  c = __fmaf_rn(x.hi, y.lo, c);
  a.c = __fmaf_rn(x.lo, y.hi, c);
}

// first term of a fresh accumulator: a = x * y
__device__ __forceinline__ acc mul_acc(dw x, dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float c = __fmaf_rn(x.hi, y.hi, -p);
  c = __fmaf_rn(x.hi, y.lo, c);
  c = __fmaf_rn(x.lo, y.hi, c);
  return acc{p, c};
}

// a * b + c (all double-word): the exact product of the high parts and its
// cross terms (a.lo * b.lo, below 2^-48 of the product, is left out), then
// TwoSum with c.hi; 15 flops instead of a DW product and a DW sum (20).
__device__ __forceinline__ dw fma(dw a, dw b, dw c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dw s = two_sum(c.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// Lightly unnormalised results.  The sums below skip the final Fast2Sum:
// they return hi + lo with hi = RN(a.hi + b.hi) and |lo| a few ulp(hi) at
// most (the TwoSum error plus the low parts).  Every consumer here (TwoSum-
// based sums, products with both cross terms, the division's residual
// correction, the float64 conversion) keeps its absolute error of order
// 2^-47 times the magnitudes involved for such inputs, because none of them
// relies on hi = RN(hi + lo).
__device__ __forceinline__ dw add_lazy(dw x, dw y) {
  const dw s = two_sum(x.hi, y.hi);
  return dw{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ dw sub_lazy(dw x, dw y) {
  const dw s = two_sum(x.hi, -y.hi);
  return dw{s.hi, __fadd_rn(s.lo, __fsub_rn(x.lo, y.lo))};
}
// a + b and a - b of two accumulators
__device__ __forceinline__ dw acc_sum(acc a, acc b) {
  const dw s = two_sum(a.s, b.s);
  return dw{s.hi, __fadd_rn(s.lo, __fadd_rn(a.c, b.c))};
}
__device__ __forceinline__ dw acc_dif(acc a, acc b) {
  const dw s = two_sum(a.s, -b.s);
  return dw{s.hi, __fadd_rn(s.lo, __fsub_rn(a.c, b.c))};
}

__device__ __forceinline__ void acc_add(acc &a, acc b) {
  const dw t = two_sum(a.s, b.s);
  a.s = t.hi;
  a.c = __fadd_rn(__fadd_rn(a.c, b.c), t.lo);
}

__device__ __forceinline__ dw fin(acc a) { return fast_two_sum(a.s, a.c); }

// x / y (DW by DW): q0 = x.hi * rcp(y.hi); r = x - q0*y (exact hi part via
// TwoProd); q = q0 + r.hi * rcp(y.hi).
__device__ __forceinline__ dw div(dw x, dw y) {
  const float inv = __frcp_rn(y.hi);
  const float q0 = __fmul_rn(x.hi, inv);
  const float p = __fmul_rn(q0, y.hi);
  const float pe = __fmaf_rn(q0, y.hi, -p);
  // r = (x.hi - p) - pe + x.lo - q0 * y.lo
  float r = __fsub_rn(x.hi, p);
  r = __fsub_rn(r, pe);
  r = __fadd_rn(r, x.lo);
  r = __fmaf_rn(-q0, y.lo, r);
  return fast_two_sum(q0, __fmul_rn(r, inv));
}

// float64 <-> double-word conversions (FP64-pipe instructions: used only at
// the boundary of a kernel).
__device__ __forceinline__ dw from_double(double v) {
  const float h = __double2float_rn(v);
  const float l = __double2float_rn(v - (double)h);
  return dw{h, l};
}
__device__ __forceinline__ double to_double(dw v) { return (double)v.hi + (double)v.lo; }
// a + b + c to float64: two TwoSums of the high parts, the low parts and
// errors summed in float, the last addition in float64 (no Fast2Sum needed)
__device__ __forceinline__ double sum3_to_double(dw a, dw b, dw c) {
  const dw s1 = two_sum(a.hi, b.hi);
  const dw s2 = two_sum(s1.hi, c.hi);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), c.lo), __fadd_rn(s1.lo, s2.lo));
  return (double)s2.hi + (double)lo;
}

// The same conversions without FP64-pipe instructions, for values inside a
// kernel's direct range.  The forms above spend four (float64 -> pair) and
// two (pair -> float64, besides the last addition) instructions per value on
// the FP64 pipe, which GB300 runs at 1/64 of the FP32 rate; here the words
// are assembled by integer instructions on the IEEE-754 bit fields.
//
// float64 -> pair: hi holds the leading 24 significand bits of v (truncated:
// the exponent re-biased from 1023 to 127, the top 23 fraction bits shifted
// into place), lo the 29 fraction bits below them, converted as an integer
// with one rounding (cvt.rn.f32.u32) and scaled by their weight
// 2^(E - 1075), E the biased exponent of v (a product by a power of two:
// exact).  |hi + lo - v| <= 2^-48 |v|, as for from_double.  Valid for |v| in
// [2^-74, 2^128), where both words are normal floats; smaller magnitudes give
// 0 (the caller reports them: tiny_nonzero), larger ones, infinities and NaNs
// meaningless words (the caller routes them to from_double).
__device__ __forceinline__ dw from_double_direct(double v) {
  const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
  const unsigned a = hw & 0x7fffffffu;
  const unsigned hb = __funnelshift_l(lw, a - (896u << 20), 3) | (hw & 0x80000000u);
  const float scale = __uint_as_float((hb & 0xff800000u) - (52u << 23));  // +-2^(E - 1075)
  const float lo = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), scale);
  const bool tiny = a < (949u << 20);  // |v| < 2^-74
  return dw{tiny ? 0.0f : __uint_as_float(hb), tiny ? 0.0f : lo};
}
// v is nonzero and below from_double_direct's range (flushed to 0 there);
// a = upper 32 bits of |v|
__device__ __forceinline__ bool tiny_nonzero(unsigned a) { return a - 1u < (949u << 20) - 1u; }
// float -> float64 by integer instructions: exact for normal floats and
// zero; subnormal floats (below 2^-126) give 0, infinities and NaNs
// meaningless values
__device__ __forceinline__ double float_to_double_direct(float f) {
  const unsigned b = __float_as_uint(f), a = b & 0x7fffffffu;
  const bool z = a < 0x00800000u;
  const unsigned hw = ((a >> 3) + (896u << 20)) | (b & 0x80000000u);
  return __hiloint2double(z ? 0 : (int)hw, z ? 0 : (int)(b << 29));
}
// sum3_to_double with the two float -> float64 conversions above: one
// FP64-pipe instruction (the last addition) per value
__device__ __forceinline__ double sum3_to_double_direct(dw a, dw b, dw c) {
  const dw s1 = two_sum(a.hi, b.hi);
  const dw s2 = two_sum(s1.hi, c.hi);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), c.lo), __fadd_rn(s1.lo, s2.lo));
  return float_to_double_direct(s2.hi) + float_to_double_direct(lo);
}

}  // namespace dw
}  // namespace ax
