// Host check of the double-word building blocks of csrc/dw.cuh against
// long-double references on seeded random operands.  Prints one line per
// operation: "name max_error_in_units_of_2^-47".  The unit is relative to the
// magnitudes involved (|a||b| for products, |a| + |b| for sums, ...), the
// scale the AxLocal error bound is stated in.
#include "cuda_runtime.h"
#include "../../paper_2504_07042_gb300/csrc/dw.cuh"

#include <cstdio>
#include <random>

using namespace ax::dw;
typedef long double LD;

static dw from_ld(LD v) {
  const float h = (float)v;
  return dw{h, (float)(v - (LD)h)};
}
static LD val(dw x) { return (LD)x.hi + (LD)x.lo; }
static LD val(acc a) { return (LD)a.s + (LD)a.c; }

int main() {
  std::mt19937_64 g(20250407);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> Ex(-20, 20);
  const LD unit = std::ldexp((LD)1, -47);
  LD e_two = 0, e_mul = 0, e_mac = 0, e_fma = 0, e_sum = 0, e_lazy = 0, e_div = 0, e_conv = 0, e_s3 = 0, e_add = 0;
  LD e_convd = 0, e_s3d = 0;
  long bad_direct = 0;  // cases the FP64-pipe-free conversions get wrong (must stay 0)
  auto upd = [](LD &m, LD err, LD scale) {
    const LD r = err / (scale > 0 ? scale : 1);
    if (r > m) m = r;
  };
  for (int it = 0; it < 300000; ++it) {
    const LD sa = std::ldexp(1.0L, Ex(g)), sb = std::ldexp(1.0L, Ex(g));
    const dw a = from_ld(U(g) * sa), b = from_ld(U(g) * sb), c = from_ld(U(g) * sa), d = from_ld(U(g) * sb);
    const LD A = val(a), B = val(b), C = val(c), D = val(d);
    // TwoSum is error-free
    const dw t = two_sum(a.hi, b.hi);
    upd(e_two, fabsl((LD)t.hi + (LD)t.lo - ((LD)a.hi + (LD)b.hi)), 1);
    upd(e_add, fabsl(val(add(a, b)) - (A + B)), fabsl(A) + fabsl(B));
    upd(e_mul, fabsl(val(mul(a, b)) - A * B), fabsl(A * B));
    upd(e_fma, fabsl(val(fma(a, b, c)) - (A * B + C)), fabsl(A * B) + fabsl(C));
    acc p = mul_acc(a, b);
    mac(p, c, d);
    mac(p, a, d);
    upd(e_mac, fabsl(val(fin(p)) - (A * B + C * D + A * D)), fabsl(A * B) + fabsl(C * D) + fabsl(A * D));
    acc q = mul_acc(b, c);
    mac(q, d, d);
    const LD P = A * B + C * D + A * D, Q = B * C + D * D;
    const LD sP = fabsl(A * B) + fabsl(C * D) + fabsl(A * D), sQ = fabsl(B * C) + D * D;
    upd(e_sum, fabsl(val(acc_sum(p, q)) - (P + Q)), sP + sQ);
    upd(e_sum, fabsl(val(acc_dif(q, p)) - (Q - P)), sP + sQ);
    const dw e = add_lazy(a, c), o = sub_lazy(a, c);
    upd(e_lazy, fabsl(val(e) - (A + C)), fabsl(A) + fabsl(C));
    upd(e_lazy, fabsl(val(o) - (A - C)), fabsl(A) + fabsl(C));
    // a product of lazy sums, as the even-odd contraction forms them
    acc r = mul_acc(e, b);
    mac(r, o, d);
    upd(e_lazy, fabsl(val(fin(r)) - ((A + C) * B + (A - C) * D)), (fabsl(A) + fabsl(C)) * (fabsl(B) + fabsl(D)));
    upd(e_div, fabsl(val(div(a, b)) - A / B), fabsl(A / B));
    const double v = (double)(U(g) * sa);
    upd(e_conv, fabsl((LD)to_double(from_double(v)) - (LD)v), fabsl((LD)v));
    upd(e_s3, fabsl((LD)sum3_to_double(a, b, c) - (A + B + C)), fabsl(A) + fabsl(B) + fabsl(C));
    upd(e_s3d, fabsl((LD)sum3_to_double_direct(a, b, c) - (A + B + C)), fabsl(A) + fabsl(B) + fabsl(C));
    // float64 -> pair without the FP64 pipe, over its whole range [2^-74, 2^128)
    // (random 53-bit significands, both signs)
    {
      const int ex = std::uniform_int_distribution<int>(-74, 127)(g);
      const double w = std::ldexp(std::uniform_real_distribution<double>(1.0, 2.0)(g), ex) * (U(g) < 0 ? -1 : 1);
      const dw p2 = from_double_direct(w);
      upd(e_convd, fabsl((LD)p2.hi + (LD)p2.lo - (LD)w), fabsl((LD)w));
      if (std::fabs(p2.lo) >= std::fabs(p2.hi) * 0x1p-23f) ++bad_direct;  // |lo| < ulp(hi)
      if (tiny_nonzero((unsigned)__double2hiint(w) & 0x7fffffffu)) ++bad_direct;
      // float -> float64 exact on normal floats
      const float f = (float)w;
      if (std::isnormal(f) && float_to_double_direct(f) != (double)f) ++bad_direct;
    }
  }
  // below the range: flushed to 0 and reported, except below 2^-1042, where the
  // upper 32 bits (all the range tests read) are zero and the value counts as
  // a zero; zeros of either sign pass as 0
  for (int ex = -1074; ex < -74; ++ex) {
    if (ex < -1042) {
      const dw p2 = from_double_direct(std::ldexp(1.5, ex));
      if (p2.hi != 0.0f || p2.lo != 0.0f) ++bad_direct;
      continue;
    }
    const double w = std::ldexp(1.5, ex);
    const dw p2 = from_double_direct(w);
    if (p2.hi != 0.0f || p2.lo != 0.0f) ++bad_direct;
    if (!tiny_nonzero((unsigned)__double2hiint(w) & 0x7fffffffu)) ++bad_direct;
  }
  for (double z : {0.0, -0.0}) {
    const dw p2 = from_double_direct(z);
    if (p2.hi != 0.0f || p2.lo != 0.0f || tiny_nonzero((unsigned)__double2hiint(z) & 0x7fffffffu)) ++bad_direct;
    if (float_to_double_direct((float)z) != 0.0) ++bad_direct;
  }
  // exact powers of two and the largest significand at both ends of the range
  for (double w : {0x1p-74, 0x1.fffffffffffffp-74, 0x1p127, 0x1.fffffffffffffp127, 1.0, -1.0, 0x1.fffffffffffffp0}) {
    const dw p2 = from_double_direct(w);
    upd(e_convd, fabsl((LD)p2.hi + (LD)p2.lo - (LD)w), fabsl((LD)w));
  }
  // float subnormals go to 0
  if (float_to_double_direct(0x1p-130f) != 0.0 || float_to_double_direct(-0x1p-149f) != 0.0) ++bad_direct;
  std::printf("two_sum %.3Lg\nadd %.3Lg\nmul %.3Lg\nfma %.3Lg\nmac %.3Lg\nacc_sum %.3Lg\nlazy %.3Lg\ndiv %.3Lg\nconv %.3Lg\nsum3 %.3Lg\n",
              e_two, e_add / unit, e_mul / unit, e_fma / unit, e_mac / unit, e_sum / unit, e_lazy / unit, e_div / unit,
              e_conv / unit, e_s3 / unit);
  std::printf("conv_direct %.3Lg\nsum3_direct %.3Lg\nbad_direct %ld\n", e_convd / unit, e_s3d / unit, bad_direct);
  return 0;
}
