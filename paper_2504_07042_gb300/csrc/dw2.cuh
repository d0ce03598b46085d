// Two double-word operations in lockstep on the packed FP32x2 instructions
// of sm_100-class GPUs (mul / fma .rn.f32x2: two independent, correctly
// rounded FP32 operations per instruction).
//
// The double-word kernels issue about 1000 instructions per node, 890 of
// them FP32: they are bound by instruction issue, not by the FP32 lanes.
// A packed instruction performs the two lanes' operations with one issue,
// so two independent double-word computations written as one sequence of
// packed instructions cost about half the issue slots.  Every packed
// operation rounds each lane exactly as the scalar operation of dw.cuh
// would, in the same order, so results are bit-identical to the scalar
// double-word code.
//
// The even-odd fiber product (ax_fiber.cuh) pairs its two dot products per
// output index, P (even part) and Q (odd part): lane 0 carries P, lane 1 Q.
#pragma once

#include <cuda_runtime.h>

#include "dw.cuh"

namespace ax {
namespace dw2 {

using f2 = float2;

// Each operation is written as PTX with an explicit .rn rounding modifier:
// like the scalar __fadd_rn / __fmul_rn, such an instruction is never
// contracted with a neighbour into a fused multiply-add, which would change
// the rounding the error-free transformations rely on.
__device__ __forceinline__ f2 mul(f2 a, f2 b) {
  f2 r;
  asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
      " mul.rn.f32x2 z, x, y;\n mov.b64 {%0, %1}, z;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("{\n .reg .b64 x, y, z, w;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n mov.b64 z, {%6, %7};\n"
      " fma.rn.f32x2 w, x, y, z;\n mov.b64 {%0, %1}, w;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
// Sums and differences as fused multiply-adds by +-1 (a * 1 + b = RN(a + b),
// the same rounding, the same issue cost).  Measured with this toolchain:
// sequences of add.rn.f32x2 / sub.rn.f32x2 mixed with the packed products
// above did not reproduce the scalar roundings of the error-free sums (the
// fiber product differed in its low words), while this form gave output
// bits identical to the scalar double-word code for every order and kind.
__device__ __forceinline__ f2 add(f2 a, f2 b) { return fma(a, make_float2(1.0f, 1.0f), b); }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return fma(b, make_float2(-1.0f, -1.0f), a); }

// Two unnormalised dot-product accumulators (dw::acc) in lockstep.
struct acc2 {
  f2 s, c;
};

// The operand pair y of a product term, with its high parts negated (nh):
// the products' rounding errors are then formed without a separate negation
// (x.hi * (-y.hi) + p = -(x.hi * y.hi - p) exactly).
struct opnd {
  f2 h, l, nh;
};

// a = x * y (dw::mul_acc in each lane)
__device__ __forceinline__ acc2 mul0(f2 xh, f2 xl, const opnd &y) {
  const f2 p = mul(xh, y.h);
  const f2 np = mul(xh, y.nh);  // -p, exactly
  f2 c = fma(xh, y.h, np);      // x.hi * y.hi - p
  c = fma(xh, y.l, c);
  c = fma(xl, y.h, c);
  return acc2{p, c};
}

// a += x * y (dw::mac in each lane)
__device__ __forceinline__ void mac(acc2 &a, f2 xh, f2 xl, const opnd &y) {
  const f2 p = mul(xh, y.h);
  const f2 npe = fma(xh, y.nh, p);  // -(x.hi * y.hi - p), exactly the negated error term
  // TwoSum(a.s, p)
  const f2 s = add(a.s, p);
  const f2 bb = sub(s, a.s);
  const f2 e = add(sub(a.s, sub(s, bb)), sub(p, bb));
  a.s = s;
  f2 c = add(a.c, sub(e, npe));  // a.c + (e + pe)
  c = fma(xh, y.l, c);
  a.c = fma(xl, y.h, c);
}

// Even-odd fiber product of even order N1 (see contract in ax_fiber.cuh)
// with the P and Q dot products of each output pair in the two lanes.
// eo2: the order's block of packed constants, entry i * c + m =
// (A.hi, B.hi, A.lo, B.lo) with A = (M[i][m] + M[i][N-m]) / 2 and
// B = (M[i][m] - M[i][N-m]) / 2.
template <int N1>
__device__ __forceinline__ void contract(const float4 *__restrict__ eo2, const dw::dw *in, dw::dw *out) {
  static_assert((N1 & 1) == 0, "packed fiber product: even orders only");
  constexpr int c = N1 / 2;
  opnd y[c];
#pragma unroll
  for (int m = 0; m < c; ++m) {
    const dw::dw e = dw::add_lazy(in[m], in[N1 - 1 - m]);
    const dw::dw o = dw::sub_lazy(in[m], in[N1 - 1 - m]);
    y[m].h = make_float2(e.hi, o.hi);
    y[m].l = make_float2(e.lo, o.lo);
    y[m].nh = make_float2(-e.hi, -o.hi);
  }
#pragma unroll
  for (int i = 0; i < c; ++i) {
    float4 k = eo2[i * c];
    acc2 pq = mul0(make_float2(k.x, k.y), make_float2(k.z, k.w), y[0]);
#pragma unroll
    for (int m = 1; m < c; ++m) {
      k = eo2[i * c + m];
      mac(pq, make_float2(k.x, k.y), make_float2(k.z, k.w), y[m]);
    }
    const dw::acc p{pq.s.x, pq.c.x}, q{pq.s.y, pq.c.y};
    if constexpr (N1 < 16) {
      out[i] = dw::acc_sum(p, q);
      out[N1 - 1 - i] = dw::acc_dif(q, p);
    } else {
      // as the scalar product at N1 = 16: finalise both sums first
      const dw::dw Pv = dw::fin(p), Qv = dw::fin(q);
      out[i] = dw::add(Pv, Qv);
      out[N1 - 1 - i] = dw::sub(Qv, Pv);
    }
  }
}

// Even-odd fiber product of even order N1 in FP32 with the P and Q dot
// products of each output pair in the two lanes (the float policy's
// contract: the same products and fused multiply-adds per lane, in the same
// order).  The constants come from the same paired table, whose high words
// are the float constants of the scalar table.
template <int N1>
__device__ __forceinline__ void contract_f32(const float4 *__restrict__ eo2, const float *in, float *out) {
  static_assert((N1 & 1) == 0, "packed fiber product: even orders only");
  constexpr int c = N1 / 2;
  f2 y[c];
#pragma unroll
  for (int m = 0; m < c; ++m) y[m] = make_float2(in[m] + in[N1 - 1 - m], in[m] - in[N1 - 1 - m]);
#pragma unroll
  for (int i = 0; i < c; ++i) {
    float4 k = eo2[i * c];
    f2 pq = mul(make_float2(k.x, k.y), y[0]);
#pragma unroll
    for (int m = 1; m < c; ++m) {
      k = eo2[i * c + m];
      pq = fma(make_float2(k.x, k.y), y[m], pq);
    }
    out[i] = pq.x + pq.y;
    out[N1 - 1 - i] = pq.y - pq.x;
  }
}

}  // namespace dw2
}  // namespace ax
