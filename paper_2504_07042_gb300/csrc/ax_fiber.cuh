// AxLocal, fiber-per-thread design (templates over an arithmetic policy:
// native FP64, native FP32, or double-word FP32 pairs).
//
// The whole element (EPB elements per CTA) sits in padded shared memory.
// Every contraction of Algorithm 1 is done by a thread that owns a whole
// fiber of the tensor in the contraction's direction, so the differentiation
// matrix is read as a uniform constant-memory operand by all threads at once
// (the constant-memory idea of Sec. 4.3.1, applied to all three directions),
// and each fiber product uses the even-odd split of the centro-antisymmetric
// D (D[N-i][N-j] = -D[i][j]): outputs i and N-i come from two half-length
// dot products of the fiber's even and odd parts, nearly halving the
// multiply-adds.
//
//   r-fibers  x0 = D_r x -> B0;   s-fibers  x1 = D_s x -> B1
//   thread (i,j): t-fiber x2 = D_t x[i,j,:]; per node k the geometry
//           (stored / Algorithm 2 / Algorithm 3 / partial) and
//           (r,s,t) = G (x0,x1,x2); r -> B0, s -> B1; Y = D_t^T t
//   r-fibers  Y += D_r^T r;   s-fibers  Y += D_s^T s;   Y to HBM.
// Five barriers per element (two per k-layer in the layer-wise design).
// Phase 3 (own t-fiber) needs no barrier after the geometry: each thread
// reads and writes only its own fiber there.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ax_internal.h"
#include "dw.cuh"
#include "dw2.cuh"
#include "tables.cuh"

namespace ax {
namespace fiber {

// ---------------------------------------------------------------------------
// arithmetic policies
// ---------------------------------------------------------------------------
template <typename T>
struct Native {
  using V = T;   // register value
  using S = T;   // shared-memory / geometry-record word
  using A = T;   // dot-product accumulator
  using C = T;   // constant-table word
  using IO = T;  // X, Y in HBM
  static constexpr bool kRoll = false;  // short code: unroll the phase and k loops
  static constexpr bool kScaleIO = false;  // native range: X and Y pass unscaled
  static constexpr int kTargetWarpsPerSM = 0;  // no cap
  static constexpr int kTiles = sizeof(T) == 4 ? 2 : 1;  // tile variants the autotuner may pick
  __device__ static __forceinline__ V ld(const S *p) { return *p; }
  __device__ static __forceinline__ S st(V v) { return v; }
  __device__ static __forceinline__ V cst(const C *p) { return *p; }
  __device__ static __forceinline__ V from_io(IO v) { return v; }
  __device__ static __forceinline__ V from_io_direct(IO v) { return v; }
  __device__ static __forceinline__ IO to_io(V v) { return v; }
  __device__ static __forceinline__ V lit(double v) { return (T)v; }
  __device__ static __forceinline__ A zero() { return T(0); }
  __device__ static __forceinline__ A mul0(V x, V y) { return x * y; }
  __device__ static __forceinline__ void mac(A &a, V x, V y) { a = fma(x, y, a); }
  __device__ static __forceinline__ V fin(A a) { return a; }
  __device__ static __forceinline__ V acc_sum(A a, A b) { return a + b; }
  __device__ static __forceinline__ V acc_dif(A a, A b) { return a - b; }
  __device__ static __forceinline__ V add(V a, V b) { return a + b; }
  __device__ static __forceinline__ V sub(V a, V b) { return a - b; }
  __device__ static __forceinline__ V add_lazy(V a, V b) { return a + b; }
  __device__ static __forceinline__ V sub_lazy(V a, V b) { return a - b; }
  __device__ static __forceinline__ V mul(V a, V b) { return a * b; }
  __device__ static __forceinline__ V fma3(V a, V b, V c) { return fma(a, b, c); }
  __device__ static __forceinline__ V twice(V a) { return a + a; }
  __device__ static __forceinline__ IO sum3_io(V a, V b, V c) { return (a + b) + c; }
  __device__ static __forceinline__ IO sum3_io_direct(V a, V b, V c) { return (a + b) + c; }
  __device__ static __forceinline__ V div(V a, V b) {
    if constexpr (sizeof(T) == 4)
      return __fdividef(a, b);  // 2-ulp quotient: the FP32 path's tolerance is 2e-5
    else
      return a / b;
  }
  __device__ static __forceinline__ V neg(V a) { return -a; }
};

struct DW {
  using V = dw::dw;
  using S = float2;
  using A = dw::acc;
  using C = float2;
  using IO = double;
  static constexpr bool kRoll = true;  // long code: keep the phase and k loops rolled (instruction cache)
  // float64 X has float64's exponent range, the float pairs only float32's:
  // each element's X is scaled by a power of two that brings its largest
  // magnitude near 1 before the conversion, and Y is scaled back (both exact)
  static constexpr bool kScaleIO = true;
  static constexpr int kTiles = 1;
  // Resident warps per SM the launcher aims at for the trilinear kinds at
  // N1 = 8 (by padding the dynamic shared memory): more warps thrash the
  // instruction cache with this long code.  Measured on GB300: 5 CTAs of 4
  // warps 2% faster than 4, and fewer (3) or longer code per warp (unrolled
  // k or phase loops) slower; at other orders and for the stored kind a cap
  // measured slower, so it is not applied there.
  static constexpr int kTargetWarpsPerSM = 20;
  __device__ static __forceinline__ V ld(const S *p) { return dw::from_float2(*p); }
  __device__ static __forceinline__ S st(V v) { return make_float2(v.hi, v.lo); }
  __device__ static __forceinline__ V cst(const C *p) { return dw::from_float2(*p); }
  __device__ static __forceinline__ V from_io(IO v) { return dw::from_double(v); }
  // inside the direct range (the main kernel): no FP64-pipe instruction
  __device__ static __forceinline__ V from_io_direct(IO v) { return dw::from_double_direct(v); }
  __device__ static __forceinline__ IO to_io(V v) { return dw::to_double(v); }
  __device__ static __forceinline__ V lit(double v) { return dw::make((float)v, 0.0f); }  // exact small literals only
  __device__ static __forceinline__ A zero() { return dw::acc_zero(); }
  __device__ static __forceinline__ A mul0(V x, V y) { return dw::mul_acc(x, y); }
  __device__ static __forceinline__ void mac(A &a, V x, V y) { dw::mac(a, x, y); }
  __device__ static __forceinline__ V fin(A a) { return dw::fin(a); }
  // sums that feed only error-tolerant consumers skip the final Fast2Sum (dw.cuh)
  __device__ static __forceinline__ V acc_sum(A a, A b) { return dw::acc_sum(a, b); }
  __device__ static __forceinline__ V acc_dif(A a, A b) { return dw::acc_dif(a, b); }
  __device__ static __forceinline__ V add(V a, V b) { return dw::add(a, b); }
  __device__ static __forceinline__ V sub(V a, V b) { return dw::sub(a, b); }
  __device__ static __forceinline__ V add_lazy(V a, V b) { return dw::add_lazy(a, b); }
  __device__ static __forceinline__ V sub_lazy(V a, V b) { return dw::sub_lazy(a, b); }
  __device__ static __forceinline__ V mul(V a, V b) { return dw::mul(a, b); }
  __device__ static __forceinline__ V fma3(V a, V b, V c) { return dw::fma(a, b, c); }
  __device__ static __forceinline__ V twice(V a) { return dw::make(2.0f * a.hi, 2.0f * a.lo); }  // exact
  __device__ static __forceinline__ IO sum3_io(V a, V b, V c) { return dw::sum3_to_double(a, b, c); }
  __device__ static __forceinline__ IO sum3_io_direct(V a, V b, V c) { return dw::sum3_to_double_direct(a, b, c); }
  __device__ static __forceinline__ V div(V a, V b) { return dw::div(a, b); }
  __device__ static __forceinline__ V neg(V a) { return dw::neg(a); }
};


template <class P>
__device__ __forceinline__ typename P::V dot3(const typename P::V a[3], const typename P::V b[3]) {
  typename P::A s = P::mul0(a[0], b[0]);
  P::mac(s, a[1], b[1]);
  P::mac(s, a[2], b[2]);
  return P::fin(s);
}

// a*b - c*d
template <class P>
__device__ __forceinline__ typename P::V det2(typename P::V a, typename P::V b, typename P::V c, typename P::V d) {
  typename P::A s = P::mul0(a, b);
  P::mac(s, P::neg(c), d);
  return P::fin(s);
}

// ---------------------------------------------------------------------------
// even-odd fiber product: out = M in, M centro-antisymmetric (D or D^T).
// Table block of order N1 (N1*N1 words), c = N1/2:
//   rows i < c: [ A(i,0..c-1) | B(i,0..c-1) | M[i][c] if N1 odd ],
//     A = (M[i][m] + M[i][N-m]) / 2,  B = (M[i][m] - M[i][N-m]) / 2
//   row c (N1 odd): M[c][0..c-1]
// out[i] = P + Q, out[N-i] = Q - P with P = sum A e + M[i][c] f[c], Q = sum B o,
// e[m] = f[m] + f[N-m], o[m] = f[m] - f[N-m].
// ---------------------------------------------------------------------------
template <class P, int N1>
__device__ __forceinline__ void contract(const typename P::C *__restrict__ eo, const typename P::V *in,
                                         typename P::V *out) {
  using V = typename P::V;
  constexpr int c = N1 / 2;
  constexpr bool odd = (N1 & 1) != 0;
  V e[c], o[c];
#pragma unroll
  for (int m = 0; m < c; ++m) {
    e[m] = P::add_lazy(in[m], in[N1 - 1 - m]);
    o[m] = P::sub_lazy(in[m], in[N1 - 1 - m]);
  }
#pragma unroll
  for (int i = 0; i < c; ++i) {
    typename P::A p = P::mul0(P::cst(eo + i * N1), e[0]), q = P::mul0(P::cst(eo + i * N1 + c), o[0]);
#pragma unroll
    for (int m = 1; m < c; ++m) {
      P::mac(p, P::cst(eo + i * N1 + m), e[m]);
      P::mac(q, P::cst(eo + i * N1 + c + m), o[m]);
    }
    if constexpr (odd) P::mac(p, P::cst(eo + i * N1 + 2 * c), in[c]);
    if constexpr (N1 < 16) {
      out[i] = P::acc_sum(p, q);
      out[N1 - 1 - i] = P::acc_dif(q, p);
    } else {
      // N1 = 16: under the 128-register cap the sums straight from the
      // accumulators spill in double-word arithmetic; finalise them first
      const V Pv = P::fin(p), Qv = P::fin(q);
      out[i] = P::add(Pv, Qv);
      out[N1 - 1 - i] = P::sub(Qv, Pv);
    }
  }
  if constexpr (odd) {
    typename P::A q = P::mul0(P::cst(eo + c * N1), o[0]);
#pragma unroll
    for (int m = 1; m < c; ++m) P::mac(q, P::cst(eo + c * N1 + m), o[m]);
    out[c] = P::fin(q);
  }
}

// The double-word fiber product at even orders runs its two dot products per
// output pair in the lanes of packed FP32x2 instructions (dw2.cuh; the same
// roundings in the same order: bit-identical results, about half the issue
// slots for the products); eo2: the order's paired table.
template <class P, int N1>
constexpr bool kPairedDW = P::kRoll && (N1 % 2) == 0;
// FP32 likewise (the same products per lane, bit-identical).  Measured on
// GB300 against the scalar product: N = 7 trilinear 238 -> 255 GDOF/s,
// parallelepiped 314 -> 324, stored 180 -> 188, N = 3, 9 trilinear +5%,
// N = 15 trilinear 172 -> 178 (with the two-CTA register bound of
// shape_min_ctas; unbounded the kernel takes 161 registers and one CTA per
// SM: 131); the partial kind at N1 = 8 measured 6% slower and keeps the
// scalar product.
template <class P, int N1, int KIND>
constexpr bool kPairedF32 = !P::kRoll && sizeof(typename P::V) == 4 && (N1 % 2) == 0 &&
                            !(N1 == 8 && KIND == AX_GEOM_TRILINEAR_PARTIAL);
template <class P, int N1, int KIND>
__device__ __forceinline__ void contract_p(const typename P::C *__restrict__ eo, const float4 *__restrict__ eo2,
                                           const typename P::V *in, typename P::V *out) {
  if constexpr (kPairedDW<P, N1>)
    dw2::contract<N1>(eo2, in, out);
  else if constexpr (kPairedF32<P, N1, KIND>)
    dw2::contract_f32<N1>(eo2, in, out);
  else
    contract<P, N1>(eo, in, out);
}

// Elements per CTA for F threads per element: at least 128 threads, and
// among up to about four times that many elements (at most 512 threads) the
// count that leaves the fewest idle lanes in the last warp (N1 = 6: 7
// elements = 252 threads instead of 3 = 108 threads in four warps).
__host__ __device__ constexpr int idle_lanes_permille(int t) { return ((t + 31) / 32 * 32 - t) * 1000 / ((t + 31) / 32 * 32); }
__host__ __device__ constexpr int pick_epb(int F) {
  int base = F >= 128 ? 1 : 128 / F, best = base, bw = idle_lanes_permille(F * base);
  for (int e = base + 1; e <= 4 * base + 3 && F * e <= 512; ++e)
    if (idle_lanes_permille(F * e) < bw) {
      best = e;
      bw = idle_lanes_permille(F * e);
    }
  return best;
}

// Measured exceptions to the shape rules below, per policy (0: double-word,
// 1: FP32), order and kind: elements per CTA and the minimum resident CTAs
// that bound the registers (0: no override).
// Double-word recompute kernels at N1 = 6 and 10, whose register counts
// (96-127) let an SM hold only one or two filled CTAs (16-18 warps, stalled
// at their barriers), measured on GB300 against the filled shapes, with the
// register bounds' few spills included: N = 5 trilinear 7 elements, 3 CTAs
// (24.0 -> 32.1 GDOF/s), partial 6, 4 (27.1 -> 32.9); N = 9 trilinear 1, 5
// (21.9 -> 24.1), partial 3, 2 (21.8 -> 26.2).  Their stored and
// parallelepiped kinds (56-96 registers) and N1 = 12 measured no faster in
// any of the shapes tried.  With the packed fiber product (dw2.cuh) the
// trilinear kernel at N1 = 8 takes 127 registers unbounded (four CTAs per
// SM); bounded to five CTAs (96 registers, no spills) it runs 2.4% faster.
// FP32 (40-64 registers, mostly faster as they are): N = 5 partial 4
// elements (153 -> 163), N = 9 parallelepiped 2 (243 -> 251), N = 11 stored
// 1 element, 4 CTAs (156 -> 172); N1 = 16 two CTAs (the packed fiber
// product, kPairedF32, would otherwise take 161 registers).
__host__ __device__ constexpr int shape_epb(int pc, int N1, int KIND) {
  return pc == 0 ? (N1 == 6    ? (KIND == AX_GEOM_TRILINEAR ? 7 : KIND == AX_GEOM_TRILINEAR_PARTIAL ? 6 : 0)
                    : N1 == 10 ? (KIND == AX_GEOM_TRILINEAR ? 1 : KIND == AX_GEOM_TRILINEAR_PARTIAL ? 3 : 0)
                               : 0)
                 : (N1 == 6 && KIND == AX_GEOM_TRILINEAR_PARTIAL) ? 4
                 : (N1 == 10 && KIND == AX_GEOM_PARALLELEPIPED)   ? 2
                                                                  : 0;
}
__host__ __device__ constexpr int shape_min_ctas(int pc, int N1, int KIND) {
  return pc == 0 ? (N1 == 8    ? (KIND == AX_GEOM_TRILINEAR ? 5 : 0)
                    : N1 == 6  ? (KIND == AX_GEOM_TRILINEAR ? 3 : KIND == AX_GEOM_TRILINEAR_PARTIAL ? 4 : 0)
                    : N1 == 10 ? (KIND == AX_GEOM_TRILINEAR ? 5 : KIND == AX_GEOM_TRILINEAR_PARTIAL ? 2 : 0)
                               : 0)
                 : (N1 == 12 && KIND == AX_GEOM_STORED) ? 4
                 : N1 == 16                              ? 2
                                                        : 0;
}
// the policy class of shape_epb / shape_min_ctas (-1: none)
template <class P>
constexpr int kShapeClass = P::kRoll ? 0 : sizeof(typename P::S) == 4 ? 1 : -1;

// Elements per CTA of the per-order kernels (0: the plain 128-thread rule).
// Measured on GB300: filling the warps (pick_epb) pays for the trilinear
// kinds in 8-byte arithmetic (double-word, FP64) and for every recompute
// kind at N1 = 6; the stored and parallelepiped kinds elsewhere, and FP32
// at N1 = 10, 12, run faster with the smaller CTAs (more of them per SM).
// The exceptions of shape_epb come first.
template <class P, int N1, int KIND>
constexpr int kEpb =
    (kShapeClass<P> >= 0 && shape_epb(kShapeClass<P>, N1, KIND)) ? shape_epb(kShapeClass<P>, N1, KIND)
    : (KIND != AX_GEOM_STORED && (N1 == 6 || (sizeof(typename P::S) == 8 && KIND != AX_GEOM_PARALLELEPIPED)))
        ? pick_epb(N1 * N1)
        : 0;

// Minimum resident CTAs for the register budget (0: no bound): the
// double-word kernels at N1 = 16 (256-thread CTAs) are held to 128 registers
// so that two CTAs fit per SM (unbounded they take about 147 and run one CTA
// per SM, 5-30% slower); the double-word trilinear kernel at N1 = 12
// (288-thread CTAs) likewise to two CTAs (96 registers and some spills
// instead of 119 registers and one CTA: 33% faster; the partial kind
// measured 5% slower so and keeps its allocation); the exceptions of
// shape_min_ctas.  Elsewhere no bound is given: even an explicit 1 changes
// the register allocation for the worse.
template <class P, int N1, int KIND>
constexpr int kMinCtas =
    (kShapeClass<P> >= 0 && shape_min_ctas(kShapeClass<P>, N1, KIND)) ? shape_min_ctas(kShapeClass<P>, N1, KIND)
    : (P::kRoll && (N1 == 16 || (N1 == 12 && KIND == AX_GEOM_TRILINEAR)))  ? 2
                                                                           : 0;

// Trilinear kinds: whether an element's first 2 N1 threads compute the axis
// terms of the geometry (Geometry::axis_terms) for all its threads.  Measured
// on GB300: native FP64 3% faster (N = 7), double-word 7% faster at N = 3 and
// 3% at N = 5 but 1-4% slower at N = 7 (where the prologue is amortised over
// more nodes), FP32 1-3% slower; so native FP64 at every order, double-word
// up to N1 = 6.
template <class P, int N1, int KIND>
constexpr bool kShareAxis = (KIND == AX_GEOM_TRILINEAR || KIND == AX_GEOM_TRILINEAR_PARTIAL) &&
                            (P::kRoll ? N1 <= 6 : sizeof(typename P::V) == 8);

template <int N1, int EM = 1, int EPB0 = 0>
struct Shape {
  static constexpr int n3 = N1 * N1 * N1;
  static constexpr int F = N1 * N1;  // fibers (threads) per element
  static constexpr int EPB = EM * (EPB0 > 0 ? EPB0 : (F >= 128 ? 1 : 128 / F));  // elements per CTA (EM: tile variant)
  static constexpr int threads = F * EPB;
  static constexpr int P = N1 + 1;            // padded row
  static constexpr int ES = N1 * N1 * P;      // padded element size (words)
  __device__ static __forceinline__ int at(int i, int j, int k) { return i + P * (j + N1 * k); }
};

// ---------------------------------------------------------------------------
// geometry (getFactors of Algorithm 4) in policy arithmetic
//
// Trilinear (Algorithm 2, true Jacobian): the element's record holds the
// map's monomial coefficients (A..G of x = x0 + Ar + Bs + Ct + Drs + Ert +
// Fst + Grst, Eq. 8), from which thread (i,j) forms the columns
//   J0(t) = E0 + t E1  (E0, E1 depend on s = xi_j),
//   J1(t) = F0 + t F1  (F0, F1 depend on r = xi_i),   J2 = Jc2(r, s),
// so along its k-fiber (t = xi_k) every entry of K = J^T J is a polynomial
// in t of degree <= 2 (K02, K12 affine, K22 constant) and so is
// det J = J2 . (J0 x J1).  The prologue computes their coefficients once;
// each node then costs 10 multiply-adds for K and det J, the adjugate
// (Eq. 12) and one division:  (r,s,t) = adj(K) (lambda x), lambda = w/det J.
// ---------------------------------------------------------------------------
template <class P, int N1, int KIND>
struct Geometry {
  using V = typename P::V;
  using S = typename P::S;
  V wij;
  V k00[3], k01[3], k11[3], k02[2], k12[2], k22, dt[3];  // polynomial coefficients in t
  V h[7];
  const S *gl = nullptr;

  // Terms of the trilinear geometry that depend on one reference coordinate
  // only, written to out[0..8]:  axis 0 (u = r = xi_idx): F0 = B + D r,
  // F1 = F + G r and the K11 coefficients (F0.F0, 2 F0.F1, F1.F1);  axis 1
  // (u = s = xi_idx): E0 = A + D s, E1 = E + G s and the K00 coefficients.
  // An element has N1 of each, which its first 2 N1 threads compute once and
  // share (kAxisWords words per set) instead of every thread recomputing them.
  static constexpr int kAxisWords = 9;
  __device__ __forceinline__ static void axis_terms(const S *sv, const typename P::C *xg, int axis, int idx,
                                                    S *out) {
    const V u = P::cst(xg + idx);
    V X0[3], X1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      auto M = [&](int m) { return P::ld(sv + 3 * m + c); };  // A B C D E F G = 0..6
      X0[c] = P::fma3(M(3), u, M(axis ? 0 : 1));
      X1[c] = P::fma3(M(6), u, M(axis ? 4 : 5));
      out[c] = P::st(X0[c]);
      out[3 + c] = P::st(X1[c]);
    }
    out[6] = P::st(dot3<P>(X0, X0));
    out[7] = P::st(P::twice(dot3<P>(X0, X1)));
    out[8] = P::st(dot3<P>(X1, X1));
  }

  // AX: read the axis terms from ax, the element's shared table
  // ([2][N1][kAxisWords], see axis_terms), instead of computing them here.
  template <bool AX = false>
  __device__ __forceinline__ void prologue(const S *sv, const typename P::C *xg, const typename P::C *wg, int i,
                                           int j, const S *G_e, const S *lam_e, const S *ax = nullptr) {
    wij = P::mul(P::cst(wg + i), P::cst(wg + j));
    if constexpr (KIND == AX_GEOM_STORED) {
      gl = G_e;
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
#pragma unroll
      for (int q = 0; q < 7; ++q) h[q] = P::ld(sv + q);
    } else {
      // columns of J from the monomial coefficients of the map (Eq. 8):
      // J0 = E0 + t E1, E0 = A + D s, E1 = E + G s;  J1 = F0 + t F1, F0 = B + D r,
      // F1 = F + G r;  J2 = C + E r + F s + G rs   (r = xi_i, s = xi_j)
      V E0[3], E1[3], F0[3], F1[3], J2[3];
      const V r = P::cst(xg + i), s = P::cst(xg + j), rs = P::mul(r, s);
      if constexpr (AX) {
        const S *fi = ax + i * kAxisWords, *ej = ax + (N1 + j) * kAxisWords;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          F0[c] = P::ld(fi + c); F1[c] = P::ld(fi + 3 + c);
          E0[c] = P::ld(ej + c); E1[c] = P::ld(ej + 3 + c);
          k11[c] = P::ld(fi + 6 + c); k00[c] = P::ld(ej + 6 + c);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        auto M = [&](int m) { return P::ld(sv + 3 * m + c); };  // A B C D E F G = 0..6
        if constexpr (!AX) {
          E0[c] = P::fma3(M(3), s, M(0));
          E1[c] = P::fma3(M(6), s, M(4));
          F0[c] = P::fma3(M(3), r, M(1));
          F1[c] = P::fma3(M(6), r, M(5));
        }
        typename P::A q = P::mul0(M(4), r);
        P::mac(q, M(5), s);
        P::mac(q, M(6), rs);
        J2[c] = P::add(M(2), P::fin(q));
      }
      if constexpr (!AX) {
        k00[0] = dot3<P>(E0, E0); k00[1] = P::twice(dot3<P>(E0, E1)); k00[2] = dot3<P>(E1, E1);
        k11[0] = dot3<P>(F0, F0); k11[1] = P::twice(dot3<P>(F0, F1)); k11[2] = dot3<P>(F1, F1);
      }
      // K = J^T J as polynomials in t
      k01[0] = dot3<P>(E0, F0); k01[1] = P::add(dot3<P>(E0, F1), dot3<P>(E1, F0)); k01[2] = dot3<P>(E1, F1);
      k02[0] = dot3<P>(E0, J2); k02[1] = dot3<P>(E1, J2);
      k12[0] = dot3<P>(F0, J2); k12[1] = dot3<P>(F1, J2);
      k22 = dot3<P>(J2, J2);
      if constexpr (KIND == AX_GEOM_TRILINEAR) {
        // det J(t) = J2 . (J0 x J1) = J0 . (J1 x J2): with w_a = F_a x J2
        V w0[3], w1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
          w0[c] = det2<P>(F0[c1], J2[c2], F0[c2], J2[c1]);
          w1[c] = det2<P>(F1[c1], J2[c2], F1[c2], J2[c1]);
        }
        dt[0] = dot3<P>(E0, w0);
        dt[1] = P::add(dot3<P>(E0, w1), dot3<P>(E1, w0));
        dt[2] = dot3<P>(E1, w1);
      }
      gl = lam_e;
    }
  }

  __device__ __forceinline__ static V quad(const V c[3], V t) { return P::fma3(t, P::fma3(t, c[2], c[1]), c[0]); }
  __device__ __forceinline__ static V lin(const V c[2], V t) { return P::fma3(t, c[1], c[0]); }

  // adjugate of K at t (symmetric: A00 A01 A02 A11 A12 A22)
  __device__ __forceinline__ void adjK(V t, V A[6]) const {
    const V K00 = quad(k00, t), K01 = quad(k01, t), K11 = quad(k11, t), K02 = lin(k02, t), K12 = lin(k12, t);
    A[0] = det2<P>(K11, k22, K12, K12);
    A[1] = det2<P>(K02, K12, K01, k22);
    A[2] = det2<P>(K01, K12, K02, K11);
    A[3] = det2<P>(K00, k22, K02, K02);
    A[4] = det2<P>(K01, K02, K00, K12);
    A[5] = det2<P>(K00, K11, K01, K01);
  }

  // (r, s, t) = G (x0, x1, x2) at local node l (t = xi_k, wk = w_k)
  __device__ __forceinline__ void apply(int l, V t, V wk, const V xv[3], V out[3]) const {
    constexpr int n3 = N1 * N1 * N1;
    V A[6];
    V y[3];
    if constexpr (KIND == AX_GEOM_STORED) {
#pragma unroll
      for (int q = 0; q < 6; ++q) A[q] = P::ld(gl + q * n3 + l);
      y[0] = xv[0]; y[1] = xv[1]; y[2] = xv[2];
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
#pragma unroll
      for (int q = 0; q < 6; ++q) A[q] = h[q];
      const V W = P::mul(wij, wk);
      y[0] = P::mul(W, xv[0]); y[1] = P::mul(W, xv[1]); y[2] = P::mul(W, xv[2]);
    } else {
      adjK(t, A);
      V lam;
      if constexpr (KIND == AX_GEOM_TRILINEAR)
        lam = P::div(P::mul(wij, wk), quad(dt, t));
      else
        lam = P::ld(gl + l);
      y[0] = P::mul(lam, xv[0]); y[1] = P::mul(lam, xv[1]); y[2] = P::mul(lam, xv[2]);
    }
    const V gr[3] = {A[0], A[1], A[2]}, gs[3] = {A[1], A[3], A[4]}, gt[3] = {A[2], A[4], A[5]};
    out[0] = dot3<P>(gr, y);
    out[1] = dot3<P>(gs, y);
    out[2] = dot3<P>(gt, y);
  }

  // g[0..5] = g00 g01 g02 g11 g12 g22 at local node l; returns the seventh factor w|J|.
  __device__ __forceinline__ V factors(int l, V t, V wk, V g[6]) const {
    constexpr int n3 = N1 * N1 * N1;
    if constexpr (KIND == AX_GEOM_STORED) {
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = P::ld(gl + q * n3 + l);
      return P::ld(gl + 6 * n3 + l);
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
      const V W = P::mul(wij, wk);
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = P::mul(W, h[q]);
      return P::mul(W, h[6]);
    } else {
      V A[6];
      adjK(t, A);
      const V W = P::mul(wij, wk);
      V lam, wdet;
      if constexpr (KIND == AX_GEOM_TRILINEAR) {
        const V det = quad(dt, t);
        lam = P::div(W, det);
        wdet = P::mul(W, det);
      } else {
        lam = P::ld(gl + l);
        wdet = P::div(P::mul(W, W), lam);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = P::mul(lam, A[q]);
      return wdet;
    }
  }
};


// Power-of-two scaling of an element's float64 values (policies with
// kScaleIO).  emax is the largest biased exponent field among the element's
// values; the shift d brings the largest magnitude into [1, 2) (clamped so
// that 2^d and 2^-d are normal doubles).  Elements with an infinity or NaN
// (emax 0x7ff) are not scaled.
__device__ __forceinline__ int io_shift(int emax) {
  if (emax == 0x7ff) return 0;
  if (emax == 0) return 1022;  // zeros and float64 subnormals: brought up by 2^1022
  const int d = 1023 - emax;
  return d < -1022 ? -1022 : (d > 1022 ? 1022 : d);
}
__device__ __forceinline__ double pow2i(int d) { return __hiloint2double((1023 + d) << 20, 0); }
__device__ __forceinline__ int exp_field(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ __forceinline__ int exp_field(float v) { return (__float_as_int(v) >> 23) & 0xff; }
// Direct range of the double-word kernels, tested per row of N1 values on
// the largest magnitude of the row, read from the upper 32 bits of the
// float64 values (sign cleared, integer order = magnitude order): a row is
// direct when it is all zero or its largest magnitude lies in
// [2^-60, 2^61), and no value of it is nonzero below 2^-74.  Within it the
// float pairs and every intermediate of the product stay normal floats for
// element extents in [2^-20, 2^24] (checked at setup), values far below their
// row's largest contribute below the accuracy, and X is converted by integer
// instructions (dw::from_double_direct, whose range ends at 2^-74); Y goes
// back the same way (dw::sum3_to_double_direct).  The fix-up kernel over the
// other blocks converts on the FP64 pipe.
__device__ __forceinline__ int mag_hi(double v) { return __double2hiint(v) & 0x7fffffff; }
__device__ __forceinline__ bool row_direct(int hmax) {
  return hmax == 0 || (hmax >= ((1023 - 60) << 20) && hmax < ((1023 + 61) << 20));
}

// Coalesced copy of a block of values (contiguous in HBM) into padded
// shared-memory rows of N1 values (pitch PITCH), converted by the policy P:
// value m goes to row m / N1 at i = m % N1.  Consecutive threads read
// consecutive 16-byte vectors when the values come in whole vectors and the
// pointer is 16-byte aligned, else consecutive words.  THREADS * N1 >= nvals.
template <class P, int N1, int PITCH, int THREADS>
__device__ __forceinline__ bool load_rows(const typename P::IO *__restrict__ src, int nvals, typename P::S *xs,
                                          int tid, const int *emax) {
  // emax (kScaleIO policies, or nullptr): per-element largest exponent field;
  // each value is scaled by its element's power of two.  Without it the
  // return value says whether a nonzero value lay outside the direct range.
  using IO = typename P::IO;
  constexpr int n3 = N1 * N1 * N1, VEC = 16 / (int)sizeof(IO);
  bool wide = false;
  auto put = [&](int m, IO v) {
    const int row = m / N1;
    if constexpr (P::kScaleIO) {
      if (emax) v = v * pow2i(io_shift(emax[m / n3]));
    }
    if constexpr (P::kScaleIO) {
      // each value alone is its own "row" here (a nonzero value is then at
      // least 2^-60: inside from_io_direct's range)
      if (!emax) wide |= !row_direct(mag_hi(v));
    }
    xs[row * PITCH + (m - row * N1)] = P::st(emax ? P::from_io(v) : P::from_io_direct(v));
  };
  if constexpr (n3 % VEC == 0) {
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      using VT = typename std::conditional<sizeof(IO) == 4, float4, double2>::type;
      const VT *srcv = reinterpret_cast<const VT *>(src);
#pragma unroll
      for (int s = 0; s < (N1 + VEC - 1) / VEC; ++s) {
        const int mv = tid + s * THREADS;
        if (mv * VEC < nvals) {
          const VT v = srcv[mv];
          const IO *pv = reinterpret_cast<const IO *>(&v);
#pragma unroll
          for (int c = 0; c < VEC; ++c) put(mv * VEC + c, pv[c]);
        }
      }
      return wide;
    }
  }
#pragma unroll
  for (int s = 0; s < N1; ++s) {
    const int m = tid + s * THREADS;
    if (m < nvals) put(m, src[m]);
  }
  return wide;
}

template <int KIND>
struct GeoWords {
  static constexpr int value = (KIND == AX_GEOM_STORED) ? 0 : (KIND == AX_GEOM_PARALLELEPIPED ? kParWords : kVertexWords);
};

// Sources of X: in place (element e's values at X[e n3 + m]), or the local
// copies of a global vector, X[m] = u[gid[m]] (the scatter Q u of Eq. 1,
// fused into the load).
template <typename IO>
struct XDirect {
  static constexpr bool kDirect = true;
  const IO *__restrict__ p;
  __device__ __forceinline__ IO operator[](int64_t m) const { return p[m]; }
};
template <typename IO>
struct XGather {
  static constexpr bool kDirect = false;
  const IO *__restrict__ u;
  const gidx *__restrict__ gid;
  __device__ __forceinline__ IO operator[](int64_t m) const { return u[gid[m]]; }
};

// Shared-memory buffers of one block of EPB elements.
// EPB0: the block shape (kEpb for the per-order kernels).
template <class P, int N1, int KIND, int EM, int EPB0 = kEpb<P, N1, KIND>>
struct FiberSmem {
  using Sh = Shape<N1, EM, EPB0>;
  using S = typename P::S;
  static constexpr int GW = GeoWords<KIND>::value, GWD = GW > 0 ? GW : 1;
  static constexpr bool AXS = kShareAxis<P, N1, KIND>;
  static constexpr int AXD = AXS ? 2 * N1 * Geometry<P, N1, KIND>::kAxisWords : 1;
  S *xs;        // [3][EPB][ES]: x, x0, x1; later t / Y_t, r / Y_r, s / Y_s
  S *sgeo;      // [EPB][GWD]: the elements' geometry records
  S *sax;       // [EPB][AXD]: per-element axis terms of the trilinear geometry (AXS)
  int *sexp;    // [EPB] largest exponent field of each element's X (scaled fix-up pass)
  __host__ __device__ static constexpr size_t a16(size_t b) { return (b + 15) / 16 * 16; }
  // all four carved from one 16-byte aligned buffer of `bytes` bytes
  static constexpr size_t bytes = a16(sizeof(S) * 3 * Sh::EPB * Sh::ES) + a16(sizeof(S) * Sh::EPB * GWD) +
                                  a16(sizeof(S) * Sh::EPB * AXD) + a16(sizeof(int) * Sh::EPB);
  __device__ static __forceinline__ FiberSmem carve(unsigned char *raw) {
    FiberSmem m;
    m.xs = (S *)raw;
    raw += a16(sizeof(S) * 3 * Sh::EPB * Sh::ES);
    m.sgeo = (S *)raw;
    raw += a16(sizeof(S) * Sh::EPB * GWD);
    m.sax = (S *)raw;
    raw += a16(sizeof(S) * Sh::EPB * AXD);
    m.sexp = (int *)raw;
    return m;
  }
};

// ---------------------------------------------------------------------------
// AxLocal of one block of elements [e0, e0 + nel), nel <= EPB, by the CTA's
// threads (Algorithm 1 with the geometry of Algorithms 2 and 3).  Tables
// (per translation unit, constant memory): c_eoD / c_eoDT even-odd blocks of
// D and D^T, c_w, c_x weights and points.  IDLE: the CTA may have more
// threads than the order's shape (a CTA shaped for several orders); those
// threads only take part in the barriers.
// ---------------------------------------------------------------------------
template <class P, int N1, int KIND, int EM, bool IDLE, int SCALE, class XS, int EPB0 = kEpb<P, N1, KIND>>
__device__ __forceinline__ bool fiber_block(const FiberSmem<P, N1, KIND, EM, EPB0> &sm, const int tid, const int64_t e0,
                                            const int nel, const typename P::S *__restrict__ geo,
                                            const typename P::S *__restrict__ lam, const XS &X,
                                            typename P::IO *__restrict__ Y) {
  using Sh = Shape<N1, EM, EPB0>;
  using Buf = FiberSmem<P, N1, KIND, EM, EPB0>;
  using V = typename P::V;
  using S = typename P::S;
  constexpr int n3 = Sh::n3, EPB = Sh::EPB, ES = Sh::ES;
  constexpr int GW = GeoWords<KIND>::value;
  static_assert(!IDLE || !P::kRoll, "idle threads are handled in the short (native) kernel body");
  static_assert(SCALE == 0 || P::kScaleIO, "X scaling belongs to the policies with kScaleIO");
  S *const xs = sm.xs;          // [EPB][ES]: x, later Y
  S *const b0 = xs + EPB * ES;  // x0, later r
  S *const b1 = b0 + EPB * ES;  // x1, later s
  int *const sexp = sm.sexp;
  constexpr bool AXS = Buf::AXS;
  constexpr int AXW = Geometry<P, N1, KIND>::kAxisWords;
  const bool act = !IDLE || tid < Sh::threads;
  const int z = tid / Sh::F, q = tid % Sh::F;
  const int qa = q % N1, qb = q / N1;
  const typename P::C *eoD = c_eoD + tab_off_D(N1);
  const typename P::C *eoDT = c_eoDT + tab_off_D(N1);
  const float4 *eo2D = c_eo2D + tab_off_P(N1), *eo2DT = c_eo2DT + tab_off_P(N1);
  const typename P::C *cw = c_w + tab_off_v(N1);
  const typename P::C *cx = c_x + tab_off_v(N1);
  const S *const sgeo_z = sm.sgeo + (act ? z : 0) * Buf::GWD;
  S *const sax_z = sm.sax + (act && AXS ? z : 0) * Buf::AXD;
  const int64_t e = e0 + z;
  const bool live = act && z < nel;

  // pass 0: the CTA's elements (contiguous in HBM) into padded shared memory.
  // Value m of the block sits in row m / N1 (row = j + N1 (k + N1 z) is also
  // the padded row index) at i = m % N1.  Float32 data at N1 = 2, 4, 8 and
  // double-word data at N1 = 16 are read coalesced (load_rows): measured on
  // GB300 4-16% faster than one row per thread for float32 at N = 3 and 7,
  // 3-10% for double-word at N = 15.  Elsewhere one i-row of N1 values per
  // thread: the coalesced form measured 10% slower for float32 N = 5 and 29%
  // for double-word N = 5 (the row and column of each value cost a division
  // there), 2% slower for double-word N = 3 and 7 and, through a register
  // increase that halves the resident CTAs, 23% slower for float32 N = 15
  // (the compiler raises the register count at every N1 >= 11 of the float32
  // kernels with it).
  // (a gathered X, X[m] = u[gid[m]], is read one row per thread)
  constexpr bool kRowsCoalesced =
      XS::kDirect && ((sizeof(typename P::IO) == 4 && (N1 == 2 || N1 == 4 || N1 == 8)) || (P::kRoll && N1 == 16));
  // Policies with kScaleIO (float64 data in float32 pairs) run in two modes.
  // SCALE = 1, the main kernel: X is converted directly and the block
  // reports whether a row's largest magnitude lies outside the direct range
  // (row_direct).  SCALE = 2, a fix-up kernel over only the reported blocks:
  // each element's X is scaled by the power of two that brings its largest
  // magnitude into [1, 2) before the conversion, and its Y is scaled back.
  bool wide = false;  // SCALE 1: a row of this thread lies outside the direct range
  int xshift = 0;     // SCALE 2: this thread's element entered as X * 2^xshift
  if constexpr (SCALE == 2) {
    if (live) {
      const int64_t srow = e * n3 + q * N1;  // row q of element z
      int mx = 0;
#pragma unroll
      for (int i = 0; i < N1; ++i) mx = max(mx, exp_field(X[srow + i]));
      atomicMax(&sexp[z], mx);
    }
    __syncthreads();
    if (live) xshift = io_shift(sexp[z]);
  }
  if (act) {
    using IO = typename P::IO;
    if constexpr (kRowsCoalesced) {
      wide = load_rows<P, N1, Sh::P, Sh::threads>(X.p + e0 * n3, nel * n3, xs, tid, SCALE == 2 ? sexp : nullptr);
    } else {
      for (int row = tid; row < nel * N1 * N1; row += Sh::threads) {
        const int64_t src = e0 * n3 + (int64_t)row * N1;
        S *dst = xs + row * Sh::P;
        // SCALE 2: one row per thread (threads = EPB N1^2), row tid of element z
        const IO sc = SCALE == 2 ? (IO)pow2i(xshift) : IO(1);
        int hmax = 0;       // SCALE 1: the row's largest magnitude (upper 32 bits)
        bool tiny = false;  // SCALE 1: a nonzero value below from_io_direct's range
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          const IO v = X[src + i];
          if constexpr (SCALE == 1) {
            hmax = max(hmax, mag_hi(v));
            if constexpr (P::kScaleIO) tiny |= dw::tiny_nonzero((unsigned)mag_hi(v));
            dst[i] = P::st(P::from_io_direct(v));
          } else {
            dst[i] = P::st(P::from_io(SCALE == 2 ? v * sc : v));
          }
        }
        if constexpr (SCALE == 1) wide |= tiny || !row_direct(hmax);
      }
    }
    if constexpr (GW > 0) {
      for (int m = tid; m < nel * GW; m += Sh::threads) sm.sgeo[(m / GW) * Buf::GWD + m % GW] = geo[e0 * GW + m];
    }
  }
  bool any_wide = false;
  if constexpr (SCALE == 1) {
    any_wide = __syncthreads_or(wide);
  } else {
    __syncthreads();
  }
  if constexpr (SCALE == 2) {
    if (tid < EPB) sexp[tid] = 0;  // every read of sexp came before the barrier
  }
  if constexpr (AXS) {
    // threads q < 2 N1 of each element: the N1 r-axis and N1 s-axis terms,
    // read by every thread's geometry prologue after the next barriers
    if (live && q < 2 * N1) Geometry<P, N1, KIND>::axis_terms(sgeo_z, cx, q / N1, q % N1, sax_z + q * AXW);
  }

  S *x_e = xs + z * ES, *r_e = b0 + z * ES, *s_e = b1 + z * ES;
  // Six fiber products in two rolled phase loops (one code copy of the fiber
  // product per matrix, D or D^T, so the constants stay immediate operands
  // and the instruction footprint fits the instruction cache):
  //   ph 0: r-fibers  D x -> B0 (x0)     ph 1: s-fibers  D x -> B1 (x1)
  //   ph 2: t-fiber   D x -> X  (x2);  then per node the geometry and
  //         (r,s,t) = G (x0,x1,x2): r -> B0, s -> B1, t -> X
  //   ph 3: t-fiber   D^T t -> registers (Y_t)
  //   ph 4: r-fibers  D^T r -> B0 (Y_r)  ph 5: s-fibers  D^T s -> B1 (Y_s)
  //   then the t-fiber owner stores Y = Y_t + Y_r + Y_s to HBM
  const int fr = Sh::at(0, qa, qb), fs = Sh::at(qa, 0, qb), ft = Sh::at(qa, qb, 0);
  constexpr int str_r = 1, str_s = Sh::P, str_t = Sh::P * N1;
  auto forward = [&](int ph) {
    if (ph == 2) __syncthreads();  // every r/s-fiber read of x is done before x is overwritten
    S *dst = ph == 0 ? r_e : (ph == 1 ? s_e : x_e);
    const int base = ph == 0 ? fr : (ph == 1 ? fs : ft);
    const int stride = ph == 0 ? str_r : (ph == 1 ? str_s : str_t);
    V fin_[N1], fout[N1];
#pragma unroll
    for (int n = 0; n < N1; ++n) fin_[n] = P::ld(x_e + base + n * stride);
    contract_p<P, N1, KIND>(eoD, eo2D, fin_, fout);
#pragma unroll
    for (int n = 0; n < N1; ++n) dst[base + n * stride] = P::st(fout[n]);
  };
  if constexpr (P::kRoll) {
#pragma unroll 1
    for (int ph = 0; ph < 3; ++ph) forward(ph);
  __syncthreads();
  {
    // thread (i, j) = (qa, qb): geometry and G x along its own t-fiber
    const int i = qa, j = qb;
    Geometry<P, N1, KIND> gm;
    gm.template prologue<AXS>(sgeo_z, cx, cw, i, j, (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * n3 : nullptr,
                              (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * n3 : nullptr, sax_z);
    auto node = [&](int k) {
      const int sidx = ft + k * str_t;
      const V xv[3] = {P::ld(r_e + sidx), P::ld(s_e + sidx), P::ld(x_e + sidx)};
      V o3[3];
      if (live) {
        gm.apply(i + j * N1 + k * N1 * N1, P::cst(cx + k), P::cst(cw + k), xv, o3);
      } else {
        o3[0] = o3[1] = o3[2] = P::lit(0.0);
      }
      r_e[sidx] = P::st(o3[0]);
      s_e[sidx] = P::st(o3[1]);
      x_e[sidx] = P::st(o3[2]);
    };
#pragma unroll 1
    for (int k = 0; k < N1; ++k) node(k);
  }
    // transposed products: D_t^T t of the own t-fiber, then the r- and
    // s-fibers in place in B0, B1 (one rolled loop: one code copy of the D^T
    // product); the t-fiber owner sums and stores Y.  Y_t stays in registers
    // up to N1 = 10; above, the 2 N1 extra registers would cost resident
    // warps, so it goes back in place into X (read only by its owner).
    constexpr bool kYtRegs = N1 <= 10;
    V yt[kYtRegs ? N1 : 1];
#pragma unroll 1
    for (int ph = 3; ph < 6; ++ph) {
      if (ph == 4) __syncthreads();  // every thread's r, s values are in B0, B1
      S *buf = ph == 3 ? x_e : (ph == 4 ? r_e : s_e);
      const int base = ph == 3 ? ft : (ph == 4 ? fr : fs);
      const int stride = ph == 3 ? str_t : (ph == 4 ? str_r : str_s);
      V fin_[N1], fout[N1];
#pragma unroll
      for (int n = 0; n < N1; ++n) fin_[n] = P::ld(buf + base + n * stride);
      contract_p<P, N1, KIND>(eoDT, eo2DT, fin_, fout);
      if (kYtRegs && ph == 3) {
#pragma unroll
        for (int n = 0; n < N1; ++n) yt[kYtRegs ? n : 0] = fout[n];
      } else {
#pragma unroll
        for (int n = 0; n < N1; ++n) buf[base + n * stride] = P::st(fout[n]);
      }
    }
    __syncthreads();  // every Y_r, Y_s value is in B0, B1
    if (live) {
      typename P::IO *ye = Y + e * n3 + qa + N1 * qb;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int sidx = ft + k * str_t;
        const V ytk = kYtRegs ? yt[kYtRegs ? k : 0] : P::ld(x_e + sidx);
        const V yr = P::ld(r_e + sidx), ys = P::ld(s_e + sidx);
        ye[k * N1 * N1] = SCALE == 1 ? P::sum3_io_direct(ytk, yr, ys) : P::sum3_io(ytk, yr, ys);
      }
      if constexpr (SCALE == 2) {
        // undo the element's input shift on the values just stored (exact)
        if (xshift != 0) {
          const typename P::IO ysc = (typename P::IO)pow2i(-xshift);
#pragma unroll 1
          for (int k = 0; k < N1; ++k) ye[k * N1 * N1] *= ysc;
        }
      }
    }
  } else {
    // Short code (native arithmetic): the thread's own t-fiber stays in
    // registers from D_t x through the geometry to D_t^T t (no shared-memory
    // round trips, x never overwritten); the r- and s-fiber transposed
    // products overwrite B0 and B1 in place (no read-modify-write of Y, no
    // barrier between them); the t-fiber owner sums Y = Y_t + Y_r + Y_s at
    // its nodes and stores it to HBM (for each k the warp writes consecutive
    // i, j: coalesced).  (IDLE threads skip every step but the barriers.)
    V tf[N1];
    if (act) {
      forward(0);
      forward(1);
      V fin_[N1];
#pragma unroll
      for (int n = 0; n < N1; ++n) fin_[n] = P::ld(x_e + ft + n * str_t);
      contract_p<P, N1, KIND>(eoD, eo2D, fin_, tf);
    }
    __syncthreads();  // every r/s fiber product is in B0, B1
    V yt[N1];
    if (act) {
      const int i = qa, j = qb;
      Geometry<P, N1, KIND> gm;
      gm.template prologue<AXS>(sgeo_z, cx, cw, i, j,
                                (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * n3 : nullptr,
                                (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * n3 : nullptr, sax_z);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int sidx = ft + k * str_t;
        const V xv[3] = {P::ld(r_e + sidx), P::ld(s_e + sidx), tf[k]};
        V o3[3];
        if (live) {
          gm.apply(i + j * N1 + k * N1 * N1, P::cst(cx + k), P::cst(cw + k), xv, o3);
        } else {
          o3[0] = o3[1] = o3[2] = P::lit(0.0);
        }
        r_e[sidx] = P::st(o3[0]);
        s_e[sidx] = P::st(o3[1]);
        tf[k] = o3[2];
      }
      contract_p<P, N1, KIND>(eoDT, eo2DT, tf, yt);
    }
    __syncthreads();  // every r, s value is in B0, B1
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (!act) break;
      S *buf = d == 0 ? r_e : s_e;
      const int base = d == 0 ? fr : fs, stride = d == 0 ? str_r : str_s;
      V fin_[N1], fout[N1];
#pragma unroll
      for (int n = 0; n < N1; ++n) fin_[n] = P::ld(buf + base + n * stride);
      contract_p<P, N1, KIND>(eoDT, eo2DT, fin_, fout);
#pragma unroll
      for (int n = 0; n < N1; ++n) buf[base + n * stride] = P::st(fout[n]);
    }
    __syncthreads();  // every Y_r, Y_s value is in B0, B1
    if (live) {
      typename P::IO *ye = Y + e * n3 + qa + N1 * qb;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int sidx = ft + k * str_t;
        ye[k * N1 * N1] = P::sum3_io(yt[k], P::ld(r_e + sidx), P::ld(s_e + sidx));
      }
    }
  }

  __syncthreads();  // the next block reuses the shared buffers
  return any_wide;
}

// ---------------------------------------------------------------------------
// the per-order kernel: blocks of EPB elements, persistent over blocks when
// the grid is capped (autotuner)
// ---------------------------------------------------------------------------
// wide: kScaleIO policies: list of the blocks whose X left the direct range
// ([0] count, [1] exit counter of the fix-up kernel, [2..] block indices).
template <class P, int N1, int KIND, int EM>
__global__ void __launch_bounds__(Shape<N1, EM, kEpb<P, N1, KIND>>::threads, kMinCtas<P, N1, KIND>)
    ax_fiber_kernel(int64_t E, const typename P::S *__restrict__ geo, const typename P::S *__restrict__ lam,
                    const typename P::IO *__restrict__ X, typename P::IO *__restrict__ Y, int *__restrict__ wide) {
  using Sh = Shape<N1, EM, kEpb<P, N1, KIND>>;
  using Buf = FiberSmem<P, N1, KIND, EM>;
  using S = typename P::S;
  constexpr int EPB = Sh::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ S sgeo[EPB][Buf::GWD];
  __shared__ S sax[Buf::AXS ? EPB : 1][Buf::AXD];
  Buf sm;
  sm.xs = (S *)smem_raw;
  sm.sgeo = &sgeo[0][0];
  sm.sax = &sax[0][0];
  sm.sexp = nullptr;
  const int tid = threadIdx.x;
  const int64_t nblk = (E + EPB - 1) / EPB;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t e0 = blk * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    const bool w = fiber_block<P, N1, KIND, EM, false, P::kScaleIO ? 1 : 0>(sm, tid, e0, nel, geo, lam,
                                                                           XDirect<typename P::IO>{X}, Y);
    if constexpr (P::kScaleIO) {
      if (w && tid == 0) wide[2 + atomicAdd(&wide[0], 1)] = (int)blk;
    }
  }
}

// The fix-up kernel of the kScaleIO policies: the listed blocks again, with X
// scaled per element; the last CTA to finish clears the list.
template <class P, int N1, int KIND, int EM>
__global__ void __launch_bounds__(Shape<N1, EM, kEpb<P, N1, KIND>>::threads)
    ax_fiber_fix_kernel(int64_t E, const typename P::S *__restrict__ geo, const typename P::S *__restrict__ lam,
                        const typename P::IO *__restrict__ X, typename P::IO *__restrict__ Y, int *__restrict__ wide) {
  using Sh = Shape<N1, EM, kEpb<P, N1, KIND>>;
  using Buf = FiberSmem<P, N1, KIND, EM>;
  using S = typename P::S;
  constexpr int EPB = Sh::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ S sgeo[EPB][Buf::GWD];
  __shared__ S sax[Buf::AXS ? EPB : 1][Buf::AXD];
  __shared__ int sexp[EPB];
  Buf sm;
  sm.xs = (S *)smem_raw;
  sm.sgeo = &sgeo[0][0];
  sm.sax = &sax[0][0];
  sm.sexp = sexp;
  const int tid = threadIdx.x;
  if (tid < EPB) sexp[tid] = 0;
  __syncthreads();
  const int cnt = *(volatile int *)&wide[0];
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int64_t e0 = (int64_t)wide[2 + i] * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    fiber_block<P, N1, KIND, EM, false, 2>(sm, tid, e0, nel, geo, lam, XDirect<typename P::IO>{X}, Y);
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&wide[1], 1) == (int)gridDim.x - 1) {
      wide[0] = 0;
      wide[1] = 0;
    }
  }
}

// Factor export through the same geometry code: G_out [E][7][n3] float64.
template <class P, int N1, int KIND>
__global__ void __launch_bounds__(Shape<N1, 1, kEpb<P, N1, KIND>>::threads)
    factors_fiber_kernel(int64_t E, const typename P::S *__restrict__ geo, const typename P::S *__restrict__ lam,
                         double *__restrict__ G) {
  using Sh = Shape<N1, 1, kEpb<P, N1, KIND>>;
  using V = typename P::V;
  using S = typename P::S;
  constexpr int n3 = Sh::n3, EPB = Sh::EPB;
  constexpr int GW = GeoWords<KIND>::value;
  __shared__ S sgeo[EPB][GW > 0 ? GW : 1];
  const int tid = threadIdx.x;
  const int z = tid / Sh::F, q = tid % Sh::F;
  const int i = q % N1, j = q / N1;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
  const int64_t e = e0 + z;
  const typename P::C *cw = c_w + tab_off_v(N1);
  const typename P::C *cx = c_x + tab_off_v(N1);
  if constexpr (GW > 0) {
    for (int m = tid; m < nel * GW; m += Sh::threads) sgeo[m / GW][m % GW] = geo[e0 * GW + m];
  }
  __syncthreads();
  if (z >= nel) return;
  Geometry<P, N1, KIND> gm;
  gm.prologue(sgeo[z], cx, cw, i, j, KIND == AX_GEOM_STORED ? geo + e * 7 * n3 : nullptr,
              KIND == AX_GEOM_TRILINEAR_PARTIAL ? lam + e * n3 : nullptr);
  for (int k = 0; k < N1; ++k) {
    const int l = i + j * N1 + k * N1 * N1;
    V g[6];
    const V gwj = gm.factors(l, P::cst(cx + k), P::cst(cw + k), g);
    for (int w = 0; w < 6; ++w) G[(e * 7 + w) * n3 + l] = (double)P::to_io(g[w]);
    G[(e * 7 + 6) * n3 + l] = (double)P::to_io(gwj);
  }
}

// CTAs of the fix-up kernel (a persistent loop over the listed blocks)
constexpr int64_t kFixGrid = 256;

template <class P, int N1, int KIND, int EM>
cudaError_t launch_ax_em(const AxArgs &a) {
  using Sh = Shape<N1, EM, kEpb<P, N1, KIND>>;
  const int64_t nblk = (a.E + Sh::EPB - 1) / Sh::EPB;
  if (nblk <= 0) return cudaSuccess;
  int64_t grid = a.grid > 0 && a.grid < nblk ? a.grid : nblk;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  size_t smem = (size_t)3 * Sh::EPB * Sh::ES * sizeof(typename P::S);
  if constexpr (P::kTargetWarpsPerSM > 0 && N1 == 8 &&
                (KIND == AX_GEOM_TRILINEAR || KIND == AX_GEOM_TRILINEAR_PARTIAL)) {
    // cap the resident CTAs by their shared memory (the kernel uses only its share)
    static int sm_smem = 0;
    if (!sm_smem) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    static int static_smem = -1;
    if (static_smem < 0) {
      cudaFuncAttributes fa;
      static_smem = cudaFuncGetAttributes(&fa, ax_fiber_kernel<P, N1, KIND, EM>) == cudaSuccess ? (int)fa.sharedSizeBytes : 4096;
    }
    const int warps = (Sh::threads + 31) / 32;
    int ctas = (P::kTargetWarpsPerSM + warps / 2) / warps;
    if (ctas < 1) ctas = 1;
    // per CTA: dynamic + static shared memory + the 1 KB the hardware
    // reserves, with 1 KB to spare (with none the driver chose a smaller
    // shared-memory carveout and only ctas - 1 CTAs fitted: measured)
    const size_t cap = sm_smem > 0 ? (size_t)sm_smem / ctas - (size_t)static_smem - 2048 : 0;
    if (cap > smem && cap <= 200 * 1024) smem = cap;
  }
  // per instantiation; static shared memory counts against the same 48 KB
  // default, so the attribute is set whatever the dynamic size
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ax_fiber_kernel<P, N1, KIND, EM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (P::kScaleIO && !a.wide) return cudaErrorInvalidValue;  // the context's block list is required
  ax_fiber_kernel<P, N1, KIND, EM><<<(unsigned)grid, Sh::threads, smem, a.stream>>>(
      a.E, (const typename P::S *)a.geo, (const typename P::S *)a.lam, (const typename P::IO *)a.X,
      (typename P::IO *)a.Y, a.wide);
  if constexpr (P::kScaleIO) {
    // the blocks whose X left the direct range, again with scaling (usually none)
    static bool fix_attr = false;
    const size_t fsmem = (size_t)3 * Sh::EPB * Sh::ES * sizeof(typename P::S);
    if (!fix_attr) {
      cudaError_t e = cudaFuncSetAttribute(ax_fiber_fix_kernel<P, N1, KIND, EM>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
      if (e != cudaSuccess) return e;
      fix_attr = true;
    }
    const int64_t fgrid = nblk < kFixGrid ? nblk : kFixGrid;
    ax_fiber_fix_kernel<P, N1, KIND, EM><<<(unsigned)fgrid, Sh::threads, fsmem, a.stream>>>(
        a.E, (const typename P::S *)a.geo, (const typename P::S *)a.lam, (const typename P::IO *)a.X,
        (typename P::IO *)a.Y, a.wide);
  }
  return cudaGetLastError();
}

template <class P, int N1, int KIND>
cudaError_t launch_fiber_n(const AxArgs &a, double *G_out) {
  using Sh = Shape<N1, 1, kEpb<P, N1, KIND>>;
  if (G_out) {
    const int64_t blocks = (a.E + Sh::EPB - 1) / Sh::EPB;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    factors_fiber_kernel<P, N1, KIND><<<(unsigned)blocks, Sh::threads, 0, a.stream>>>(
        a.E, (const typename P::S *)a.geo, (const typename P::S *)a.lam, G_out);
    return cudaGetLastError();
  }
  if constexpr (P::kTiles > 1) {
    if (a.tile == 1) return launch_ax_em<P, N1, KIND, 2>(a);
  }
  return launch_ax_em<P, N1, KIND, 1>(a);
}

template <class P, int N1>
cudaError_t launch_fiber_kinds(const AxArgs &a, double *G_out) {
  switch (a.kind) {
    case AX_GEOM_STORED: return launch_fiber_n<P, N1, AX_GEOM_STORED>(a, G_out);
    case AX_GEOM_TRILINEAR: return launch_fiber_n<P, N1, AX_GEOM_TRILINEAR>(a, G_out);
    case AX_GEOM_PARALLELEPIPED: return launch_fiber_n<P, N1, AX_GEOM_PARALLELEPIPED>(a, G_out);
    case AX_GEOM_TRILINEAR_PARTIAL: return launch_fiber_n<P, N1, AX_GEOM_TRILINEAR_PARTIAL>(a, G_out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fiber
}  // namespace ax
