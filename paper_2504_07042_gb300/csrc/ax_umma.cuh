// AxLocal with the six contractions of Algorithm 1 on the 5th-generation
// tensor cores (tcgen05.mma kind::tf32 for TF32 operands, kind::f16 for
// BF16 and FP16 operands; accumulation in tensor memory): the kernel tuned
// for order N = 7 (N1 = 8) described first, and below it the same structure
// sized to every other order (ax_umma_gen_kernel).
//
// A contraction along one direction is a [fibers x 8] by [8 x 8] product.
// Two elements' 64 fibers of one direction make the M = 128 rows of one
// MMA (M = 128, N = 16 with D padded by 8 zero columns, K = 8):
//   forward    x_d[f][a] = sum_m X[f][m] D[a][m]     B = D   (row a, K = m)
//   transposed y_d[f][m] = sum_a t_d[f][a] D[a][m]   B = D^T (row m, K = a)
// with the fibers of direction d as rows: r-fibers (j, k), s-fibers (i, k),
// t-fibers (i, j).  All operands are K-major in shared memory in the
// canonical core-matrix layout without swizzle (8 rows x 16 bytes
// contiguous, LBO between the two K halves, SBO between 8-row groups); each
// operand buffer has its own LBO and SBO, chosen so that the threads'
// stores into it are free of bank conflicts (the t buffer: at most 2-way).
//
// One CTA of 128 threads (thread = TMEM lane = row of the MMA) per tile of
// two elements, persistent over tiles:
//   1. X (coalesced float4 loads) into the three operand buffers, one per
//      fiber direction; the geometry records into shared memory
//   2. one thread issues the three forward MMAs into TMEM columns 0, 16, 32
//      and commits them to an mbarrier
//   3. every thread reads its rows (tcgen05.ld): thread (j,k) the x0 row
//      over i, (i,k) the x1 row over j, (i,j) the x2 row over k; x0 and x1
//      go through shared memory to the t-fiber owner (i,j)
//   4. thread (i,j): per node the FP32 geometry of the fiber kernels
//      (Algorithm 2 / 3, stored or partial) and (r,s,t) = G (x0,x1,x2)
//   5. r, s, t into the operand buffers; the three transposed MMAs
//   6. the three partial products are summed through shared memory by the
//      t-fiber owners, which store Y coalesced.
// Operands: X, r, s, t are rounded to the operand format (to nearest) when
// staged (for TF32 the tensor core would otherwise drop the low mantissa
// bits); D is rounded once per CTA.
// Every mbarrier wait is bounded; one that runs out sets the kernel's error
// word, and the CTA stops and frees its tensor memory.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ax_fiber.cuh"

namespace ax {
namespace umma {

constexpr int kN1 = 8, kN3 = 512, kEPB = 2, kThreads = 128, kTmemCols = 32;

// Operand formats: OP 0 = TF32 (tcgen05.mma kind::tf32, 4-byte operands,
// K = 8 per instruction: the 8 values of a row fill it), OP 1 = BF16 and
// OP 2 = FP16 (kind::f16, 2-byte operands, K = 16 per instruction: a row's 8
// values fill the first K half; the second K half of each A operand is the
// first one again (LBO = 0) and that of each B operand is zero, so it adds
// nothing).  Per format: the operand buffers r (rows (j,k,e), K = i),
// s (rows (i,k,e), K = j), t (rows (i,j,e), K = k) with their LBO and SBO,
// the B buffers of D and D^T, and the instruction descriptor: D float32
// (bits 4-5 = 1), A and B types (bits 7-9, 10-12: TF32 = 2 in kind::tf32;
// F16 = 0, BF16 = 1 in kind::f16), both K-major, N = 16 (bits 17-22 =
// N >> 3), M = 128 (bits 24-28 = M >> 4).
template <int OP>
struct Fmt;
template <>
struct Fmt<0> {
  static constexpr int kEsz = 4;  // bytes per operand value
  // strides from a search over the threads' store patterns: r free of bank
  // conflicts, s and t at most 2-way (a dense r, also 2-way, measured 3% slower)
  static constexpr uint32_t kLboR = 448, kSboR = 288, kLboS = 128, kSboS = 272, kLboT = 128, kSboT = 272;
  static constexpr uint32_t kBytesR = 4896, kBytesS = 4336, kBytesT = 4336;
  // B buffers: 24 rows x K 8 (two K cores of 4 values)
  static constexpr uint32_t kLboB = 128, kSboB = 256, kBytesB = 768;
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
};
template <int OP>
struct Fmt16 {
  static constexpr int kEsz = 2;
  // one K core per row group: r dense (its 8-byte staging stores cover
  // whole rows), s with SBO = 160 bytes (staging and r/s stores free of bank
  // conflicts), t with SBO = 144 (2-way staging stores, conflict-free 16-byte
  // row stores)
  static constexpr uint32_t kLboR = 0, kSboR = 128, kLboS = 0, kSboS = 160, kLboT = 0, kSboT = 144;
  static constexpr uint32_t kBytesR = 16 * 128, kBytesS = 16 * 160, kBytesT = 16 * 144;
  // B buffers: 24 rows x the first K half (three row groups of 128 bytes),
  // then the zero second K half at LBO = 384
  static constexpr uint32_t kLboB = 384, kSboB = 128, kBytesB = 768;
  static constexpr uint32_t kIdesc =
      (1u << 4) | ((OP == 1 ? 1u : 0u) << 7) | ((OP == 1 ? 1u : 0u) << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
};
template <>
struct Fmt<1> : Fmt16<1> {};
template <>
struct Fmt<2> : Fmt16<2> {};
// exchange buffers (x0, x1, then Y_r, Y_s): [e][k][j][i] float32 with pitches
// 576, 72, 8, 1 floats (the k pitch 72 = 8 mod 32 keeps the stride-8 row
// writes and the t-fiber reads free of bank conflicts); apart from the
// operand buffers, so that staging a tile's operands needs no barrier after
// the reads of the previous exchange
constexpr int kXe = 576, kXk = 72;
constexpr uint32_t kBytesX = 2 * kXe * 4;
// D and D^T, each in a 24-row B buffer (rows 8..15 hold it, the rest zero):
// the 16-row descriptor window starting at row 8 puts a product in columns
// 0-7 of its 16-column accumulator, the window starting at row 0 in columns
// 8-15.  So the r and s products share one accumulator (x0 | x1, then
// Y_r | Y_s) and t has the next: 32 TMEM columns per CTA
// shared memory: r, s, t operand buffers, the two exchange buffers, the D
// and D^T B buffers, geometry records, mbarrier, TMEM address
template <int OP>
struct Smem {
  using F = Fmt<OP>;
  static constexpr uint32_t kOffR = 0, kOffS = kOffR + F::kBytesR, kOffT = kOffS + F::kBytesS,
                            kOffX0 = kOffT + F::kBytesT, kOffX1 = kOffX0 + kBytesX, kOffBD = kOffX1 + kBytesX,
                            kOffBDT = kOffBD + F::kBytesB, kOffGeo = kOffBDT + F::kBytesB;
  static constexpr uint32_t kBytes = kOffGeo + kEPB * kVertexWords * 4 + 64;
};
constexpr long long kWaitCycles = 1ll << 32;  // SM clocks (about 2 s) before a wait gives up
// resident CTAs per SM, per kind: the shared memory (about 25 KB each)
// allows eight, the tensor memory 512 / 32 = 16, and the launch bounds size
// the registers for them (at most 64 per thread at eight, 73 at seven).
// Measured on GB300 (GDOF/s at 7 / 8 CTAs): trilinear 208 / 197, stored
// 193 / 156, parallelepiped 244 / 277, partial 157 / 167.
template <int KIND>
constexpr int kCtasPerSm = (KIND == AX_GEOM_TRILINEAR || KIND == AX_GEOM_STORED) ? 7 : 8;

// byte offset of (row, k) in a K-major no-swizzle core-matrix layout of
// ESZ-byte values (16 bytes of K per core-matrix row)
template <int ESZ = 4>
__host__ __device__ constexpr uint32_t cm_off(int row, int k, uint32_t lbo, uint32_t sbo) {
  constexpr int per = 16 / ESZ;  // values per core-matrix row
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k / per) * lbo + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k % per) * ESZ;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory descriptor: K-major, no swizzle, descriptor version 1
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
template <int OP>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  if constexpr (OP == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(Fmt<OP>::kIdesc), "r"(accumulate));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(Fmt<OP>::kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63u) == 63u && clock64() - t0 > kWaitCycles) return false;
  }
}
// 16 float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
// 8 float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ float tf32_rn(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// a value in the operand format (rounded to nearest): the TF32 bits, or the
// 16-bit code in the low half
template <int OP>
__device__ __forceinline__ uint32_t code(float v) {
  if constexpr (OP == 0)
    return __float_as_uint(tf32_rn(v));
  else if constexpr (OP == 1)
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
  else
    return (uint32_t)__half_as_ushort(__float2half_rn(v));
}
// one coded value stored at base + off
template <int OP>
__device__ __forceinline__ void st_code(unsigned char *base, uint32_t off, uint32_t c) {
  if constexpr (OP == 0)
    *(uint32_t *)(base + off) = c;
  else
    *(uint16_t *)(base + off) = (uint16_t)c;
}
// four coded consecutive K values of one row (16-byte aligned for TF32, 8-byte for 16-bit)
template <int OP>
__device__ __forceinline__ void st_code4(unsigned char *base, uint32_t off, const uint32_t c[4]) {
  if constexpr (OP == 0)
    *(uint4 *)(base + off) = make_uint4(c[0], c[1], c[2], c[3]);
  else
    *(uint2 *)(base + off) = make_uint2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
}
template <int OP>
__device__ __forceinline__ void st_op(unsigned char *base, uint32_t off, float v) {
  st_code<OP>(base, off, code<OP>(v));
}

template <int KIND, int OP>
__global__ void __launch_bounds__(kThreads, kCtasPerSm<KIND>)
    ax_umma_kernel(int64_t E, const float *__restrict__ geo, const float *__restrict__ lam,
                   const float *__restrict__ X, float *__restrict__ Y, const float *__restrict__ Dp,
                   int *__restrict__ err) {
  using P = fiber::Native<float>;
  using F = Fmt<OP>;
  using L = Smem<OP>;
  constexpr int ESZ = F::kEsz;
  constexpr int GW = fiber::GeoWords<KIND>::value;
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char *bufR = sm + L::kOffR, *bufS = sm + L::kOffS, *bufT = sm + L::kOffT;
  float *sgeo = (float *)(sm + L::kOffGeo);
  uint64_t *bar = (uint64_t *)(sm + L::kOffGeo + kEPB * kVertexWords * 4);
  uint32_t *tslot = (uint32_t *)(bar + 1);
  __shared__ int abort_cta;
  const int tid = threadIdx.x, warp = tid >> 5;
  const float *cw = fiber::c_w + tab_off_v(kN1);
  const float *cx = fiber::c_x + tab_off_v(kN1);

  // D (rows a, K = m) and D^T (rows m, K = a), in the operand format, at
  // rows 8..15 of their 24-row buffers, zero elsewhere (and in the second K
  // half of the 16-bit formats)
  constexpr int kKB = OP == 0 ? 8 : 16;  // K values per B row
  for (int q = tid; q < 2 * 24 * kKB; q += kThreads) {
    const int which = q / (24 * kKB), row = (q % (24 * kKB)) / kKB, k = q % kKB, a = row - 8;
    float v = 0.0f;
    if (a >= 0 && a < kN1 && k < kN1) v = which == 0 ? Dp[a * kN1 + k] : Dp[k * kN1 + a];
    st_op<OP>(sm + (which == 0 ? L::kOffBD : L::kOffBDT), cm_off<ESZ>(row, k, F::kLboB, F::kSboB), v);
  }
  if (tid == 0) {
    abort_cta = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
  const uint32_t aR = smem_u32(bufR), aS = smem_u32(bufS), aT = smem_u32(bufT);
  const uint32_t aBD = smem_u32(sm + L::kOffBD), aBDT = smem_u32(sm + L::kOffBDT);
  // this thread as a row of each direction: L = a + 8 b + 64 e
  const int la = tid & 7, lb = (tid >> 3) & 7, le = tid >> 6;
  uint32_t phase = 0;

  // float4 loads need a 16-byte aligned X (element offsets are 2048-byte multiples)
  const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  const int64_t ntile = (E + kEPB - 1) / kEPB;
  // X of a tile: two float4 per thread (float4 index f = i0/4 + 2 j + 16 k + 128 e),
  // loaded one tile ahead so that the loads overlap the previous tile's work
  auto load_x = [&](int64_t tt, float4 xv[2]) {
    const int64_t b0 = tt * kEPB;
    const int nl = (int)((E - b0) < kEPB ? (E - b0) : kEPB);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int f = tid + kThreads * s;
      xv[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tt < ntile && (f >> 7) < nl) {
        if (vec) {
          xv[s] = reinterpret_cast<const float4 *>(X + b0 * kN3)[f];
        } else {
          const float *src = X + b0 * kN3 + 4 * f;
          xv[s] = make_float4(src[0], src[1], src[2], src[3]);
        }
      }
    }
  };
  float4 xnext[2];
  load_x(blockIdx.x, xnext);
  for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
    const int64_t e0 = t * kEPB;
    const int nel = (int)((E - e0) < kEPB ? (E - e0) : kEPB);
    // 1. X into the three operand buffers (zeros beyond the last element)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int f = tid + kThreads * s;
      const int i0 = 4 * (f & 1), j = (f >> 1) & 7, k = (f >> 4) & 7, e = f >> 7;
      const float4 v = xnext[s];
      // rounded to the format once (to nearest, not truncated)
      const uint32_t c[4] = {code<OP>(v.x), code<OP>(v.y), code<OP>(v.z), code<OP>(v.w)};
      st_code4<OP>(bufR, cm_off<ESZ>(j + 8 * k + 64 * e, i0, F::kLboR, F::kSboR), c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        st_code<OP>(bufS, cm_off<ESZ>(i0 + q + 8 * k + 64 * e, j, F::kLboS, F::kSboS), c[q]);
        st_code<OP>(bufT, cm_off<ESZ>(i0 + q + 8 * j + 64 * e, k, F::kLboT, F::kSboT), c[q]);
      }
    }
    if constexpr (GW > 0) {
      for (int m = tid; m < nel * GW; m += kThreads) sgeo[m] = geo[e0 * GW + m];
    }
    load_x(t + gridDim.x, xnext);  // the next tile's X, in flight meanwhile
    proxy_fence();
    __syncthreads();
    // 2. forward MMAs
    if (tid == 0 && !abort_cta) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      mma<OP>(tmem, desc(aR, F::kLboR, F::kSboR), desc(aBD + F::kSboB, F::kLboB, F::kSboB), 0u);
      mma<OP>(tmem, desc(aS, F::kLboS, F::kSboS), desc(aBD, F::kLboB, F::kSboB), 1u);
      mma<OP>(tmem + 16, desc(aT, F::kLboT, F::kSboT), desc(aBD + F::kSboB, F::kLboB, F::kSboB), 0u);
      commit(smem_u32(bar));
    }
    // thread 0 waits for the MMAs (bounded); the others sleep in the barrier
    if (tid == 0 && !mbar_wait(smem_u32(bar), phase)) abort_cta = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_cta) {
      if (tid == 0) mbar_wait(smem_u32(bar), phase);  // bounded: the MMAs in flight before TMEM is freed
      break;
    }
    phase ^= 1u;
    // 3. rows out of TMEM; x0 (over i) and x1 (over j) to the t-fiber owners
    float x01[16], x2[8];  // x0 in columns 0-7, x1 in 8-15, x2 in 16-23
    tmem_ld16(tlane + 0, x01);
    tmem_ld8(tlane + 16, x2);
    tmem_wait_ld();
    const float *x0 = x01, *x1 = x01 + 8;
    float *ex0 = (float *)(sm + L::kOffX0), *ex1 = (float *)(sm + L::kOffX1);  // [e][k][j][i]
    const int xrow = le * kXe + kXk * lb + 8 * la;   // as r-row (j, k) = (la, lb): x0[i] at (i, j, k)
    const int xcol = le * kXe + kXk * lb + la;       // as s-row (i, k) = (la, lb): x1[j] at (i, j, k)
    const int xown = le * kXe + 8 * lb + la;         // as t-fiber owner (i, j) = (la, lb): + kXk k
    // the two 16-byte halves of a row in an order that differs between lanes
    // la and la + 4 (they share banks otherwise)
    auto put_row = [&](float *b, const float v[8]) {
      const int h = (la >> 2) & 1;
      float4 *p = (float4 *)(b + xrow);
      p[h] = h ? make_float4(v[4], v[5], v[6], v[7]) : make_float4(v[0], v[1], v[2], v[3]);
      p[h ^ 1] = h ? make_float4(v[0], v[1], v[2], v[3]) : make_float4(v[4], v[5], v[6], v[7]);
    };
    put_row(ex0, x0);
#pragma unroll
    for (int q = 0; q < 8; ++q) ex1[xcol + 8 * q] = x1[q];
    __syncthreads();
    // 4. geometry along the t-fiber of (i, j) = (la, lb), element le
    uint32_t tt[8];  // the t values, coded in the operand format
    {
      const bool live = le < nel;
      const int64_t e = e0 + le;
      fiber::Geometry<P, kN1, KIND> gm;
      gm.template prologue<false>(sgeo + le * (GW > 0 ? GW : 1), cx, cw, la, lb,
                                  (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * kN3 : nullptr,
                                  (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * kN3 : nullptr, nullptr);
#pragma unroll
      for (int k = 0; k < kN1; ++k) {
        const int o = xown + kXk * k;
        const float xv[3] = {ex0[o], ex1[o], x2[k]};
        float o3[3] = {0.f, 0.f, 0.f};
        if (live) gm.apply(la + lb * kN1 + k * kN1 * kN1, cx[k], cw[k], xv, o3);
        // 5. r, s into their operand buffers at once (the forward MMAs are
        // done and the exchange buffers are apart), t after the loop
        st_op<OP>(bufR, cm_off<ESZ>(lb + 8 * k + 64 * le, la, F::kLboR, F::kSboR), o3[0]);
        st_op<OP>(bufS, cm_off<ESZ>(la + 8 * k + 64 * le, lb, F::kLboS, F::kSboS), o3[1]);
        tt[k] = code<OP>(o3[2]);
      }
    }
    st_code4<OP>(bufT, cm_off<ESZ>(tid, 0, F::kLboT, F::kSboT), tt);
    st_code4<OP>(bufT, cm_off<ESZ>(tid, 4, F::kLboT, F::kSboT), tt + 4);
    proxy_fence();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      mma<OP>(tmem, desc(aR, F::kLboR, F::kSboR), desc(aBDT + F::kSboB, F::kLboB, F::kSboB), 0u);
      mma<OP>(tmem, desc(aS, F::kLboS, F::kSboS), desc(aBDT, F::kLboB, F::kSboB), 1u);
      mma<OP>(tmem + 16, desc(aT, F::kLboT, F::kSboT), desc(aBDT + F::kSboB, F::kLboB, F::kSboB), 0u);
      commit(smem_u32(bar));
    }
    if (tid == 0 && !mbar_wait(smem_u32(bar), phase)) abort_cta = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_cta) {
      if (tid == 0) mbar_wait(smem_u32(bar), phase);
      break;
    }
    phase ^= 1u;
    // 6. Y = Y_r + Y_s + Y_t
    float yrs[16], yt[8];  // Y_r in columns 0-7, Y_s in 8-15, Y_t in 16-23
    tmem_ld16(tlane + 0, yrs);
    tmem_ld8(tlane + 16, yt);
    tmem_wait_ld();
    const float *yr = yrs, *ys = yrs + 8;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    put_row(ex0, yr);
#pragma unroll
    for (int q = 0; q < 8; ++q) ex1[xcol + 8 * q] = ys[q];
    __syncthreads();
    if (le < nel) {
      float *ye = Y + (e0 + le) * kN3 + la + 8 * lb;
#pragma unroll
      for (int k = 0; k < kN1; ++k) {
        const int o = xown + kXk * k;
        ye[64 * k] = ex0[o] + ex1[o] + yt[k];
      }
    }
    // no barrier here: the next tile writes the operand buffers (free since
    // the MMA wait) and its exchange only after two more barriers
  }
  if (tid == 0 && abort_cta && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// Orders N = 1..15 but 7 (N1 = 2..16): the same six-MMA structure with the
// tile sized to the order.  A tile is EPB = 128 / N1^2 elements (N1 = 4, 6,
// 10: 8, 3, 1; one above N1 = 11), whose ROWS = EPB N1^2 fibers of a
// direction (128, 108, 100; 144 to 256 above N1 = 11) are the MMA rows in
// use, in one or two 128-row MMA blocks with one thread per row (two
// blocks: 256 threads, the second block's accumulators CPB columns to the
// right in the same TMEM lanes); unused rows stay zero and their results
// are not read.
// The contraction index K is padded with zeros to whole MMA instructions
// (TF32: K = 8 per instruction, the 16-bit formats K = 16): the operand
// buffers are zeroed once per CTA and only their data positions are written
// afterwards, so every pad holds zero.  N1 <= 8: the r and s products share
// one 16-column accumulator (the D windows of the order-7 kernel) and t has
// the next (32 columns); N1 > 8: D fills rows 0..N1-1 of a 16-row B buffer
// and each direction has its own 16-column accumulator (64 columns).  Operand
// buffers are dense core-matrix layouts (K core columns 128 bytes apart)
// with 16 bytes of padding per 8-row group; X is read with scalar coalesced
// loads.  Thread L is row L of every direction: r-fiber (j, k, e), s-fiber
// (i, k, e) and t-fiber (i, j, e) with (a, b, e) = (L % N1, L / N1 % N1,
// L / N1^2); x0 and x1 reach the t-fiber owners through the exchange
// buffers [e][k][j][i] (k pitch XK), as in the order-7 kernel.
// ---------------------------------------------------------------------------
// Shared-memory layouts of the order-sized kernel, per order and operand
// width (TF32 / 16-bit), from a search over a bank-conflict model of the
// kernel's shared-memory accesses (every access pattern of a tile, counted
// in wavefronts as the hardware serves 4-, 8- and 16-byte accesses): the
// exchange buffers' j and k pitches (floats) and each operand buffer's LBO
// and SBO (bytes).  Measured by the model at N1 = 16, 16-bit: 2432 wavefronts
// per tile against 7168 for dense layouts with scalar staging.
struct GenLayout {
  int n1, op, pj, xk, lbo_r, sbo_r, lbo_s, sbo_s, lbo_t, sbo_t;
};
constexpr GenLayout kGenLayouts[] = {
    {2, 0, 2, 6, 128, 272, 128, 272, 128, 256},
    {2, 1, 2, 6, 128, 272, 128, 272, 128, 256},
    {3, 0, 3, 35, 128, 272, 128, 272, 128, 256},
    {3, 1, 3, 35, 128, 272, 128, 272, 128, 256},
    {4, 0, 8, 35, 128, 288, 128, 288, 128, 256},
    {4, 1, 8, 35, 128, 288, 128, 288, 128, 256},
    {5, 0, 5, 25, 2112, 128, 2288, 144, 128, 256},
    {5, 1, 5, 25, 128, 320, 128, 256, 128, 256},
    {6, 0, 7, 42, 2112, 128, 128, 256, 128, 256},
    {6, 1, 7, 42, 128, 272, 128, 256, 128, 256},
    {7, 0, 7, 49, 128, 256, 128, 256, 128, 256},
    {7, 1, 7, 49, 128, 256, 128, 256, 128, 256},
    {9, 0, 9, 81, 2096, 128, 128, 512, 128, 512},
    {9, 1, 9, 81, 2128, 128, 128, 256, 128, 256},
    {10, 0, 10, 101, 2080, 128, 128, 512, 128, 512},
    {10, 1, 10, 101, 2112, 128, 128, 256, 128, 256},
    {11, 0, 11, 121, 2096, 128, 128, 512, 128, 512},
    {11, 1, 11, 121, 2112, 128, 128, 256, 128, 256},
    {12, 0, 17, 204, 4144, 128, 128, 512, 128, 512},
    {12, 1, 17, 204, 4160, 128, 128, 256, 128, 256},
    {13, 0, 13, 169, 4128, 128, 128, 512, 128, 512},
    {13, 1, 13, 169, 4160, 128, 128, 256, 128, 256},
    {14, 0, 14, 199, 4128, 128, 128, 512, 128, 512},
    {14, 1, 14, 199, 4144, 128, 128, 256, 128, 256},
    {15, 0, 15, 225, 4128, 128, 128, 512, 128, 512},
    {15, 1, 15, 225, 4144, 128, 128, 256, 128, 256},
    {16, 0, 17, 272, 4128, 128, 128, 512, 128, 512},
    {16, 1, 17, 272, 4128, 128, 128, 256, 128, 256},
};
constexpr GenLayout gen_layout(int n1, int op) {
  for (const GenLayout &g : kGenLayouts)
    if (g.n1 == n1 && g.op == (op == 0 ? 0 : 1)) return g;
  return GenLayout{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
}

template <int N1, int OP>
struct GShape {
  static constexpr int F = N1 * N1, EPB = F > 128 ? 1 : 128 / F, ROWS = EPB * F, N3 = N1 * N1 * N1, TN = EPB * N3;
  static constexpr int MB = (ROWS + 127) / 128;                // 128-row MMA blocks (two above N1 = 11)
  static constexpr int THREADS = 128 * MB;                      // one thread per row
  static constexpr int ESZ = OP == 0 ? 4 : 2, PER = 16 / ESZ;   // bytes per value, K values per core row
  static constexpr int KI = OP == 0 ? 8 : 16;                   // K per MMA instruction
  static constexpr int NI = (N1 + KI - 1) / KI;                 // instructions per contraction
  static constexpr int NC = NI * KI / PER;                      // K core columns of every operand buffer
  static constexpr int NCD = (N1 + PER - 1) / PER;              // core columns holding data
  static constexpr GenLayout LY = gen_layout(N1, OP);
  static_assert(LY.n1 == N1, "no layout for this order");
  static constexpr uint32_t LBO_R = LY.lbo_r, SBO_R = LY.sbo_r, LBO_S = LY.lbo_s, SBO_S = LY.sbo_s,
                            LBO_T = LY.lbo_t, SBO_T = LY.sbo_t;
  // bytes of an operand buffer: its last core matrix ends there
  static constexpr uint32_t span(uint32_t lbo, uint32_t sbo) { return (16 * MB - 1) * sbo + (NC - 1) * lbo + 128; }
  static constexpr uint32_t BYTES_R = span(LBO_R, SBO_R), BYTES_S = span(LBO_S, SBO_S),
                            BYTES_T = span(LBO_T, SBO_T);
  static constexpr bool SPLIT = N1 > 8;                          // one accumulator per direction
  static constexpr int BROWS = SPLIT ? 16 : 24, BROW0 = SPLIT ? 0 : 8;  // B buffer rows, first row of D
  static constexpr uint32_t LBOB = 128, SBOB = NC * 128, BBYTES = (BROWS / 8) * SBOB;
  // tensor-memory columns: per M-block CPB (32, or 64 with an accumulator per direction)
  static constexpr int CPB = SPLIT ? 64 : 32, TCOLS = CPB * MB;
  // exchange buffers [e][k][j][i]: i pitch 1, j pitch PJ, k pitch XK floats
  static constexpr int PJ = LY.pj, XK = LY.xk, XE = N1 * XK, XF = EPB * XE;
  static constexpr uint32_t OFF_R = 0, OFF_S = BYTES_R, OFF_T = OFF_S + BYTES_S, OFF_X0 = OFF_T + BYTES_T,
                            OFF_X1 = OFF_X0 + (uint32_t)(XF * 4 + 15) / 16 * 16,
                            OFF_BD = OFF_X1 + (uint32_t)(XF * 4 + 15) / 16 * 16, OFF_BDT = OFF_BD + BBYTES,
                            OFF_GEO = OFF_BDT + BBYTES, BYTES = OFF_GEO + EPB * kVertexWords * 4 + 64;
  static_assert(EPB >= 1 && N1 <= 16 - BROW0 && N1 <= 16, "tile shape");
  static_assert((N1 - 1) * PJ + N1 <= XK, "exchange rows fit the k pitch");
  static_assert(BYTES_R % 16 == 0 && BYTES_S % 16 == 0 && BYTES_T % 16 == 0 && BBYTES % 16 == 0,
                "16-byte aligned operand buffers");
};
// resident CTAs per SM: as the order-7 kernel up to N1 = 8; at N1 = 9..11
// five of 128 threads (up to 102 registers); above, three of 256 threads
// (85 registers) where their shared memory fits, else two (and two for the
// stored kind, which spills at 85 registers)
template <int N1, int KIND, int OP>
constexpr int kCtasGen =
    N1 * N1 > 128 ? ((KIND == AX_GEOM_STORED || 3 * (GShape<N1, OP>::BYTES + 1024) > 228 * 1024) ? 2 : 3)
                  : (N1 > 8 ? 5 : kCtasPerSm<KIND>);

template <int N1, int KIND, int OP>
__global__ void __launch_bounds__(GShape<N1, OP>::THREADS, kCtasGen<N1, KIND, OP>)
    ax_umma_gen_kernel(int64_t E, const float *__restrict__ geo, const float *__restrict__ lam,
                       const float *__restrict__ X, float *__restrict__ Y, const float *__restrict__ Dp,
                       int *__restrict__ err) {
  using P = fiber::Native<float>;
  using G = GShape<N1, OP>;
  constexpr int ESZ = G::ESZ, F = G::F, EPB = G::EPB, N3 = G::N3, NT = G::THREADS;
  constexpr int GW = fiber::GeoWords<KIND>::value;
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char *bufR = sm + G::OFF_R, *bufS = sm + G::OFF_S, *bufT = sm + G::OFF_T;
  float *ex0 = (float *)(sm + G::OFF_X0), *ex1 = (float *)(sm + G::OFF_X1);
  float *sgeo = (float *)(sm + G::OFF_GEO);
  uint64_t *bar = (uint64_t *)(sm + G::OFF_GEO + EPB * kVertexWords * 4);
  uint32_t *tslot = (uint32_t *)(bar + 1);
  __shared__ int abort_cta;
  const int tid = threadIdx.x, warp = tid >> 5;
  const float *cw = fiber::c_w + tab_off_v(N1);
  const float *cx = fiber::c_x + tab_off_v(N1);

  // the three operand buffers zeroed (pads stay zero), then D and D^T in
  // their B buffers (rows a, K = m and rows m, K = a), zero elsewhere
  for (uint32_t q = tid; q < (G::BYTES_R + G::BYTES_S + G::BYTES_T) / 16; q += NT)
    ((uint4 *)sm)[q] = make_uint4(0u, 0u, 0u, 0u);
  constexpr int KB = G::NC * G::PER;  // K positions per B row
  for (int q = tid; q < 2 * G::BROWS * KB; q += NT) {
    const int which = q / (G::BROWS * KB), row = (q % (G::BROWS * KB)) / KB, k = q % KB, a = row - G::BROW0;
    float v = 0.0f;
    if (a >= 0 && a < N1 && k < N1) v = which == 0 ? Dp[a * N1 + k] : Dp[k * N1 + a];
    st_op<OP>(sm + (which == 0 ? G::OFF_BD : G::OFF_BDT), cm_off<ESZ>(row, k, G::LBOB, G::SBOB), v);
  }
  if (tid == 0) {
    abort_cta = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(G::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  // TMEM lane 32 (warp % 4) + lane of the thread's M-block (tid / 128), whose columns start at CPB (tid / 128)
  const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(G::CPB * (tid >> 7));
  const uint32_t aR = smem_u32(bufR), aS = smem_u32(bufS), aT = smem_u32(bufT);
  const uint32_t aBD = smem_u32(sm + G::OFF_BD), aBDT = smem_u32(sm + G::OFF_BDT);
  const int la = tid % N1, lb = (tid / N1) % N1, le = tid / F;
  const bool row_in_use = tid < G::ROWS;
  uint32_t phase = 0;
  constexpr int kStepC = G::KI / G::PER;  // K core columns per instruction

  // the six (forward or transposed) contractions of a tile, issued by one thread
  auto issue = [&](uint32_t aB) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int mb = 0; mb < G::MB; ++mb) {
      const uint32_t ta = tmem + (uint32_t)(G::CPB * mb), m16 = (uint32_t)(mb * 16);  // 128 rows down
      const uint64_t dR = desc(aR + m16 * G::SBO_R, G::LBO_R, G::SBO_R), dS = desc(aS + m16 * G::SBO_S, G::LBO_S, G::SBO_S),
                     dT = desc(aT + m16 * G::SBO_T, G::LBO_T, G::SBO_T);
      if constexpr (!G::SPLIT) {
        mma<OP>(ta, dR, desc(aB + G::SBOB, G::LBOB, G::SBOB), 0u);
        mma<OP>(ta, dS, desc(aB, G::LBOB, G::SBOB), 1u);
        mma<OP>(ta + 16, dT, desc(aB + G::SBOB, G::LBOB, G::SBOB), 0u);
      } else {
        const uint32_t aA[3] = {aR + m16 * G::SBO_R, aS + m16 * G::SBO_S, aT + m16 * G::SBO_T};
        const uint32_t lA[3] = {G::LBO_R, G::LBO_S, G::LBO_T}, sA[3] = {G::SBO_R, G::SBO_S, G::SBO_T};
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int q = 0; q < G::NI; ++q)
            mma<OP>(ta + 16 * d, desc(aA[d] + q * kStepC * lA[d], lA[d], sA[d]),
                    desc(aB + q * kStepC * G::LBOB, G::LBOB, G::SBOB), q > 0 ? 1u : 0u);
      }
    }
    commit(smem_u32(bar));
  };
  // this thread's TMEM row: the r-, s- and t-direction results (N1 values each)
  auto read_rows = [&](float v0[N1], float v1[N1], float v2[N1]) {
    if constexpr (!G::SPLIT) {
      float a16[16], a8[8];
      tmem_ld16(tlane + 0, a16);
      tmem_ld8(tlane + 16, a8);
      tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        v0[q] = a16[q];
        v1[q] = a16[8 + q];
        v2[q] = a8[q];
      }
    } else {
      float a[16], b[16], c[16];
      tmem_ld16(tlane + 0, a);
      tmem_ld16(tlane + 16, b);
      tmem_ld16(tlane + 32, c);
      tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        v0[q] = a[q];
        v1[q] = b[q];
        v2[q] = c[q];
      }
    }
  };
  // r-row values (over i) and s-row values (over j) to the t-fiber owners
  const int xrow = le * G::XE + G::XK * lb + G::PJ * la;  // r-row (j, k) = (la, lb): value i at + i
  const int xcol = le * G::XE + G::XK * lb + la;          // s-row (i, k) = (la, lb): value j at + PJ j
  const int xown = le * G::XE + G::PJ * lb + la;          // t-fiber owner (i, j) = (la, lb): node k at + XK k
  auto exchange = [&](const float v0[N1], const float v1[N1]) {
    if (row_in_use) {
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        ex0[xrow + q] = v0[q];
        ex1[xcol + G::PJ * q] = v1[q];
      }
    }
  };

  const int64_t ntile = (E + EPB - 1) / EPB;
  // X of a tile, staged by the t-fiber owners: thread (i, j, e) = (la, lb, le)
  // reads its N1 values X[e][k][j][i] (for each k the warp reads consecutive
  // i, j: coalesced), one tile ahead so that the loads overlap the previous
  // tile's work; zeros beyond the last element
  auto load_x = [&](int64_t tt, float xv[N1]) {
    const int64_t eg = tt * EPB + le;
    const bool ok = row_in_use && tt < ntile && eg < E;
    const float *src = X + eg * N3 + la + N1 * lb;
#pragma unroll
    for (int k = 0; k < N1; ++k) xv[k] = ok ? src[F * k] : 0.0f;
  };
  // the thread's own T row (t-fiber, K = k) in 16-byte stores, the pad of the
  // last core column zero
  auto st_trow = [&](const uint32_t c[N1]) {
#pragma unroll
    for (int cc = 0; cc < G::NCD; ++cc) {
      uint32_t w[G::PER];
#pragma unroll
      for (int p = 0; p < G::PER; ++p) w[p] = cc * G::PER + p < N1 ? c[cc * G::PER + p] : 0u;
      uint4 v;
      if constexpr (OP == 0)
        v = make_uint4(w[0], w[1], w[2], w[3]);
      else
        v = make_uint4(w[0] | (w[1] << 16), w[2] | (w[3] << 16), w[4] | (w[5] << 16), w[6] | (w[7] << 16));
      *(uint4 *)(bufT + cm_off<ESZ>(tid, cc * G::PER, G::LBO_T, G::SBO_T)) = v;
    }
  };
  float xnext[N1];
  load_x(blockIdx.x, xnext);
  for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
    const int64_t e0 = t * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    // 1. X into the three operand buffers: r-row (j, k) and s-row (i, k) at
    // K = i and j value by value, the own t-row whole
    if (row_in_use) {
      uint32_t c[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        c[k] = code<OP>(xnext[k]);
        st_code<OP>(bufR, cm_off<ESZ>(lb + N1 * k + F * le, la, G::LBO_R, G::SBO_R), c[k]);
        st_code<OP>(bufS, cm_off<ESZ>(la + N1 * k + F * le, lb, G::LBO_S, G::SBO_S), c[k]);
      }
      st_trow(c);
    }
    if constexpr (GW > 0) {
      for (int m = tid; m < nel * GW; m += NT) sgeo[m] = geo[e0 * GW + m];
    }
    load_x(t + gridDim.x, xnext);  // the next tile's X, in flight meanwhile
    proxy_fence();
    __syncthreads();
    // 2. forward MMAs; thread 0 waits for them (bounded), the others sleep in the barrier
    if (tid == 0 && !abort_cta) issue(aBD);
    if (tid == 0 && !mbar_wait(smem_u32(bar), phase)) abort_cta = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_cta) {
      if (tid == 0) mbar_wait(smem_u32(bar), phase);  // bounded: the MMAs in flight before TMEM is freed
      break;
    }
    phase ^= 1u;
    // 3. rows out of TMEM; x0 and x1 to the t-fiber owners
    float x0[N1], x1[N1], x2[N1];
    read_rows(x0, x1, x2);
    exchange(x0, x1);
    __syncthreads();
    // 4. geometry along the t-fiber of (i, j) = (la, lb), element le; 5. r, s, t into the operand buffers
    if (row_in_use) {
      uint32_t tt[N1];  // the t values, coded in the operand format
      const bool live = le < nel;
      const int64_t e = e0 + le;
      fiber::Geometry<P, N1, KIND> gm;
      gm.template prologue<false>(sgeo + le * (GW > 0 ? GW : 1), cx, cw, la, lb,
                                  (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * N3 : nullptr,
                                  (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * N3 : nullptr, nullptr);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int o = xown + G::XK * k;
        const float xv[3] = {ex0[o], ex1[o], x2[k]};
        float o3[3] = {0.f, 0.f, 0.f};
        if (live) gm.apply(la + lb * N1 + k * F, cx[k], cw[k], xv, o3);
        st_op<OP>(bufR, cm_off<ESZ>(lb + N1 * k + F * le, la, G::LBO_R, G::SBO_R), o3[0]);
        st_op<OP>(bufS, cm_off<ESZ>(la + N1 * k + F * le, lb, G::LBO_S, G::SBO_S), o3[1]);
        tt[k] = code<OP>(o3[2]);
      }
      st_trow(tt);
    }
    proxy_fence();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) issue(aBDT);
    if (tid == 0 && !mbar_wait(smem_u32(bar), phase)) abort_cta = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_cta) {
      if (tid == 0) mbar_wait(smem_u32(bar), phase);
      break;
    }
    phase ^= 1u;
    // 6. Y = Y_r + Y_s + Y_t
    float yr[N1], ys[N1], yt[N1];
    read_rows(yr, ys, yt);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    exchange(yr, ys);
    __syncthreads();
    if (row_in_use && le < nel) {
      float *ye = Y + (e0 + le) * N3 + la + N1 * lb;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int o = xown + G::XK * k;
        ye[F * k] = ex0[o] + ex1[o] + yt[k];
      }
    }
    // no barrier here: the next tile writes the operand buffers (free since
    // the MMA wait) and its exchange only after two more barriers
  }
  if (tid == 0 && abort_cta && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G::TCOLS) : "memory");
}

// Launch over a.E elements of order N1 - 1: kCtasGen CTAs per SM,
// persistent over the tiles.
template <int N1, int KIND, int OP>
cudaError_t launch_gen(const AxArgs &a, const float *Dp) {
  using G = GShape<N1, OP>;
  const int64_t ntile = (a.E + G::EPB - 1) / G::EPB;
  if (ntile <= 0) return cudaSuccess;
  static int grid_cap = 0;
  if (!grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(ax_umma_gen_kernel<N1, KIND, OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::BYTES);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid_cap = kCtasGen<N1, KIND, OP> * sms;
  }
  const int64_t cap = a.grid > 0 && a.grid < grid_cap ? a.grid : grid_cap;
  const int64_t grid = ntile < cap ? ntile : cap;
  ax_umma_gen_kernel<N1, KIND, OP><<<(unsigned)grid, G::THREADS, G::BYTES, a.stream>>>(
      a.E, (const float *)a.geo, (const float *)a.lam, (const float *)a.X, (float *)a.Y, Dp, a.err);
  return cudaGetLastError();
}

// Launch over a.E elements of order 7: kCtasPerSm CTAs per SM, persistent
// over the tiles of two elements.
template <int KIND, int OP>
cudaError_t launch_kind(const AxArgs &a, const float *Dp) {
  const int64_t ntile = (a.E + kEPB - 1) / kEPB;
  if (ntile <= 0) return cudaSuccess;
  static int grid_cap = 0;
  if (!grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(ax_umma_kernel<KIND, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Smem<OP>::kBytes);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid_cap = kCtasPerSm<KIND> * sms;
  }
  const int64_t cap = a.grid > 0 && a.grid < grid_cap ? a.grid : grid_cap;
  const int64_t grid = ntile < cap ? ntile : cap;
  ax_umma_kernel<KIND, OP><<<(unsigned)grid, kThreads, Smem<OP>::kBytes, a.stream>>>(
      a.E, (const float *)a.geo, (const float *)a.lam, (const float *)a.X, (float *)a.Y, Dp, a.err);
  return cudaGetLastError();
}

}  // namespace umma
}  // namespace ax
