// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the learned
// preconditioner's MLP:  C[m][n] = sum_k A[m][k] B[n][k]  (both operands
// K-contiguous, "TN"), FP32 accumulation in tensor memory, fused epilogues.
//
// Persistent and warp-specialised: one CTA per SM walks the 128 x 256 tiles
// of C (tile t, t + gridDim.x, ...; the two N-tiles of a row block are
// neighbours, so A is read from HBM once):
//   * warp 0, lane 0 streams 128 x 64 tiles of A and 256 x 64 tiles of B into
//     a 4-stage shared-memory ring with TMA (128-byte swizzle, zero fill
//     outside the tensor: ragged M and K need no special case);
//   * warp 1, lane 0 issues tcgen05.mma (M = 128, N = 256, K = 16) from the
//     two shared-memory descriptors into one of two 256-column TMEM
//     accumulators, releases each stage with tcgen05.commit and signals the
//     finished accumulator;
//   * warps 2..9 drain the other accumulator meanwhile: warp w reads TMEM
//     lanes 32 (w % 4).. (rows of the tile) and half of the columns
//     (tcgen05.ld), stages each 32 x 32 block in shared memory, and writes
//     coalesced rows of C with the fused epilogue; then it frees the buffer.
// Every mbarrier wait is bounded; a wait that runs out records an error code
// in *err, the CTA stops issuing work, drains what it issued (bounded) and
// frees its TMEM before returning.
// Requirements: K % 8 == 0, lda == ldb == K (row pitch 16-byte multiple),
// 16-byte aligned A and B, N % 32 == 0, ldc % 4 == 0, 16-byte aligned outputs.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ax {
namespace mlp {

enum Epi {
  kEpiF32 = 0,    // Cf[m][n] = acc (+ bias[n])
  kEpiGelu = 1,   // z = acc + bias[n]; Zf[m][n] = z (when Cf is set); Hb[m][n] = bf16(gelu(z))
  kEpiDGelu = 2,  // Hb[m][n] = bf16(acc * gelu'(Zf[m][n]))
  kEpiBf16 = 3    // Hb[m][n] = bf16(acc (+ bias[n]))
};

struct GemmOut {
  float *Cf = nullptr;           // kEpiF32 output / kEpiGelu pre-activation
  __nv_bfloat16 *Hb = nullptr;   // bf16 output
  const float *Zin = nullptr;    // kEpiDGelu: pre-activation of the same shape
  const float *bias = nullptr;
  const double *skip = nullptr;  // when set and nonzero at launch, the GEMM does nothing
  int ldc = 0;
};

// gelu(z) = z Phi(z) with the normal CDF written through erf
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

}  // namespace mlp

namespace tc {

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 4;
constexpr int kEpiWarps = 8, kThreads = 32 * (2 + kEpiWarps);
constexpr int kABytes = kBM * kBK * 2, kBBytes = kBN * kBK * 2, kStageBytes = kABytes + kBBytes;
constexpr int kTmemCols = 2 * kBN;  // two accumulators
// epilogue staging: a 32 x 32 float block per warp, rows of 128 bytes whose
// 16-byte chunks are XOR-swizzled by (row % 8): conflict-free row writes and
// row-segment reads
constexpr int kStageTile = 32 * 32 * 4;
constexpr int kNumBars = 2 * kStages + 4;  // full[s], empty[s], tmem_full[2], tmem_empty[2]
// ring, epilogue staging, mbarriers, TMEM address slot; 1 KB for alignment
constexpr int kSmemBytes = kStages * kStageBytes + kEpiWarps * kStageTile + 8 * kNumBars + 16 + 1024;
constexpr long long kWaitCycles = 1ll << 32;  // SM clocks (about 2 s) before a wait gives up

enum TcError { kErrFull = 1, kErrEmpty = 2, kErrAccum = 3, kErrAccumFree = 4 };

// Instruction descriptor of tcgen05.mma kind::f16: D float32, A and B bf16,
// both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1, base offset 0 (tiles are
// 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after kWaitCycles
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

// 32 consecutive float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void record_error(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

template <int EPI>
__device__ __forceinline__ float4 epi_op(float4 x, float4 z) {
  auto f = [](float a, float zz) {
    if constexpr (EPI == mlp::kEpiGelu) return mlp::gelu_f(a);
    else if constexpr (EPI == mlp::kEpiDGelu) return a * mlp::gelu_grad_f(zz);
    else return a;
  };
  return make_float4(f(x.x, z.x), f(x.y, z.y), f(x.z, z.z), f(x.w, z.w));
}
__device__ __forceinline__ void store_bf16x4(__nv_bfloat16 *p, float4 v) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t *>(&lo);
  u.y = *reinterpret_cast<uint32_t *>(&hi);
  *reinterpret_cast<uint2 *>(p) = u;
}

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
                   int K, mlp::GemmOut out, int *err) {
  if (out.skip && *out.skip != 0.0) return;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned ring (128-byte swizzle atoms)
  uint8_t *gbase = smem_raw + (base - raw);
  const uint32_t sA = base, sB = base + kStages * kABytes;
  float *stage_tiles = reinterpret_cast<float *>(gbase + kStages * kStageBytes);
  const uint32_t bars = base + kStages * kStageBytes + kEpiWarps * kStageTile;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + kStages * kStageBytes + kEpiWarps * kStageTile +
                                                     8 * kNumBars);
  __shared__ int abort_flag;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (kStages + s); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * kStages + b); };
  auto acc_free = [&](int b) { return bars + 8u * (2 * kStages + 2 + b); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = (K + kBK - 1) / kBK;
  const int ntn = (N + kBN - 1) / kBN, ntiles = ((M + kBM - 1) / kBM) * ntn;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_free(b), kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: one k-block of A and B per stage, across all tiles of this CTA
      asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&ta) : "memory");
      asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&tb) : "memory");
      int g = 0;  // k-blocks issued
      for (int t = blockIdx.x; t < ntiles && !*(volatile int *)&abort_flag; t += gridDim.x) {
        const int m0 = (t / ntn) * kBM, n0 = (t % ntn) * kBN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % kStages, round = g / kStages;
          if (round > 0 && !mbar_wait(empty(s), (uint32_t)((round - 1) & 1))) {
            record_error(err, kErrEmpty);
            atomicExch(&abort_flag, 1);
            break;
          }
          mbar_expect_tx(full(s), (uint32_t)kStageBytes);
          tma_load_2d(sA + s * kABytes, &ta, kb * kBK, m0, full(s));
          tma_load_2d(sB + s * kBBytes, &tb, kb * kBK, n0, full(s));
        }
      }
      // drain: the copies of the last stages issued have landed before teardown
      for (int q = (g > kStages ? g - kStages : 0); q < g; ++q)
        if (!mbar_wait(full(q % kStages), (uint32_t)((q / kStages) & 1))) record_error(err, kErrFull);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int g = 0, i = 0;  // k-blocks consumed, tiles accumulated
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int b = i & 1, use = i >> 1;
        if (use > 0 && !mbar_wait(acc_free(b), (uint32_t)((use - 1) & 1))) {
          record_error(err, kErrAccumFree);
          atomicExch(&abort_flag, 1);
        }
        if (*(volatile int *)&abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * kBN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % kStages;
          if (!mbar_wait(full(s), (uint32_t)((g / kStages) & 1))) {
            record_error(err, kErrFull);
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint64_t ad = sw128_desc(sA + s * kABytes + kk * 32);
            const uint64_t bd = sw128_desc(sB + s * kBBytes + kk * 32);
            umma_bf16(d, ad, bd, (kb | kk) != 0 ? 1u : 0u);
          }
          umma_commit(empty(s));
        }
        umma_commit(acc_full(b));  // arrives when every MMA issued so far has completed
        if (!ok) break;
      }
    }
  } else {
    // epilogue warps: lane quarter q = warp % 4 (TMEM lanes = tile rows), column half h
    const int ew = warp - 2, q = warp & 3, h = ew >> 2;
    float *tile = stage_tiles + ew * (kStageTile / 4);
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1, use = i >> 1;
      const bool ok = mbar_wait(acc_full(b), (uint32_t)(use & 1));
      if (!ok) record_error(err, kErrAccum);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (!__all_sync(0xffffffffu, ok && !*(volatile int *)&abort_flag)) break;
      const int m0 = (t / ntn) * kBM, n0 = (t % ntn) * kBN;
      const int mw = m0 + 32 * q;  // first row of this warp's 32-row block
#pragma unroll 1
      for (int c = h * (kBN / 64); c < (h + 1) * (kBN / 64); ++c) {
        const int nc = n0 + 32 * c;
        if (nc >= N) break;  // N % 32 == 0: whole 32-column chunks
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kBN + 32 * c), v);
        float4 *trow = reinterpret_cast<float4 *>(tile + lane * 32);
#pragma unroll
        for (int j = 0; j < 8; ++j) trow[j ^ (lane & 7)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        __syncwarp();
        // lane -> (row lane / 8 + 4 r, columns 4 (lane % 8) .. +3)
        const int cn = nc + 4 * (lane & 7);
        float4 bias = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (EPI != mlp::kEpiDGelu)
          if (out.bias) bias = *reinterpret_cast<const float4 *>(out.bias + cn);
#pragma unroll 2
        for (int r = 0; r < 8; ++r) {
          const int rr = 4 * r + (lane >> 3), m = mw + rr;
          if (m < M) {
            float4 x = reinterpret_cast<const float4 *>(tile + rr * 32)[(lane & 7) ^ (rr & 7)];
            x.x += bias.x; x.y += bias.y; x.z += bias.z; x.w += bias.w;
            const size_t o = (size_t)m * out.ldc + cn;
            if constexpr (EPI == mlp::kEpiF32) {
              *reinterpret_cast<float4 *>(out.Cf + o) = x;
            } else if constexpr (EPI == mlp::kEpiGelu) {
              if (out.Cf) *reinterpret_cast<float4 *>(out.Cf + o) = x;
              store_bf16x4(out.Hb + o, epi_op<EPI>(x, x));
            } else if constexpr (EPI == mlp::kEpiDGelu) {
              store_bf16x4(out.Hb + o, epi_op<EPI>(x, *reinterpret_cast<const float4 *>(out.Zin + o)));
            } else {
              store_bf16x4(out.Hb + o, x);
            }
          }
        }
        __syncwarp();
      }
      // this warp's reads of buffer b are complete: hand it back to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acc_free(b)) : "memory");
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 2-D bf16 tensor [rows][K] (K contiguous), boxes of kBK x box_rows, 128-byte swizzle, zero fill outside
inline bool make_map(CUtensorMap *map, const void *ptr, int rows, int K, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// once per process and device, outside any stream capture
inline cudaError_t gemm_init() {
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<mlp::kEpiF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<mlp::kEpiGelu>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<mlp::kEpiDGelu>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<mlp::kEpiBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e == cudaSuccess && !encode_fn()) e = cudaErrorNotSupported;
  return e;
}

// C = A B^T with A [M][K], B [N][K] bf16 (row pitch K), epilogue EPI.
template <int EPI>
inline cudaError_t gemm(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B,
                        const mlp::GemmOut &out, int *err, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0 || K % 8 || N % 32 || out.ldc % 4 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) ||
      ((uintptr_t)out.Cf & 15) || ((uintptr_t)out.Hb & 15) || ((uintptr_t)out.Zin & 15) || ((uintptr_t)out.bias & 15))
    return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K, kBM) || !make_map(&tb, B, N, K, kBN)) return cudaErrorInvalidValue;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  const int ntiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
  const int grid = ntiles < sms ? ntiles : sms;
  gemm_tc_kernel<EPI><<<grid, kThreads, kSmemBytes, s>>>(ta, tb, M, N, K, out, err);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace ax
