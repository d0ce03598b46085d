// BF16 tensor-core GEMM with FP32 accumulation for the learned
// preconditioner's MLP:  C[m][n] = sum_k A[m][k] B[n][k]  (both operands
// K-contiguous, "TN"), with fused epilogues (bias, GELU, GELU derivative).
//
// CTA tile 128 x 128 x 32, 8 warps (2 along M x 4 along N), each warp 64 x 32
// as 4 x 4 mma.sync.m16n8k16 tiles.  Global -> shared by cp.async (16 B,
// zero-fill outside M/N), double-buffered; shared -> registers by ldmatrix.
// Shared rows are padded to 40 bf16 (80 B) so the 8 row addresses of every
// ldmatrix phase fall in distinct bank groups.
// Requirements: K % 32 == 0, lda, ldb % 8 == 0, 16-byte aligned A and B.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ax {
namespace mlp {

constexpr int kBM = 128, kBN = 128, kBK = 32, kLDS = kBK + 8;
constexpr int kGemmThreads = 256;

enum Epi {
  kEpiF32 = 0,    // Cf[m][n] = acc (+ bias[n])
  kEpiGelu = 1,   // z = acc + bias[n]; Zf[m][n] = z; Hb[m][n] = bf16(gelu(z))
  kEpiDGelu = 2,  // Hb[m][n] = bf16(acc * gelu'(Zf[m][n]))
  kEpiBf16 = 3    // Hb[m][n] = bf16(acc (+ bias[n]))
};

struct GemmOut {
  float *Cf = nullptr;          // kEpiF32 output / kEpiGelu pre-activation
  __nv_bfloat16 *Hb = nullptr;  // bf16 output
  const float *Zin = nullptr;   // kEpiDGelu: pre-activation of the same shape
  const float *bias = nullptr;
  int ldc = 0;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all_but1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda, const __nv_bfloat16 *__restrict__ B,
                 int ldb, GemmOut out) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][kBM][kLDS];
  __shared__ __align__(16) __nv_bfloat16 sB[2][kBN][kLDS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // warp tile origin: (wm*64, wn*32)
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;

  // each thread copies 2 chunks of A and 2 of B per K-tile: chunk c -> row c/4, col (c%4)*8
  auto load_tile = [&](int stage, int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + h * kGemmThreads;
      const int row = c >> 2, col = (c & 3) * 8;
      const int gm = m0 + row, gn = n0 + row;
      const bool pa = gm < M, pb = gn < N;
      cp_async16(&sA[stage][row][col], A + (size_t)(pa ? gm : 0) * lda + k0 + col, pa);
      cp_async16(&sB[stage][row][col], B + (size_t)(pb ? gn : 0) * ldb + k0 + col, pb);
    }
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

  const int nk = K / kBK;
  load_tile(0, 0);
  cp_async_commit();
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    if (kt + 1 < nk) {
      load_tile(st ^ 1, (kt + 1) * kBK);
      cp_async_commit();
      cp_async_wait_all_but1();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      unsigned a[4][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = wm * 64 + i * 16 + (lane & 15);
        const int c = kk + (lane >> 4) * 8;
        ldmatrix_x4(a[i][0], a[i][1], a[i][2], a[i][3], &sA[st][r][c]);
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        // matrices: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
        const int r = wn * 32 + j * 8 + (lane & 7) + ((lane >> 4) << 3);
        const int c = kk + ((lane >> 3) & 1) * 8;
        ldmatrix_x4(b[j][0], b[j][1], b[j + 1][0], b[j + 1][1], &sB[st][r][c]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
    }
    __syncthreads();
  }

  // epilogue: acc[i][j] holds rows g, g+8 and columns 2t, 2t+1 of its 16x8 tile
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 64 + i * 16 + g + h * 8;
        const int n = n0 + wn * 32 + j * 8 + 2 * t;
        if (m >= M) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int nn = n + q;
          if (nn >= N) continue;
          float v = acc[i][j][2 * h + q];
          const size_t o = (size_t)m * out.ldc + nn;
          if constexpr (EPI == kEpiF32) {
            if (out.bias) v += out.bias[nn];
            out.Cf[o] = v;
          } else if constexpr (EPI == kEpiGelu) {
            v += out.bias[nn];
            out.Cf[o] = v;
            out.Hb[o] = __float2bfloat16_rn(gelu_f(v));
          } else if constexpr (EPI == kEpiDGelu) {
            out.Hb[o] = __float2bfloat16_rn(v * gelu_grad_f(out.Zin[o]));
          } else {
            if (out.bias) v += out.bias[nn];
            out.Hb[o] = __float2bfloat16_rn(v);
          }
        }
      }
}

template <int EPI>
inline cudaError_t gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                        const GemmOut &out, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K % kBK || lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return cudaErrorInvalidValue;
  const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  gemm_bf16_tn<EPI><<<grid, kGemmThreads, 0, s>>>(M, N, K, A, lda, B, ldb, out);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ax
