// Learned per-element preconditioner: a small MLP, trained and run on the GPU
// with the BF16 tensor-core GEMM of gemm_bf16.cuh (FP32 accumulation, FP32
// master weights, Adam), and the flexible PCG that uses it.
//
// Network: in_dim -> hidden (GELU) -> hidden (GELU) -> out_dim (linear).
// The element input is its local residual scaled by s_e = max |r_e| and its
// 24 vertex coordinates relative to vertex 0 divided by h_e = |v1 - v0|; the
// output, times s_e / h_e, is a correction added to the Jacobi step, then
// gather-scatter averaged (Eq. 1's Q^T with multiplicity weights):
//   z = D^-1 r + Q^T(c) / multiplicity,   c_e = (s_e / h_e) MLP(r_e / s_e, geo_e).
// Training pairs come from solves: target_e = (h_e / s_e) (e - D^-1 r)_e with
// e = x* - x_k the error of an iterate x_k and r = b - A x_k its residual.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ax_internal.h"
#include "gemm_bf16.cuh"

namespace ax {
namespace mlp {

constexpr int kIn = 536, kInPad = 544, kHid = 512, kOut = 512;

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void f32_to_bf16(int64_t n, const float *__restrict__ a, __nv_bfloat16 *__restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// out[c][r] = in[r][c]  (R x C bf16), 32x32 tiles
__global__ void transpose_bf16(int R, int C, const __nv_bfloat16 *__restrict__ in, int ldi, __nv_bfloat16 *__restrict__ out,
                               int ldo) {
  __shared__ __nv_bfloat16 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * ldi + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (c < C && r < R) out[(size_t)c * ldo + r] = t[threadIdx.x][y];
  }
}

// dY = (Y - T) / (M * O) as bf16; partial sums of (Y - T)^2 per block
__global__ void loss_grad(int M, int O, const float *__restrict__ Y, const float *__restrict__ T,
                          __nv_bfloat16 *__restrict__ dY, float *__restrict__ part) {
  __shared__ float sh[256];
  float s = 0.0f;
  const float inv = 1.0f / ((float)M * (float)O);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)M * O; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    s += d * d;
    dY[i] = __float2bfloat16_rn(d * inv);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// db[n] = sum_m dZ[m][n] (fixed order: one thread per column, rows in order)
__global__ void colsum_bf16(int M, int N, const __nv_bfloat16 *__restrict__ dZ, float *__restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int m = 0; m < M; ++m) s += __bfloat162float(dZ[(size_t)m * N + n]);
  db[n] = s;
}

// Adam on a flat FP32 parameter vector; w, m, v updated in place
__global__ void adam(int64_t n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                     float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// rows idx[i] of X (bf16, ldx) and T (f32, ldt) -> packed Xb [n][ldx], Tb [n][ldt]
__global__ void gather_rows(int64_t n, const int64_t *__restrict__ idx, const __nv_bfloat16 *__restrict__ X, int ldx,
                            const float *__restrict__ T, int ldt, __nv_bfloat16 *__restrict__ Xb,
                            float *__restrict__ Tb) {
  const int64_t r = blockIdx.x;
  if (r >= n) return;
  const int64_t src = idx[r];
  for (int c = threadIdx.x; c < ldx; c += blockDim.x) Xb[r * ldx + c] = X[src * ldx + c];
  for (int c = threadIdx.x; c < ldt; c += blockDim.x) Tb[r * ldt + c] = T[src * ldt + c];
}

// Element inputs: one CTA (256 threads) per listed element (all elements when
// list is null).  rl: local residual [E][512] float64; V: vertices [E][24].
// Writes F[i][0..543] (bf16) and scale[i] = s_e / h_e.
__global__ void __launch_bounds__(256)
    element_inputs(int64_t n, const int64_t *__restrict__ list, const double *__restrict__ rl,
                   const double *__restrict__ V, __nv_bfloat16 *__restrict__ F, double *__restrict__ scale) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t e = list ? list[i] : i;
  const double *r = rl + e * kOut;
  __shared__ double red[256];
  double mx = 0.0;
  for (int l = threadIdx.x; l < kOut; l += 256) mx = fmax(mx, fabs(r[l]));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double se = red[0] > 0.0 ? red[0] : 1.0;
  const double *v = V + e * 24;
  const double dx = v[3] - v[0], dy = v[4] - v[1], dz = v[5] - v[2];
  const double he = sqrt(dx * dx + dy * dy + dz * dz);
  __nv_bfloat16 *f = F + i * kInPad;
  for (int l = threadIdx.x; l < kOut; l += 256) f[l] = __float2bfloat16_rn((float)(r[l] / se));
  for (int q = threadIdx.x; q < kInPad - kOut; q += 256)
    f[kOut + q] = __float2bfloat16_rn(q < 24 ? (float)((v[q] - v[q % 3]) / he) : 0.0f);
  if (threadIdx.x == 0 && scale) scale[i] = se / he;
}

// T[i][l] = (e_l - d_l r_l) / scale[i]   (local copies; el, dl, rl [E][512])
__global__ void element_targets(int64_t n, const int64_t *__restrict__ list, const double *__restrict__ el,
                                const double *__restrict__ dl, const double *__restrict__ rl,
                                const double *__restrict__ scale, float *__restrict__ T) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t e = list ? list[i] : i;
  const double inv = 1.0 / scale[i];
  for (int l = threadIdx.x; l < kOut; l += blockDim.x) {
    const int64_t q = e * kOut + l;
    T[i * kOut + l] = (float)((el[q] - dl[q] * rl[q]) * inv);
  }
}

// correction of every element: cl[e][l] = Y[e][l] * scale[e]
__global__ void element_correction(int64_t n, const float *__restrict__ Y, const double *__restrict__ scale,
                                   double *__restrict__ cl) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * kOut; q += (int64_t)gridDim.x * blockDim.x)
    cl[q] = (double)Y[q] * scale[q / kOut];
}

// z[g] = dinv[g] r[g] + omega (sum of the local corrections of g) / (number of copies); 0 on masked nodes
__global__ void precond_combine(int64_t n, const gidx *__restrict__ off, const gidx *__restrict__ idx,
                                const double *__restrict__ cl, const double *__restrict__ dinv,
                                const double *__restrict__ r, const uint8_t *__restrict__ mask, double omega,
                                double *__restrict__ z) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    if (mask && mask[g]) {
      z[g] = 0.0;
      continue;
    }
    double s = 0.0;
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += cl[idx[q]];
    const int64_t cnt = off[g + 1] - off[g];
    z[g] = dinv[g] * r[g] + (cnt ? omega * s / (double)cnt : 0.0);
  }
}

// z = dinv r (the Jacobi step, also the fallback)
__global__ void jacobi_d(int64_t n, const double *__restrict__ dinv, const double *__restrict__ r, double *__restrict__ z) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    z[g] = dinv[g] * r[g];
}

__global__ void scatter_d(int64_t n, const gidx *__restrict__ gid, const double *__restrict__ u, double *__restrict__ U) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
    U[m] = u[gid[m]];
}
__global__ void gather_d(int64_t n, const gidx *__restrict__ off, const gidx *__restrict__ idx,
                         const double *__restrict__ Y, double *__restrict__ y, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
    y[g] = (mask && mask[g]) ? 0.0 : s;
  }
}
// out = a - b (masked to 0), or out = a - b without mask
__global__ void sub_d(int64_t n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out,
                      const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = (mask && mask[g]) ? 0.0 : a[g] - b[g];
}
__global__ void inv_d(int64_t n, const double *__restrict__ d, double *__restrict__ inv, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    inv[g] = (mask && mask[g]) ? 0.0 : 1.0 / d[g];
}
// fixed-order dot: partial per block, then host sum of the 1024 partials
__global__ void __launch_bounds__(256) dot_d(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                                             double *__restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    s += a[g] * b[g];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// y += a x
__global__ void axpy_d(int64_t n, double a, const double *__restrict__ x, double *__restrict__ y) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] += a * x[g];
}
// p = z + beta p
__global__ void xpby_d(int64_t n, const double *__restrict__ z, double beta, double *__restrict__ p) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    p[g] = z[g] + beta * p[g];
}

inline unsigned gfor(int64_t n, int b = 256) {
  int64_t g = (n + b - 1) / b;
  return (unsigned)(g < 1 ? 1 : (g > (1 << 20) ? (1 << 20) : g));
}

}  // namespace mlp
}  // namespace ax

using namespace ax;
using namespace ax::mlp;

struct ax_mlp {
  int device = 0;
  // FP32 master parameters, flat: W1 [H][InPad], b1 [H], W2 [H][H], b2 [H], W3 [O][H], b3 [O]
  float *p = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;
  int64_t np = 0;
  int64_t off[6] = {0, 0, 0, 0, 0, 0};
  // bf16 copies: W and W^T per layer
  __nv_bfloat16 *Wb[3] = {nullptr, nullptr, nullptr}, *WTb[3] = {nullptr, nullptr, nullptr};
  // activations for a batch of up to cap rows
  int64_t cap = 0;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *part = nullptr;
  __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *dY = nullptr, *dZ1 = nullptr, *dZ2 = nullptr, *T1 = nullptr,
                *T2 = nullptr;
  int64_t adam_t = 0;
  std::string err;
};

namespace {

thread_local std::string g_mlp_err;

ax_status mfail(ax_mlp *m, ax_status st, const std::string &msg) {
  if (m)
    m->err = msg;
  else
    g_mlp_err = msg;
  return st;
}
ax_status mcuda(ax_mlp *m, cudaError_t e, const char *what) {
  (void)cudaGetLastError();
  return mfail(m, e == cudaErrorMemoryAllocation ? AX_ENOMEM : AX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

const int kRows[3] = {kHid, kHid, kOut}, kCols[3] = {kInPad, kHid, kHid};

// splitmix64 (Steele, Lea, Flood 2014) and Box-Muller: deterministic host initialisation
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

// refresh bf16 W and W^T of every layer from the FP32 masters
cudaError_t refresh_bf16(ax_mlp *m, cudaStream_t s) {
  for (int l = 0; l < 3; ++l) {
    const int R = kRows[l], C = kCols[l];
    f32_to_bf16<<<gfor((int64_t)R * C), 256, 0, s>>>((int64_t)R * C, m->p + m->off[2 * l], m->Wb[l]);
    transpose_bf16<<<dim3((C + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, s>>>(R, C, m->Wb[l], C, m->WTb[l], R);
  }
  return cudaGetLastError();
}

cudaError_t ensure_cap(ax_mlp *m, int64_t rows) {
  if (rows <= m->cap) return cudaSuccess;
  cudaFree(m->Z1); cudaFree(m->Z2); cudaFree(m->Y); cudaFree(m->part);
  cudaFree(m->H1); cudaFree(m->H2); cudaFree(m->dY); cudaFree(m->dZ1); cudaFree(m->dZ2); cudaFree(m->T1); cudaFree(m->T2);
  m->cap = 0;
  const int64_t r = (rows + 127) / 128 * 128;
  cudaError_t e = cudaMalloc(&m->Z1, sizeof(float) * r * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&m->Z2, sizeof(float) * r * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&m->Y, sizeof(float) * r * kOut);
  if (e == cudaSuccess) e = cudaMalloc(&m->part, sizeof(float) * 1024);
  if (e == cudaSuccess) e = cudaMalloc(&m->H1, sizeof(__nv_bfloat16) * r * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&m->H2, sizeof(__nv_bfloat16) * r * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&m->dY, sizeof(__nv_bfloat16) * r * kOut);
  if (e == cudaSuccess) e = cudaMalloc(&m->dZ1, sizeof(__nv_bfloat16) * r * kHid);
  if (e == cudaSuccess) e = cudaMalloc(&m->dZ2, sizeof(__nv_bfloat16) * r * kHid);
  // transposes: the largest is [kInPad][r]
  if (e == cudaSuccess) e = cudaMalloc(&m->T1, sizeof(__nv_bfloat16) * r * kInPad);
  if (e == cudaSuccess) e = cudaMalloc(&m->T2, sizeof(__nv_bfloat16) * r * kInPad);
  if (e == cudaSuccess) m->cap = r;
  return e;
}

// forward of M rows of X (bf16 [M][kInPad]) -> m->Y (f32 [M][kOut])
cudaError_t forward(ax_mlp *m, const __nv_bfloat16 *X, int64_t M, cudaStream_t s) {
  GemmOut o1;
  o1.Cf = m->Z1; o1.Hb = m->H1; o1.bias = m->p + m->off[1]; o1.ldc = kHid;
  cudaError_t e = gemm<kEpiGelu>((int)M, kHid, kInPad, X, kInPad, m->Wb[0], kInPad, o1, s);
  GemmOut o2;
  o2.Cf = m->Z2; o2.Hb = m->H2; o2.bias = m->p + m->off[3]; o2.ldc = kHid;
  if (e == cudaSuccess) e = gemm<kEpiGelu>((int)M, kHid, kHid, m->H1, kHid, m->Wb[1], kHid, o2, s);
  GemmOut o3;
  o3.Cf = m->Y; o3.bias = m->p + m->off[5]; o3.ldc = kOut;
  if (e == cudaSuccess) e = gemm<kEpiF32>((int)M, kOut, kHid, m->H2, kHid, m->Wb[2], kHid, o3, s);
  return e;
}

// forward + backward of M rows (M a multiple of 32): gradients into m->g; loss partials in m->part
cudaError_t forward_backward(ax_mlp *m, const __nv_bfloat16 *X, const float *T, int64_t M, cudaStream_t s) {
  cudaError_t e = forward(m, X, M, s);
  if (e != cudaSuccess) return e;
  loss_grad<<<1024, 256, 0, s>>>((int)M, kOut, m->Y, T, m->dY, m->part);
  const dim3 tb(32, 8);
  auto tr = [&](int R, int C, const __nv_bfloat16 *in, __nv_bfloat16 *out) {
    transpose_bf16<<<dim3((C + 31) / 32, (R + 31) / 32), tb, 0, s>>>(R, C, in, C, out, R);
  };
  float *g = m->g;
  // layer 3: dW3 = dY^T H2, db3 = colsum dY, dZ2 = (dY W3) * gelu'(Z2)
  tr((int)M, kOut, m->dY, m->T1);
  tr((int)M, kHid, m->H2, m->T2);
  GemmOut w3;
  w3.Cf = g + m->off[4]; w3.ldc = kHid;
  e = gemm<kEpiF32>(kOut, kHid, (int)M, m->T1, (int)M, m->T2, (int)M, w3, s);
  colsum_bf16<<<gfor(kOut), 256, 0, s>>>((int)M, kOut, m->dY, g + m->off[5]);
  GemmOut d2;
  d2.Hb = m->dZ2; d2.Zin = m->Z2; d2.ldc = kHid;
  if (e == cudaSuccess) e = gemm<kEpiDGelu>((int)M, kHid, kOut, m->dY, kOut, m->WTb[2], kOut, d2, s);
  // layer 2
  tr((int)M, kHid, m->dZ2, m->T1);
  tr((int)M, kHid, m->H1, m->T2);
  GemmOut w2;
  w2.Cf = g + m->off[2]; w2.ldc = kHid;
  if (e == cudaSuccess) e = gemm<kEpiF32>(kHid, kHid, (int)M, m->T1, (int)M, m->T2, (int)M, w2, s);
  colsum_bf16<<<gfor(kHid), 256, 0, s>>>((int)M, kHid, m->dZ2, g + m->off[3]);
  GemmOut d1;
  d1.Hb = m->dZ1; d1.Zin = m->Z1; d1.ldc = kHid;
  if (e == cudaSuccess) e = gemm<kEpiDGelu>((int)M, kHid, kHid, m->dZ2, kHid, m->WTb[1], kHid, d1, s);
  // layer 1
  tr((int)M, kHid, m->dZ1, m->T1);
  tr((int)M, kInPad, X, m->T2);
  GemmOut w1;
  w1.Cf = g + m->off[0]; w1.ldc = kInPad;
  if (e == cudaSuccess) e = gemm<kEpiF32>(kHid, kInPad, (int)M, m->T1, (int)M, m->T2, (int)M, w1, s);
  colsum_bf16<<<gfor(kHid), 256, 0, s>>>((int)M, kHid, m->dZ1, g + m->off[1]);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace

extern "C" {

const char *ax_mlp_last_error(const ax_mlp *m) { return m ? m->err.c_str() : g_mlp_err.c_str(); }

ax_status ax_mlp_create(ax_mlp **out, uint64_t seed, void *stream) {
  if (!out) return mfail(nullptr, AX_EINVAL, "ax_mlp_create: out is NULL");
  *out = nullptr;
  ax_mlp *m = new (std::nothrow) ax_mlp;
  if (!m) return mfail(nullptr, AX_ENOMEM, "ax_mlp_create: host allocation failed");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&m->device);
  int64_t o = 0;
  for (int l = 0; l < 3; ++l) {
    m->off[2 * l] = o;
    o += (int64_t)kRows[l] * kCols[l];
    m->off[2 * l + 1] = o;
    o += kRows[l];
  }
  m->np = o;
  // He-style initialisation N(0, 2/fan_in) for the GELU layers, N(0, 1/fan_in)
  // scaled by 0.1 for the output layer (start close to the Jacobi step);
  // biases zero; padded input columns zero
  std::vector<float> h((size_t)o, 0.0f);
  SplitMix rng{seed};
  for (int l = 0; l < 3; ++l) {
    const int fan = l == 0 ? kIn : kHid;
    const double sd = l < 2 ? std::sqrt(2.0 / fan) : 0.1 / std::sqrt((double)fan);
    for (int r = 0; r < kRows[l]; ++r)
      for (int c = 0; c < kCols[l]; ++c)
        h[m->off[2 * l] + (int64_t)r * kCols[l] + c] = (l == 0 && c >= kIn) ? 0.0f : (float)(sd * rng.normal());
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->p, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMalloc(&m->g, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMalloc(&m->am, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMalloc(&m->av, sizeof(float) * o);
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = cudaMalloc(&m->Wb[l], sizeof(__nv_bfloat16) * kRows[l] * kCols[l]);
    if (e == cudaSuccess) e = cudaMalloc(&m->WTb[l], sizeof(__nv_bfloat16) * kRows[l] * kCols[l]);
  }
  if (e == cudaSuccess) e = cudaMemcpy(m->p, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->am, 0, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMemset(m->av, 0, sizeof(float) * o);
  if (e == cudaSuccess) e = cudaMemset(m->g, 0, sizeof(float) * o);
  if (e == cudaSuccess) e = refresh_bf16(m, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ax_status st = mcuda(nullptr, e, "ax_mlp_create");
    ax_mlp_destroy(m);
    return st;
  }
  *out = m;
  return AX_OK;
}

// Parameter count and layout: W1 [512][544] (columns >= 536 are zero), b1 [512],
// W2 [512][512], b2 [512], W3 [512][512], b3 [512], flat float32.
int64_t ax_mlp_num_params(const ax_mlp *m) { return m ? m->np : 0; }

ax_status ax_mlp_get_params(ax_mlp *m, float *params, void *stream) {
  if (!m || !params) return mfail(m, AX_EINVAL, "ax_mlp_get_params: NULL argument");
  cudaError_t e = cudaMemcpyAsync(params, m->p, sizeof(float) * m->np, cudaMemcpyDefault, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? AX_OK : mcuda(m, e, "ax_mlp_get_params");
}

ax_status ax_mlp_set_params(ax_mlp *m, const float *params, void *stream) {
  if (!m || !params) return mfail(m, AX_EINVAL, "ax_mlp_set_params: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(m->p, params, sizeof(float) * m->np, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = refresh_bf16(m, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? AX_OK : mcuda(m, e, "ax_mlp_set_params");
}

ax_status ax_mlp_forward(ax_mlp *m, const void *X_bf16, float *Y, int64_t M, void *stream) {
  if (!m || !X_bf16 || !Y || M < 0) return mfail(m, AX_EINVAL, "ax_mlp_forward: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = ensure_cap(m, M);
  if (e == cudaSuccess) e = forward(m, (const __nv_bfloat16 *)X_bf16, M, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Y, m->Y, sizeof(float) * M * kOut, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? AX_OK : mcuda(m, e, "ax_mlp_forward");
}

ax_status ax_mlp_grad(ax_mlp *m, const void *X_bf16, const float *T, int64_t M, float *loss, float *grads,
                      void *stream) {
  if (!m || !X_bf16 || !T || !loss || !grads || M < 32 || M % 32)
    return mfail(m, AX_EINVAL, "ax_mlp_grad: bad arguments (M must be a positive multiple of 32)");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = ensure_cap(m, M);
  if (e == cudaSuccess) e = forward_backward(m, (const __nv_bfloat16 *)X_bf16, T, M, s);
  std::vector<float> part(1024);
  if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), m->part, sizeof(float) * 1024, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grads, m->g, sizeof(float) * m->np, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mcuda(m, e, "ax_mlp_grad");
  double acc = 0.0;
  for (float v : part) acc += v;
  *loss = (float)(0.5 * acc / ((double)M * kOut));
  return AX_OK;
}

ax_status ax_mlp_train(ax_mlp *m, const void *X_bf16, const float *T, int64_t n_samples, int epochs, int batch,
                       float lr, uint64_t seed, float *loss_history, void *stream) {
  if (!m || !X_bf16 || !T || n_samples < batch || epochs < 1 || batch < 32 || batch % 32 || !(lr > 0.0f))
    return mfail(m, AX_EINVAL, "ax_mlp_train: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = ensure_cap(m, batch);
  __nv_bfloat16 *Xb = nullptr;
  float *Tb = nullptr;
  int64_t *idx = nullptr;
  const int64_t steps = n_samples / batch;
  if (e == cudaSuccess) e = cudaMalloc(&Xb, sizeof(__nv_bfloat16) * batch * kInPad);
  if (e == cudaSuccess) e = cudaMalloc(&Tb, sizeof(float) * batch * kOut);
  if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(int64_t) * steps * batch);
  std::vector<int64_t> perm((size_t)n_samples);
  std::vector<float> part(1024);
  SplitMix rng{seed};
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int64_t i = 0; i < n_samples; ++i) perm[i] = i;
    for (int64_t i = n_samples - 1; i > 0; --i) std::swap(perm[i], perm[rng.next() % (uint64_t)(i + 1)]);  // Fisher-Yates
    e = cudaMemcpyAsync(idx, perm.data(), sizeof(int64_t) * steps * batch, cudaMemcpyHostToDevice, s);
    double ep_loss = 0.0;
    for (int64_t st = 0; st < steps && e == cudaSuccess; ++st) {
      gather_rows<<<batch, 256, 0, s>>>(batch, idx + st * batch, (const __nv_bfloat16 *)X_bf16, kInPad, T, kOut, Xb, Tb);
      e = forward_backward(m, Xb, Tb, batch, s);
      if (e != cudaSuccess) break;
      ++m->adam_t;
      const float c1 = 1.0f - powf(b1, (float)m->adam_t), c2 = 1.0f - powf(b2, (float)m->adam_t);
      adam<<<gfor(m->np), 256, 0, s>>>(m->np, m->p, m->g, m->am, m->av, lr, b1, b2, eps, c1, c2);
      e = refresh_bf16(m, s);
      if (e == cudaSuccess && (st == steps - 1)) {
        e = cudaMemcpyAsync(part.data(), m->part, sizeof(float) * 1024, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        double acc = 0.0;
        for (float v : part) acc += v;
        ep_loss = 0.5 * acc / ((double)batch * kOut);
      }
    }
    if (loss_history) loss_history[ep] = (float)ep_loss;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(Xb);
  cudaFree(Tb);
  cudaFree(idx);
  return e == cudaSuccess ? AX_OK : mcuda(m, e, "ax_mlp_train");
}

}  // extern "C"

namespace {

// Work buffers shared by ax_mlp_pairs and pcg_solve_learned.
struct LearnWork {
  int64_t n = 0, nl = 0, E = 0;
  double *r = nullptr, *w = nullptr, *Ul = nullptr, *Yl = nullptr, *dinv = nullptr, *diag_l = nullptr,
         *scale = nullptr, *cl = nullptr, *part = nullptr;
  __nv_bfloat16 *F = nullptr;
  float *Y = nullptr;
  cudaError_t alloc(int64_t n_, int64_t nl_, int64_t E_) {
    n = n_;
    nl = nl_;
    E = E_;
    cudaError_t e = cudaMalloc(&r, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dinv, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Ul, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&Yl, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&diag_l, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&cl, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&scale, sizeof(double) * E);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 1024);
    if (e == cudaSuccess) e = cudaMalloc(&F, sizeof(__nv_bfloat16) * E * kInPad);
    if (e == cudaSuccess) e = cudaMalloc(&Y, sizeof(float) * E * kOut);
    return e;
  }
  void release() {
    cudaFree(r); cudaFree(w); cudaFree(dinv); cudaFree(Ul); cudaFree(Yl); cudaFree(diag_l); cudaFree(cl);
    cudaFree(scale); cudaFree(part); cudaFree(F); cudaFree(Y);
  }
};

cudaError_t (*ax_launcher(int prec))(const AxArgs &) {
  switch (prec) {
    case AX_FP64: return launch_ax_fp64;
    case AX_F64DW: return launch_ax_dw;
    default: return nullptr;
  }
}

// w = A x (assembled, masked), through the local vectors of W
cudaError_t apply_A(const ax_ctx *c, LearnWork &W, const double *x, double *w, cudaStream_t s) {
  const GsPlan &P = ax_ctx_core(c).gs;
  scatter_d<<<gfor(P.n_local), 256, 0, s>>>(P.n_local, P.gid, x, W.Ul);
  AxArgs a = ax_ctx_args(c);
  a.X = W.Ul;
  a.Y = W.Yl;
  a.stream = s;
  cudaError_t e = ax_launcher(ax_ctx_core(c).prec)(a);
  if (e != cudaSuccess) return e;
  gather_d<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, P.off, P.idx, W.Yl, w, P.mask);
  return cudaGetLastError();
}

cudaError_t jacobi_inverse(ax_ctx *c, LearnWork &W, cudaStream_t s) {
  const GsPlan &P = ax_ctx_core(c).gs;
  const void *dg = nullptr;
  cudaError_t e = assembled_diag(c, true, &dg, s);
  if (e != cudaSuccess) return e;
  inv_d<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, (const double *)dg, W.dinv, P.mask);
  return cudaGetLastError();
}

double host_dot(LearnWork &W, const double *a, const double *b, int64_t n, cudaStream_t s, cudaError_t *err) {
  std::vector<double> h(1024);
  dot_d<<<1024, 256, 0, s>>>(n, a, b, W.part);
  cudaError_t e = cudaMemcpyAsync(h.data(), W.part, sizeof(double) * 1024, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) *err = e;
  double acc = 0.0;
  for (double v : h) acc += v;
  return acc;
}

// z = D^-1 r + omega Q^T(c) / multiplicity with c from the MLP on every element
cudaError_t apply_learned(const ax_ctx *c, ax_mlp *m, LearnWork &W, const double *r, double *z, double omega,
                          cudaStream_t s) {
  const GsPlan &P = ax_ctx_core(c).gs;
  const int64_t E = ax_ctx_core(c).E;
  scatter_d<<<gfor(P.n_local), 256, 0, s>>>(P.n_local, P.gid, r, W.Ul);
  element_inputs<<<(unsigned)E, 256, 0, s>>>(E, nullptr, W.Ul, ax_ctx_vertices(c), W.F, W.scale);
  cudaError_t e = forward(m, W.F, E, s);
  if (e != cudaSuccess) return e;
  element_correction<<<gfor(E * kOut), 256, 0, s>>>(E, m->Y, W.scale, W.cl);
  precond_combine<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, P.off, P.idx, W.cl, W.dinv, r, P.mask, omega, z);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

ax_status ax_mlp_pairs(ax_ctx *c, const double *b_global, const double *x_star, const double *x_k,
                       const int64_t *elements, int64_t n, void *F_bf16, float *T, void *stream) {
  if (!c || !b_global || !x_star || !x_k || !elements || n < 0 || !F_bf16 || !T)
    return mfail(nullptr, AX_EINVAL, "ax_mlp_pairs: bad arguments");
  const Ctx &C = ax_ctx_core(c);
  if (C.N != 7) return mfail(nullptr, AX_EUNSUPPORTED, "ax_mlp_pairs: the learned preconditioner is for N = 7");
  if (!C.gs.off) return mfail(nullptr, AX_EINVAL, "ax_mlp_pairs: call gs_setup first");
  if (!ax_launcher(C.prec)) return mfail(nullptr, AX_EUNSUPPORTED, "ax_mlp_pairs: needs an AX_FP64 or AX_F64DW context");
  if (n == 0) return AX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  LearnWork W;
  double *e_glob = nullptr, *el = nullptr, *dl = nullptr, *sc = nullptr;
  cudaError_t e = W.alloc(C.gs.n_global, C.gs.n_local, C.E);
  if (e == cudaSuccess) e = cudaMalloc(&e_glob, sizeof(double) * C.gs.n_global);
  if (e == cudaSuccess) e = cudaMalloc(&el, sizeof(double) * C.gs.n_local);
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(double) * C.gs.n_local);
  if (e == cudaSuccess) e = cudaMalloc(&sc, sizeof(double) * n);
  if (e == cudaSuccess) e = jacobi_inverse(c, W, s);
  if (e == cudaSuccess) e = apply_A(c, W, x_k, W.w, s);
  if (e == cudaSuccess) {
    const GsPlan &P = C.gs;
    sub_d<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, b_global, W.w, W.r, P.mask);    // r = b - A x_k
    sub_d<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, x_star, x_k, e_glob, P.mask);  // e = x* - x_k
    scatter_d<<<gfor(P.n_local), 256, 0, s>>>(P.n_local, P.gid, W.r, W.Ul);
    scatter_d<<<gfor(P.n_local), 256, 0, s>>>(P.n_local, P.gid, e_glob, el);
    scatter_d<<<gfor(P.n_local), 256, 0, s>>>(P.n_local, P.gid, W.dinv, dl);
    element_inputs<<<(unsigned)n, 256, 0, s>>>(n, elements, W.Ul, ax_ctx_vertices(c), (__nv_bfloat16 *)F_bf16, sc);
    element_targets<<<(unsigned)n, 256, 0, s>>>(n, elements, el, dl, W.Ul, sc, T);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  W.release();
  cudaFree(e_glob);
  cudaFree(el);
  cudaFree(dl);
  cudaFree(sc);
  return e == cudaSuccess ? AX_OK : mcuda(nullptr, e, "ax_mlp_pairs");
}

ax_status pcg_solve_learned(ax_ctx *c, ax_mlp *m, const double *b_global, double *x, double rtol, int maxit,
                            double omega, int *iters, double *relres, int *fell_back, void *stream) {
  if (!c || !m || !b_global || !x || !iters || !relres || !fell_back || maxit < 0 || !(rtol >= 0.0) ||
      !(omega >= 0.0))
    return mfail(m, AX_EINVAL, "pcg_solve_learned: bad arguments");
  *fell_back = 0;
  const Ctx &C = ax_ctx_core(c);
  if (C.N != 7) return mfail(m, AX_EUNSUPPORTED, "pcg_solve_learned: the learned preconditioner is for N = 7");
  if (!C.gs.off) return mfail(m, AX_EINVAL, "pcg_solve_learned: call gs_setup first");
  if (!ax_launcher(C.prec)) return mfail(m, AX_EUNSUPPORTED, "pcg_solve_learned: needs an AX_FP64 or AX_F64DW context");
  cudaStream_t s = (cudaStream_t)stream;
  const GsPlan &P = C.gs;
  const int64_t n = P.n_global;
  *iters = 0;
  *relres = 0.0;
  LearnWork W;
  double *z = nullptr, *p = nullptr, *rold = nullptr, *bm = nullptr;
  cudaError_t e = W.alloc(n, P.n_local, C.E);
  if (e == cudaSuccess) e = ensure_cap(m, C.E);
  if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&rold, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&bm, sizeof(double) * n);
  if (e == cudaSuccess) e = jacobi_inverse(c, W, s);
  int conv = 0;
  if (e == cudaSuccess) {
    // masked b and x; r = b - A x
    e = cudaMemsetAsync(W.w, 0, sizeof(double) * n, s);
    sub_d<<<gfor(n), 256, 0, s>>>(n, b_global, W.w, bm, P.mask);
    sub_d<<<gfor(n), 256, 0, s>>>(n, x, W.w, x, P.mask);
    if (e == cudaSuccess) e = apply_A(c, W, x, W.w, s);
    sub_d<<<gfor(n), 256, 0, s>>>(n, bm, W.w, W.r, P.mask);
    const double bnorm = std::sqrt(host_dot(W, bm, bm, n, s, &e));
    double rnorm = std::sqrt(host_dot(W, W.r, W.r, n, s, &e));
    int it = 0;
    if (bnorm == 0.0 || rnorm <= rtol * bnorm) conv = 1;
    // preconditioner with safeguards: a learned step that is not a descent
    // direction (r . z <= 0) is replaced by the Jacobi step; after the
    // residual has failed to halve for `patience` iterations the solve falls
    // back to Jacobi for good (then it is plain Jacobi-PCG).
    const int patience = 200;
    double best = rnorm;
    int best_it = 0;
    bool learned_on = true;
    auto precond = [&](double &rz_out) {
      if (learned_on) {
        e = apply_learned(c, m, W, W.r, z, omega, s);
        if (e != cudaSuccess) return;
        rz_out = host_dot(W, W.r, z, n, s, &e);
        if (rz_out > 0.0 && rz_out == rz_out) return;
      }
      jacobi_d<<<gfor(n), 256, 0, s>>>(n, W.dinv, W.r, z);
      rz_out = host_dot(W, W.r, z, n, s, &e);
    };
    double rz = 0.0;
    if (!conv && e == cudaSuccess) precond(rz);
    if (!conv && e == cudaSuccess) e = cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    while (!conv && e == cudaSuccess && it < maxit) {
      e = apply_A(c, W, p, W.w, s);
      if (e != cudaSuccess) break;
      const double pw = host_dot(W, p, W.w, n, s, &e);
      const double alpha = pw != 0.0 ? rz / pw : 0.0;
      axpy_d<<<gfor(n), 256, 0, s>>>(n, alpha, p, x);
      e = cudaMemcpyAsync(rold, W.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
      axpy_d<<<gfor(n), 256, 0, s>>>(n, -alpha, W.w, W.r);
      ++it;
      rnorm = std::sqrt(host_dot(W, W.r, W.r, n, s, &e));
      if (!(rnorm == rnorm)) break;
      if (rnorm <= rtol * bnorm) {
        conv = 1;
        break;
      }
      if (rnorm < 0.5 * best) {
        best = rnorm;
        best_it = it;
      } else if (learned_on && it - best_it >= patience) {
        learned_on = false;
        *fell_back = 1;
      }
      double rz_new = 0.0;
      if (e == cudaSuccess) precond(rz_new);
      // flexible (Polak-Ribiere) beta = z . (r - r_old) / rz
      sub_d<<<gfor(n), 256, 0, s>>>(n, W.r, rold, rold, nullptr);
      const double zdr = host_dot(W, z, rold, n, s, &e);
      const double beta = rz != 0.0 ? zdr / rz : 0.0;
      rz = rz_new;
      xpby_d<<<gfor(n), 256, 0, s>>>(n, z, beta, p);
    }
    *iters = it;
    *relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  W.release();
  cudaFree(z);
  cudaFree(p);
  cudaFree(rold);
  cudaFree(bm);
  if (e != cudaSuccess) return mcuda(m, e, "pcg_solve_learned");
  if (!conv) return mfail(m, AX_ENOTCONV, "pcg_solve_learned: not converged");
  return AX_OK;
}

void ax_mlp_destroy(ax_mlp *m) {
  if (!m) return;
  cudaFree(m->p); cudaFree(m->g); cudaFree(m->am); cudaFree(m->av);
  for (int l = 0; l < 3; ++l) {
    cudaFree(m->Wb[l]);
    cudaFree(m->WTb[l]);
  }
  cudaFree(m->Z1); cudaFree(m->Z2); cudaFree(m->Y); cudaFree(m->part);
  cudaFree(m->H1); cudaFree(m->H2); cudaFree(m->dY); cudaFree(m->dZ1); cudaFree(m->dZ2); cudaFree(m->T1); cudaFree(m->T2);
  delete m;
}

}  // extern "C"
