// Learned per-element preconditioner: a small MLP, trained and run on the GPU
// with the tcgen05 BF16 GEMM of gemm_tc.cuh (FP32 accumulation in TMEM, FP32
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
#include "gemm_tc.cuh"
#include "reduce.cuh"

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

// Element inputs: one warp per listed element (all elements when list is
// null), 8 warps per CTA.  rl: local residual [E][512] float64; V: vertices
// [E][24].  Writes F[i][0..543] (bf16) and scale[i] = s_e / h_e (float).  The
// residual is converted to float once and everything after runs on the FP32
// pipe (a float64 division per value would bind the kernel to GB300's FP64
// rate).
constexpr int kInputWarps = 8;
__global__ void __launch_bounds__(32 * kInputWarps)
    element_inputs(int64_t n, const int64_t *__restrict__ list, const double *__restrict__ rl,
                   const double *__restrict__ V, __nv_bfloat16 *__restrict__ F, float *__restrict__ scale,
                   const double *__restrict__ skip) {
  const int64_t i = (int64_t)blockIdx.x * kInputWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n || (skip && *skip != 0.0)) return;
  const int64_t e = list ? list[i] : i;
  const double2 *r2 = reinterpret_cast<const double2 *>(rl + e * kOut);
  float v[16];
  float mx = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {  // pairs (2 lane + 64 k, +1): coalesced 16-byte loads
    const double2 d = r2[lane + 32 * k];
    v[2 * k] = (float)d.x;
    v[2 * k + 1] = (float)d.y;
    mx = fmaxf(mx, fmaxf(fabsf(v[2 * k]), fabsf(v[2 * k + 1])));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float se = mx > 0.0f ? mx : 1.0f, inv_se = 1.0f / se;
  const double *vt = V + e * 24;
  const float dx = (float)(vt[3] - vt[0]), dy = (float)(vt[4] - vt[1]), dz = (float)(vt[5] - vt[2]);
  const float he = sqrtf(dx * dx + dy * dy + dz * dz), inv_he = 1.0f / he;
  __nv_bfloat162 *f2 = reinterpret_cast<__nv_bfloat162 *>(F + i * kInPad);
#pragma unroll
  for (int k = 0; k < 8; ++k) f2[lane + 32 * k] = __floats2bfloat162_rn(v[2 * k] * inv_se, v[2 * k + 1] * inv_se);
  // 32 trailing inputs: 24 relative vertex coordinates / h_e, then zero padding
  F[i * kInPad + kOut + lane] = __float2bfloat16_rn(lane < 24 ? (float)(vt[lane] - vt[lane % 3]) * inv_he : 0.0f);
  if (lane == 0 && scale) scale[i] = se * inv_he;
}
inline unsigned input_blocks(int64_t n) { return (unsigned)((n + kInputWarps - 1) / kInputWarps); }

// T[i][l] = (e_g - dinv_g r_l) / scale[i] with g = gid[e][l] (e, dinv global; rl local [E][512])
__global__ void element_targets(int64_t n, const int64_t *__restrict__ list, const gidx *__restrict__ gid,
                                const double *__restrict__ eg, const double *__restrict__ dinv,
                                const double *__restrict__ rl, const float *__restrict__ scale, float *__restrict__ T) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t e = list ? list[i] : i;
  const double inv = 1.0 / (double)scale[i];
  for (int l = threadIdx.x; l < kOut; l += blockDim.x) {
    const int64_t q = e * kOut + l;
    const gidx g = gid[q];
    T[i * kOut + l] = (float)((eg[g] - dinv[g] * rl[q]) * inv);
  }
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
// ---------------------------------------------------------------------------
// learned flexible PCG: every scalar stays on the device; one iteration is
//   lp_direction   p = z + beta p (z = D^-1 r when the Jacobi step was chosen); U = Q p
//   AxLocal        W = A_e U
//   lp_gather      w = mask(Q^T W); alpha = rz / (p . w)
//   lp_update      x += alpha p; r -= alpha w; U = Q r; test ||r||; patience
//   element_inputs, 3 GEMMs (the MLP on every element's residual)
//   lp_precond     z = D^-1 r + omega Q^T(c)/multiplicity; safeguard; beta
// with the flexible (Polak-Ribiere) beta = z_new . (r_new - r_old) / rz_old
// = -alpha (z_new . w) / rz_old.
// ---------------------------------------------------------------------------
enum LpScalar {
  kRz = 0, kPw = 1, kRr = 2, kBb = 3, kUseJac = 5, kDone = 6, kConvIt = 7, kTol2 = 8, kIter = 9, kAlpha = 10,
  kBeta = 11, kBestRr = 12, kBestIt = 13, kLearnOff = 14, kMlpSkip = 15, kPatience = 16, kLpScalars = 24
};
constexpr int kLpBlocks = 1024;
// lp_precond: nodes per thread whose gathers are in flight together (measured
// 248 -> 213 us per launch at 32^3 elements; the same unrolling made lp_gather,
// which gathers float64, slower: 136 -> 227 us, so it keeps the plain loop)
constexpr int kLpU = 4;

__global__ void __launch_bounds__(red::kThreads)
    lp_init(int64_t n, const double *__restrict__ b, const double *__restrict__ w, double *__restrict__ bm,
            double *__restrict__ r, double *__restrict__ p, const uint8_t *__restrict__ mask, double rtol,
            double patience, double *__restrict__ part, unsigned *__restrict__ cnt, double *__restrict__ S) {
  double bb = 0.0, rr = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const bool m = mask && mask[g];
    const double bg = m ? 0.0 : b[g];
    const double rg = m ? 0.0 : bg - w[g];
    bm[g] = bg;
    r[g] = rg;
    p[g] = 0.0;
    bb += bg * bg;
    rr += rg * rg;
  }
  red::block_reduce_store(bb, part + blockIdx.x);
  __syncthreads();
  red::block_reduce_store(rr, part + kLpBlocks + blockIdx.x);
  if (!red::arrive_last(cnt)) return;
  const double bbt = red::sum_partials(part, gridDim.x);
  const double rrt = red::sum_partials(part + kLpBlocks, gridDim.x);
  if (threadIdx.x == 0) {
    for (int q = 0; q < kLpScalars; ++q) S[q] = 0.0;
    S[kBb] = bbt;
    S[kRr] = rrt;
    S[kBestRr] = rrt;
    S[kTol2] = rtol * rtol * bbt;
    S[kPatience] = patience;
  }
}

// U = Q r (the local copies of the residual, the network's input)
__global__ void lp_scatter(int64_t n, const double *__restrict__ r, const gidx *__restrict__ off,
                           const gidx *__restrict__ idx, double *__restrict__ U) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double rg = r[g];
    for (gidx q = off[g]; q < off[g + 1]; ++q) U[idx[q]] = rg;
  }
}

__global__ void lp_direction(int64_t n, const double *__restrict__ S, const double *__restrict__ z,
                             const double *__restrict__ r, const double *__restrict__ dinv, double *__restrict__ p,
                             const gidx *__restrict__ off, const gidx *__restrict__ idx, double *__restrict__ U) {
  if (S[kDone] != 0.0) return;
  const double beta = S[kBeta];
  const bool jac = S[kUseJac] != 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double zg = jac ? dinv[g] * r[g] : z[g];
    const double pg = zg + beta * p[g];
    p[g] = pg;
    for (gidx q = off[g]; q < off[g + 1]; ++q) U[idx[q]] = pg;
  }
}

__global__ void __launch_bounds__(red::kThreads)
    lp_gather(int64_t n, const gidx *__restrict__ off, const gidx *__restrict__ idx, const double *__restrict__ Y,
              double *__restrict__ w, const uint8_t *__restrict__ mask, const double *__restrict__ p,
              double *__restrict__ part, unsigned *__restrict__ cnt, double *__restrict__ S) {
  if (S[kDone] != 0.0) return;
  double d = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
    if (mask && mask[g]) s = 0.0;
    w[g] = s;
    d += p[g] * s;
  }
  red::block_reduce_store(d, part + blockIdx.x);
  if (!red::arrive_last(cnt)) return;
  const double pw = red::sum_partials(part, gridDim.x);
  if (threadIdx.x == 0) {
    S[kPw] = pw;
    S[kAlpha] = pw != 0.0 ? S[kRz] / pw : 0.0;
  }
}

// After the update the residual either converged (done), or the patience
// test runs: ||r|| must halve (rr drop to a quarter) within `patience`
// iterations of the last halving, else the learned step is switched off for
// good (the solve continues as Jacobi-PCG).
__global__ void __launch_bounds__(red::kThreads)
    lp_update(int64_t n, double *__restrict__ S, const double *__restrict__ p, const double *__restrict__ w,
              double *__restrict__ x, double *__restrict__ r, const gidx *__restrict__ off,
              const gidx *__restrict__ idx, double *__restrict__ U, double *__restrict__ part,
              unsigned *__restrict__ cnt) {
  if (S[kDone] != 0.0) return;
  const double alpha = S[kAlpha];
  double rr = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    x[g] += alpha * p[g];
    const double rg = r[g] - alpha * w[g];
    r[g] = rg;
    for (gidx q = off[g]; q < off[g + 1]; ++q) U[idx[q]] = rg;
    rr += rg * rg;
  }
  red::block_reduce_store(rr, part + blockIdx.x);
  if (!red::arrive_last(cnt)) return;
  const double rrt = red::sum_partials(part, gridDim.x);
  if (threadIdx.x == 0) {
    const double it = S[kIter] + 1.0;
    S[kIter] = it;
    S[kRr] = rrt;
    if (rrt <= S[kTol2]) {
      S[kDone] = 1.0;
      S[kConvIt] = it;
    } else if (!(rrt == rrt)) {
      S[kDone] = 1.0;
      S[kConvIt] = -it;
    } else if (rrt < 0.25 * S[kBestRr]) {
      S[kBestRr] = rrt;
      S[kBestIt] = it;
    } else if (S[kLearnOff] == 0.0 && it - S[kBestIt] >= S[kPatience]) {
      S[kLearnOff] = 1.0;
    }
    S[kMlpSkip] = (S[kDone] != 0.0 || S[kLearnOff] != 0.0) ? 1.0 : 0.0;
  }
}

constexpr int kRcpTable = 33;
__constant__ float c_rcp[kRcpTable] = {
    0.0f,        1.0f,        1.0f / 2,  1.0f / 3,  1.0f / 4,  1.0f / 5,  1.0f / 6,  1.0f / 7,  1.0f / 8,
    1.0f / 9,    1.0f / 10,   1.0f / 11, 1.0f / 12, 1.0f / 13, 1.0f / 14, 1.0f / 15, 1.0f / 16, 1.0f / 17,
    1.0f / 18,   1.0f / 19,   1.0f / 20, 1.0f / 21, 1.0f / 22, 1.0f / 23, 1.0f / 24, 1.0f / 25, 1.0f / 26,
    1.0f / 27,   1.0f / 28,   1.0f / 29, 1.0f / 30, 1.0f / 31, 1.0f / 32};

// z = D^-1 r + omega (sum of the local corrections c = scale_e Y_e of g) / multiplicity,
// the correction summed in float; partial dots r.z and w.z.  When the
// network is off (converged, or switched off by the patience test) z is the
// Jacobi step.  The last block sets beta and rz, or, when the learned step is
// not a descent direction (r.z <= 0), flags the iteration for lp_jacobi_fix.
__global__ void __launch_bounds__(red::kThreads)
    lp_precond(int64_t n, const gidx *__restrict__ off, const gidx *__restrict__ idx, const float *__restrict__ Y,
               const float *__restrict__ scale, const double *__restrict__ dinv, const double *__restrict__ r,
               const double *__restrict__ w, const uint8_t *__restrict__ mask, float omega, double *__restrict__ z,
               double *__restrict__ part, unsigned *__restrict__ cnt, double *__restrict__ S) {
  if (S[kDone] != 0.0) return;
  const bool learned = S[kMlpSkip] == 0.0;
  double rz = 0.0, wz = 0.0;
  // kLpU nodes per thread at a time (their gathers in flight together); the
  // averaged correction in float: omega / multiplicity from a table (no
  // int -> float conversion or division on the slow pipes)
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g0 < n; g0 += kLpU * step) {
    gidx b[kLpU], c[kLpU];
    float sc[kLpU];
#pragma unroll
    for (int u = 0; u < kLpU; ++u) {
      const int64_t g = g0 + u * step;
      const bool on = g < n && learned && !(mask && mask[g]);
      b[u] = on ? off[g] : 0;
      c[u] = on ? off[g + 1] - b[u] : 0;
      sc[u] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int u = 0; u < kLpU; ++u)
        if (q < c[u]) {
          const gidx l = idx[b[u] + q];
          sc[u] += Y[l] * scale[l >> 9];  // 512 nodes per element at N = 7
        }
#pragma unroll
    for (int u = 0; u < kLpU; ++u) {
      const int64_t g = g0 + u * step;
      if (g >= n) break;
      for (int q = 8; q < c[u]; ++q) {
        const gidx l = idx[b[u] + q];
        sc[u] += Y[l] * scale[l >> 9];
      }
      const int k = c[u];
      if (k > 0) sc[u] *= omega * (k < kRcpTable ? c_rcp[k] : __frcp_rn((float)k));
      const double rg = r[g];
      const double zg = fma(dinv[g], rg, (double)sc[u]);
      z[g] = zg;
      rz += rg * zg;
      wz += w[g] * zg;
    }
  }
  red::block_reduce_store(rz, part + blockIdx.x);
  __syncthreads();
  red::block_reduce_store(wz, part + kLpBlocks + blockIdx.x);
  if (!red::arrive_last(cnt)) return;
  const double RZ = red::sum_partials(part, gridDim.x);
  const double WZ = red::sum_partials(part + kLpBlocks, gridDim.x);
  if (threadIdx.x == 0) {
    const bool jac = learned && !(RZ > 0.0);
    S[kUseJac] = jac ? 1.0 : 0.0;
    if (!jac) {
      const double rz_old = S[kRz];
      S[kBeta] = rz_old != 0.0 ? -S[kAlpha] * WZ / rz_old : 0.0;
      S[kRz] = RZ;
    }
  }
}

// The safeguard: when lp_precond rejected the learned step, z = D^-1 r
// (lp_direction recomputes it), rz = r.z, beta from w.z.  Otherwise a no-op.
__global__ void __launch_bounds__(red::kThreads)
    lp_jacobi_fix(int64_t n, const double *__restrict__ dinv, const double *__restrict__ r,
                  const double *__restrict__ w, double *__restrict__ part, unsigned *__restrict__ cnt,
                  double *__restrict__ S) {
  if (S[kDone] != 0.0 || S[kUseJac] == 0.0) return;
  double rz = 0.0, wz = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double zg = dinv[g] * r[g];
    rz += r[g] * zg;
    wz += w[g] * zg;
  }
  red::block_reduce_store(rz, part + blockIdx.x);
  __syncthreads();
  red::block_reduce_store(wz, part + kLpBlocks + blockIdx.x);
  if (!red::arrive_last(cnt)) return;
  const double RZ = red::sum_partials(part, gridDim.x);
  const double WZ = red::sum_partials(part + kLpBlocks, gridDim.x);
  if (threadIdx.x == 0) {
    const double rz_old = S[kRz];
    S[kBeta] = rz_old != 0.0 ? -S[kAlpha] * WZ / rz_old : 0.0;
    S[kRz] = RZ;
  }
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
  int *derr = nullptr;  // device error word of the GEMM kernels (bounded waits that ran out)
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

// After a synchronising point: AX_ETIMEOUT when a GEMM wait ran out (the
// word is cleared for the next call).
ax_status gemm_status(ax_mlp *m, const char *what) {
  int h = 0;
  if (cudaMemcpy(&h, m->derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return AX_ECUDA;
  if (!h) return AX_OK;
  cudaMemset(m->derr, 0, sizeof(int));
  m->err = std::string(what) + ": a tensor-core GEMM wait timed out (code " + std::to_string(h) + ")";
  return AX_ETIMEOUT;
}

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
// (skip: optional device flag; when nonzero the three GEMMs do nothing;
// keep_z: store the pre-activations for a backward pass)
cudaError_t forward(ax_mlp *m, const __nv_bfloat16 *X, int64_t M, cudaStream_t s, const double *skip = nullptr,
                    bool keep_z = false) {
  GemmOut o1;
  o1.Cf = keep_z ? m->Z1 : nullptr; o1.Hb = m->H1; o1.bias = m->p + m->off[1]; o1.ldc = kHid; o1.skip = skip;
  cudaError_t e = tc::gemm<kEpiGelu>((int)M, kHid, kInPad, X, m->Wb[0], o1, m->derr, s);
  GemmOut o2;
  o2.Cf = keep_z ? m->Z2 : nullptr; o2.Hb = m->H2; o2.bias = m->p + m->off[3]; o2.ldc = kHid; o2.skip = skip;
  if (e == cudaSuccess) e = tc::gemm<kEpiGelu>((int)M, kHid, kHid, m->H1, m->Wb[1], o2, m->derr, s);
  GemmOut o3;
  o3.Cf = m->Y; o3.bias = m->p + m->off[5]; o3.ldc = kOut; o3.skip = skip;
  if (e == cudaSuccess) e = tc::gemm<kEpiF32>((int)M, kOut, kHid, m->H2, m->Wb[2], o3, m->derr, s);
  return e;
}

// forward + backward of M rows (M a multiple of 32): gradients into m->g; loss partials in m->part
cudaError_t forward_backward(ax_mlp *m, const __nv_bfloat16 *X, const float *T, int64_t M, cudaStream_t s) {
  cudaError_t e = forward(m, X, M, s, nullptr, true);
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
  e = tc::gemm<kEpiF32>(kOut, kHid, (int)M, m->T1, m->T2, w3, m->derr, s);
  colsum_bf16<<<gfor(kOut), 256, 0, s>>>((int)M, kOut, m->dY, g + m->off[5]);
  GemmOut d2;
  d2.Hb = m->dZ2; d2.Zin = m->Z2; d2.ldc = kHid;
  if (e == cudaSuccess) e = tc::gemm<kEpiDGelu>((int)M, kHid, kOut, m->dY, m->WTb[2], d2, m->derr, s);
  // layer 2
  tr((int)M, kHid, m->dZ2, m->T1);
  tr((int)M, kHid, m->H1, m->T2);
  GemmOut w2;
  w2.Cf = g + m->off[2]; w2.ldc = kHid;
  if (e == cudaSuccess) e = tc::gemm<kEpiF32>(kHid, kHid, (int)M, m->T1, m->T2, w2, m->derr, s);
  colsum_bf16<<<gfor(kHid), 256, 0, s>>>((int)M, kHid, m->dZ2, g + m->off[3]);
  GemmOut d1;
  d1.Hb = m->dZ1; d1.Zin = m->Z1; d1.ldc = kHid;
  if (e == cudaSuccess) e = tc::gemm<kEpiDGelu>((int)M, kHid, kHid, m->dZ2, m->WTb[1], d1, m->derr, s);
  // layer 1
  tr((int)M, kHid, m->dZ1, m->T1);
  tr((int)M, kInPad, X, m->T2);
  GemmOut w1;
  w1.Cf = g + m->off[0]; w1.ldc = kInPad;
  if (e == cudaSuccess) e = tc::gemm<kEpiF32>(kHid, kInPad, (int)M, m->T1, m->T2, w1, m->derr, s);
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
  if (e == cudaSuccess) e = tc::gemm_init();
  if (e == cudaSuccess) e = cudaMalloc(&m->derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->derr, 0, sizeof(int));
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
  return gemm_status(m, "ax_mlp_grad");
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
  return e == cudaSuccess ? gemm_status(m, "ax_mlp_train") : mcuda(m, e, "ax_mlp_train");
}

}  // extern "C"

namespace {

// Work buffers shared by ax_mlp_pairs and pcg_solve_learned.
struct LearnWork {
  int64_t n = 0, nl = 0, E = 0;
  double *r = nullptr, *w = nullptr, *z = nullptr, *p = nullptr, *bm = nullptr, *Ul = nullptr, *Yl = nullptr,
         *dinv = nullptr, *part = nullptr, *S = nullptr, *hS = nullptr;
  float *scale = nullptr;
  unsigned *cnt = nullptr;
  __nv_bfloat16 *F = nullptr;
  cudaError_t alloc(int64_t n_, int64_t nl_, int64_t E_) {
    n = n_;
    nl = nl_;
    E = E_;
    cudaError_t e = cudaMalloc(&r, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bm, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dinv, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Ul, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&Yl, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&scale, sizeof(float) * E);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 4 * kLpBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(double) * kLpScalars);
    if (e == cudaSuccess) e = cudaMemset(S, 0, sizeof(double) * kLpScalars);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&hS, sizeof(double) * kLpScalars);
    if (e == cudaSuccess) e = cudaMalloc(&F, sizeof(__nv_bfloat16) * E * kInPad);
    return e;
  }
  void release() {
    cudaFree(r); cudaFree(w); cudaFree(z); cudaFree(p); cudaFree(bm); cudaFree(dinv); cudaFree(Ul); cudaFree(Yl);
    cudaFree(scale); cudaFree(part); cudaFree(S); cudaFree(cnt); cudaFreeHost(hS); cudaFree(F);
  }
};

void delete_learn(void *p) {
  LearnWork *W = static_cast<LearnWork *>(p);
  W->release();
  delete W;
}

// The context's learned-solver work (kept between calls, freed with the context).
cudaError_t learn_work(ax_ctx *c, LearnWork **out) {
  Ctx &C = ax_ctx_core_mut(c);
  LearnWork *W = static_cast<LearnWork *>(C.ws[Ctx::kWsLearn]);
  if (!W) {
    W = new (std::nothrow) LearnWork;
    if (!W) return cudaErrorMemoryAllocation;
    cudaError_t e = W->alloc(C.gs.n_global, C.gs.n_local, C.E);
    if (e != cudaSuccess) {
      delete_learn(W);
      return e;
    }
    C.ws[Ctx::kWsLearn] = W;
    C.ws_del[Ctx::kWsLearn] = delete_learn;
  }
  *out = W;
  return cudaSuccess;
}

// the learned solver runs FP64-accurate operators only
cudaError_t (*ax_launcher(int prec))(const AxArgs &) {
  return (prec == AX_FP64 || prec == AX_F64DW) ? ax_launcher_of(prec) : nullptr;
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

// The preconditioner on the current residual W.r: U = Q r, the network on
// every element, z and beta (lp_precond).  skip: S[kMlpSkip].
cudaError_t lp_apply(const ax_ctx *c, ax_mlp *m, LearnWork &W, double omega, bool scatter, cudaStream_t s) {
  const GsPlan &P = ax_ctx_core(c).gs;
  const int64_t E = ax_ctx_core(c).E, n = P.n_global;
  const double *skip = W.S + kMlpSkip;
  if (scatter) lp_scatter<<<gfor(n), 256, 0, s>>>(n, W.r, P.off, P.idx, W.Ul);
  element_inputs<<<input_blocks(E), 32 * kInputWarps, 0, s>>>(E, nullptr, W.Ul, ax_ctx_vertices(c), W.F, W.scale, skip);
  cudaError_t e = forward(m, W.F, E, s, skip);
  if (e != cudaSuccess) return e;
  lp_precond<<<kLpBlocks, red::kThreads, 0, s>>>(n, P.off, P.idx, m->Y, W.scale, W.dinv, W.r, W.w, P.mask,
                                                 (float)omega, W.z, W.part, W.cnt + 3, W.S);
  lp_jacobi_fix<<<kLpBlocks, red::kThreads, 0, s>>>(n, W.dinv, W.r, W.w, W.part + 2 * kLpBlocks, W.cnt + 3, W.S);
  return cudaGetLastError();
}

// One flexible-PCG iteration on stream s (x: the solution vector).
cudaError_t lp_iteration(const ax_ctx *c, ax_mlp *m, LearnWork &W, double *x, double omega, cudaStream_t s) {
  const GsPlan &P = ax_ctx_core(c).gs;
  const int64_t n = P.n_global;
  lp_direction<<<gfor(n), 256, 0, s>>>(n, W.S, W.z, W.r, W.dinv, W.p, P.off, P.idx, W.Ul);
  AxArgs a = ax_ctx_args(c);
  a.X = W.Ul;
  a.Y = W.Yl;
  a.stream = s;
  cudaError_t e = ax_launcher(ax_ctx_core(c).prec)(a);
  if (e != cudaSuccess) return e;
  lp_gather<<<kLpBlocks, red::kThreads, 0, s>>>(n, P.off, P.idx, W.Yl, W.w, P.mask, W.p, W.part, W.cnt, W.S);
  lp_update<<<kLpBlocks, red::kThreads, 0, s>>>(n, W.S, W.p, W.w, x, W.r, P.off, P.idx, W.Ul, W.part, W.cnt + 1);
  return lp_apply(c, m, W, omega, false, s);
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
  LearnWork *Wp = nullptr;
  cudaError_t e = learn_work(c, &Wp);
  if (e != cudaSuccess) return mcuda(nullptr, e, "ax_mlp_pairs");
  LearnWork &W = *Wp;
  if (n > C.E) return mfail(nullptr, AX_EINVAL, "ax_mlp_pairs: more samples than elements");
  e = jacobi_inverse(c, W, s);
  if (e == cudaSuccess) e = apply_A(c, W, x_k, W.w, s);
  if (e == cudaSuccess) {
    const GsPlan &P = C.gs;
    sub_d<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, b_global, W.w, W.r, P.mask);  // r = b - A x_k
    sub_d<<<gfor(P.n_global), 256, 0, s>>>(P.n_global, x_star, x_k, W.z, P.mask);    // e = x* - x_k
    scatter_d<<<gfor(P.n_local), 256, 0, s>>>(P.n_local, P.gid, W.r, W.Ul);
    element_inputs<<<input_blocks(n), 32 * kInputWarps, 0, s>>>(n, elements, W.Ul, ax_ctx_vertices(c),
                                                                (__nv_bfloat16 *)F_bf16, W.scale, nullptr);
    element_targets<<<(unsigned)n, 256, 0, s>>>(n, elements, P.gid, W.z, W.dinv, W.Ul, W.scale, T);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
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
  constexpr int kCheck = 16;   // iterations per graph launch (between host checks)
  constexpr int kPatience = 200;
  *iters = 0;
  *relres = 0.0;
  LearnWork *Wp = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = learn_work(c, &Wp);
  if (e != cudaSuccess) return mcuda(m, e, "pcg_solve_learned");
  LearnWork &W = *Wp;
  e = ensure_cap(m, C.E);
  if (e == cudaSuccess) e = jacobi_inverse(c, W, s);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  int conv = 0;
  double bb = 0.0, rr = 0.0;
  if (e == cudaSuccess) {
    // masked x; r = b - A x (masked); p = 0; ||b||, ||r||
    e = cudaMemsetAsync(W.w, 0, sizeof(double) * n, s);
    sub_d<<<gfor(n), 256, 0, s>>>(n, x, W.w, x, P.mask);  // x = 0 on Dirichlet nodes
    if (e == cudaSuccess) e = apply_A(c, W, x, W.w, s);
    lp_init<<<kLpBlocks, red::kThreads, 0, s>>>(n, b_global, W.w, W.bm, W.r, W.p, P.mask, rtol, (double)kPatience,
                                                W.part, W.cnt + 2, W.S);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W.hS, W.S, sizeof(double) * kLpScalars, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      bb = W.hS[kBb];
      rr = W.hS[kRr];
      if (bb == 0.0 || rr <= W.hS[kTol2]) conv = 1;
    }
  }
  int it = 0;
  if (e == cudaSuccess && !conv && maxit > 0) {
    e = lp_apply(c, m, W, omega, true, s);  // z0, rz0 (beta = 0: p = z0)
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    if (e == cudaSuccess && maxit >= kCheck) {
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      for (int q = 0; q < kCheck && e == cudaSuccess; ++q) e = lp_iteration(c, m, W, x, omega, cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = ec;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    int issued = 0;
    while (e == cudaSuccess && issued < maxit) {
      const int block = (maxit - issued) < kCheck ? (maxit - issued) : kCheck;
      if (block == kCheck)
        e = cudaGraphLaunch(exec, cs);
      else
        for (int q = 0; q < block && e == cudaSuccess; ++q) e = lp_iteration(c, m, W, x, omega, cs);
      issued += block;
      if (e == cudaSuccess) e = cudaMemcpyAsync(W.hS, W.S, sizeof(double) * kLpScalars, cudaMemcpyDeviceToHost, cs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
      if (e != cudaSuccess) break;
      rr = W.hS[kRr];
      it = issued;
      if (W.hS[kDone] != 0.0) {
        conv = W.hS[kConvIt] > 0.0;
        it = (int)std::fabs(W.hS[kConvIt]);
        break;
      }
    }
    *fell_back = W.hS[kLearnOff] != 0.0 ? 1 : 0;
    const cudaError_t e2 = cudaEventRecord(ev, cs);
    if (e2 == cudaSuccess) cudaStreamWaitEvent(s, ev, 0);
    if (e == cudaSuccess) e = e2;
  }
  *iters = it;
  *relres = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  if (ev) cudaEventDestroy(ev);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) return mcuda(m, e, "pcg_solve_learned");
  const ax_status gst = gemm_status(m, "pcg_solve_learned");
  if (gst != AX_OK) return gst;
  if (!conv) return mfail(m, AX_ENOTCONV, "pcg_solve_learned: not converged");
  return AX_OK;
}

void ax_mlp_destroy(ax_mlp *m) {
  if (!m) return;
  cudaFree(m->p); cudaFree(m->g); cudaFree(m->am); cudaFree(m->av); cudaFree(m->derr);
  for (int l = 0; l < 3; ++l) {
    cudaFree(m->Wb[l]);
    cudaFree(m->WTb[l]);
  }
  cudaFree(m->Z1); cudaFree(m->Z2); cudaFree(m->Y); cudaFree(m->part);
  cudaFree(m->H1); cudaFree(m->H2); cudaFree(m->dY); cudaFree(m->dZ1); cudaFree(m->dZ2); cudaFree(m->T1); cudaFree(m->T2);
  delete m;
}

}  // extern "C"
