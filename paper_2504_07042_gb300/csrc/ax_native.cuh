// AxLocal kernels in native arithmetic (T = double on the FP64 pipe, or
// T = float on the FP32 pipe).  Included by exactly one .cu per T.
//
// Mapping (Sec. 4.1, Algorithm 4, kept because it still fits sm_103a): a CTA
// holds EPB elements; thread (i,j) of element z owns the k-fiber X[i,j,:] in
// registers and walks k; one k-slice of x and of the intermediates r, s lives
// in shared memory at a time.  Per k-layer:
//   x0 = sum_n D[i][n] x[n,j,k]   x1 = sum_n D[j][n] x[i,n,k]   x2 = sum_n D[k][n] x[i,j,n]
//   (r,s,t) = G (x0,x1,x2)                                    (Algorithm 1, a4)
//   y[i,j,k] += sum_n D[n][i] r[n,j,k] + sum_n D[n][j] s[i,n,k]
//   y[i,j,n] += D[k][n] t[i,j,k]  for all n       (D_t^T accumulated along k)
// The D_t rows are uniform across the CTA and come from constant memory
// (Sec. 4.3.1); the per-thread rows/columns D[i][:], D[j][:] from shared memory.
//
// Geometry (getFactors of Algorithm 4) by kind:
//   STORED          g_q = G[e][q][node]                        (6 loads / node)
//   PARALLELEPIPED  g_q = w_i w_j w_k h_q[e]                   (Algorithm 3)
//   TRILINEAR       Algorithm 2 with the true Jacobian: columns
//                     J0 = E0[j] + t E1[j], J1 = F0[i] + t F1[i], J2 = Jc2[i,j],
//                   K = J^T J, G = (w_i w_j w_k / det J) adj(K)   (Eq. 12)
//   PARTIAL         as TRILINEAR with the per-node scalar w/det J read from HBM
//                   (Sec. 4.2.2), so no division in the kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ax_internal.h"
#include "tables.cuh"

namespace ax {
namespace native {

template <int N1>
struct Shape {
  static constexpr int n3 = N1 * N1 * N1;
  static constexpr int EPB = (N1 * N1 >= 128) ? 1 : (128 / (N1 * N1));
  static constexpr int threads = N1 * N1 * EPB;
  static constexpr int P = N1 + 1;  // padded row length of shared 2-D arrays
};

// Per-element geometry prologue + per-node factors, by kind.
template <typename T, int N1, int KIND>
struct Geometry {
  // trilinear state
  T E0[3], E1[3], F0[3], F1[3], J2[3], K22;
  T wij;
  T h[7];
  const T *gl = nullptr;  // stored factors of this element, or lam of this element

  __device__ __forceinline__ void prologue(const T *sv, const T *xg, const T *wg, int i, int j, const T *G_e,
                                           const T *lam_e) {
    constexpr int n3 = Shape<N1>::n3;
    wij = wg[i] * wg[j];
    if constexpr (KIND == AX_GEOM_STORED) {
      gl = G_e;
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
#pragma unroll
      for (int q = 0; q < 7; ++q) h[q] = sv[q];
    } else {
      (void)n3;
      const T r = xg[i], s = xg[j];
      const T u0 = (T(1) - s) * T(0.125), u1 = (T(1) + s) * T(0.125);
      const T v0 = (T(1) - r) * T(0.125), v1 = (T(1) + r) * T(0.125);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // edges along r (a_bc), s (b_ac), t (c_ab); V[v][c] at sv[3 v + c]
        const T a00 = sv[3 * 1 + c] - sv[3 * 0 + c], a10 = sv[3 * 3 + c] - sv[3 * 2 + c];
        const T a01 = sv[3 * 5 + c] - sv[3 * 4 + c], a11 = sv[3 * 7 + c] - sv[3 * 6 + c];
        const T b00 = sv[3 * 2 + c] - sv[3 * 0 + c], b10 = sv[3 * 3 + c] - sv[3 * 1 + c];
        const T b01 = sv[3 * 6 + c] - sv[3 * 4 + c], b11 = sv[3 * 7 + c] - sv[3 * 5 + c];
        const T c00 = sv[3 * 4 + c] - sv[3 * 0 + c], c10 = sv[3 * 5 + c] - sv[3 * 1 + c];
        const T c01 = sv[3 * 6 + c] - sv[3 * 2 + c], c11 = sv[3 * 7 + c] - sv[3 * 3 + c];
        E0[c] = u0 * (a00 + a01) + u1 * (a10 + a11);
        E1[c] = u0 * (a01 - a00) + u1 * (a11 - a10);
        F0[c] = v0 * (b00 + b01) + v1 * (b10 + b11);
        F1[c] = v0 * (b01 - b00) + v1 * (b11 - b10);
        J2[c] = T(0.125) * ((T(1) - r) * (T(1) - s) * c00 + (T(1) + r) * (T(1) - s) * c10 +
                            (T(1) - r) * (T(1) + s) * c01 + (T(1) + r) * (T(1) + s) * c11);
      }
      K22 = J2[0] * J2[0] + J2[1] * J2[1] + J2[2] * J2[2];
      gl = lam_e;
    }
  }

  // factors g[0..5] = g00 g01 g02 g11 g12 g22 at node (i,j,k), local index l;
  // returns w|J| (the seventh factor) for the factor export.
  __device__ __forceinline__ T at(int k, int l, T t, T wk, T g[6]) const {
    constexpr int n3 = Shape<N1>::n3;
    if constexpr (KIND == AX_GEOM_STORED) {
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = gl[q * n3 + l];
      return gl[6 * n3 + l];
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
      const T W = wij * wk;
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = W * h[q];
      return W * h[6];
    } else {
      T J0[3], J1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        J0[c] = E0[c] + t * E1[c];
        J1[c] = F0[c] + t * F1[c];
      }
      const T K00 = J0[0] * J0[0] + J0[1] * J0[1] + J0[2] * J0[2];
      const T K01 = J0[0] * J1[0] + J0[1] * J1[1] + J0[2] * J1[2];
      const T K02 = J0[0] * J2[0] + J0[1] * J2[1] + J0[2] * J2[2];
      const T K11 = J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2];
      const T K12 = J1[0] * J2[0] + J1[1] * J2[1] + J1[2] * J2[2];
      const T A00 = K11 * K22 - K12 * K12;
      const T A01 = K02 * K12 - K01 * K22;
      const T A02 = K01 * K12 - K02 * K11;
      const T A11 = K00 * K22 - K02 * K02;
      const T A12 = K01 * K02 - K00 * K12;
      const T A22 = K00 * K11 - K01 * K01;
      T lam, wdet;
      if constexpr (KIND == AX_GEOM_TRILINEAR) {
        // det J = J0 . (J1 x J2)
        const T det = J0[0] * (J1[1] * J2[2] - J1[2] * J2[1]) + J0[1] * (J1[2] * J2[0] - J1[0] * J2[2]) +
                      J0[2] * (J1[0] * J2[1] - J1[1] * J2[0]);
        const T W = wij * wk;
        lam = W / det;
        wdet = W * det;
      } else {
        lam = gl[l];
        const T W = wij * wk;
        wdet = W * W / lam;
      }
      g[0] = lam * A00; g[1] = lam * A01; g[2] = lam * A02;
      g[3] = lam * A11; g[4] = lam * A12; g[5] = lam * A22;
      return wdet;
    }
  }
};


// ---------------------------------------------------------------------------
// The kernels reference the constant tables c_D, c_w, c_x of the including
// translation unit (declared there with element type T before this header).
// ---------------------------------------------------------------------------
template <typename T, int N1, int KIND>
__global__ void __launch_bounds__(Shape<N1>::threads)
    ax_native_kernel(int64_t E, const T *__restrict__ geo, const T *__restrict__ lam, const T *__restrict__ X,
                     T *__restrict__ Y) {
  using S = Shape<N1>;
  constexpr int n3 = S::n3, EPB = S::EPB, P = S::P;
  constexpr int GW = (KIND == AX_GEOM_STORED) ? 0 : (KIND == AX_GEOM_PARALLELEPIPED ? kParWords : kVertexWords);
  __shared__ T sD[N1][P];
  __shared__ T sx[EPB][N1][P];
  __shared__ T sr[EPB][N1][P];
  __shared__ T ss[EPB][N1][P];
  __shared__ T sgeo[EPB][GW > 0 ? GW : 1];

  const int i = threadIdx.x, j = threadIdx.y, z = threadIdx.z;
  const int tid = i + N1 * (j + N1 * z);
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int64_t e = e0 + z;
  const bool live = e < E;
  const T *cD = c_D + tab_off_D(N1);
  const T *cw = c_w + tab_off_v(N1);
  const T *cx = c_x + tab_off_v(N1);

  for (int q = tid; q < N1 * N1; q += S::threads) sD[q / N1][q % N1] = cD[q];
  if constexpr (GW > 0) {
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int q = tid; q < nel * GW; q += S::threads) sgeo[q / GW][q % GW] = geo[e0 * GW + q];
  }
  T xf[N1], y[N1];
  const int64_t base = e * n3 + i + j * N1;
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    xf[k] = live ? X[base + k * N1 * N1] : T(0);
    y[k] = T(0);
  }
  __syncthreads();

  Geometry<T, N1, KIND> gm;
  gm.prologue(sgeo[z], cx, cw, i, j, (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * n3 : nullptr,
              (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * n3 : nullptr);

#pragma unroll
  for (int k = 0; k < N1; ++k) {
    sx[z][j][i] = xf[k];
    __syncthreads();
    T x0 = T(0), x1 = T(0), x2 = T(0);
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      x0 += sD[i][n] * sx[z][j][n];
      x1 += sD[j][n] * sx[z][n][i];
      x2 += cD[k * N1 + n] * xf[n];
    }
    T g[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (live) gm.at(k, i + j * N1 + k * N1 * N1, cx[k], cw[k], g);
    const T r = g[0] * x0 + g[1] * x1 + g[2] * x2;
    const T s = g[1] * x0 + g[3] * x1 + g[4] * x2;
    const T t = g[2] * x0 + g[4] * x1 + g[5] * x2;
    sr[z][j][i] = r;
    ss[z][j][i] = s;
    __syncthreads();
    T acc = T(0);
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      acc += sD[n][i] * sr[z][j][n];
      acc += sD[n][j] * ss[z][n][i];
      y[n] += cD[k * N1 + n] * t;
    }
    y[k] += acc;
  }
  if (live) {
#pragma unroll
    for (int k = 0; k < N1; ++k) Y[base + k * N1 * N1] = y[k];
  }
}

// Factor export through the same geometry code: G_out [E][7][n3] float64.
template <typename T, int N1, int KIND>
__global__ void __launch_bounds__(Shape<N1>::threads)
    factors_native_kernel(int64_t E, const T *__restrict__ geo, const T *__restrict__ lam, double *__restrict__ G) {
  using S = Shape<N1>;
  constexpr int n3 = S::n3, EPB = S::EPB;
  constexpr int GW = (KIND == AX_GEOM_STORED) ? 0 : (KIND == AX_GEOM_PARALLELEPIPED ? kParWords : kVertexWords);
  __shared__ T sgeo[EPB][GW > 0 ? GW : 1];
  const int i = threadIdx.x, j = threadIdx.y, z = threadIdx.z;
  const int tid = i + N1 * (j + N1 * z);
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int64_t e = e0 + z;
  const bool live = e < E;
  const T *cw = c_w + tab_off_v(N1);
  const T *cx = c_x + tab_off_v(N1);
  if constexpr (GW > 0) {
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int q = tid; q < nel * GW; q += S::threads) sgeo[q / GW][q % GW] = geo[e0 * GW + q];
  }
  __syncthreads();
  if (!live) return;
  Geometry<T, N1, KIND> gm;
  gm.prologue(sgeo[z], cx, cw, i, j, KIND == AX_GEOM_STORED ? geo + e * 7 * n3 : nullptr,
              KIND == AX_GEOM_TRILINEAR_PARTIAL ? lam + e * n3 : nullptr);
  for (int k = 0; k < N1; ++k) {
    const int l = i + j * N1 + k * N1 * N1;
    T g[6];
    const T gwj = gm.at(k, l, cx[k], cw[k], g);
    for (int q = 0; q < 6; ++q) G[(e * 7 + q) * n3 + l] = (double)g[q];
    G[(e * 7 + 6) * n3 + l] = (double)gwj;
  }
}

template <typename T, int N1, int KIND>
cudaError_t launch_native_n(const AxArgs &a, double *G_out) {
  using S = Shape<N1>;
  const int64_t blocks = (a.E + S::EPB - 1) / S::EPB;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 block(N1, N1, S::EPB);
  if (G_out)
    factors_native_kernel<T, N1, KIND><<<(unsigned)blocks, block, 0, a.stream>>>(
        a.E, (const T *)a.geo, (const T *)a.lam, G_out);
  else
    ax_native_kernel<T, N1, KIND><<<(unsigned)blocks, block, 0, a.stream>>>(
        a.E, (const T *)a.geo, (const T *)a.lam, (const T *)a.X, (T *)a.Y);
  return cudaGetLastError();
}

// All geometry kinds for one order (one translation unit instantiates a few orders).
template <typename T, int N1>
cudaError_t launch_native_kinds(const AxArgs &a, double *G_out) {
  switch (a.kind) {
    case AX_GEOM_STORED: return launch_native_n<T, N1, AX_GEOM_STORED>(a, G_out);
    case AX_GEOM_TRILINEAR: return launch_native_n<T, N1, AX_GEOM_TRILINEAR>(a, G_out);
    case AX_GEOM_PARALLELEPIPED: return launch_native_n<T, N1, AX_GEOM_PARALLELEPIPED>(a, G_out);
    case AX_GEOM_TRILINEAR_PARTIAL: return launch_native_n<T, N1, AX_GEOM_TRILINEAR_PARTIAL>(a, G_out);
    default: return cudaErrorInvalidValue;
  }
}

// Upload constant tables (converted to T) once per device.  The symbols are
// passed in: every translation unit has its own static copies, and this
// function is shared between them.
template <typename T>
cudaError_t upload_native_tables(UploadOnce &once, const void *symD, const void *symw, const void *symx) {
  std::lock_guard<std::mutex> lock(once.mu);
  int device = 0;
  cudaError_t err = cudaGetDevice(&device);
  if (err != cudaSuccess) return err;
  if (device < 64 && (once.done >> device) & 1ull) return cudaSuccess;
  std::vector<double> D(kTabD), w(kTabV), x(kTabV);
  if (!build_packed_tables(D.data(), w.data(), x.data())) return cudaErrorInvalidValue;
  std::vector<T> Dt(kTabD), wt(kTabV), xt(kTabV);
  for (int q = 0; q < kTabD; ++q) Dt[q] = (T)D[q];
  for (int q = 0; q < kTabV; ++q) { wt[q] = (T)w[q]; xt[q] = (T)x[q]; }
  err = cudaMemcpyToSymbol(symD, Dt.data(), kTabD * sizeof(T));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(symw, wt.data(), kTabV * sizeof(T));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(symx, xt.data(), kTabV * sizeof(T));
  if (err == cudaSuccess && device < 64) once.done |= 1ull << device;
  return err;
}

}  // namespace native
}  // namespace ax
