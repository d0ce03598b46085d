// Double-word AxLocal kernels (templates); instantiated per group of orders
// by the ax_dw_g*.cu translation units through inst_dw.inc.
//
// float64 inputs/outputs, double-word (FP32-pair) arithmetic on the FP32 pipe
// (about 47 bits; see dw.cuh).  Same mapping and geometry steps as the native
// kernels (ax_native.cuh): 2-D thread layer per element, k-fiber per thread,
// one k-slice of x, r, s in shared memory, D_t from constant memory; the
// geometry of Algorithm 2 / Algorithm 3 / stored factors evaluated in
// double-word arithmetic.
#pragma once

#include <cstdint>
#include <vector>

#include "ax_internal.h"
#include "dw.cuh"
#include "tables.cuh"

namespace ax {
namespace dwk {

using dw::acc;
using ddw = dw::dw;

// c_D, c_w, c_x: constant tables (float2 hi/lo) of the including translation unit.

template <int N1>
struct Shape {
  static constexpr int n3 = N1 * N1 * N1;
  static constexpr int EPB = (N1 * N1 >= 128) ? 1 : (128 / (N1 * N1));
  static constexpr int threads = N1 * N1 * EPB;
  static constexpr int P = N1 + 1;
};

__device__ __forceinline__ ddw ld(const float2 *p) { return dw::from_float2(*p); }
__device__ __forceinline__ ddw dot3(const ddw a[3], const ddw b[3]) {
  acc s = dw::mul_acc(a[0], b[0]);
  dw::mac(s, a[1], b[1]);
  dw::mac(s, a[2], b[2]);
  return dw::fin(s);
}
// a*b - c*d
__device__ __forceinline__ ddw det2(ddw a, ddw b, ddw c, ddw d) {
  acc s = dw::mul_acc(a, b);
  dw::mac(s, dw::neg(c), d);
  return dw::fin(s);
}

template <int N1, int KIND>
struct Geometry {
  ddw E0[3], E1[3], F0[3], F1[3], J2[3], K22, wij;
  ddw h[7];
  const float2 *gl = nullptr;

  __device__ __forceinline__ void prologue(const float2 *sv, const float2 *xg, const float2 *wg, int i, int j,
                                           const float2 *G_e, const float2 *lam_e) {
    wij = dw::mul(ld(wg + i), ld(wg + j));
    if constexpr (KIND == AX_GEOM_STORED) {
      gl = G_e;
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
#pragma unroll
      for (int q = 0; q < 7; ++q) h[q] = ld(sv + q);
    } else {
      const ddw r = ld(xg + i), s = ld(xg + j);
      const ddw one = dw::make(1.0f, 0.0f), eighth = dw::make(0.125f, 0.0f);
      const ddw u0 = dw::mul(dw::sub(one, s), eighth), u1 = dw::mul(dw::add(one, s), eighth);
      const ddw v0 = dw::mul(dw::sub(one, r), eighth), v1 = dw::mul(dw::add(one, r), eighth);
      const ddw w00 = dw::mul(v0, dw::sub(one, s)), w10 = dw::mul(v1, dw::sub(one, s));
      const ddw w01 = dw::mul(v0, dw::add(one, s)), w11 = dw::mul(v1, dw::add(one, s));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        auto V = [&](int v) { return ld(sv + 3 * v + c); };
        const ddw a00 = dw::sub(V(1), V(0)), a10 = dw::sub(V(3), V(2));
        const ddw a01 = dw::sub(V(5), V(4)), a11 = dw::sub(V(7), V(6));
        const ddw b00 = dw::sub(V(2), V(0)), b10 = dw::sub(V(3), V(1));
        const ddw b01 = dw::sub(V(6), V(4)), b11 = dw::sub(V(7), V(5));
        const ddw c00 = dw::sub(V(4), V(0)), c10 = dw::sub(V(5), V(1));
        const ddw c01 = dw::sub(V(6), V(2)), c11 = dw::sub(V(7), V(3));
        E0[c] = dw::add(dw::mul(u0, dw::add(a00, a01)), dw::mul(u1, dw::add(a10, a11)));
        E1[c] = dw::add(dw::mul(u0, dw::sub(a01, a00)), dw::mul(u1, dw::sub(a11, a10)));
        F0[c] = dw::add(dw::mul(v0, dw::add(b00, b01)), dw::mul(v1, dw::add(b10, b11)));
        F1[c] = dw::add(dw::mul(v0, dw::sub(b01, b00)), dw::mul(v1, dw::sub(b11, b10)));
        acc q = dw::mul_acc(w00, c00);
        dw::mac(q, w10, c10);
        dw::mac(q, w01, c01);
        dw::mac(q, w11, c11);
        J2[c] = dw::fin(q);
      }
      K22 = dot3(J2, J2);
      gl = lam_e;
    }
  }

  // g[0..5] at node (i,j,k) (local index l); returns w|J|.
  __device__ __forceinline__ ddw at(int l, ddw t, ddw wk, ddw g[6]) const {
    constexpr int n3 = N1 * N1 * N1;
    if constexpr (KIND == AX_GEOM_STORED) {
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = ld(gl + q * n3 + l);
      return ld(gl + 6 * n3 + l);
    } else if constexpr (KIND == AX_GEOM_PARALLELEPIPED) {
      const ddw W = dw::mul(wij, wk);
#pragma unroll
      for (int q = 0; q < 6; ++q) g[q] = dw::mul(W, h[q]);
      return dw::mul(W, h[6]);
    } else {
      ddw J0[3], J1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        J0[c] = dw::add(E0[c], dw::mul(t, E1[c]));
        J1[c] = dw::add(F0[c], dw::mul(t, F1[c]));
      }
      const ddw K00 = dot3(J0, J0), K01 = dot3(J0, J1), K02 = dot3(J0, J2);
      const ddw K11 = dot3(J1, J1), K12 = dot3(J1, J2);
      const ddw A00 = det2(K11, K22, K12, K12);
      const ddw A01 = det2(K02, K12, K01, K22);
      const ddw A02 = det2(K01, K12, K02, K11);
      const ddw A11 = det2(K00, K22, K02, K02);
      const ddw A12 = det2(K01, K02, K00, K12);
      const ddw A22 = det2(K00, K11, K01, K01);
      const ddw W = dw::mul(wij, wk);
      ddw lam, wdet;
      if constexpr (KIND == AX_GEOM_TRILINEAR) {
        ddw cr[3];
        cr[0] = det2(J1[1], J2[2], J1[2], J2[1]);
        cr[1] = det2(J1[2], J2[0], J1[0], J2[2]);
        cr[2] = det2(J1[0], J2[1], J1[1], J2[0]);
        const ddw det = dot3(J0, cr);
        lam = dw::div(W, det);
        wdet = dw::mul(W, det);
      } else {
        lam = ld(gl + l);
        wdet = dw::div(dw::mul(W, W), lam);
      }
      g[0] = dw::mul(lam, A00); g[1] = dw::mul(lam, A01); g[2] = dw::mul(lam, A02);
      g[3] = dw::mul(lam, A11); g[4] = dw::mul(lam, A12); g[5] = dw::mul(lam, A22);
      return wdet;
    }
  }
};

template <int N1, int KIND>
__global__ void __launch_bounds__(Shape<N1>::threads)
    ax_dw_kernel(int64_t E, const float2 *__restrict__ geo, const float2 *__restrict__ lam,
                 const double *__restrict__ X, double *__restrict__ Y) {
  using S = Shape<N1>;
  constexpr int n3 = S::n3, EPB = S::EPB, P = S::P;
  constexpr int GW = (KIND == AX_GEOM_STORED) ? 0 : (KIND == AX_GEOM_PARALLELEPIPED ? kParWords : kVertexWords);
  __shared__ float2 sD[N1][P];
  __shared__ float2 sx[EPB][N1][P];
  __shared__ float2 sr[EPB][N1][P];
  __shared__ float2 ss[EPB][N1][P];
  __shared__ float2 sgeo[EPB][GW > 0 ? GW : 1];

  const int i = threadIdx.x, j = threadIdx.y, z = threadIdx.z;
  const int tid = i + N1 * (j + N1 * z);
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int64_t e = e0 + z;
  const bool live = e < E;
  const float2 *cD = c_D + tab_off_D(N1);
  const float2 *cw = c_w + tab_off_v(N1);
  const float2 *cx = c_x + tab_off_v(N1);

  for (int q = tid; q < N1 * N1; q += S::threads) sD[q / N1][q % N1] = cD[q];
  if constexpr (GW > 0) {
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int q = tid; q < nel * GW; q += S::threads) sgeo[q / GW][q % GW] = geo[e0 * GW + q];
  }
  ddw xf[N1];
  acc y[N1];
  const int64_t base = e * n3 + i + j * N1;
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    xf[k] = dw::from_double(live ? X[base + k * N1 * N1] : 0.0);
    y[k] = dw::acc_zero();
  }
  __syncthreads();

  Geometry<N1, KIND> gm;
  gm.prologue(sgeo[z], cx, cw, i, j, (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * n3 : nullptr,
              (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * n3 : nullptr);

#pragma unroll
  for (int k = 0; k < N1; ++k) {
    sx[z][j][i] = make_float2(xf[k].hi, xf[k].lo);
    __syncthreads();
    acc a0 = dw::acc_zero(), a1 = dw::acc_zero(), a2 = dw::acc_zero();
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      dw::mac(a0, dw::from_float2(sD[i][n]), dw::from_float2(sx[z][j][n]));
      dw::mac(a1, dw::from_float2(sD[j][n]), dw::from_float2(sx[z][n][i]));
      dw::mac(a2, dw::from_float2(cD[k * N1 + n]), xf[n]);
    }
    ddw xg[3] = {dw::fin(a0), dw::fin(a1), dw::fin(a2)};
    ddw g[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) g[q] = dw::make(0.0f, 0.0f);
    if (live) gm.at(i + j * N1 + k * N1 * N1, ld(cx + k), ld(cw + k), g);
    const ddw gr[3] = {g[0], g[1], g[2]}, gs[3] = {g[1], g[3], g[4]}, gt[3] = {g[2], g[4], g[5]};
    const ddw r = dot3(gr, xg), s = dot3(gs, xg), t = dot3(gt, xg);
    sr[z][j][i] = make_float2(r.hi, r.lo);
    ss[z][j][i] = make_float2(s.hi, s.lo);
    __syncthreads();
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      dw::mac(y[k], dw::from_float2(sD[n][i]), dw::from_float2(sr[z][j][n]));
      dw::mac(y[k], dw::from_float2(sD[n][j]), dw::from_float2(ss[z][n][i]));
      dw::mac(y[n], dw::from_float2(cD[k * N1 + n]), t);
    }
  }
  if (live) {
#pragma unroll
    for (int k = 0; k < N1; ++k) Y[base + k * N1 * N1] = dw::to_double(dw::fin(y[k]));
  }
}

template <int N1, int KIND>
__global__ void __launch_bounds__(Shape<N1>::threads)
    factors_dw_kernel(int64_t E, const float2 *__restrict__ geo, const float2 *__restrict__ lam, double *__restrict__ G) {
  using S = Shape<N1>;
  constexpr int n3 = S::n3, EPB = S::EPB;
  constexpr int GW = (KIND == AX_GEOM_STORED) ? 0 : (KIND == AX_GEOM_PARALLELEPIPED ? kParWords : kVertexWords);
  __shared__ float2 sgeo[EPB][GW > 0 ? GW : 1];
  const int i = threadIdx.x, j = threadIdx.y, z = threadIdx.z;
  const int tid = i + N1 * (j + N1 * z);
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int64_t e = e0 + z;
  const bool live = e < E;
  const float2 *cw = c_w + tab_off_v(N1);
  const float2 *cx = c_x + tab_off_v(N1);
  if constexpr (GW > 0) {
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int q = tid; q < nel * GW; q += S::threads) sgeo[q / GW][q % GW] = geo[e0 * GW + q];
  }
  __syncthreads();
  if (!live) return;
  Geometry<N1, KIND> gm;
  gm.prologue(sgeo[z], cx, cw, i, j, KIND == AX_GEOM_STORED ? geo + e * 7 * n3 : nullptr,
              KIND == AX_GEOM_TRILINEAR_PARTIAL ? lam + e * n3 : nullptr);
  for (int k = 0; k < N1; ++k) {
    const int l = i + j * N1 + k * N1 * N1;
    ddw g[6];
    const ddw gwj = gm.at(l, ld(cx + k), ld(cw + k), g);
    for (int q = 0; q < 6; ++q) G[(e * 7 + q) * n3 + l] = dw::to_double(g[q]);
    G[(e * 7 + 6) * n3 + l] = dw::to_double(gwj);
  }
}

template <int N1, int KIND>
cudaError_t launch_n(const AxArgs &a, double *G_out) {
  using S = Shape<N1>;
  const int64_t blocks = (a.E + S::EPB - 1) / S::EPB;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 block(N1, N1, S::EPB);
  if (G_out)
    factors_dw_kernel<N1, KIND><<<(unsigned)blocks, block, 0, a.stream>>>(a.E, (const float2 *)a.geo,
                                                                           (const float2 *)a.lam, G_out);
  else
    ax_dw_kernel<N1, KIND><<<(unsigned)blocks, block, 0, a.stream>>>(a.E, (const float2 *)a.geo,
                                                                      (const float2 *)a.lam, (const double *)a.X,
                                                                      (double *)a.Y);
  return cudaGetLastError();
}

template <int N1>
cudaError_t launch_kinds(const AxArgs &a, double *G_out) {
  switch (a.kind) {
    case AX_GEOM_STORED: return launch_n<N1, AX_GEOM_STORED>(a, G_out);
    case AX_GEOM_TRILINEAR: return launch_n<N1, AX_GEOM_TRILINEAR>(a, G_out);
    case AX_GEOM_PARALLELEPIPED: return launch_n<N1, AX_GEOM_PARALLELEPIPED>(a, G_out);
    case AX_GEOM_TRILINEAR_PARTIAL: return launch_n<N1, AX_GEOM_TRILINEAR_PARTIAL>(a, G_out);
    default: return cudaErrorInvalidValue;
  }
}

// Upload this translation unit's constant tables (double-word pairs) once per device.
inline cudaError_t upload_dw_tables_impl(UploadOnce &once, const void *symD, const void *symw, const void *symx) {
  std::lock_guard<std::mutex> lock(once.mu);
  int device = 0;
  cudaError_t err = cudaGetDevice(&device);
  if (err != cudaSuccess) return err;
  if (device < 64 && (once.done >> device) & 1ull) return cudaSuccess;
  std::vector<double> D(kTabD), w(kTabV), x(kTabV);
  if (!build_packed_tables(D.data(), w.data(), x.data())) return cudaErrorInvalidValue;
  std::vector<float2> D2(kTabD), w2(kTabV), x2(kTabV);
  auto split = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  for (int q = 0; q < kTabD; ++q) D2[q] = split(D[q]);
  for (int q = 0; q < kTabV; ++q) {
    w2[q] = split(w[q]);
    x2[q] = split(x[q]);
  }
  err = cudaMemcpyToSymbol(symD, D2.data(), kTabD * sizeof(float2));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(symw, w2.data(), kTabV * sizeof(float2));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(symx, x2.data(), kTabV * sizeof(float2));
  if (err == cudaSuccess && device < 64) once.done |= 1ull << device;
  return err;
}

}  // namespace dwk
}  // namespace ax
