// AxLocal with the six sum-factorised contractions of Algorithm 1 on the
// tensor cores (mma.sync m16n8k8, operands TF32, BF16 or FP16, accumulation
// in FP32); X, Y, the geometry and (r,s,t) = G (x0,x1,x2) stay FP32.  The
// tcgen05 kernels of ax_umma.cuh run every order by default; this warp-level
// kernel is the second tile variant, which the batch autotuner compares with
// them.
//
// A contraction along direction d maps the element's N1^2 fibers of that
// direction through D (forward) or D^T (transposed).  Written as a product
// of a [fibers x N1] slab and an N1 x N1 matrix, it is a small GEMM with
// M = fibers (16 per MMA row tile), K = N = N1 padded to 8 (N1 <= 8) or 16:
//   forward    out[f][a] = sum_m x[f][m] D[a][m]   (B[k][n] = D[n][k])
//   transposed y[f][m]   = sum_a t[f][a] D[a][m]   (B[k][n] = D[k][n])
// A warp owns one (element, 16-fiber tile) unit at a time: it gathers the A
// fragments of its fibers from the padded shared element, multiplies by the
// B fragments of D held in registers for the whole kernel, and scatters the
// C fragments back.  The geometry step between the passes is the FP32 code
// of the fiber kernel (one thread per t-fiber).
//
// Shared buffers per element: x (input), and b0, b1, b2 holding x0, x1, x2,
// then r, s, t (in place), then the three transposed partial sums (in place:
// a unit reads all of its fibers' values before it writes them), summed on
// the way to HBM.  Five barriers per block of elements.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ax_fiber.cuh"
#include "ax_umma.cuh"

namespace ax {
namespace tcx {

enum Mode { kTF32 = 0, kBF16 = 1, kFP16 = 2 };

template <int N1>
struct TcShape {
  static constexpr int F = N1 * N1;                     // fibers per direction and element
  static constexpr int EPB = N1 == 6 ? fiber::pick_epb(F) : (F >= 128 ? 1 : 128 / F);  // elements per CTA
  static constexpr int GT = F * EPB;                    // geometry threads (one per t-fiber)
  static constexpr int threads = (GT + 31) / 32 * 32;   // whole warps for mma.sync
  static constexpr int warps = threads / 32;
  static constexpr int P = N1 + 1;                      // padded row
  static constexpr int ES = N1 * N1 * P;                // padded element (words)
  static constexpr int KP = N1 <= 8 ? 8 : 16;           // contraction length padded to the MMA K
  static constexpr int KS = KP / 8;                     // k steps of 8
  static constexpr int NT = KP / 8;                     // n tiles of 8
  static constexpr int FT = (F + 15) / 16;              // 16-fiber row tiles per element
  static constexpr int UNITS = EPB * FT;                // warp work units per direction
  __device__ static __forceinline__ int at(int i, int j, int k) { return i + P * (j + N1 * k); }
  // first node and stride of fiber f in direction d (0: r, 1: s, 2: t)
  __device__ static __forceinline__ int base(int d, int f) {
    return d == 0 ? P * f : (d == 1 ? (f % N1) + P * N1 * (f / N1) : (f % N1) + P * (f / N1));
  }
  __device__ static __forceinline__ int stride(int d) { return d == 0 ? 1 : (d == 1 ? P : P * N1); }
};

// ---------------------------------------------------------------------------
// fragments (PTX ISA layouts of mma.m16n8k8; g = lane / 4, t = lane % 4)
//   tf32  A: a0 (g, t) a1 (g+8, t) a2 (g, t+4) a3 (g+8, t+4);  B: b0 (t, g) b1 (t+4, g)
//   16-bit A: a0 (g, 2t..2t+1) a1 (g+8, 2t..2t+1);  B: b0 (2t..2t+1, g)  (low half: lower index)
//   C (f32): c0 c1 (g, 2t..2t+1)  c2 c3 (g+8, 2t..2t+1)
// ---------------------------------------------------------------------------
template <int MODE>
struct Frag {
  static constexpr int A = MODE == kTF32 ? 4 : 2;
  static constexpr int B = MODE == kTF32 ? 2 : 1;
};

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(v));
  return r;
}
template <int MODE>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (MODE == kBF16) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
  } else {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
  }
}

template <int MODE>
__device__ __forceinline__ void mma(float c[4], const uint32_t *a, const uint32_t *b) {
  if constexpr (MODE == kTF32) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else if constexpr (MODE == kBF16) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]));
  }
}

// B fragment of the 8 x 8 block (ks, nt) of B[k][n] = tr ? D[k][n] : D[n][k] (zero outside N1)
template <int MODE, int N1>
__device__ __forceinline__ void load_b(const float *D, bool tr, int ks, int nt, int lane, uint32_t *b) {
  const int g = lane >> 2, t = lane & 3;
  auto B = [&](int k, int n) -> float {
    if (k >= N1 || n >= N1) return 0.0f;
    return tr ? D[k * N1 + n] : D[n * N1 + k];
  };
  const int n = 8 * nt + g;
  if constexpr (MODE == kTF32) {
    b[0] = to_tf32(B(8 * ks + t, n));
    b[1] = to_tf32(B(8 * ks + t + 4, n));
  } else {
    b[0] = pack2<MODE>(B(8 * ks + 2 * t, n), B(8 * ks + 2 * t + 1, n));
  }
}

// One (element, 16-fiber tile) unit of a contraction in direction d:
// dst[fibers][0..N1) = src[fibers][0..N1) x B, with bf the B fragments.
template <int MODE, int N1>
__device__ __forceinline__ void unit(const float *src, float *dst, int d, int ft, int lane,
                                     const uint32_t (&bf)[TcShape<N1>::KS][TcShape<N1>::NT][Frag<MODE>::B]) {
  using Sh = TcShape<N1>;
  const int g = lane >> 2, t = lane & 3;
  const int f0 = 16 * ft + g, f1 = f0 + 8;
  const bool v0 = f0 < Sh::F, v1 = f1 < Sh::F;
  const int b0 = v0 ? Sh::base(d, f0) : 0, b1 = v1 ? Sh::base(d, f1) : 0, st = Sh::stride(d);
  auto ld = [&](bool v, int b, int col) -> float { return (v && col < N1) ? src[b + col * st] : 0.0f; };
  uint32_t a[Sh::KS][Frag<MODE>::A];
#pragma unroll
  for (int ks = 0; ks < Sh::KS; ++ks) {
    if constexpr (MODE == kTF32) {
      const int c0 = 8 * ks + t, c1 = c0 + 4;
      a[ks][0] = to_tf32(ld(v0, b0, c0));
      a[ks][1] = to_tf32(ld(v1, b1, c0));
      a[ks][2] = to_tf32(ld(v0, b0, c1));
      a[ks][3] = to_tf32(ld(v1, b1, c1));
    } else {
      const int c0 = 8 * ks + 2 * t;
      a[ks][0] = pack2<MODE>(ld(v0, b0, c0), ld(v0, b0, c0 + 1));
      a[ks][1] = pack2<MODE>(ld(v1, b1, c0), ld(v1, b1, c0 + 1));
    }
  }
  __syncwarp();  // every lane has read its operands before any lane writes (in-place units)
#pragma unroll
  for (int nt = 0; nt < Sh::NT; ++nt) {
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int ks = 0; ks < Sh::KS; ++ks) mma<MODE>(c, a[ks], bf[ks][nt]);
    const int col = 8 * nt + 2 * t;
    if (v0 && col < N1) dst[b0 + col * st] = c[0];
    if (v0 && col + 1 < N1) dst[b0 + (col + 1) * st] = c[1];
    if (v1 && col < N1) dst[b1 + col * st] = c[2];
    if (v1 && col + 1 < N1) dst[b1 + (col + 1) * st] = c[3];
  }
}

// Tables (per translation unit, constant memory): c_Dp plain D (float) of every order.
template <int MODE, int N1, int KIND>
__global__ void __launch_bounds__(TcShape<N1>::threads)
    ax_tc_kernel(int64_t E, const float *__restrict__ geo, const float *__restrict__ lam, const float *__restrict__ X,
                 float *__restrict__ Y, const float *__restrict__ Dp) {
  using Sh = TcShape<N1>;
  using P = fiber::Native<float>;
  constexpr int n3 = N1 * N1 * N1, EPB = Sh::EPB, ES = Sh::ES;
  constexpr int GW = fiber::GeoWords<KIND>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *xs = (float *)smem_raw;  // [EPB][ES] x
  float *bb = xs + EPB * ES;      // b0, b1, b2: [3][EPB][ES]
  __shared__ float sgeo[EPB][GW > 0 ? GW : 1];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float *cw = fiber::c_w + tab_off_v(N1);
  const float *cx = fiber::c_x + tab_off_v(N1);
  uint32_t bf[Sh::KS][Sh::NT][Frag<MODE>::B], bt[Sh::KS][Sh::NT][Frag<MODE>::B];
#pragma unroll
  for (int ks = 0; ks < Sh::KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < Sh::NT; ++nt) {
      load_b<MODE, N1>(Dp, false, ks, nt, lane, bf[ks][nt]);
      load_b<MODE, N1>(Dp, true, ks, nt, lane, bt[ks][nt]);
    }
  const int64_t nblk = (E + EPB - 1) / EPB;

  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t e0 = blk * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    // X into the padded element (row = j + N1 (k + N1 z) is also the padded
    // row): coalesced at N1 = 2, 4, 8 (row and column by shifts), one row per
    // thread elsewhere (the same rule as the fiber kernels, measured there)
    if constexpr (N1 == 2 || N1 == 4 || N1 == 8) {
      fiber::load_rows<P, N1, Sh::P, Sh::threads>(X + e0 * n3, nel * n3, xs, tid, nullptr);
    } else {
      for (int row = tid; row < nel * N1 * N1; row += Sh::threads) {
        const float *src = X + e0 * n3 + (int64_t)row * N1;
        float *dst = xs + row * Sh::P;
#pragma unroll
        for (int i = 0; i < N1; ++i) dst[i] = src[i];
      }
    }
    if constexpr (GW > 0) {
      for (int m = tid; m < nel * GW; m += Sh::threads) sgeo[m / GW][m % GW] = geo[e0 * GW + m];
    }
    __syncthreads();
    // forward: x0, x1, x2 = D_r x, D_s x, D_t x
    for (int d = 0; d < 3; ++d)
      for (int u = warp; u < Sh::UNITS; u += Sh::warps) {
        const int z = u / Sh::FT, ft = u % Sh::FT;
        if (z < nel) unit<MODE, N1>(xs + z * ES, bb + (d * EPB + z) * ES, d, ft, lane, bf);
      }
    __syncthreads();
    // geometry and (r, s, t) = G (x0, x1, x2) along each thread's t-fiber (FP32)
    if (tid < Sh::GT) {
      const int z = tid / Sh::F, q = tid % Sh::F, i = q % N1, j = q / N1;
      const bool live = z < nel;
      const int64_t e = e0 + z;
      float *r_e = bb + z * ES, *s_e = bb + (EPB + z) * ES, *t_e = bb + (2 * EPB + z) * ES;
      fiber::Geometry<P, N1, KIND> gm;
      gm.prologue(sgeo[z], cx, cw, i, j, (KIND == AX_GEOM_STORED && live) ? geo + e * 7 * n3 : nullptr,
                  (KIND == AX_GEOM_TRILINEAR_PARTIAL && live) ? lam + e * n3 : nullptr);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const int sidx = Sh::at(i, j, k);
        const float xv[3] = {r_e[sidx], s_e[sidx], t_e[sidx]};
        float o3[3] = {0.0f, 0.0f, 0.0f};
        if (live) gm.apply(i + j * N1 + k * N1 * N1, cx[k], cw[k], xv, o3);
        r_e[sidx] = o3[0];
        s_e[sidx] = o3[1];
        t_e[sidx] = o3[2];
      }
    }
    __syncthreads();
    // transposed, in place: b0 = D_r^T r, b1 = D_s^T s, b2 = D_t^T t
    for (int d = 0; d < 3; ++d)
      for (int u = warp; u < Sh::UNITS; u += Sh::warps) {
        const int z = u / Sh::FT, ft = u % Sh::FT;
        float *buf = bb + (d * EPB + z) * ES;
        if (z < nel) unit<MODE, N1>(buf, buf, d, ft, lane, bt);
      }
    __syncthreads();
    // Y = b0 + b1 + b2 to HBM (coalesced at N1 = 2, 4, 8: value m of the
    // block from row m / N1 at i = m % N1)
    if constexpr (N1 == 2 || N1 == 4 || N1 == 8) {
      float *dst = Y + e0 * n3;
      const int nvals = nel * n3;
#pragma unroll 4
      for (int s = 0; s < N1; ++s) {
        const int m = tid + s * Sh::threads;
        if (m < nvals) {
          const int row = m / N1, off = row * Sh::P + (m - row * N1);
          dst[m] = bb[off] + bb[EPB * ES + off] + bb[2 * EPB * ES + off];
        }
      }
    } else {
      for (int row = tid; row < nel * N1 * N1; row += Sh::threads) {
        float *dst = Y + e0 * n3 + (int64_t)row * N1;
        const int off = row * Sh::P;
        const float *y0 = bb + off, *y1 = bb + EPB * ES + off, *y2 = bb + 2 * EPB * ES + off;
#pragma unroll
        for (int i = 0; i < N1; ++i) dst[i] = y0[i] + y1[i] + y2[i];
      }
    }
    __syncthreads();  // the next block reuses the shared buffers
  }
}

template <int MODE, int N1, int KIND>
cudaError_t launch_tc_kind(const AxArgs &a, const float *Dp) {
  using Sh = TcShape<N1>;
  const int64_t nblk = (a.E + Sh::EPB - 1) / Sh::EPB;
  if (nblk <= 0) return cudaSuccess;
  const int64_t grid = a.grid > 0 && a.grid < nblk ? a.grid : nblk;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  const size_t smem = (size_t)4 * Sh::EPB * Sh::ES * sizeof(float);
  // per instantiation; static shared memory counts against the same 48 KB
  // default, so the attribute is set whatever the dynamic size
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(ax_tc_kernel<MODE, N1, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  ax_tc_kernel<MODE, N1, KIND><<<(unsigned)grid, Sh::threads, smem, a.stream>>>(
      a.E, (const float *)a.geo, (const float *)a.lam, (const float *)a.X, (float *)a.Y, Dp);
  return cudaGetLastError();
}

template <int MODE, int N1>
cudaError_t launch_tc_n(const AxArgs &a, const float *Dp) {
  if constexpr (N1 >= 2 && N1 != 8) {
    // every order but 7: the tcgen05 kernel sized to the order (tile
    // variant 1 selects the mma.sync kernel below)
    if (a.tile != 1) {
      switch (a.kind) {
        case AX_GEOM_STORED: return umma::launch_gen<N1, AX_GEOM_STORED, MODE>(a, Dp);
        case AX_GEOM_TRILINEAR: return umma::launch_gen<N1, AX_GEOM_TRILINEAR, MODE>(a, Dp);
        case AX_GEOM_PARALLELEPIPED: return umma::launch_gen<N1, AX_GEOM_PARALLELEPIPED, MODE>(a, Dp);
        case AX_GEOM_TRILINEAR_PARTIAL: return umma::launch_gen<N1, AX_GEOM_TRILINEAR_PARTIAL, MODE>(a, Dp);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  if constexpr (N1 == 8) {
    // order 7: tcgen05 in every format (operand format = MODE; tile variant 1
    // selects the mma.sync kernel below)
    if (a.tile != 1) {
      switch (a.kind) {
        case AX_GEOM_STORED: return umma::launch_kind<AX_GEOM_STORED, MODE>(a, Dp);
        case AX_GEOM_TRILINEAR: return umma::launch_kind<AX_GEOM_TRILINEAR, MODE>(a, Dp);
        case AX_GEOM_PARALLELEPIPED: return umma::launch_kind<AX_GEOM_PARALLELEPIPED, MODE>(a, Dp);
        case AX_GEOM_TRILINEAR_PARTIAL: return umma::launch_kind<AX_GEOM_TRILINEAR_PARTIAL, MODE>(a, Dp);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  switch (a.kind) {
    case AX_GEOM_STORED: return launch_tc_kind<MODE, N1, AX_GEOM_STORED>(a, Dp);
    case AX_GEOM_TRILINEAR: return launch_tc_kind<MODE, N1, AX_GEOM_TRILINEAR>(a, Dp);
    case AX_GEOM_PARALLELEPIPED: return launch_tc_kind<MODE, N1, AX_GEOM_PARALLELEPIPED>(a, Dp);
    case AX_GEOM_TRILINEAR_PARTIAL: return launch_tc_kind<MODE, N1, AX_GEOM_TRILINEAR_PARTIAL>(a, Dp);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tcx
}  // namespace ax
