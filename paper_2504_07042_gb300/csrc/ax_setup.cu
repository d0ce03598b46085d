// Setup-stage kernels (FP64 arithmetic; run once per context):
//   - validation: det J > 0 at every GLL node (analytic trilinear Jacobian),
//   - STORED: the seven factors per node from the standard discrete Jacobian
//     of Sec. 3.2 (nodal coordinates, then the discrete gradient D of
//     Table 1), then Eq. 7,
//   - PARALLELEPIPED: h0..h6 of Algorithm 3 from the constant Jacobian, plus
//     a check that every element is affine,
//   - TRILINEAR kinds: vertex coordinates relative to vertex 0 (24 words),
//   - PARTIAL: the per-node scalar w_i w_j w_k / det J (Sec. 4.2.2),
//   - node coordinates (Eq. 8 at the GLL points).
// Results are written in the storage format of the context's precision:
// float64, float32, or a double-word pair (float hi, float lo).
#include <cstdint>

#include "ax_internal.h"
#include "tables.cuh"

namespace ax {
namespace setup {

static __constant__ double c_D[kTabD];
static __constant__ double c_w[kTabV];
static __constant__ double c_x[kTabV];

enum Store { kF64 = 0, kF32 = 1, kDW = 2 };

// Write v in the storage format.  FP32-based formats: values above 1e30 are
// counted as out of range (products of them could overflow); values below
// 1e-30 are stored as zero (an absolute error far below the tolerances).
__device__ __forceinline__ void store(void *base, int64_t idx, double v, int fmt, int *flags) {
  if (fmt == kF64) {
    ((double *)base)[idx] = v;
    return;
  }
  const double a = fabs(v);
  if (!(a <= 1e30)) atomicAdd(&flags[2], 1);
  if (a < 1e-30) v = 0.0;
  if (fmt == kF32) {
    ((float *)base)[idx] = (float)v;
  } else {
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    ((float2 *)base)[idx] = make_float2(hi, lo);
  }
}

// Trilinear map (Eq. 8) at reference point (r,s,t).
__device__ void map_point(const double *V, double r, double s, double t, double X[3]) {
  for (int c = 0; c < 3; ++c) X[c] = 0.0;
  for (int v = 0; v < 8; ++v) {
    const double wv = (1.0 + ((v & 1) ? r : -r)) * (1.0 + ((v & 2) ? s : -s)) * (1.0 + ((v & 4) ? t : -t)) * 0.125;
    for (int c = 0; c < 3; ++c) X[c] += wv * V[3 * v + c];
  }
}

// Analytic Jacobian of the trilinear map, J[c][d] = d x_c / d ref_d.
__device__ void map_jacobian(const double *V, double r, double s, double t, double J[9]) {
  for (int q = 0; q < 9; ++q) J[q] = 0.0;
  for (int v = 0; v < 8; ++v) {
    const double sr = (v & 1) ? 1.0 : -1.0, ss = (v & 2) ? 1.0 : -1.0, st = (v & 4) ? 1.0 : -1.0;
    const double fr = 1.0 + sr * r, fs = 1.0 + ss * s, ft = 1.0 + st * t;
    const double d[3] = {sr * fs * ft * 0.125, fr * ss * ft * 0.125, fr * fs * st * 0.125};
    for (int c = 0; c < 3; ++c)
      for (int q = 0; q < 3; ++q) J[3 * c + q] += d[q] * V[3 * v + c];
  }
}

__device__ double det3(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

// G = W |J| J^-1 J^-T = W adj(J) adj(J)^T / det J  (6 entries), gwj = W det J.
__device__ void factors_from_J(const double J[9], double W, double g[7]) {
  const double det = det3(J);
  double A[9];  // adjugate (transpose of the cofactor matrix): J^-1 = A / det
  A[0] = J[4] * J[8] - J[5] * J[7];
  A[1] = J[2] * J[7] - J[1] * J[8];
  A[2] = J[1] * J[5] - J[2] * J[4];
  A[3] = J[5] * J[6] - J[3] * J[8];
  A[4] = J[0] * J[8] - J[2] * J[6];
  A[5] = J[2] * J[3] - J[0] * J[5];
  A[6] = J[3] * J[7] - J[4] * J[6];
  A[7] = J[1] * J[6] - J[0] * J[7];
  A[8] = J[0] * J[4] - J[1] * J[3];
  const int pr[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  for (int q = 0; q < 6; ++q) {
    const int p = pr[q][0], m = pr[q][1];
    const double dot = A[3 * p] * A[3 * m] + A[3 * p + 1] * A[3 * m + 1] + A[3 * p + 2] * A[3 * m + 2];
    g[q] = W * dot / det;
  }
  g[6] = W * det;
}

// Element extents the FP32-based formats (float32, double-word pairs) handle
// at full accuracy: the trilinear geometry forms products of up to four
// Jacobian entries (adj(J^T J)); with entries of size L/2 these stay inside
// float32's normal range, low words and error terms included, for element
// extents L in [2^-20, 2^24] (adj ~ L^4 between about 2^-84 and 2^92).
constexpr double kMinExtent = 0x1p-20, kMaxExtent = 0x1p24;

// One thread per node.  flags[0] += nodes with det J <= 0; for the
// FP32-based formats flags[3] += elements whose extent (largest vertex
// coordinate difference from vertex 0) lies outside [kMinExtent, kMaxExtent].
__global__ void validate_kernel(int64_t E, int N1, const double *__restrict__ V, int fmt, int *flags) {
  const int64_t n3 = (int64_t)N1 * N1 * N1;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * n3) return;
  const int64_t e = gidx / n3;
  const int l = (int)(gidx % n3), i = l % N1, j = (l / N1) % N1, k = l / (N1 * N1);
  const double *cx = c_x + tab_off_v(N1);
  double J[9];
  map_jacobian(V + 24 * e, cx[i], cx[j], cx[k], J);
  if (!(det3(J) > 0.0)) atomicAdd(&flags[0], 1);
  if (fmt != kF64 && l == 0) {
    const double *Ve = V + 24 * e;
    double ext = 0.0;
    for (int v = 1; v < 8; ++v)
      for (int c = 0; c < 3; ++c) ext = fmax(ext, fabs(Ve[3 * v + c] - Ve[c]));
    if (!(ext >= kMinExtent && ext <= kMaxExtent)) atomicAdd(&flags[3], 1);
  }
}

// STORED: discrete Jacobian of Sec. 3.2 -- the derivative along each reference
// direction is D applied to the nodal coordinates on the line through the node.
__global__ void stored_factors_kernel(int64_t E, int N1, const double *__restrict__ V, void *G, int fmt, int *flags) {
  const int64_t n3 = (int64_t)N1 * N1 * N1;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * n3) return;
  const int64_t e = gidx / n3;
  const int l = (int)(gidx % n3), i = l % N1, j = (l / N1) % N1, k = l / (N1 * N1);
  const double *cD = c_D + tab_off_D(N1), *cx = c_x + tab_off_v(N1), *cw = c_w + tab_off_v(N1);
  const double *Ve = V + 24 * e;
  double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int n = 0; n < N1; ++n) {
    double Xr[3], Xs[3], Xt[3];
    map_point(Ve, cx[n], cx[j], cx[k], Xr);
    map_point(Ve, cx[i], cx[n], cx[k], Xs);
    map_point(Ve, cx[i], cx[j], cx[n], Xt);
    for (int c = 0; c < 3; ++c) {
      J[3 * c + 0] += cD[i * N1 + n] * Xr[c];
      J[3 * c + 1] += cD[j * N1 + n] * Xs[c];
      J[3 * c + 2] += cD[k * N1 + n] * Xt[c];
    }
  }
  double g[7];
  factors_from_J(J, cw[i] * cw[j] * cw[k], g);
  for (int q = 0; q < 7; ++q) store(G, (e * 7 + q) * n3 + l, g[q], fmt, flags);
}

// Vertices relative to vertex 0 (24 words per element; row 0 is zero).
// TRILINEAR record: the trilinear map of Eq. 8 written in the monomial basis,
//   x(r,s,t) = x0 + A r + B s + C t + D rs + E rt + F st + G rst,
// each coefficient (1/8) sum_v sigma(v) (V_v - V_0) with the sign pattern of
// its monomial (sigma = +-1 from the vertex's corner, v = a + 2b + 4c); the
// vertex-0 offset cancels in every sign sum, and subtracting it first keeps
// the sums free of cancellation far from the origin.  Words: A B C D E F G
// (3 coordinates each) and 3 zero pads.  Then the Jacobian's columns are
//   J0 = (A + D s) + t (E + G s),  J1 = (B + D r) + t (F + G r),
//   J2 = C + E r + F s + G r s.
__global__ void trilinear_coeffs_kernel(int64_t E, const double *__restrict__ V, void *out, int fmt, int *flags) {
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * 24) return;
  const int64_t e = gidx / 24;
  const int q = (int)(gidx % 24), m = q / 3, c = q % 3;
  double acc = 0.0;
  if (m < 7) {
    // monomials r, s, t, rs, rt, st, rst: which of (a, b, c) enter the sign
    const int use[7] = {1, 2, 4, 3, 5, 6, 7};
    for (int v = 0; v < 8; ++v) {
      int sgn = 1;
      for (int d = 0; d < 3; ++d)
        if ((use[m] >> d) & 1) sgn *= ((v >> d) & 1) ? 1 : -1;
      acc += sgn * (V[24 * e + 3 * v + c] - V[24 * e + c]);
    }
    acc *= 0.125;
  }
  store(out, gidx, acc, fmt, flags);
}

// PARALLELEPIPED: J = [v1-v0, v2-v0, v4-v0] / 2 (columns) is constant;
// h0..h5 = |J| J^-1 J^-T, h6 = |J| (Algorithm 3 input, without GLL weights).
// flags[1] += elements whose vertices deviate from v0 + a e1 + b e2 + c e3.
__global__ void parallelepiped_kernel(int64_t E, const double *__restrict__ V, void *out, int fmt, int *flags) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double *Ve = V + 24 * e;
  double J[9], scale = 0.0;
  for (int c = 0; c < 3; ++c) {
    J[3 * c + 0] = 0.5 * (Ve[3 + c] - Ve[c]);
    J[3 * c + 1] = 0.5 * (Ve[6 + c] - Ve[c]);
    J[3 * c + 2] = 0.5 * (Ve[12 + c] - Ve[c]);
    for (int d = 0; d < 3; ++d) scale = fmax(scale, fabs(J[3 * c + d]));
  }
  double dev = 0.0;
  for (int v = 0; v < 8; ++v) {
    const int a = v & 1, b = (v >> 1) & 1, cc = (v >> 2) & 1;
    for (int c = 0; c < 3; ++c) {
      const double pred = Ve[c] + 2.0 * (a * J[3 * c] + b * J[3 * c + 1] + cc * J[3 * c + 2]);
      dev = fmax(dev, fabs(pred - Ve[3 * v + c]));
    }
  }
  if (dev > 1e-12 * scale) atomicAdd(&flags[1], 1);
  double g[7];
  factors_from_J(J, 1.0, g);
  for (int q = 0; q < 7; ++q) store(out, e * kParWords + q, g[q], fmt, flags);
  store(out, e * kParWords + 7, 0.0, fmt, flags);
}

// PARTIAL: lam = w_i w_j w_k / det J at every node.
__global__ void partial_lam_kernel(int64_t E, int N1, const double *__restrict__ V, void *out, int fmt, int *flags) {
  const int64_t n3 = (int64_t)N1 * N1 * N1;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * n3) return;
  const int64_t e = gidx / n3;
  const int l = (int)(gidx % n3), i = l % N1, j = (l / N1) % N1, k = l / (N1 * N1);
  const double *cx = c_x + tab_off_v(N1), *cw = c_w + tab_off_v(N1);
  double J[9];
  map_jacobian(V + 24 * e, cx[i], cx[j], cx[k], J);
  store(out, gidx, cw[i] * cw[j] * cw[k] / det3(J), fmt, flags);
}

__global__ void node_coords_kernel(int64_t E, int N1, const double *__restrict__ V, double *xyz) {
  const int64_t n3 = (int64_t)N1 * N1 * N1;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * n3) return;
  const int64_t e = gidx / n3;
  const int l = (int)(gidx % n3), i = l % N1, j = (l / N1) % N1, k = l / (N1 * N1);
  const double *cx = c_x + tab_off_v(N1);
  double X[3];
  map_point(V + 24 * e, cx[i], cx[j], cx[k], X);
  for (int c = 0; c < 3; ++c) xyz[(e * 3 + c) * n3 + l] = X[c];
}

// Y = w_i w_j w_k det J * F at every node (the seventh factor times F).
template <typename T>
__global__ void mass_kernel(int64_t E, int N1, const double *__restrict__ V, const T *__restrict__ F, T *__restrict__ Y) {
  const int64_t n3 = (int64_t)N1 * N1 * N1;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * n3) return;
  const int64_t e = gidx / n3;
  const int l = (int)(gidx % n3), i = l % N1, j = (l / N1) % N1, k = l / (N1 * N1);
  const double *cx = c_x + tab_off_v(N1), *cw = c_w + tab_off_v(N1);
  double J[9];
  map_jacobian(V + 24 * e, cx[i], cx[j], cx[k], J);
  Y[gidx] = (T)(cw[i] * cw[j] * cw[k] * det3(J) * (double)F[gidx]);
}

// Diagonal of the element matrix D^T G D at node l = (i,j,k):
//   sum_n (D[n][i]^2 g00(n,j,k) + D[n][j]^2 g11(i,n,k) + D[n][k]^2 g22(i,j,n))
//   + 2 (D[i][i] D[j][j] g01 + D[i][i] D[k][k] g02 + D[j][j] D[k][k] g12)(l)
template <typename T>
__global__ void diag_kernel(int64_t E, int N1, const double *__restrict__ G, T *__restrict__ out) {
  const int64_t n3 = (int64_t)N1 * N1 * N1;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= E * n3) return;
  const int64_t e = gidx / n3;
  const int l = (int)(gidx % n3), i = l % N1, j = (l / N1) % N1, k = l / (N1 * N1);
  const double *cD = c_D + tab_off_D(N1);
  const double *Ge = G + e * 7 * n3;
  double d = 0.0;
  for (int n = 0; n < N1; ++n) {
    const double a = cD[n * N1 + i], b = cD[n * N1 + j], c = cD[n * N1 + k];
    d += a * a * Ge[0 * n3 + n + j * N1 + k * N1 * N1];
    d += b * b * Ge[3 * n3 + i + n * N1 + k * N1 * N1];
    d += c * c * Ge[5 * n3 + i + j * N1 + n * N1 * N1];
  }
  const double di = cD[i * N1 + i], dj = cD[j * N1 + j], dk = cD[k * N1 + k];
  d += 2.0 * (di * dj * Ge[1 * n3 + l] + di * dk * Ge[2 * n3 + l] + dj * dk * Ge[4 * n3 + l]);
  out[gidx] = (T)d;
}

static unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace setup

static UploadOnce g_once_setup;

cudaError_t upload_tables_setup(int device) {
  std::lock_guard<std::mutex> lock(g_once_setup.mu);
  if (device < 64 && (g_once_setup.done >> device) & 1ull) return cudaSuccess;
  static double D[kTabD], w[kTabV], x[kTabV];
  if (!build_packed_tables(D, w, x)) return cudaErrorInvalidValue;
  cudaError_t err = cudaMemcpyToSymbol(setup::c_D, D, sizeof(D));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(setup::c_w, w, sizeof(w));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(setup::c_x, x, sizeof(x));
  if (err == cudaSuccess && device < 64) g_once_setup.done |= 1ull << device;
  return err;
}

cudaError_t setup_geometry(const Ctx &c, const double *V, void *geo, void *lam, int *flags, cudaStream_t s) {
  using namespace setup;
  const int fmt = (c.prec == AX_FP64) ? kF64 : (c.prec == AX_F64DW ? kDW : kF32);
  const int64_t nodes = c.E * (int64_t)c.n3;
  const int B = 256;
  if (c.E == 0) return cudaSuccess;
  if ((nodes + B - 1) / B > 0x7fffffffLL) return cudaErrorInvalidValue;
  validate_kernel<<<grid_for(nodes, B), B, 0, s>>>(c.E, c.N1, V, fmt, flags);
  switch (c.kind) {
    case AX_GEOM_STORED:
      stored_factors_kernel<<<grid_for(nodes, B), B, 0, s>>>(c.E, c.N1, V, geo, fmt, flags);
      break;
    case AX_GEOM_PARALLELEPIPED:
      parallelepiped_kernel<<<grid_for(c.E, B), B, 0, s>>>(c.E, V, geo, fmt, flags);
      break;
    case AX_GEOM_TRILINEAR_PARTIAL:
      partial_lam_kernel<<<grid_for(nodes, B), B, 0, s>>>(c.E, c.N1, V, lam, fmt, flags);
      trilinear_coeffs_kernel<<<grid_for(c.E * 24, B), B, 0, s>>>(c.E, V, geo, fmt, flags);
      break;
    case AX_GEOM_TRILINEAR:
      trilinear_coeffs_kernel<<<grid_for(c.E * 24, B), B, 0, s>>>(c.E, V, geo, fmt, flags);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t setup_node_coords(const Ctx &c, const double *V, double *xyz, cudaStream_t s) {
  const int64_t nodes = c.E * (int64_t)c.n3;
  if (nodes == 0) return cudaSuccess;
  setup::node_coords_kernel<<<setup::grid_for(nodes, 256), 256, 0, s>>>(c.E, c.N1, V, xyz);
  return cudaGetLastError();
}

}  // namespace ax

namespace ax {

cudaError_t setup_mass(const Ctx &c, const double *V, const void *F, void *Y, bool f64, cudaStream_t s) {
  const int64_t nodes = c.E * (int64_t)c.n3;
  if (nodes == 0) return cudaSuccess;
  if (f64)
    setup::mass_kernel<double><<<setup::grid_for(nodes, 256), 256, 0, s>>>(c.E, c.N1, V, (const double *)F, (double *)Y);
  else
    setup::mass_kernel<float><<<setup::grid_for(nodes, 256), 256, 0, s>>>(c.E, c.N1, V, (const float *)F, (float *)Y);
  return cudaGetLastError();
}

cudaError_t setup_diag(const Ctx &c, const double *V, void *diag, bool f64, cudaStream_t s) {
  const int64_t nodes = c.E * (int64_t)c.n3;
  if (nodes == 0) return cudaSuccess;
  double *G = nullptr;
  int *flags = nullptr;
  cudaError_t e = cudaMalloc(&G, sizeof(double) * 7 * nodes);
  if (e == cudaSuccess) e = cudaMalloc(&flags, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s);
  if (e == cudaSuccess) {
    setup::stored_factors_kernel<<<setup::grid_for(nodes, 256), 256, 0, s>>>(c.E, c.N1, V, G, setup::kF64, flags);
    if (f64)
      setup::diag_kernel<double><<<setup::grid_for(nodes, 256), 256, 0, s>>>(c.E, c.N1, G, (double *)diag);
    else
      setup::diag_kernel<float><<<setup::grid_for(nodes, 256), 256, 0, s>>>(c.E, c.N1, G, (float *)diag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(G);
  cudaFree(flags);
  return e;
}

}  // namespace ax
