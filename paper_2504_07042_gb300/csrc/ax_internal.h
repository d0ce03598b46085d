// Internal declarations shared by the C-ABI layer (ax_api.cu) and the kernel
// translation units.  Not installed; the public interface is include/ax.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/ax.h"
#include "gll.h"

namespace ax {

// Per-element geometry record sizes (words of the storage type).
constexpr int kVertexWords = 24;  // trilinear record: 7 monomial coefficients x 3 (Eq. 8) + 3 pad
constexpr int kParWords = 8;      // h0..h6 of Algorithm 3 + one pad word

// Device tables for one polynomial order, uploaded once per device by each
// kernel translation unit into its own constant memory.
struct GllHost {
  int N = 0;
  double x[kMaxN1], w[kMaxN1], D[kMaxN1 * kMaxN1];
};

// Gather-scatter plan (Eq. 1's Q): CSR from global node to local copies.
// Gather-scatter plans index with 32-bit integers (half the index traffic of
// every gather and scatter); gs_setup refuses larger problems with AX_ERANGE.
using gidx = int32_t;
constexpr int64_t kMaxGsIndex = 2147483647;

struct GsPlan {
  int64_t n_global = 0, n_local = 0;
  gidx *off = nullptr;  // [n_global + 1]
  gidx *idx = nullptr;  // [n_local], local indices grouped by global node, increasing within a group
  gidx *gid = nullptr;  // [n_local], global id of every local node
  uint8_t *mask = nullptr; // [n_global] Dirichlet mask or nullptr
};

struct Ctx {
  int64_t E = 0;
  int N = 0, N1 = 0, n3 = 0;
  ax_geom_kind kind = AX_GEOM_STORED;
  ax_precision prec = AX_FP64;
  int device = 0;
  // geometry record, in the storage type of the precision:
  //   STORED: factors [E][7][n3]; TRILINEAR(_PARTIAL): vertices [E][24];
  //   PARALLELEPIPED: constants [E][8]; PARTIAL additionally lam [E][n3].
  void *geo = nullptr;
  size_t geo_bytes = 0;
  void *lam = nullptr;
  size_t lam_bytes = 0;
  int *wide = nullptr;  // AX_F64DW: block list of the scaled fix-up pass (int[2 + E], zeroed)
  int *kerr = nullptr;  // AX_TF32: error word of the tensor-core AxLocal's bounded waits
  // device staging buffers for ax_local_host
  void *hx = nullptr, *hy = nullptr;
  size_t hbytes = 0;
  GsPlan gs;
  // assembled (gathered, masked) diagonal of the operator, double and float,
  // computed on first use after gs_setup (Jacobi preconditioning)
  double *diag64 = nullptr;
  float *diag32 = nullptr;
  // solver workspaces kept between calls (work vectors, streams, captured
  // graphs), each with its deleter; freed by gs_setup and ax_destroy
  enum { kWsCg64 = 0, kWsCg32 = 1, kWsMixed = 2, kWsLearn = 3, kWsHost = 4, kNumWs = 5 };
  void *ws[kNumWs] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  void (*ws_del[kNumWs])(void *) = {nullptr, nullptr, nullptr, nullptr, nullptr};
  void free_ws() {
    for (int q = 0; q < kNumWs; ++q) {
      if (ws[q] && ws_del[q]) ws_del[q](ws[q]);
      ws[q] = nullptr;
      ws_del[q] = nullptr;
    }
  }
  std::string err;
};

// Argument bundle handed to every AxLocal launcher.
struct AxArgs {
  int64_t E = 0;
  int N = 0;
  ax_geom_kind kind = AX_GEOM_STORED;
  const void *geo = nullptr;
  const void *lam = nullptr;
  const void *X = nullptr;
  void *Y = nullptr;
  cudaStream_t stream = nullptr;
  int tile = 0;      // tile variant (elements per CTA: 0 = base, 1 = twice; FP32 only)
  int64_t grid = 0;  // CTAs to launch (0 = one per block of elements; fewer = persistent loop)
  // double-word precision: the context's list of element blocks whose X left
  // the kernel's direct range (int[2 + E], zero at rest; see ax_fiber.cuh)
  int *wide = nullptr;
  // kernels with bounded waits (tensor-core AxLocal): error word, nonzero
  // once a wait ran out (read by the context's synchronising calls)
  int *err = nullptr;
};

// Launchers (return cudaSuccess or the launch error).
cudaError_t launch_ax_fp64(const AxArgs &a);
cudaError_t launch_ax_fp32(const AxArgs &a);
cudaError_t launch_ax_dw(const AxArgs &a);
// tensor-core contractions (TF32, BF16, FP16 operands; FP32 accumulation, io and geometry)
cudaError_t launch_ax_tf32(const AxArgs &a);
cudaError_t launch_ax_bf16(const AxArgs &a);
cudaError_t launch_ax_fp16(const AxArgs &a);
cudaError_t upload_tables_tf32(int device);
cudaError_t upload_tables_bf16(int device);
cudaError_t upload_tables_fp16(int device);
// AxLocal launcher of a precision (nullptr if none)
cudaError_t (*ax_launcher_of(int prec))(const AxArgs &);

// Factor export through the kernel's own geometry code (G_out [E][7][n3] float64).
cudaError_t launch_factors_fp64(const AxArgs &a, double *G_out);
cudaError_t launch_factors_fp32(const AxArgs &a, double *G_out);
cudaError_t launch_factors_dw(const AxArgs &a, double *G_out);

// Per-device table upload of each translation unit (idempotent per device).
cudaError_t upload_tables_fp64(int device);
cudaError_t upload_tables_fp32(int device);
cudaError_t upload_tables_dw(int device);
cudaError_t upload_tables_setup(int device);

// Binding-pipe instructions per node of the AxLocal kernel (design count).
double pipe_ops_per_node(int N1, int kind, int prec);

// Setup kernels (FP64, ax_setup.cu).  flags: device int[4] zeroed by the caller:
//   [0] count of GLL nodes with det J <= 0, [1] count of non-affine elements,
//   [2] count of values outside the precision's number range.
cudaError_t setup_geometry(const Ctx &c, const double *vertices, void *geo, void *lam, int *flags,
                           cudaStream_t s);
cudaError_t setup_node_coords(const Ctx &c, const double *vertices, double *xyz, cudaStream_t s);
// Y = w|J| F per node (GLL-lumped mass); F, Y float64 when f64 else float32.
cudaError_t setup_mass(const Ctx &c, const double *vertices, const void *F, void *Y, bool f64, cudaStream_t s);
// diag[e][l] = e_l^T A^(e) e_l from the factors (computed in FP64 into a temporary).
cudaError_t setup_diag(const Ctx &c, const double *vertices, void *diag, bool f64, cudaStream_t s);

// Gather-scatter and CG (ax_gs.cu).
cudaError_t gs_build(GsPlan &plan, const int64_t *gid_dev, int64_t n_local, int64_t n_global, const uint8_t *mask_dev,
                     cudaStream_t s, int64_t *bad_ids);
void gs_free(GsPlan &plan);
cudaError_t gs_assemble_run(const GsPlan &p, bool f64, void *Y, cudaStream_t s);
cudaError_t gs_gather_run(const GsPlan &p, bool f64, const void *Y, void *y, cudaStream_t s);
cudaError_t gs_scatter_run(const GsPlan &p, bool f64, const void *u, void *U, cudaStream_t s);
// (P)CG on ctx's gs plan; the work buffers live in ctx.ws (kept between calls)
cudaError_t pcg_run(Ctx &ctx, bool f64, const AxArgs &base, cudaError_t (*launch)(const AxArgs &), const void *b,
                    void *x, const void *diag_global, double rtol, int maxit, int *iters, double *relres,
                    int *converged, cudaStream_t s);
cudaError_t pcg_mixed_run(Ctx &ctx, const AxArgs &hi, cudaError_t (*launch_hi)(const AxArgs &), const AxArgs &lo,
                          cudaError_t (*launch_lo)(const AxArgs &), const double *b, double *x, const float *diag_lo,
                          double rtol, double inner_rtol, int max_outer, int max_inner, int *outer, int *inner_total,
                          double *relres, int *converged, cudaStream_t s);

// Assembled diagonal of the context's operator on its gs plan (cached), as
// float64 or float32 (ax_api.cu).
cudaError_t assembled_diag(ax_ctx *c, bool f64, const void **out, cudaStream_t s);

// Access to a context's internals for the batch layer (ax_api.cu).
AxArgs ax_ctx_args(const ax_ctx *c);
const Ctx &ax_ctx_core(const ax_ctx *c);
Ctx &ax_ctx_core_mut(ax_ctx *c);
const double *ax_ctx_vertices(const ax_ctx *c);

}  // namespace ax
