// Routes a launch to the translation unit that instantiates its order.
#include "ax_internal.h"

namespace ax {

cudaError_t upload_tables_fp64_g0(int device);
cudaError_t launch_fp64_g0(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp64_g1(int device);
cudaError_t launch_fp64_g1(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp64_g2(int device);
cudaError_t launch_fp64_g2(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp64_g3(int device);
cudaError_t launch_fp64_g3(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp64_g4(int device);
cudaError_t launch_fp64_g4(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp64_g5(int device);
cudaError_t launch_fp64_g5(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp64_g6(int device);
cudaError_t launch_fp64_g6(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g0(int device);
cudaError_t launch_fp32_g0(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g1(int device);
cudaError_t launch_fp32_g1(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g2(int device);
cudaError_t launch_fp32_g2(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g3(int device);
cudaError_t launch_fp32_g3(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g4(int device);
cudaError_t launch_fp32_g4(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g5(int device);
cudaError_t launch_fp32_g5(const AxArgs &a, double *G_out);
cudaError_t upload_tables_fp32_g6(int device);
cudaError_t launch_fp32_g6(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g0(int device);
cudaError_t launch_dw_g0(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g1(int device);
cudaError_t launch_dw_g1(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g2(int device);
cudaError_t launch_dw_g2(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g3(int device);
cudaError_t launch_dw_g3(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g4(int device);
cudaError_t launch_dw_g4(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g5(int device);
cudaError_t launch_dw_g5(const AxArgs &a, double *G_out);
cudaError_t upload_tables_dw_g6(int device);
cudaError_t launch_dw_g6(const AxArgs &a, double *G_out);

cudaError_t upload_tables_tf32_g0(int device);
cudaError_t launch_tf32_g0(const AxArgs &a);
cudaError_t upload_tables_tf32_g1(int device);
cudaError_t launch_tf32_g1(const AxArgs &a);
cudaError_t upload_tables_tf32_g2(int device);
cudaError_t launch_tf32_g2(const AxArgs &a);
cudaError_t upload_tables_bf16_g0(int device);
cudaError_t launch_bf16_g0(const AxArgs &a);
cudaError_t upload_tables_bf16_g1(int device);
cudaError_t launch_bf16_g1(const AxArgs &a);
cudaError_t upload_tables_bf16_g2(int device);
cudaError_t launch_bf16_g2(const AxArgs &a);
cudaError_t upload_tables_fp16_g0(int device);
cudaError_t launch_fp16_g0(const AxArgs &a);
cudaError_t upload_tables_fp16_g1(int device);
cudaError_t launch_fp16_g1(const AxArgs &a);
cudaError_t upload_tables_fp16_g2(int device);
cudaError_t launch_fp16_g2(const AxArgs &a);

static int group_of(int N) {
  switch (N) {
    case 1: return 0;
    case 2: return 0;
    case 3: return 0;
    case 4: return 0;
    case 5: return 0;
    case 6: return 1;
    case 7: return 1;
    case 8: return 2;
    case 9: return 2;
    case 10: return 3;
    case 11: return 3;
    case 12: return 4;
    case 13: return 4;
    case 14: return 5;
    case 15: return 6;
    default: return -1;
  }
}

static cudaError_t launch_fp64(const AxArgs &a, double *G_out) {
  switch (group_of(a.N)) {
    case 0: return launch_fp64_g0(a, G_out);
    case 1: return launch_fp64_g1(a, G_out);
    case 2: return launch_fp64_g2(a, G_out);
    case 3: return launch_fp64_g3(a, G_out);
    case 4: return launch_fp64_g4(a, G_out);
    case 5: return launch_fp64_g5(a, G_out);
    case 6: return launch_fp64_g6(a, G_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t upload_tables_fp64(int device) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload_tables_fp64_g0(device);
  if (e == cudaSuccess) e = upload_tables_fp64_g1(device);
  if (e == cudaSuccess) e = upload_tables_fp64_g2(device);
  if (e == cudaSuccess) e = upload_tables_fp64_g3(device);
  if (e == cudaSuccess) e = upload_tables_fp64_g4(device);
  if (e == cudaSuccess) e = upload_tables_fp64_g5(device);
  if (e == cudaSuccess) e = upload_tables_fp64_g6(device);
  return e;
}

cudaError_t launch_ax_fp64(const AxArgs &a) { return launch_fp64(a, nullptr); }
cudaError_t launch_factors_fp64(const AxArgs &a, double *G_out) { return launch_fp64(a, G_out); }

static cudaError_t launch_fp32(const AxArgs &a, double *G_out) {
  switch (group_of(a.N)) {
    case 0: return launch_fp32_g0(a, G_out);
    case 1: return launch_fp32_g1(a, G_out);
    case 2: return launch_fp32_g2(a, G_out);
    case 3: return launch_fp32_g3(a, G_out);
    case 4: return launch_fp32_g4(a, G_out);
    case 5: return launch_fp32_g5(a, G_out);
    case 6: return launch_fp32_g6(a, G_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t upload_tables_fp32(int device) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload_tables_fp32_g0(device);
  if (e == cudaSuccess) e = upload_tables_fp32_g1(device);
  if (e == cudaSuccess) e = upload_tables_fp32_g2(device);
  if (e == cudaSuccess) e = upload_tables_fp32_g3(device);
  if (e == cudaSuccess) e = upload_tables_fp32_g4(device);
  if (e == cudaSuccess) e = upload_tables_fp32_g5(device);
  if (e == cudaSuccess) e = upload_tables_fp32_g6(device);
  return e;
}

cudaError_t launch_ax_fp32(const AxArgs &a) { return launch_fp32(a, nullptr); }
cudaError_t launch_factors_fp32(const AxArgs &a, double *G_out) { return launch_fp32(a, G_out); }

static cudaError_t launch_dw(const AxArgs &a, double *G_out) {
  switch (group_of(a.N)) {
    case 0: return launch_dw_g0(a, G_out);
    case 1: return launch_dw_g1(a, G_out);
    case 2: return launch_dw_g2(a, G_out);
    case 3: return launch_dw_g3(a, G_out);
    case 4: return launch_dw_g4(a, G_out);
    case 5: return launch_dw_g5(a, G_out);
    case 6: return launch_dw_g6(a, G_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t upload_tables_dw(int device) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload_tables_dw_g0(device);
  if (e == cudaSuccess) e = upload_tables_dw_g1(device);
  if (e == cudaSuccess) e = upload_tables_dw_g2(device);
  if (e == cudaSuccess) e = upload_tables_dw_g3(device);
  if (e == cudaSuccess) e = upload_tables_dw_g4(device);
  if (e == cudaSuccess) e = upload_tables_dw_g5(device);
  if (e == cudaSuccess) e = upload_tables_dw_g6(device);
  return e;
}

cudaError_t launch_ax_dw(const AxArgs &a) { return launch_dw(a, nullptr); }
cudaError_t launch_factors_dw(const AxArgs &a, double *G_out) { return launch_dw(a, G_out); }

// tensor-core contraction kernels: order groups {1..5}, {6..9}, {10..15}
static int tc_group(int N) { return N >= 1 && N <= 5 ? 0 : (N >= 6 && N <= 9 ? 1 : (N >= 10 && N <= 15 ? 2 : -1)); }

cudaError_t launch_ax_tf32(const AxArgs &a) {
  switch (tc_group(a.N)) {
    case 0: return launch_tf32_g0(a);
    case 1: return launch_tf32_g1(a);
    case 2: return launch_tf32_g2(a);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t upload_tables_tf32(int device) {
  cudaError_t e = upload_tables_tf32_g0(device);
  if (e == cudaSuccess) e = upload_tables_tf32_g1(device);
  if (e == cudaSuccess) e = upload_tables_tf32_g2(device);
  return e;
}

cudaError_t launch_ax_bf16(const AxArgs &a) {
  switch (tc_group(a.N)) {
    case 0: return launch_bf16_g0(a);
    case 1: return launch_bf16_g1(a);
    case 2: return launch_bf16_g2(a);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t upload_tables_bf16(int device) {
  cudaError_t e = upload_tables_bf16_g0(device);
  if (e == cudaSuccess) e = upload_tables_bf16_g1(device);
  if (e == cudaSuccess) e = upload_tables_bf16_g2(device);
  return e;
}

cudaError_t launch_ax_fp16(const AxArgs &a) {
  switch (tc_group(a.N)) {
    case 0: return launch_fp16_g0(a);
    case 1: return launch_fp16_g1(a);
    case 2: return launch_fp16_g2(a);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t upload_tables_fp16(int device) {
  cudaError_t e = upload_tables_fp16_g0(device);
  if (e == cudaSuccess) e = upload_tables_fp16_g1(device);
  if (e == cudaSuccess) e = upload_tables_fp16_g2(device);
  return e;
}

}  // namespace ax
