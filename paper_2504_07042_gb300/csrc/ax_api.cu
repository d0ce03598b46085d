// C-ABI layer of libax (include/ax.h): argument checks, context ownership,
// dispatch to the kernel translation units, status and error strings.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "ax_internal.h"

struct ax_ctx {
  ax::Ctx c;
  double *vtx = nullptr;  // copy of the caller's vertices (node coordinates, exports)
  void *static_stage = nullptr;  // device address of the file-scope staging array (ax_local_host_static)
};

namespace {
cudaError_t static_stage_address(void **out);  // defined beside the array, at the end of this file
}

namespace {

thread_local std::string g_create_err;

ax_status fail(ax_ctx *c, ax_status st, const std::string &msg) {
  if (c)
    c->c.err = msg;
  else
    g_create_err = msg;
  return st;
}

ax_status cuda_fail(ax_ctx *c, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();  // clear a sticky launch error where possible
  return fail(c, e == cudaErrorMemoryAllocation ? AX_ENOMEM : AX_ECUDA, m);
}

bool is_f64_io(ax_precision p) { return p == AX_FP64 || p == AX_F64DW; }

size_t storage_word(ax_precision p) {
  // bytes per geometry value: float64, double-word pair, or float32
  return (p == AX_FP64 || p == AX_F64DW) ? 8 : 4;
}

size_t io_word(ax_precision p) { return is_f64_io(p) ? 8 : 4; }

void release(ax_ctx *c) {
  if (!c) return;
  cudaFree(c->c.geo);
  cudaFree(c->c.lam);
  cudaFree(c->c.hx);
  cudaFree(c->c.hy);
  cudaFree(c->c.wide);
  c->c.wide = nullptr;
  cudaFree(c->c.kerr);
  c->c.kerr = nullptr;
  c->c.free_ws();
  cudaFree(c->vtx);
  cudaFree(c->c.diag64);
  cudaFree(c->c.diag32);
  c->c.diag64 = nullptr;
  c->c.diag32 = nullptr;
  ax::gs_free(c->c.gs);
  c->c.geo = c->c.lam = c->c.hx = c->c.hy = nullptr;
  c->vtx = nullptr;
}

ax::AxArgs make_args(ax_ctx *c, const void *X, void *Y, void *stream) {
  ax::AxArgs a;
  a.E = c->c.E;
  a.N = c->c.N;
  a.kind = c->c.kind;
  a.geo = c->c.geo;
  a.lam = c->c.lam;
  a.wide = c->c.wide;
  a.err = c->c.kerr;
  a.X = X;
  a.Y = Y;
  a.stream = (cudaStream_t)stream;
  return a;
}

cudaError_t run_ax(ax_ctx *c, const ax::AxArgs &a) {
  cudaError_t (*launch)(const ax::AxArgs &) = ax::ax_launcher_of(c->c.prec);
  return launch ? launch(a) : cudaErrorNotSupported;
}

bool same_device(ax_ctx *c) {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == c->c.device;
}

}  // namespace

namespace ax {
cudaError_t (*ax_launcher_of(int prec))(const AxArgs &) {
  switch (prec) {
    case AX_FP64: return launch_ax_fp64;
    case AX_FP32: return launch_ax_fp32;
    case AX_F64DW: return launch_ax_dw;
    case AX_TF32: return launch_ax_tf32;
    case AX_BF16: return launch_ax_bf16;
    case AX_FP16: return launch_ax_fp16;
    default: return nullptr;
  }
}

cudaError_t assembled_diag(ax_ctx *c, bool f64, const void **out, cudaStream_t s) {
  void **slot = f64 ? (void **)&c->c.diag64 : (void **)&c->c.diag32;
  if (*slot) {
    *out = *slot;
    return cudaSuccess;
  }
  const size_t w = f64 ? 8 : 4;
  void *dl = nullptr, *dg = nullptr;
  cudaError_t e = cudaMalloc(&dl, w * c->c.gs.n_local + 8);
  if (e == cudaSuccess) e = cudaMalloc(&dg, w * c->c.gs.n_global + 8);
  if (e == cudaSuccess) e = setup_diag(c->c, c->vtx, dl, f64, s);
  if (e == cudaSuccess) e = gs_gather_run(c->c.gs, f64, dl, dg, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dl);
  if (e != cudaSuccess) {
    cudaFree(dg);
    return e;
  }
  *slot = dg;
  *out = dg;
  return cudaSuccess;
}

AxArgs ax_ctx_args(const ax_ctx *c) { return make_args(const_cast<ax_ctx *>(c), nullptr, nullptr, nullptr); }
const Ctx &ax_ctx_core(const ax_ctx *c) { return c->c; }
Ctx &ax_ctx_core_mut(ax_ctx *c) { return c->c; }
const double *ax_ctx_vertices(const ax_ctx *c) { return c->vtx; }
}  // namespace ax

extern "C" {

const char *ax_status_string(ax_status s) {
  switch (s) {
    case AX_OK: return "AX_OK";
    case AX_EINVAL: return "AX_EINVAL";
    case AX_ENOMEM: return "AX_ENOMEM";
    case AX_ECUDA: return "AX_ECUDA";
    case AX_EINVERTED: return "AX_EINVERTED";
    case AX_ENOTPARALLELEPIPED: return "AX_ENOTPARALLELEPIPED";
    case AX_ENOTCONV: return "AX_ENOTCONV";
    case AX_ETIMEOUT: return "AX_ETIMEOUT";
    case AX_EUNSUPPORTED: return "AX_EUNSUPPORTED";
    case AX_ERANGE: return "AX_ERANGE";
  }
  return "AX_UNKNOWN";
}

const char *ax_last_error(const ax_ctx *c) { return c ? c->c.err.c_str() : g_create_err.c_str(); }

ax_status ax_setup(ax_ctx **out, int64_t E, int N, const double *vertices, ax_geom_kind kind, ax_precision prec,
                   void *stream) {
  if (!out) return fail(nullptr, AX_EINVAL, "ax_setup: out is NULL");
  *out = nullptr;
  if (E < 0) return fail(nullptr, AX_EINVAL, "ax_setup: E < 0");
  if (N < 1 || N > ax::kMaxN) return fail(nullptr, AX_EINVAL, "ax_setup: N must be in [1, 15]");
  if (E > 0 && !vertices) return fail(nullptr, AX_EINVAL, "ax_setup: vertices is NULL");
  if ((int)kind < 0 || (int)kind > 3) return fail(nullptr, AX_EINVAL, "ax_setup: bad geometry kind");
  if ((int)prec < 0 || (int)prec > 5) return fail(nullptr, AX_EINVAL, "ax_setup: bad precision");
  const int64_t N1 = N + 1, n3 = N1 * N1 * N1;
  if (E > (int64_t)1 << 40 || E * n3 > ((int64_t)1 << 46))
    return fail(nullptr, AX_EINVAL, "ax_setup: problem too large");
  if (prec == AX_F64DW && E > 2147483645LL)
    return fail(nullptr, AX_ERANGE, "ax_setup: AX_F64DW takes at most 2^31 - 3 elements");

  ax_ctx *c = new (std::nothrow) ax_ctx;
  if (!c) return fail(nullptr, AX_ENOMEM, "ax_setup: host allocation failed");
  c->c.E = E;
  c->c.N = N;
  c->c.N1 = (int)N1;
  c->c.n3 = (int)n3;
  c->c.kind = kind;
  c->c.prec = prec;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->c.device);
  if (e == cudaSuccess) e = ax::upload_tables_setup(c->c.device);
  if (e == cudaSuccess) {
    switch (prec) {
      case AX_FP64: e = ax::upload_tables_fp64(c->c.device); break;
      case AX_FP32: e = ax::upload_tables_fp32(c->c.device); break;
      case AX_F64DW: e = ax::upload_tables_dw(c->c.device); break;
      // tensor-core contractions; the FP32 tables serve their factor export
      case AX_TF32: e = ax::upload_tables_tf32(c->c.device); break;
      case AX_BF16: e = ax::upload_tables_bf16(c->c.device); break;
      case AX_FP16: e = ax::upload_tables_fp16(c->c.device); break;
      default: break;
    }
    if (e == cudaSuccess && (prec == AX_TF32 || prec == AX_BF16 || prec == AX_FP16))
      e = ax::upload_tables_fp32(c->c.device);
  }
  // The device address of ax_local_host_static's staging array, looked up
  // here with the context's device current: the lookup loads this file's
  // module (committing the array) during set-up, never inside that call.
  if (e == cudaSuccess) e = static_stage_address(&c->static_stage);
  if (e != cudaSuccess) {
    ax_status st = cuda_fail(nullptr, e, "ax_setup: table upload");
    delete c;
    return st;
  }
  const size_t gw = storage_word(prec);
  size_t geo_words = 0;
  switch (kind) {
    case AX_GEOM_STORED: geo_words = (size_t)E * 7 * n3; break;
    case AX_GEOM_PARALLELEPIPED: geo_words = (size_t)E * ax::kParWords; break;
    default: geo_words = (size_t)E * ax::kVertexWords; break;
  }
  c->c.geo_bytes = geo_words * gw;
  c->c.lam_bytes = kind == AX_GEOM_TRILINEAR_PARTIAL ? (size_t)E * n3 * gw : 0;
  int *flags = nullptr;
  if (E > 0) {
    e = cudaMalloc(&c->c.geo, c->c.geo_bytes);
    if (e == cudaSuccess && c->c.lam_bytes) e = cudaMalloc(&c->c.lam, c->c.lam_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->vtx, (size_t)E * 24 * sizeof(double));
    if (e == cudaSuccess && prec == AX_TF32) {
      // error word of the tensor-core kernel's bounded waits
      e = cudaMalloc(&c->c.kerr, sizeof(int));
      if (e == cudaSuccess) e = cudaMemsetAsync(c->c.kerr, 0, sizeof(int), s);
    }
    if (e == cudaSuccess && prec == AX_F64DW) {
      // block list of the double-word kernel's scaled fix-up pass, zero at rest
      e = cudaMalloc(&c->c.wide, (size_t)(E + 2) * sizeof(int));
      if (e == cudaSuccess) e = cudaMemsetAsync(c->c.wide, 0, (size_t)(E + 2) * sizeof(int), s);
    }
    if (e == cudaSuccess) e = cudaMalloc(&flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->vtx, vertices, (size_t)E * 24 * sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s);
    if (e == cudaSuccess) e = ax::setup_geometry(c->c, c->vtx, c->c.geo, c->c.lam, flags, s);
    int hflags[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flags);
    if (e != cudaSuccess) {
      ax_status st = cuda_fail(nullptr, e, "ax_setup");
      release(c);
      delete c;
      return st;
    }
    ax_status st = AX_OK;
    char msg[160];
    if (hflags[0]) {
      snprintf(msg, sizeof msg, "ax_setup: det J <= 0 at %d GLL nodes", hflags[0]);
      st = fail(nullptr, AX_EINVERTED, msg);
    } else if (kind == AX_GEOM_PARALLELEPIPED && hflags[1]) {
      snprintf(msg, sizeof msg, "ax_setup: %d elements are not parallelepipeds", hflags[1]);
      st = fail(nullptr, AX_ENOTPARALLELEPIPED, msg);
    } else if (hflags[3]) {
      snprintf(msg, sizeof msg,
               "ax_setup: %d elements have an extent outside [2^-20, 2^24], the range the FP32-based "
               "precisions handle at full accuracy (scale the mesh, or use AX_FP64)", hflags[3]);
      st = fail(nullptr, AX_ERANGE, msg);
    } else if (hflags[2]) {
      snprintf(msg, sizeof msg, "ax_setup: %d geometry values above 1e30 (or not finite) for an FP32-based precision", hflags[2]);
      st = fail(nullptr, AX_ERANGE, msg);
    }
    if (st != AX_OK) {
      release(c);
      delete c;
      return st;
    }
  }
  *out = c;
  return AX_OK;
}

ax_status ax_local(ax_ctx *c, const void *X, void *Y, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_local: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!X || !Y) return fail(c, AX_EINVAL, "ax_local: X or Y is NULL");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_local: current device differs from the context's");
  const size_t bytes = (size_t)c->c.E * c->c.n3 * io_word(c->c.prec);
  const char *x = (const char *)X, *y = (const char *)Y;
  if (x < y + bytes && y < x + bytes) return fail(c, AX_EINVAL, "ax_local: X and Y overlap");
  cudaError_t e = run_ax(c, make_args(c, X, Y, stream));
  if (e == cudaErrorNotSupported) return fail(c, AX_EUNSUPPORTED, "ax_local: precision not supported");
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_local launch");
  return AX_OK;
}

// Host-buffer pipeline of ax_local_host: the elements are cut into chunks;
// chunk i's host-to-device copy, AxLocal and device-to-host copy run on three
// streams ordered by events, so the copies of one chunk overlap the kernels
// and the opposite copies of its neighbours.
namespace {
constexpr int kHostChunks = 16;
struct HostPipe {
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};  // h2d, compute, d2h
  cudaEvent_t start = nullptr, done = nullptr;
  cudaEvent_t in[kHostChunks] = {}, out[kHostChunks] = {};
  cudaError_t create() {
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaStreamCreateWithFlags(&st[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    for (int q = 0; q < kHostChunks && e == cudaSuccess; ++q) {
      e = cudaEventCreateWithFlags(&in[q], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&out[q], cudaEventDisableTiming);
    }
    return e;
  }
};
void delete_host_pipe(void *p) {
  HostPipe *h = static_cast<HostPipe *>(p);
  for (int q = 0; q < 3; ++q)
    if (h->st[q]) cudaStreamDestroy(h->st[q]);
  if (h->start) cudaEventDestroy(h->start);
  if (h->done) cudaEventDestroy(h->done);
  for (int q = 0; q < kHostChunks; ++q) {
    if (h->in[q]) cudaEventDestroy(h->in[q]);
    if (h->out[q]) cudaEventDestroy(h->out[q]);
  }
  delete h;
}

// geometry words of one element in the context's record
size_t geo_words_per_element(const ax_ctx *c) {
  switch (c->c.kind) {
    case AX_GEOM_STORED: return (size_t)7 * c->c.n3;
    case AX_GEOM_PARALLELEPIPED: return ax::kParWords;
    default: return ax::kVertexWords;
  }
}
}  // namespace

ax_status ax_local_host(ax_ctx *c, const void *X_host, void *Y_host, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_local_host: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!X_host || !Y_host) return fail(c, AX_EINVAL, "ax_local_host: X or Y is NULL");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_local_host: current device differs from the context's");
  const size_t word = io_word(c->c.prec), bytes = (size_t)c->c.E * c->c.n3 * word;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  // Float32 X and Y in page-locked host buffers the device can address
  // (mapped memory): the kernel reads X and writes Y over the host link
  // itself, so both directions stay busy for the whole call and no staging
  // copies are made.  Measured on GB300 (order 7, 131072 elements): FP32
  // 1.84 -> 1.60 ms per call, 0.98 of the link's two-way bound; the
  // float64-IO kernels (double-word, FP64), which compute longer per byte
  // with fewer resident warps, slowed down reading over the link (3.55 ->
  // 4.58 ms) and keep the chunked copy pipeline below, as does other host
  // memory.
  if (word == 4) {
    cudaPointerAttributes px{}, py{};
    const bool mapped = cudaPointerGetAttributes(&px, X_host) == cudaSuccess &&
                        cudaPointerGetAttributes(&py, Y_host) == cudaSuccess && px.type == cudaMemoryTypeHost &&
                        py.type == cudaMemoryTypeHost && px.devicePointer && py.devicePointer;
    (void)cudaGetLastError();  // an attribute query that failed leaves no error behind
    if (mapped) {
      const char *xd = (const char *)px.devicePointer;
      char *yd = (char *)py.devicePointer;
      if (xd < yd + bytes && yd < xd + bytes) return fail(c, AX_EINVAL, "ax_local_host: X and Y overlap");
      e = run_ax(c, make_args(c, xd, yd, s));
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(c, e, "ax_local_host");
      return AX_OK;
    }
  }
  if (c->c.hbytes < bytes) {
    cudaFree(c->c.hx);
    cudaFree(c->c.hy);
    c->c.hx = c->c.hy = nullptr;
    c->c.hbytes = 0;
    e = cudaMalloc(&c->c.hx, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->c.hy, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "ax_local_host: staging allocation");
    c->c.hbytes = bytes;
  }
  HostPipe *hp = static_cast<HostPipe *>(c->c.ws[ax::Ctx::kWsHost]);
  if (!hp) {
    hp = new (std::nothrow) HostPipe;
    if (!hp) return fail(c, AX_ENOMEM, "ax_local_host: host allocation failed");
    e = hp->create();
    if (e != cudaSuccess) {
      delete_host_pipe(hp);
      return cuda_fail(c, e, "ax_local_host: streams");
    }
    c->c.ws[ax::Ctx::kWsHost] = hp;
    c->c.ws_del[ax::Ctx::kWsHost] = delete_host_pipe;
  }
  // chunks of at least 2048 elements (small problems: one chunk)
  int64_t per = (c->c.E + kHostChunks - 1) / kHostChunks;
  if (per < 2048) per = 2048;
  const int nch = (int)((c->c.E + per - 1) / per);
  const size_t gw = storage_word(c->c.prec), gpe = geo_words_per_element(c), n3 = (size_t)c->c.n3;
  e = cudaEventRecord(hp->start, s);
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(hp->st[q], hp->start, 0);
  for (int i = 0; i < nch && e == cudaSuccess; ++i) {
    const int64_t e0 = i * per, ne = (c->c.E - e0) < per ? (c->c.E - e0) : per;
    const size_t off = (size_t)e0 * n3 * word, len = (size_t)ne * n3 * word;
    e = cudaMemcpyAsync((char *)c->c.hx + off, (const char *)X_host + off, len, cudaMemcpyHostToDevice, hp->st[0]);
    if (e == cudaSuccess) e = cudaEventRecord(hp->in[i], hp->st[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->st[1], hp->in[i], 0);
    if (e == cudaSuccess) {
      ax::AxArgs a = make_args(c, (const char *)c->c.hx + off, (char *)c->c.hy + off, hp->st[1]);
      a.E = ne;
      a.geo = (const char *)c->c.geo + (size_t)e0 * gpe * gw;
      if (c->c.lam) a.lam = (const char *)c->c.lam + (size_t)e0 * n3 * gw;
      e = run_ax(c, a);
    }
    if (e == cudaSuccess) e = cudaEventRecord(hp->out[i], hp->st[1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->st[2], hp->out[i], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)Y_host + off, (const char *)c->c.hy + off, len, cudaMemcpyDeviceToHost, hp->st[2]);
  }
  if (e == cudaSuccess) e = cudaEventRecord(hp->done, hp->st[2]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hp->done, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_local_host");
  return AX_OK;
}

ax_status ax_factors(ax_ctx *c, double *G_out, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_factors: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!G_out) return fail(c, AX_EINVAL, "ax_factors: G_out is NULL");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_factors: current device differs from the context's");
  ax::AxArgs a = make_args(c, nullptr, nullptr, stream);
  cudaError_t e;
  switch (c->c.prec) {
    case AX_FP64: e = ax::launch_factors_fp64(a, G_out); break;
    case AX_FP32:
    case AX_TF32:
    case AX_BF16:
    case AX_FP16: e = ax::launch_factors_fp32(a, G_out); break;  // FP32 geometry in every float32 context
    case AX_F64DW: e = ax::launch_factors_dw(a, G_out); break;
    default: return fail(c, AX_EUNSUPPORTED, "ax_factors: precision not supported");
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_factors launch");
  return AX_OK;
}

ax_status ax_node_coords(ax_ctx *c, double *XYZ_out, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_node_coords: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!XYZ_out) return fail(c, AX_EINVAL, "ax_node_coords: XYZ_out is NULL");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_node_coords: current device differs from the context's");
  cudaError_t e = ax::setup_node_coords(c->c, c->vtx, XYZ_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_node_coords launch");
  return AX_OK;
}

ax_status ax_query(const ax_ctx *c, ax_info *info) {
  if (!c || !info) return AX_EINVAL;
  const double N1 = c->c.N1, n3 = c->c.n3;
  const double io = (double)io_word(c->c.prec), gw = (double)storage_word(c->c.prec);
  info->E = c->c.E;
  info->N = c->c.N;
  info->kind = (int)c->c.kind;
  info->prec = (int)c->c.prec;
  double geo_bytes = 0.0;
  switch (c->c.kind) {
    case AX_GEOM_STORED: geo_bytes = 6.0 * n3 * gw; break;  // the Poisson kernel reads 6 of 7
    case AX_GEOM_PARALLELEPIPED: geo_bytes = ax::kParWords * gw; break;
    case AX_GEOM_TRILINEAR: geo_bytes = ax::kVertexWords * gw; break;
    case AX_GEOM_TRILINEAR_PARTIAL: geo_bytes = (ax::kVertexWords + n3) * gw; break;
  }
  info->bytes_per_element = 2.0 * n3 * io + geo_bytes;
  info->flops_ax_per_element = 12.0 * N1 * N1 * N1 * N1 + 15.0 * n3;
  // arithmetic instructions per node on the binding pipe (design counts)
  const double per_node = ax::pipe_ops_per_node(c->c.N1, (int)c->c.kind, (int)c->c.prec);
  info->pipe = (c->c.prec == AX_FP64) ? 0 : 1;
  info->pipe_ops_per_element = per_node * n3;
  return AX_OK;
}

ax_status gs_setup(ax_ctx *c, const int64_t *global_id, int64_t n_global, const uint8_t *dirichlet_mask,
                   void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "gs_setup: context is NULL");
  const int64_t n_local = c->c.E * (int64_t)c->c.n3;
  if (n_global < 0 || (n_local > 0 && !global_id)) return fail(c, AX_EINVAL, "gs_setup: bad global ids");
  if (!same_device(c)) return fail(c, AX_EINVAL, "gs_setup: current device differs from the context's");
  if (n_local >= ax::kMaxGsIndex || n_global >= ax::kMaxGsIndex)
    return fail(c, AX_ERANGE, "gs_setup: more than 2^31 - 1 local or global nodes");
  c->c.free_ws();
  ax::gs_free(c->c.gs);
  cudaFree(c->c.diag64);
  cudaFree(c->c.diag32);
  c->c.diag64 = nullptr;
  c->c.diag32 = nullptr;
  int64_t bad = 0;
  cudaError_t e = ax::gs_build(c->c.gs, global_id, n_local, n_global, dirichlet_mask, (cudaStream_t)stream, &bad);
  if (e != cudaSuccess) {
    ax::gs_free(c->c.gs);
    return cuda_fail(c, e, "gs_setup");
  }
  if (bad) {
    ax::gs_free(c->c.gs);
    char msg[120];
    snprintf(msg, sizeof msg, "gs_setup: %lld global ids outside [0, n_global)", (long long)bad);
    return fail(c, AX_EINVAL, msg);
  }
  return AX_OK;
}

static bool has_gs(ax_ctx *c) { return c->c.gs.off != nullptr; }

ax_status gs_assemble(ax_ctx *c, void *Y_local, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "gs_assemble: context is NULL");
  if (!has_gs(c)) return fail(c, AX_EINVAL, "gs_assemble: call gs_setup first");
  if (c->c.gs.n_local && !Y_local) return fail(c, AX_EINVAL, "gs_assemble: Y is NULL");
  cudaError_t e = ax::gs_assemble_run(c->c.gs, is_f64_io(c->c.prec), Y_local, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "gs_assemble");
  return AX_OK;
}

ax_status gs_gather(ax_ctx *c, const void *Y_local, void *y_global, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "gs_gather: context is NULL");
  if (!has_gs(c)) return fail(c, AX_EINVAL, "gs_gather: call gs_setup first");
  if (c->c.gs.n_global && (!Y_local || !y_global)) return fail(c, AX_EINVAL, "gs_gather: NULL vector");
  cudaError_t e = ax::gs_gather_run(c->c.gs, is_f64_io(c->c.prec), Y_local, y_global, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "gs_gather");
  return AX_OK;
}

ax_status gs_scatter(ax_ctx *c, const void *u_global, void *U_local, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "gs_scatter: context is NULL");
  if (!has_gs(c)) return fail(c, AX_EINVAL, "gs_scatter: call gs_setup first");
  if (c->c.gs.n_local && (!u_global || !U_local)) return fail(c, AX_EINVAL, "gs_scatter: NULL vector");
  cudaError_t e = ax::gs_scatter_run(c->c.gs, is_f64_io(c->c.prec), u_global, U_local, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "gs_scatter");
  return AX_OK;
}

ax_status ax_mass(ax_ctx *c, const void *F_local, void *Y_local, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_mass: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!F_local || !Y_local) return fail(c, AX_EINVAL, "ax_mass: NULL vector");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_mass: current device differs from the context's");
  cudaError_t e = ax::setup_mass(c->c, c->vtx, F_local, Y_local, is_f64_io(c->c.prec), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_mass");
  return AX_OK;
}

ax_status ax_diag(ax_ctx *c, void *diag_local, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_diag: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!diag_local) return fail(c, AX_EINVAL, "ax_diag: NULL vector");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_diag: current device differs from the context's");
  cudaError_t e = ax::setup_diag(c->c, c->vtx, diag_local, is_f64_io(c->c.prec), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_diag");
  return AX_OK;
}

ax_status pcg_solve(ax_ctx *c, const void *b_global, void *x_global, double rtol, int maxit, int precond, int *iters,
                    double *relres, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "pcg_solve: context is NULL");
  if (!has_gs(c)) return fail(c, AX_EINVAL, "pcg_solve: call gs_setup first");
  if (!iters || !relres) return fail(c, AX_EINVAL, "pcg_solve: iters or relres is NULL");
  if (precond == 2)
    return fail(c, AX_EINVAL,
                "pcg_solve: precond 2 (learned) needs a network handle: call pcg_solve_learned(ctx, mlp, ...)");
  if (precond != 0 && precond != 1) return fail(c, AX_EUNSUPPORTED, "pcg_solve: precond must be 0 (none) or 1 (Jacobi)");
  if (!(rtol >= 0.0) || maxit < 0) return fail(c, AX_EINVAL, "pcg_solve: bad rtol or maxit");
  if (c->c.gs.n_global && (!b_global || !x_global)) return fail(c, AX_EINVAL, "pcg_solve: NULL vector");
  if (!same_device(c)) return fail(c, AX_EINVAL, "pcg_solve: current device differs from the context's");
  *iters = 0;
  *relres = 0.0;
  if (c->c.gs.n_global == 0) return AX_OK;
  const bool f64 = is_f64_io(c->c.prec);
  const size_t w = f64 ? 8 : 4;
  cudaStream_t s = (cudaStream_t)stream;
  (void)w;
  const void *diag_g = nullptr;
  cudaError_t e = cudaSuccess;
  if (precond == 1) e = ax::assembled_diag(c, f64, &diag_g, s);
  int conv = 0;
  cudaError_t (*launch)(const ax::AxArgs &) = ax::ax_launcher_of(c->c.prec);
  if (e == cudaSuccess && !launch) e = cudaErrorNotSupported;
  if (e == cudaSuccess)
    e = ax::pcg_run(c->c, f64, make_args(c, nullptr, nullptr, stream), launch, b_global, x_global, diag_g, rtol,
                    maxit, iters, relres, &conv, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pcg_solve");
  if (!conv) {
    char msg[120];
    snprintf(msg, sizeof msg, "pcg_solve: not converged after %d iterations (relres %.3e)", *iters, *relres);
    return fail(c, AX_ENOTCONV, msg);
  }
  return AX_OK;
}

ax_status pcg_solve_mixed(ax_ctx *hi, ax_ctx *lo, const double *b_global, double *x_global, double rtol,
                          double inner_rtol, int max_outer, int max_inner, int *outer_iters, int *inner_iters,
                          double *relres, void *stream) {
  if (!hi || !lo) return fail(nullptr, AX_EINVAL, "pcg_solve_mixed: context is NULL");
  if (!is_f64_io(hi->c.prec)) return fail(hi, AX_EINVAL, "pcg_solve_mixed: hi must be AX_FP64 or AX_F64DW");
  if (is_f64_io(lo->c.prec)) return fail(lo, AX_EINVAL, "pcg_solve_mixed: lo must be a float32 precision");
  if (!has_gs(hi)) return fail(hi, AX_EINVAL, "pcg_solve_mixed: call gs_setup on hi first");
  if (hi->c.E != lo->c.E || hi->c.N != lo->c.N) return fail(hi, AX_EINVAL, "pcg_solve_mixed: contexts differ in E or N");
  if (!outer_iters || !inner_iters || !relres) return fail(hi, AX_EINVAL, "pcg_solve_mixed: NULL output pointer");
  if (!(rtol >= 0.0) || !(inner_rtol > 0.0) || max_outer < 0 || max_inner < 1)
    return fail(hi, AX_EINVAL, "pcg_solve_mixed: bad tolerances or iteration limits");
  if (hi->c.gs.n_global && (!b_global || !x_global)) return fail(hi, AX_EINVAL, "pcg_solve_mixed: NULL vector");
  if (!same_device(hi) || !same_device(lo)) return fail(hi, AX_EINVAL, "pcg_solve_mixed: device mismatch");
  *outer_iters = *inner_iters = 0;
  *relres = 0.0;
  if (hi->c.gs.n_global == 0) return AX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t (*lh)(const ax::AxArgs &) = hi->c.prec == AX_FP64 ? ax::launch_ax_fp64 : ax::launch_ax_dw;
  cudaError_t (*ll)(const ax::AxArgs &) = ax::ax_launcher_of(lo->c.prec);
  if (!ll) return fail(lo, AX_EUNSUPPORTED, "pcg_solve_mixed: lo precision has no AxLocal kernel");
  // the inner solve's Jacobi diagonal: the same mesh's operator, in float32
  const void *diag_g = nullptr;
  cudaError_t e = ax::assembled_diag(hi, false, &diag_g, s);
  int conv = 0;
  if (e == cudaSuccess)
    e = ax::pcg_mixed_run(hi->c, make_args(hi, nullptr, nullptr, stream), lh, make_args(lo, nullptr, nullptr, stream),
                          ll, b_global, x_global, (const float *)diag_g, rtol, inner_rtol, max_outer, max_inner,
                          outer_iters, inner_iters, relres, &conv, s);
  if (e != cudaSuccess) return cuda_fail(hi, e, "pcg_solve_mixed");
  if (!conv) {
    char msg[160];
    snprintf(msg, sizeof msg, "pcg_solve_mixed: not converged after %d outer / %d inner iterations (relres %.3e)",
             *outer_iters, *inner_iters, *relres);
    return fail(hi, AX_ENOTCONV, msg);
  }
  return AX_OK;
}

ax_status ax_check(ax_ctx *c, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_check: context is NULL");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_check: current device differs from the context's");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  int h = 0;
  if (e == cudaSuccess && c->c.kerr) {
    e = cudaMemcpy(&h, c->c.kerr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(c->c.kerr, 0, sizeof(int));
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_check");
  if (h) return fail(c, AX_ETIMEOUT, "ax_check: a bounded wait of the tensor-core AxLocal ran out; its output is void");
  return AX_OK;
}

void ax_destroy(ax_ctx *c) {
  if (!c) return;
  release(c);
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ax_local_host_static: ax_local_host without any device allocation.
//
// Some callers cannot call cudaMalloc at the time they need the operator:
// processes whose device-memory budget is fixed once start-up is over (every
// allocation is made up front), and pipelines that must not let
// cudaMalloc/cudaFree synchronise the device in the middle of their work.
// ax_local_host allocates its device staging buffers on first use, which
// such callers cannot allow.  This entry point stages X and Y through one
// file-scope device array instead, of a fixed size (kStaticStageBytes).  The
// array lives in this file's module: ax_setup looks up its device address
// (which loads the module, and so commits the array, on that device), so
// every GPU on which a context was set up holds it until the process exits,
// and the entry point itself never triggers a module load.  The address is
// kept in the context, which does not outlive a device reset.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticStageBytes = (size_t)32 << 20;     // whole array: 32 MiB
constexpr size_t kStaticStageHalf = kStaticStageBytes / 2;  // X half, Y half

static __device__ __align__(256) unsigned char g_static_stage[kStaticStageBytes];

cudaError_t static_stage_address(void **out) {
  *out = nullptr;
  return cudaGetSymbolAddress(out, g_static_stage);
}

}  // namespace

extern "C" ax_status ax_local_host_static(ax_ctx *c, const void *X_host, void *Y_host, void *stream) {
  if (!c) return fail(nullptr, AX_EINVAL, "ax_local_host_static: context is NULL");
  if (c->c.E == 0) return AX_OK;
  if (!X_host || !Y_host) return fail(c, AX_EINVAL, "ax_local_host_static: X or Y is NULL");
  if (!same_device(c)) return fail(c, AX_EINVAL, "ax_local_host_static: current device differs from the context's");
  const size_t bytes = (size_t)c->c.E * c->c.n3 * io_word(c->c.prec);
  if (bytes > kStaticStageHalf) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "ax_local_host_static: X needs %zu bytes; the static staging array holds at most %zu bytes per vector "
             "(use ax_local_host or ax_local)",
             bytes, kStaticStageHalf);
    return fail(c, AX_EINVAL, msg);
  }
  void *base = c->static_stage;  // looked up by ax_setup on this context's device
  if (!base) return fail(c, AX_EINVAL, "ax_local_host_static: staging array address unknown");
  void *xd = base;
  void *yd = (unsigned char *)base + kStaticStageHalf;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(xd, X_host, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = run_ax(c, make_args(c, xd, yd, stream));
  if (e == cudaSuccess) e = cudaMemcpyAsync(Y_host, yd, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "ax_local_host_static");
  return AX_OK;
}
