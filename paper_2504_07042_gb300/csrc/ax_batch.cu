// Batched AxLocal and batched independent CG solves over many meshes of
// uneven size and order.
//
// Layout of a batch of B meshes:
//   - meshes are grouped by order N; each group is one AxLocal context over
//     the union of its meshes' elements (elements are independent in
//     AxLocal, Algorithm 1), so AxLocal over the whole batch is one launch
//     per distinct order;
//   - the batch's local vector is the concatenation of the groups' local
//     vectors; its global vector is the concatenation of the meshes' global
//     vectors; one gather-scatter plan (Eq. 1) covers the union;
//   - every CG scalar (alpha, beta, norms, convergence flag) is per mesh;
//     reductions are segmented by mesh with a fixed block layout
//     (deterministic);
//   - one CG iteration of all meshes is captured once in a CUDA graph and
//     then launched once per iteration (the per-mesh reference runs each
//     mesh's solve with its own launches).
// Autotuning picks, per group (order, geometry kind), the tile variant
// (FP32: elements per CTA) and the grid (one CTA per element block, or a
// persistent grid of k CTAs per SM) by timing the group's AxLocal.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "ax_internal.h"
#include "ax_persist.h"

namespace ax {
namespace batch {

constexpr int kThreads = 256;
constexpr int kChunk = kThreads * 8;  // global nodes per reduction block
constexpr int kS = 16;                // scalars per mesh (same meaning as the single-mesh CG)

__device__ __forceinline__ void block_sum(double v, double *out) {
  __shared__ double sh[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < kThreads / 32 ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *out = v;
  }
  __syncthreads();
}

// Block k covers global nodes [blo[k], bhi[k]) of mesh bmesh[k].
struct Seg {
  const int *bmesh;
  const int64_t *blo, *bhi;
  const int *pbeg;  // [B+1]: partial range of each mesh
};

template <typename T>
__global__ void __launch_bounds__(kThreads)
    seg_gather_dot(Seg sg, const gidx *__restrict__ off, const gidx *__restrict__ idx, const T *__restrict__ Y,
                   T *__restrict__ w, const uint8_t *__restrict__ mask, const T *__restrict__ p,
                   double *__restrict__ part, const double *__restrict__ S) {
  const int m = sg.bmesh[blockIdx.x];
  T d = T(0);
  if (S[m * kS + 6] == 0.0) {
    for (int64_t g = sg.blo[blockIdx.x] + threadIdx.x; g < sg.bhi[blockIdx.x]; g += kThreads) {
      T s = T(0);
      for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
      if (mask && mask[g]) s = T(0);
      w[g] = s;
      d += p[g] * s;
    }
  }
  block_sum((double)d, part + blockIdx.x);
}

// one block per mesh: S[m][slot] = sum of the mesh's partials (+ alpha when slot == 1)
__global__ void __launch_bounds__(kThreads) seg_finish(Seg sg, const double *__restrict__ part, double *__restrict__ S,
                                                       int slot) {
  const int m = blockIdx.x;
  double s = 0.0;
  for (int q = sg.pbeg[m] + threadIdx.x; q < sg.pbeg[m + 1]; q += kThreads) s += part[q];
  __shared__ double res;
  block_sum(s, &res);
  if (threadIdx.x == 0 && S[m * kS + 6] == 0.0) {
    S[m * kS + slot] = res;
    if (slot == 1) S[m * kS + 10] = res != 0.0 ? S[m * kS + 0] / res : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    seg_update(Seg sg, const double *__restrict__ S, const T *__restrict__ p, const T *__restrict__ w,
               T *__restrict__ x, T *__restrict__ r, T *__restrict__ z, const T *__restrict__ inv,
               const uint8_t *__restrict__ mask, double *__restrict__ part_rz, double *__restrict__ part_rr) {
  const int m = sg.bmesh[blockIdx.x];
  T rz = T(0), rr = T(0);
  if (S[m * kS + 6] == 0.0) {
    const T alpha = (T)S[m * kS + 10];
    for (int64_t g = sg.blo[blockIdx.x] + threadIdx.x; g < sg.bhi[blockIdx.x]; g += kThreads) {
      const T rg = r[g] - alpha * w[g];
      T zg = inv ? rg * inv[g] : rg;
      if (mask && mask[g]) zg = T(0);
      x[g] += alpha * p[g];
      r[g] = rg;
      z[g] = zg;
      rz += rg * zg;
      rr += rg * rg;
    }
  }
  block_sum((double)rz, part_rz + blockIdx.x);
  block_sum((double)rr, part_rr + blockIdx.x);
}

// one thread per mesh: count, test convergence, beta
__global__ void seg_check(int B, double *S) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= B) return;
  double *s = S + m * kS;
  if (s[6] != 0.0) return;
  s[11] = s[0] != 0.0 ? s[4] / s[0] : 0.0;
  const double it = s[9] + 1.0;
  s[9] = it;
  if (s[2] <= s[8]) {
    s[6] = 1.0;
    s[7] = it;
  } else if (!(s[2] == s[2])) {
    s[6] = 1.0;
    s[7] = -it;
  } else {
    s[0] = s[4];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    seg_direction(Seg sg, const double *__restrict__ S, const T *__restrict__ z, T *__restrict__ p) {
  const int m = sg.bmesh[blockIdx.x];
  if (S[m * kS + 6] != 0.0) return;
  const T beta = (T)S[m * kS + 11];
  for (int64_t g = sg.blo[blockIdx.x] + threadIdx.x; g < sg.bhi[blockIdx.x]; g += kThreads) p[g] = z[g] + beta * p[g];
}

// r = b - w (masked), z = r inv, p = z; partials of r.z, r.r, b.b
template <typename T>
__global__ void __launch_bounds__(kThreads)
    seg_init(Seg sg, const T *__restrict__ b, const T *__restrict__ w, T *__restrict__ r, T *__restrict__ z,
             T *__restrict__ p, const T *__restrict__ inv, const uint8_t *__restrict__ mask, double *__restrict__ prz,
             double *__restrict__ prr, double *__restrict__ pbb) {
  T rz = T(0), rr = T(0), bb = T(0);
  for (int64_t g = sg.blo[blockIdx.x] + threadIdx.x; g < sg.bhi[blockIdx.x]; g += kThreads) {
    const bool mk = mask && mask[g];
    const T bg = mk ? T(0) : b[g];
    const T rg = mk ? T(0) : bg - w[g];
    const T zg = mk ? T(0) : (inv ? rg * inv[g] : rg);
    r[g] = rg;
    z[g] = zg;
    p[g] = zg;
    rz += rg * zg;
    rr += rg * rg;
    bb += bg * bg;
  }
  block_sum((double)rz, prz + blockIdx.x);
  block_sum((double)rr, prr + blockIdx.x);
  block_sum((double)bb, pbb + blockIdx.x);
}

// per mesh after the init reductions: tol^2, done when already converged
__global__ void seg_start(int B, double *S, double rtol) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= B) return;
  double *s = S + m * kS;
  s[8] = rtol * rtol * s[3];
  s[9] = 0.0;
  s[7] = 0.0;
  s[6] = (s[3] == 0.0 || s[2] <= s[8]) ? 1.0 : 0.0;
}

template <typename T>
__global__ void scatter_u(int64_t n, const gidx *__restrict__ gid, const T *__restrict__ u, T *__restrict__ U) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
    U[m] = u[gid[m]];
}
template <typename T>
__global__ void gather_u(int64_t n, const gidx *__restrict__ off, const gidx *__restrict__ idx,
                         const T *__restrict__ Y, T *__restrict__ y, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
    y[g] = (mask && mask[g]) ? T(0) : s;
  }
}
template <typename T>
__global__ void invert_u(int64_t n, const T *__restrict__ d, T *__restrict__ inv, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    inv[g] = (mask && mask[g]) ? T(0) : T(1) / d[g];
}
template <typename T>
__global__ void mask_zero_u(int64_t n, T *__restrict__ x, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (mask[g]) x[g] = T(0);
}
__global__ void offset_ids(int64_t n, const int64_t *__restrict__ src, int64_t add, int64_t *__restrict__ dst) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
    dst[m] = src[m] + add;
}

inline unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 1 << 20));
}

}  // namespace batch
}  // namespace ax

using namespace ax;

struct ax_batch {
  int B = 0;
  ax_geom_kind kind = AX_GEOM_TRILINEAR;
  ax_precision prec = AX_FP32;
  int device = 0;
  std::vector<int64_t> E;
  std::vector<int> N;
  std::vector<int64_t> loc_off, glob_off;  // per mesh, into the union local / global vectors ([B+1] for global)
  int64_t n_local = 0, n_global = 0;
  struct Group {
    int N = 0;
    std::vector<int> meshes;
    ax_ctx *ctx = nullptr;
    int64_t loc_begin = 0, E = 0;
    int tile = 0;
    int64_t grid = 0;
  };
  std::vector<Group> groups;
  std::vector<ax_ctx *> mesh_ctx;  // per-mesh contexts: the per-mesh reference solve
  GsPlan gs;
  // reduction segmentation
  int nblk = 0;
  int *bmesh = nullptr;
  int64_t *blo = nullptr, *bhi = nullptr;
  int *pbeg = nullptr;
  cudaStream_t cs = nullptr;  // private stream: graph capture needs a non-legacy stream
  // one persistent launch for AxLocal and per CG iteration (float32, N <= 9)
  persist::Plan *ps = nullptr;
  bool use_persist = false;
  std::string err;
};

namespace {

thread_local std::string g_batch_err;

ax_status bfail(ax_batch *b, ax_status st, const std::string &m) {
  if (b)
    b->err = m;
  else
    g_batch_err = m;
  return st;
}

ax_status bcuda(ax_batch *b, cudaError_t e, const char *what) {
  (void)cudaGetLastError();
  return bfail(b, e == cudaErrorMemoryAllocation ? AX_ENOMEM : AX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool f64_prec(ax_precision p) { return p == AX_FP64 || p == AX_F64DW; }

void batch_release(ax_batch *b) {
  if (b->ps) {
    persist::plan_free(*b->ps);
    delete b->ps;
    b->ps = nullptr;
  }
  for (auto &g : b->groups) ax_destroy(g.ctx);
  for (auto *c : b->mesh_ctx) ax_destroy(c);
  b->groups.clear();
  b->mesh_ctx.clear();
  gs_free(b->gs);
  cudaFree(b->bmesh);
  cudaFree(b->blo);
  cudaFree(b->bhi);
  cudaFree(b->pbeg);
  if (b->cs) cudaStreamDestroy(b->cs);
  b->bmesh = nullptr;
  b->blo = b->bhi = nullptr;
  b->pbeg = nullptr;
  b->cs = nullptr;
}

cudaError_t (*launcher(ax_precision p))(const AxArgs &) { return ax_launcher_of((int)p); }

AxArgs group_args(const ax_batch *b, const ax_batch::Group &g, const void *X, void *Y, cudaStream_t s) {
  const size_t w = f64_prec(b->prec) ? 8 : 4;
  AxArgs a = ax_ctx_args(g.ctx);
  a.X = (const char *)X + g.loc_begin * w;
  a.Y = (char *)Y + g.loc_begin * w;
  a.stream = s;
  a.tile = g.tile;
  a.grid = g.grid;
  return a;
}

}  // namespace

extern "C" {

const char *ax_batch_last_error(const ax_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

ax_status ax_batch_setup(ax_batch **out, int B, const int64_t *E, const int *N, const double *const *vertices,
                         const int64_t *const *global_id, const int64_t *n_global, const uint8_t *const *mask,
                         ax_geom_kind kind, ax_precision prec, void *stream) {
  if (!out) return bfail(nullptr, AX_EINVAL, "ax_batch_setup: out is NULL");
  *out = nullptr;
  if (B < 1 || !E || !N || !vertices || !global_id || !n_global)
    return bfail(nullptr, AX_EINVAL, "ax_batch_setup: bad arguments");
  if (!launcher(prec)) return bfail(nullptr, AX_EUNSUPPORTED, "ax_batch_setup: precision has no AxLocal kernel");
  ax_batch *b = new (std::nothrow) ax_batch;
  if (!b) return bfail(nullptr, AX_ENOMEM, "ax_batch_setup: host allocation failed");
  b->B = B;
  b->kind = kind;
  b->prec = prec;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&b->device);
  for (int m = 0; m < B; ++m) {
    if (E[m] < 1 || N[m] < 1 || N[m] > kMaxN || n_global[m] < 1 || !vertices[m] || !global_id[m]) {
      delete b;
      return bfail(nullptr, AX_EINVAL, "ax_batch_setup: bad mesh " + std::to_string(m));
    }
    b->E.push_back(E[m]);
    b->N.push_back(N[m]);
  }
  // groups by order, meshes in batch order within a group
  std::map<int, int> group_of;
  for (int m = 0; m < B; ++m) {
    if (!group_of.count(N[m])) {
      group_of[N[m]] = (int)b->groups.size();
      b->groups.emplace_back();
      b->groups.back().N = N[m];
    }
    b->groups[group_of[N[m]]].meshes.push_back(m);
  }
  b->loc_off.assign(B, 0);
  b->glob_off.assign(B + 1, 0);
  for (int m = 0; m < B; ++m) b->glob_off[m + 1] = b->glob_off[m] + n_global[m];
  b->n_global = b->glob_off[B];
  int64_t loc = 0;
  for (auto &g : b->groups) {
    g.loc_begin = loc;
    const int64_t n3 = (int64_t)(g.N + 1) * (g.N + 1) * (g.N + 1);
    for (int m : g.meshes) {
      b->loc_off[m] = loc;
      g.E += E[m];
      loc += E[m] * n3;
    }
  }
  b->n_local = loc;
  if (b->n_local >= kMaxGsIndex || b->n_global >= kMaxGsIndex) {
    delete b;
    return bfail(nullptr, AX_ERANGE, "ax_batch_setup: more than 2^31 - 1 local or global nodes");
  }
  // group contexts over the union of their meshes' elements
  double *vtx = nullptr;
  int64_t *gid_u = nullptr;
  uint8_t *mask_u = nullptr;
  ax_status st = AX_OK;
  for (auto &g : b->groups) {
    if (e != cudaSuccess) break;
    e = cudaMalloc(&vtx, sizeof(double) * 24 * g.E);
    int64_t at = 0;
    for (int m : g.meshes) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(vtx + 24 * at, vertices[m], sizeof(double) * 24 * E[m], cudaMemcpyDefault, s);
      at += E[m];
    }
    if (e == cudaSuccess) {
      st = ax_setup(&g.ctx, g.E, g.N, vtx, kind, prec, stream);
      if (st != AX_OK) {
        std::string m = ax_last_error(nullptr);
        cudaFree(vtx);
        batch_release(b);
        delete b;
        return bfail(nullptr, st, "ax_batch_setup: " + m);
      }
    }
    cudaFree(vtx);
    vtx = nullptr;
  }
  // per-mesh contexts (reference path)
  for (int m = 0; m < B && e == cudaSuccess; ++m) {
    ax_ctx *c = nullptr;
    st = ax_setup(&c, E[m], N[m], vertices[m], kind, prec, stream);
    if (st == AX_OK) st = gs_setup(c, global_id[m], n_global[m], mask ? mask[m] : nullptr, stream);
    if (st != AX_OK) {
      std::string msg = ax_last_error(c);
      ax_destroy(c);
      batch_release(b);
      delete b;
      return bfail(nullptr, st, "ax_batch_setup (mesh " + std::to_string(m) + "): " + msg);
    }
    b->mesh_ctx.push_back(c);
  }
  // union gather-scatter plan
  if (e == cudaSuccess) e = cudaMalloc(&gid_u, sizeof(int64_t) * b->n_local);
  if (e == cudaSuccess) e = cudaMalloc(&mask_u, b->n_global);
  for (int m = 0; m < B && e == cudaSuccess; ++m) {
    const int64_t n3 = (int64_t)(N[m] + 1) * (N[m] + 1) * (N[m] + 1);
    batch::offset_ids<<<batch::grid_for(E[m] * n3), 256, 0, s>>>(E[m] * n3, global_id[m], b->glob_off[m],
                                                                  gid_u + b->loc_off[m]);
    if (mask && mask[m])
      e = cudaMemcpyAsync(mask_u + b->glob_off[m], mask[m], n_global[m], cudaMemcpyDefault, s);
    else
      e = cudaMemsetAsync(mask_u + b->glob_off[m], 0, n_global[m], s);
  }
  int64_t bad = 0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = gs_build(b->gs, gid_u, b->n_local, b->n_global, mask_u, s, &bad);
  cudaFree(gid_u);
  cudaFree(mask_u);
  if (e == cudaSuccess && bad) {
    batch_release(b);
    delete b;
    return bfail(nullptr, AX_EINVAL, "ax_batch_setup: global ids out of range");
  }
  // reduction segmentation: blocks of kChunk global nodes, never crossing meshes
  if (e == cudaSuccess) {
    std::vector<int> bm, pb(B + 1, 0);
    std::vector<int64_t> lo, hi;
    for (int m = 0; m < B; ++m) {
      pb[m] = (int)bm.size();
      for (int64_t g = b->glob_off[m]; g < b->glob_off[m + 1]; g += batch::kChunk) {
        bm.push_back(m);
        lo.push_back(g);
        hi.push_back(std::min<int64_t>(g + batch::kChunk, b->glob_off[m + 1]));
      }
    }
    pb[B] = (int)bm.size();
    b->nblk = (int)bm.size();
    e = cudaMalloc(&b->bmesh, sizeof(int) * bm.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->blo, sizeof(int64_t) * lo.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->bhi, sizeof(int64_t) * hi.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->pbeg, sizeof(int) * pb.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->bmesh, bm.data(), sizeof(int) * bm.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->blo, lo.data(), sizeof(int64_t) * lo.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->bhi, hi.data(), sizeof(int64_t) * hi.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->pbeg, pb.data(), sizeof(int) * pb.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
  // the persistent plan: groups, meshes' element ranges, the segmentation
  if (e == cudaSuccess && persist::supported(prec, b->N)) {
    b->ps = new (std::nothrow) persist::Plan;
    if (!b->ps) e = cudaErrorMemoryAllocation;
  }
  if (e == cudaSuccess && b->ps) {
    persist::Plan &pl = *b->ps;
    pl.kind = (int)kind;
    pl.B = B;
    pl.mesh_group.assign(B, 0);
    pl.mesh_e0.assign(B, 0);
    pl.mesh_E.assign(B, 0);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      const auto &g = b->groups[gi];
      const Ctx &core = ax_ctx_core(g.ctx);
      persist::Group pg;
      pg.N1 = g.N + 1;
      pg.E = g.E;
      pg.loc = g.loc_begin;
      pg.geo = core.geo;
      pg.lam = core.lam;
      pl.groups.push_back(pg);
      int64_t at = 0;
      for (int m : g.meshes) {
        pl.mesh_group[m] = (int)gi;
        pl.mesh_e0[m] = at;
        pl.mesh_E[m] = E[m];
        at += E[m];
      }
    }
    pl.glob_off = b->glob_off;
    e = persist::plan_build(pl, s);
    b->use_persist = e == cudaSuccess;
  }
  if (e != cudaSuccess) {
    ax_status r = bcuda(nullptr, e, "ax_batch_setup");
    batch_release(b);
    delete b;
    return r;
  }
  *out = b;
  return AX_OK;
}

ax_status ax_batch_sizes(const ax_batch *b, int64_t *n_local, int64_t *n_global, int64_t *local_offsets,
                         int64_t *global_offsets) {
  if (!b) return AX_EINVAL;
  if (n_local) *n_local = b->n_local;
  if (n_global) *n_global = b->n_global;
  if (local_offsets)
    for (int m = 0; m < b->B; ++m) local_offsets[m] = b->loc_off[m];
  if (global_offsets)
    for (int m = 0; m <= b->B; ++m) global_offsets[m] = b->glob_off[m];
  return AX_OK;
}

ax_status ax_batch_local(ax_batch *b, const void *X, void *Y, void *stream) {
  if (!b) return bfail(nullptr, AX_EINVAL, "ax_batch_local: batch is NULL");
  if (!X || !Y) return bfail(b, AX_EINVAL, "ax_batch_local: NULL vector");
  if (b->use_persist) {
    cudaError_t e = persist::launch_local(*b->ps, (const float *)X, (float *)Y, (cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(b, e, "ax_batch_local");
    return AX_OK;
  }
  cudaError_t (*L)(const AxArgs &) = launcher(b->prec);
  for (auto &g : b->groups) {
    cudaError_t e = L(group_args(b, g, X, Y, (cudaStream_t)stream));
    if (e != cudaSuccess) return bcuda(b, e, "ax_batch_local");
  }
  return AX_OK;
}

namespace {

// Persistent mode: element blocks per AxLocal item for each order group
// (coordinate descent over {1, 2, 4, 8}, groups in turn) and the grid (CTAs
// per SM: the occupancy limit or 1, 2, 4), by timing the whole batch's
// single AxLocal launch.
ax_status tune_persist(ax_batch *b, int *tiles, int64_t *grids, cudaStream_t s) {
  persist::Plan &pl = *b->ps;
  void *X = nullptr, *Y = nullptr;
  cudaError_t e = cudaMalloc(&X, sizeof(float) * b->n_local);
  if (e == cudaSuccess) e = cudaMalloc(&Y, sizeof(float) * b->n_local);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, sizeof(float) * b->n_local, s);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  auto time_it = [&](float *ms) -> cudaError_t {
    cudaError_t r = persist::plan_build(pl, s);
    for (int q = 0; q < 2 && r == cudaSuccess; ++q) r = persist::launch_local(pl, (const float *)X, (float *)Y, s);
    if (r == cudaSuccess) r = cudaEventRecord(t0, s);
    for (int q = 0; q < 5 && r == cudaSuccess; ++q) r = persist::launch_local(pl, (const float *)X, (float *)Y, s);
    if (r == cudaSuccess) r = cudaEventRecord(t1, s);
    if (r == cudaSuccess) r = cudaEventSynchronize(t1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, t0, t1);
    return r;
  };
  float best = 0.0f;
  if (e == cudaSuccess) {
    pl.tile_blocks.assign(pl.groups.size(), 1);
    pl.grid_mult = 0;
    e = time_it(&best);
  }
  const int tile_opts[] = {1, 2, 4, 8};
  for (size_t g = 0; g < pl.groups.size() && e == cudaSuccess; ++g) {
    const int keep = pl.tile_blocks[g];
    int pick = keep;
    for (int t : tile_opts) {
      if (t == keep) continue;
      pl.tile_blocks[g] = t;
      float ms = 0.0f;
      e = time_it(&ms);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        pick = t;
      }
    }
    pl.tile_blocks[g] = pick;
  }
  const int grid_opts[] = {1, 2, 4};
  int gpick = 0;
  for (int gm : grid_opts) {
    if (e != cudaSuccess) break;
    pl.grid_mult = gm;
    float ms = 0.0f;
    e = time_it(&ms);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      gpick = gm;
    }
  }
  pl.grid_mult = gpick;
  if (e == cudaSuccess) e = persist::plan_build(pl, s);
  for (size_t g = 0; g < pl.groups.size(); ++g) {
    if (tiles) tiles[g] = pl.tile_blocks[g];
    if (grids) grids[g] = persist::plan_grid(pl);
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(X);
  cudaFree(Y);
  if (e != cudaSuccess) return bcuda(b, e, "ax_batch_tune");
  return AX_OK;
}

}  // namespace

ax_status ax_batch_tune(ax_batch *b, int *tiles, int64_t *grids, void *stream) {
  if (!b) return bfail(nullptr, AX_EINVAL, "ax_batch_tune: batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->use_persist) return tune_persist(b, tiles, grids, s);
  const size_t w = f64_prec(b->prec) ? 8 : 4;
  void *X = nullptr, *Y = nullptr;
  cudaError_t e = cudaMalloc(&X, w * b->n_local);
  if (e == cudaSuccess) e = cudaMalloc(&Y, w * b->n_local);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, w * b->n_local, s);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  cudaError_t (*L)(const AxArgs &) = launcher(b->prec);
  // tile variants: FP32 one or two element blocks per CTA; one elsewhere
  const int max_tile = (b->prec == AX_FP32) ? 2 : 1;
  const int mults[] = {0, 1, 2, 4, 8};
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    auto &g = b->groups[gi];
    float best = 1e30f;
    int best_tile = 0;
    int64_t best_grid = 0;
    for (int tile = 0; tile < max_tile && e == cudaSuccess; ++tile) {
      for (int mult : mults) {
        g.tile = tile;
        g.grid = (int64_t)mult * sms;
        AxArgs a = group_args(b, g, X, Y, s);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = L(a);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(t0, s);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = L(a);
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) break;
        if (ms < best) {
          best = ms;
          best_tile = tile;
          best_grid = g.grid;
        }
      }
    }
    g.tile = best_tile;
    g.grid = best_grid;
    if (tiles) tiles[gi] = best_tile;
    if (grids) grids[gi] = best_grid;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(X);
  cudaFree(Y);
  if (e != cudaSuccess) return bcuda(b, e, "ax_batch_tune");
  return AX_OK;
}

}  // extern "C"

namespace {

template <typename T>
struct BWork {
  T *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr, *Ul = nullptr, *Yl = nullptr, *inv = nullptr,
    *dl = nullptr;
  double *S = nullptr, *part = nullptr, *hS = nullptr;
};

// one CG iteration of every mesh, on stream s (captured into the graph)
template <typename T>
cudaError_t batch_iteration(ax_batch *b, BWork<T> &W, T *x, cudaStream_t s) {
  using namespace batch;
  const GsPlan &P = b->gs;
  Seg sg{b->bmesh, b->blo, b->bhi, b->pbeg};
  const int RB = b->nblk;
  scatter_u<T><<<grid_for(P.n_local), 256, 0, s>>>(P.n_local, P.gid, W.p, W.Ul);
  cudaError_t (*L)(const AxArgs &) = launcher(b->prec);
  for (auto &g : b->groups) {
    cudaError_t e = L(group_args(b, g, W.Ul, W.Yl, s));
    if (e != cudaSuccess) return e;
  }
  seg_gather_dot<T><<<RB, kThreads, 0, s>>>(sg, P.off, P.idx, W.Yl, W.w, P.mask, W.p, W.part, W.S);
  seg_finish<<<b->B, kThreads, 0, s>>>(sg, W.part, W.S, 1);
  seg_update<T><<<RB, kThreads, 0, s>>>(sg, W.S, W.p, W.w, x, W.r, W.z, W.inv, P.mask, W.part, W.part + RB);
  seg_finish<<<b->B, kThreads, 0, s>>>(sg, W.part, W.S, 4);
  seg_finish<<<b->B, kThreads, 0, s>>>(sg, W.part + RB, W.S, 2);
  seg_check<<<(b->B + 127) / 128, 128, 0, s>>>(b->B, W.S);
  seg_direction<T><<<RB, kThreads, 0, s>>>(sg, W.S, W.z, W.p);
  return cudaGetLastError();
}

template <typename T>
ax_status batch_pcg(ax_batch *b, const T *bvec, T *x, double rtol, int maxit, int *iters, double *relres,
                    cudaStream_t user) {
  using namespace batch;
  const GsPlan &P = b->gs;
  const int64_t n = P.n_global, nl = P.n_local;
  const int RB = b->nblk, B = b->B;
  cudaStream_t s = b->cs;
  BWork<T> W;
  cudaError_t e = cudaMalloc(&W.r, sizeof(T) * n);
  if (e == cudaSuccess) e = cudaMalloc(&W.z, sizeof(T) * n);
  if (e == cudaSuccess) e = cudaMalloc(&W.p, sizeof(T) * n);
  if (e == cudaSuccess) e = cudaMalloc(&W.w, sizeof(T) * n);
  if (e == cudaSuccess) e = cudaMalloc(&W.inv, sizeof(T) * n);
  if (e == cudaSuccess) e = cudaMalloc(&W.Ul, sizeof(T) * nl);
  if (e == cudaSuccess) e = cudaMalloc(&W.Yl, sizeof(T) * nl);
  if (e == cudaSuccess) e = cudaMalloc(&W.dl, sizeof(T) * nl);
  if (e == cudaSuccess) e = cudaMalloc(&W.S, sizeof(double) * kS * B);
  if (e == cudaSuccess) e = cudaMalloc(&W.part, sizeof(double) * 3 * RB);
  if (e == cudaSuccess) e = cudaMallocHost(&W.hS, sizeof(double) * kS * B);
  cudaEvent_t ev = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  // the solve runs on the batch's private stream, ordered after the caller's work
  if (e == cudaSuccess) e = cudaEventRecord(ev, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(W.S, 0, sizeof(double) * kS * B, s);
  // Jacobi diagonal of every group, gathered over the union
  for (auto &g : b->groups) {
    if (e != cudaSuccess) break;
    const size_t w = sizeof(T);
    e = setup_diag(ax_ctx_core(g.ctx), ax_ctx_vertices(g.ctx), (char *)W.dl + g.loc_begin * w, sizeof(T) == 8, s);
  }
  if (e == cudaSuccess) {
    gather_u<T><<<grid_for(n), 256, 0, s>>>(n, P.off, P.idx, W.dl, W.w, P.mask);
    invert_u<T><<<grid_for(n), 256, 0, s>>>(n, W.w, W.inv, P.mask);
    // w = A x0, with x0 zero on the Dirichlet nodes
    if (P.mask) mask_zero_u<T><<<grid_for(n), 256, 0, s>>>(n, x, P.mask);
    scatter_u<T><<<grid_for(nl), 256, 0, s>>>(nl, P.gid, x, W.Ul);
    cudaError_t (*L)(const AxArgs &) = launcher(b->prec);
    for (auto &g : b->groups)
      if (e == cudaSuccess) e = L(group_args(b, g, W.Ul, W.Yl, s));
  }
  Seg sg{b->bmesh, b->blo, b->bhi, b->pbeg};
  if (e == cudaSuccess) {
    gather_u<T><<<grid_for(n), 256, 0, s>>>(n, P.off, P.idx, W.Yl, W.w, P.mask);
    seg_init<T><<<RB, kThreads, 0, s>>>(sg, bvec, W.w, W.r, W.z, W.p, W.inv, P.mask, W.part, W.part + RB,
                                        W.part + 2 * RB);
    seg_finish<<<B, kThreads, 0, s>>>(sg, W.part, W.S, 0);
    seg_finish<<<B, kThreads, 0, s>>>(sg, W.part + RB, W.S, 2);
    seg_finish<<<B, kThreads, 0, s>>>(sg, W.part + 2 * RB, W.S, 3);
    seg_start<<<(B + 127) / 128, 128, 0, s>>>(B, W.S, rtol);
    e = cudaGetLastError();
  }
  // capture one iteration: one persistent launch (float32, N <= 9) or the
  // per-phase launches
  const bool one_launch = sizeof(T) == 4 && b->use_persist;
  persist::Vecs pv;
  if (one_launch) {
    pv.p = (float *)W.p;
    pv.z = (float *)W.z;
    pv.r = (float *)W.r;
    pv.x = (float *)x;
    pv.w = (float *)W.w;
    pv.Yl = (float *)W.Yl;
    pv.inv = (const float *)W.inv;
    pv.gid = P.gid;
    pv.off = P.off;
    pv.idx = P.idx;
    pv.mask = P.mask;
    pv.S = W.S;
    pv.part = W.part;
    if (e == cudaSuccess) e = persist::plan_reset(*b->ps, s);
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = one_launch ? persist::launch_iteration(*b->ps, pv, s) : batch_iteration<T>(b, W, x, s);
    e = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
  int issued = 0;
  bool all_done = false;
  int pstatus = 0;  // persistent kernel: status word (AX_ETIMEOUT after a wait ran out)
  while (e == cudaSuccess && issued < maxit && !all_done && pstatus == 0) {
    const int block = std::min(16, maxit - issued);
    for (int q = 0; q < block && e == cudaSuccess; ++q) e = cudaGraphLaunch(gexec, s);
    issued += block;
    if (e == cudaSuccess) e = cudaMemcpyAsync(W.hS, W.S, sizeof(double) * kS * B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && one_launch)
      e = cudaMemcpyAsync(&pstatus, b->ps->sc.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    all_done = true;
    for (int m = 0; m < B && e == cudaSuccess; ++m)
      if (W.hS[m * kS + 6] == 0.0) all_done = false;
  }
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(W.hS, W.S, sizeof(double) * kS * B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  int not_conv = 0;
  for (int m = 0; m < B && e == cudaSuccess; ++m) {
    const double *sm = W.hS + m * kS;
    const bool done = sm[6] != 0.0;
    iters[m] = done ? (int)std::fabs(sm[7]) : issued;
    relres[m] = sm[3] > 0.0 ? std::sqrt(sm[2] / sm[3]) : 0.0;
    if (!done || sm[7] < 0.0) ++not_conv;
  }
  if (pstatus != 0 && e == cudaSuccess) {
    // clear the status and abort words so the batch's next calls run
    e = persist::plan_reset(*b->ps, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (e == cudaSuccess) e = cudaEventRecord(ev, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev, 0);
  if (ev) cudaEventDestroy(ev);
  cudaFree(W.r); cudaFree(W.z); cudaFree(W.p); cudaFree(W.w); cudaFree(W.inv); cudaFree(W.Ul); cudaFree(W.Yl);
  cudaFree(W.dl); cudaFree(W.S); cudaFree(W.part); cudaFreeHost(W.hS);
  if (e != cudaSuccess) return bcuda(b, e, "ax_batch_pcg");
  if (pstatus != 0)
    return bfail(b, AX_ETIMEOUT,
                 "ax_batch_pcg: a dependency wait of the persistent iteration ran past its budget; the solve stopped");
  if (not_conv) return bfail(b, AX_ENOTCONV, "ax_batch_pcg: " + std::to_string(not_conv) + " meshes not converged");
  return AX_OK;
}

}  // namespace

extern "C" {

ax_status ax_batch_pcg(ax_batch *b, const void *b_global, void *x_global, double rtol, int maxit, int graph,
                       int *iters, double *relres, void *stream) {
  if (!b) return bfail(nullptr, AX_EINVAL, "ax_batch_pcg: batch is NULL");
  if (!b_global || !x_global || !iters || !relres || maxit < 0 || !(rtol >= 0.0))
    return bfail(b, AX_EINVAL, "ax_batch_pcg: bad arguments");
  const size_t w = f64_prec(b->prec) ? 8 : 4;
  if (graph) {
    if (f64_prec(b->prec))
      return batch_pcg<double>(b, (const double *)b_global, (double *)x_global, rtol, maxit, iters, relres,
                               (cudaStream_t)stream);
    return batch_pcg<float>(b, (const float *)b_global, (float *)x_global, rtol, maxit, iters, relres,
                            (cudaStream_t)stream);
  }
  // reference: every mesh solved on its own, with its own launches
  int not_conv = 0;
  for (int m = 0; m < b->B; ++m) {
    ax_status st = pcg_solve(b->mesh_ctx[m], (const char *)b_global + b->glob_off[m] * w,
                             (char *)x_global + b->glob_off[m] * w, rtol, maxit, 1, &iters[m], &relres[m], stream);
    if (st == AX_ENOTCONV)
      ++not_conv;
    else if (st != AX_OK)
      return bfail(b, st, std::string("ax_batch_pcg (per mesh): ") + ax_last_error(b->mesh_ctx[m]));
  }
  if (not_conv) return bfail(b, AX_ENOTCONV, "ax_batch_pcg: " + std::to_string(not_conv) + " meshes not converged");
  return AX_OK;
}

ax_status ax_batch_set_persistent(ax_batch *b, int on) {
  if (!b) return bfail(nullptr, AX_EINVAL, "ax_batch_set_persistent: batch is NULL");
  if (on && !b->ps)
    return bfail(b, AX_EUNSUPPORTED,
                 "ax_batch_set_persistent: the persistent kernel takes AX_FP32 batches of orders N <= 9");
  b->use_persist = on != 0;
  return AX_OK;
}

ax_status ax_batch_info(const ax_batch *b, int *persistent, int *local_launches, int *iteration_launches) {
  if (!b) return AX_EINVAL;
  const int groups = (int)b->groups.size();
  if (persistent) *persistent = b->use_persist ? 1 : 0;
  if (local_launches) *local_launches = b->use_persist ? 1 : groups;
  // grouped iteration: scatter, one AxLocal per group, gather + dot, 3 segmented
  // sums, update, convergence test, direction
  if (iteration_launches) *iteration_launches = b->use_persist ? 1 : groups + 7;
  return AX_OK;
}

ax_status ax_batch_set_wait(ax_batch *b, int64_t budget_ns, int stuck_mesh) {
  if (!b) return bfail(nullptr, AX_EINVAL, "ax_batch_set_wait: batch is NULL");
  if (!b->ps) return bfail(b, AX_EUNSUPPORTED, "ax_batch_set_wait: the batch has no persistent kernel");
  if (budget_ns <= 0 || stuck_mesh < -1 || stuck_mesh >= b->B)
    return bfail(b, AX_EINVAL, "ax_batch_set_wait: budget must be positive, stuck_mesh in [-1, B)");
  b->ps->sc.budget_ns = budget_ns;
  b->ps->sc.stuck_mesh = stuck_mesh;
  return AX_OK;
}

void ax_batch_destroy(ax_batch *b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

}  // extern "C"
