// One persistent launch over a batch of meshes of uneven size and order
// (float32 arithmetic, orders N = 1..9).
//
// AxLocal of a batch (Algorithm 1 on every element of every mesh) is one
// kernel: a device work queue of (mesh, element tile) items, dequeued by the
// CTAs with an atomic ticket, each item run by the fiber-per-thread block
// code of ax_fiber.cuh for its order (a runtime switch over the orders; the
// CTA is shaped for the widest of them, threads beyond an order's shape take
// part in the barriers only).
//
// One CG iteration of every mesh of the batch (Eq. 1: A = Q^T blkdiag(A^e) Q,
// Jacobi-preconditioned) is the same kernel with four kinds of items, queued
// phase after phase:
//   AX  AxLocal tiles, X read as the local copies of the search direction
//       (X[m] = p[gid[m]]: the scatter Q p fused into the load)
//   GD  chunks of global nodes: w = mask(Q^T Y), partial p.w; the last chunk
//       of a mesh to finish sums the partials in a fixed order and sets alpha
//   UP  chunks: x += alpha p, r -= alpha w, z = D^-1 r, partial r.z, r.r; the
//       last one sets beta, counts the iteration and tests convergence
//   DI  chunks: p = z + beta p
// An item waits (thread 0, bounded spin on a per-mesh arrival counter) until
// the items of the previous phase of its mesh have arrived.  Items are
// dequeued in queue order and an item only waits on items queued before it,
// which running CTAs already hold, so the waits end without any CTA having
// to be co-resident.  A wait that exceeds its time budget records
// AX_ETIMEOUT, raises an abort flag that every other wait and the dequeue
// loop test, and returns; the host reads the status after the launch.  The
// last CTA to exit resets the ticket and the counters for the next launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "ax_internal.h"
#include "ax_persist.h"

// float32 tables of this translation unit (no per-order launcher)
#define AX_POLICY fiber::Native<float>
#define AX_CT float
#define AX_TAG fp32_persist
#define AX_N_LIST(X)
#include "inst_fiber.inc"

namespace ax {
namespace persist {

using P = fiber::Native<float>;
constexpr int kS = 16;  // per-mesh scalars, same slots as the batched CG of ax_batch.cu
constexpr int kU = 4;   // gather-dot: nodes per thread whose gathers are in flight together

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: wait until *cnt >= target, at most budget_ns.  false when the
// batch aborted (another wait timed out) or this wait timed out.
__device__ bool wait_count(const int *cnt, int target, const Sched &sc) {
  const unsigned long long t0 = now_ns();
  for (;;) {
    if (ld_acquire(cnt) >= target) return true;
    if (*(volatile int *)sc.abortf) return false;
    if (now_ns() - t0 > (unsigned long long)sc.budget_ns) {
      atomicCAS(sc.status, 0, (int)AX_ETIMEOUT);
      atomicExch(sc.abortf, 1);
      return false;
    }
    __nanosleep(128);
  }
}

// CTA-wide wait (all threads call it): true when the dependency is met.
__device__ bool cta_wait(const int *cnt, int target, const Sched &sc) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = wait_count(cnt, target, sc) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  const bool r = ok != 0;
  __syncthreads();
  return r;
}

// Thread 0 after the CTA's writes: publish them, then count the arrival.
// Returns (to every thread) whether this CTA was the last of `need`.
__device__ bool cta_arrive(int *cnt, int need) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(cnt, 1) == need - 1) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  const bool r = last != 0;
  __syncthreads();
  return r;
}

// Sum over the CTA (fixed order: deterministic); result valid in every thread.
__device__ double cta_sum(double v) {
  __shared__ double sh[kThreads / 32];
  __shared__ double res;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += sh[q];
    res = s;
  }
  __syncthreads();
  const double r = res;
  __syncthreads();
  return r;
}

// One AxLocal tile: elements [e0, e0 + cnt) of group g, in blocks of EPB.
// Not inlined: each order keeps its own register allocation (inlined into
// one body, the nine orders' code took every register there is).
template <int N1, int KIND, bool PCG>
__device__ __noinline__ void ax_tile(unsigned char *smem, const Group &g, int64_t e0, int cnt, const float *X, const float *p,
                        const gidx *gid, float *Y) {
  using Sh = fiber::Shape<N1, 1, 0>;
  using Buf = fiber::FiberSmem<P, N1, KIND, 1, 0>;
  static_assert(Sh::threads <= kThreads, "order shape wider than the persistent CTA");
  const Buf sm = Buf::carve(smem);
  const int tid = threadIdx.x;
  float *Yg = Y + g.loc;
  for (int64_t b = e0; b < e0 + cnt; b += Sh::EPB) {
    const int nel = (int)((e0 + cnt - b) < Sh::EPB ? (e0 + cnt - b) : Sh::EPB);
    if constexpr (PCG) {
      fiber::fiber_block<P, N1, KIND, 1, true, 0, fiber::XGather<float>, 0>(
          sm, tid, b, nel, (const float *)g.geo, (const float *)g.lam, fiber::XGather<float>{p, gid + g.loc}, Yg);
    } else {
      fiber::fiber_block<P, N1, KIND, 1, true, 0, fiber::XDirect<float>, 0>(
          sm, tid, b, nel, (const float *)g.geo, (const float *)g.lam, fiber::XDirect<float>{X + g.loc}, Yg);
    }
  }
}

template <int KIND, bool PCG>
__device__ void run_ax(unsigned char *smem, const Sched &sc, const Vecs &v, int item, const float *X, float *Y) {
  const AxItem t = sc.ax[item];
  const Group g = sc.groups[t.group];
  const bool skip = PCG && __ldcg(&v.S[t.mesh * kS + 6]) != 0.0;  // mesh converged in an earlier launch
  if (!skip) {
    switch (g.N1) {
#define PX_CASE(n1) \
  case n1: ax_tile<n1, KIND, PCG>(smem, g, t.e0, t.cnt, X, v.p, v.gid, Y); break;
      PX_CASE(2) PX_CASE(3) PX_CASE(4) PX_CASE(5) PX_CASE(6) PX_CASE(7) PX_CASE(8) PX_CASE(9) PX_CASE(10)
#undef PX_CASE
      default: break;
    }
  }
  if (PCG) cta_arrive(&sc.cnt[t.mesh], 1 << 30);
}

// GD: w = mask(Q^T Y) on the chunk, partial p.w; the mesh's last chunk sets
// S[1] = p.w and alpha = S[0] / p.w (slot 10).
__device__ void run_gd(const Sched &sc, const Vecs &v, int c) {
  const int m = sc.cmesh[c];
  const int stuck = m == sc.stuck_mesh ? 1 : 0;  // test hook: a dependency nothing completes
  if (!cta_wait(&sc.cnt[m], sc.ax_need[m] + stuck, sc)) return;
  const bool done = __ldcg(&v.S[m * kS + 6]) != 0.0;
  float d = 0.0f;
  if (!done) {
    // kU nodes per thread at a time, their gathers issued together (a hexahedral
    // node has at most 8 local copies; more are summed by the tail loop)
    const int64_t hi = sc.chi[c];
    for (int64_t g0 = sc.clo[c] + threadIdx.x; g0 < hi; g0 += kU * kThreads) {
      gidx b[kU], n[kU];
      float s[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t g = g0 + u * kThreads;
        b[u] = g < hi ? v.off[g] : 0;
        n[u] = g < hi ? v.off[g + 1] - b[u] : 0;
        s[u] = 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (q < n[u]) s[u] += __ldcg(&v.Yl[v.idx[b[u] + q]]);
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t g = g0 + u * kThreads;
        if (g >= hi) break;
        for (int q = 8; q < n[u]; ++q) s[u] += __ldcg(&v.Yl[v.idx[b[u] + q]]);
        if (v.mask && v.mask[g]) s[u] = 0.0f;
        v.w[g] = s[u];
        d += v.p[g] * s[u];
      }
    }
  }
  const double ds = cta_sum((double)d);
  if (threadIdx.x == 0) v.part[c] = ds;
  const int need = sc.pbeg[m + 1] - sc.pbeg[m];
  if (cta_arrive(&sc.cnt[sc.B + m], need)) {
    double s = 0.0;
    for (int q = sc.pbeg[m] + threadIdx.x; q < sc.pbeg[m + 1]; q += kThreads) s += __ldcg(&v.part[q]);
    s = cta_sum(s);
    if (threadIdx.x == 0 && !done) {
      v.S[m * kS + 1] = s;
      v.S[m * kS + 10] = s != 0.0 ? __ldcg(&v.S[m * kS + 0]) / s : 0.0;
    }
    cta_arrive(&sc.cnt[sc.B + m], 1 << 30);  // need + 1: alpha is set
  }
}

// UP: x, r, z on the chunk, partial r.z and r.r; the mesh's last chunk sets
// r.z (slot 4), r.r (slot 2), beta (slot 11), counts the iteration and tests
// convergence (the batched CG's seg_check).
__device__ void run_up(const Sched &sc, const Vecs &v, int c) {
  const int m = sc.cmesh[c];
  const int need = sc.pbeg[m + 1] - sc.pbeg[m];
  if (!cta_wait(&sc.cnt[sc.B + m], need + 1, sc)) return;
  const bool done = __ldcg(&v.S[m * kS + 6]) != 0.0;
  float rz = 0.0f, rr = 0.0f;
  if (!done) {
    const float alpha = (float)__ldcg(&v.S[m * kS + 10]);
#pragma unroll 4
    for (int64_t g = sc.clo[c] + threadIdx.x; g < sc.chi[c]; g += kThreads) {
      const float rg = v.r[g] - alpha * __ldcg(&v.w[g]);
      float zg = v.inv ? rg * v.inv[g] : rg;
      if (v.mask && v.mask[g]) zg = 0.0f;
      v.x[g] += alpha * v.p[g];
      v.r[g] = rg;
      v.z[g] = zg;
      rz += rg * zg;
      rr += rg * rg;
    }
  }
  const double rzs = cta_sum((double)rz);
  const double rrs = cta_sum((double)rr);
  if (threadIdx.x == 0) {
    v.part[sc.n_chunks + c] = rzs;
    v.part[2 * sc.n_chunks + c] = rrs;
  }
  if (cta_arrive(&sc.cnt[2 * sc.B + m], need)) {
    double a = 0.0, b = 0.0;
    for (int q = sc.pbeg[m] + threadIdx.x; q < sc.pbeg[m + 1]; q += kThreads) {
      a += __ldcg(&v.part[sc.n_chunks + q]);
      b += __ldcg(&v.part[2 * sc.n_chunks + q]);
    }
    a = cta_sum(a);
    b = cta_sum(b);
    if (threadIdx.x == 0 && !done) {
      double *s = v.S + m * kS;
      s[4] = a;
      s[2] = b;
      const double s0 = __ldcg(&s[0]);
      s[11] = s0 != 0.0 ? a / s0 : 0.0;
      const double it = __ldcg(&s[9]) + 1.0;
      s[9] = it;
      if (b <= __ldcg(&s[8])) {
        s[6] = 1.0;
        s[7] = it;
      } else if (!(b == b)) {
        s[6] = 1.0;
        s[7] = -it;
      } else {
        s[0] = a;
      }
    }
    cta_arrive(&sc.cnt[2 * sc.B + m], 1 << 30);  // need + 1: beta and the test are set
  }
}

// DI: p = z + beta p on the chunk (meshes that converged keep p)
__device__ void run_di(const Sched &sc, const Vecs &v, int c) {
  const int m = sc.cmesh[c];
  const int need = sc.pbeg[m + 1] - sc.pbeg[m];
  if (!cta_wait(&sc.cnt[2 * sc.B + m], need + 1, sc)) return;
  if (__ldcg(&v.S[m * kS + 6]) != 0.0) return;
  const float beta = (float)__ldcg(&v.S[m * kS + 11]);
#pragma unroll 4
  for (int64_t g = sc.clo[c] + threadIdx.x; g < sc.chi[c]; g += kThreads) v.p[g] = __ldcg(&v.z[g]) + beta * v.p[g];
}

// Resident CTAs the register budget is sized for (64 registers a thread, as
// the per-order float32 kernels of these orders use).
constexpr int kMinCtasPersist = 8;

// The persistent kernel.  PCG false: AX items only, X and Y given.  PCG
// true: one CG iteration of every mesh (AX, GD, UP, DI items).
template <int KIND, bool PCG>
__global__ void __launch_bounds__(kThreads, kMinCtasPersist) persist_kernel(Sched sc, Vecs v, const float *__restrict__ X,
                                                           float *__restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const int total = sc.n_ax + (PCG ? 3 * sc.n_chunks : 0);
  for (;;) {
    if (threadIdx.x == 0) s_item = *(volatile int *)sc.abortf ? total : atomicAdd(sc.ticket, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= total) break;
    if (it < sc.n_ax) {
      run_ax<KIND, PCG>(smem, sc, v, it, X, PCG ? v.Yl : Y);
    } else if (PCG) {
      const int k = it - sc.n_ax, ph = k / sc.n_chunks, c = k - ph * sc.n_chunks;
      if (ph == 0)
        run_gd(sc, v, c);
      else if (ph == 1)
        run_up(sc, v, c);
      else
        run_di(sc, v, c);
    }
  }
  // the last CTA out resets the queue for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sc.exitc, 1) == (int)gridDim.x - 1) {
      *sc.ticket = 0;
      for (int q = 0; q < 3 * sc.B; ++q) sc.cnt[q] = 0;
      __threadfence();
      *sc.exitc = 0;
    }
  }
}

}  // namespace persist

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace persist {

namespace {

template <int N1, int KIND>
constexpr size_t smem_of() {
  return fiber::FiberSmem<P, N1, KIND, 1, 0>::bytes;
}
template <int KIND>
size_t smem_max() {
  const size_t v[] = {smem_of<2, KIND>(), smem_of<3, KIND>(), smem_of<4, KIND>(), smem_of<5, KIND>(),
                      smem_of<6, KIND>(), smem_of<7, KIND>(), smem_of<8, KIND>(), smem_of<9, KIND>(),
                      smem_of<10, KIND>()};
  return *std::max_element(v, v + 9);
}

template <bool PCG>
const void *kernel_of(int kind) {
  switch (kind) {
    case AX_GEOM_STORED: return (const void *)persist_kernel<AX_GEOM_STORED, PCG>;
    case AX_GEOM_TRILINEAR: return (const void *)persist_kernel<AX_GEOM_TRILINEAR, PCG>;
    case AX_GEOM_PARALLELEPIPED: return (const void *)persist_kernel<AX_GEOM_PARALLELEPIPED, PCG>;
    case AX_GEOM_TRILINEAR_PARTIAL: return (const void *)persist_kernel<AX_GEOM_TRILINEAR_PARTIAL, PCG>;
    default: return nullptr;
  }
}

size_t smem_for(int kind) {
  switch (kind) {
    case AX_GEOM_STORED: return smem_max<AX_GEOM_STORED>();
    case AX_GEOM_TRILINEAR: return smem_max<AX_GEOM_TRILINEAR>();
    case AX_GEOM_PARALLELEPIPED: return smem_max<AX_GEOM_PARALLELEPIPED>();
    default: return smem_max<AX_GEOM_TRILINEAR_PARTIAL>();
  }
}

cudaError_t prepare_kernel(const void *k, size_t smem, int *occ) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, kThreads, smem);
  return e;
}

}  // namespace

int epb_of(int N1) {
  const int F = N1 * N1;
  return F >= 128 ? 1 : 128 / F;
}

bool supported(ax_precision prec, const std::vector<int> &orders) {
  if (prec != AX_FP32) return false;
  for (int N : orders)
    if (N < 1 || N > kMaxOrder) return false;
  return true;
}

int plan_grid(const Plan &pl) {
  const int per_sm = pl.grid_mult > 0 ? std::min(pl.grid_mult, std::max(pl.occ, 1)) : std::max(pl.occ, 1);
  return per_sm * pl.sms;
}

void plan_free(Plan &pl) {
  cudaFree(pl.cmesh_d);
  cudaFree(pl.clo_d);
  cudaFree(pl.chi_d);
  cudaFree(pl.pbeg_d);
  pl.cmesh_d = nullptr;
  pl.clo_d = pl.chi_d = nullptr;
  pl.pbeg_d = nullptr;
  cudaFree(pl.groups_d);
  cudaFree(pl.ax_d);
  cudaFree(pl.ax_need_d);
  cudaFree(pl.ctl_d);
  pl.groups_d = nullptr;
  pl.ax_d = nullptr;
  pl.ax_need_d = nullptr;
  pl.ctl_d = nullptr;
}

cudaError_t plan_build(Plan &pl, cudaStream_t s) {
  cudaError_t e = upload_tables_fp32_persist(0);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pl.sms, cudaDevAttrMultiProcessorCount, dev);
  pl.smem = smem_for(pl.kind);
  int occ_a = 0, occ_b = 0;
  if (e == cudaSuccess) e = prepare_kernel(kernel_of<false>(pl.kind), pl.smem, &occ_a);
  if (e == cudaSuccess) e = prepare_kernel(kernel_of<true>(pl.kind), pl.smem, &occ_b);
  pl.occ = std::min(occ_a, occ_b);
  if (e != cudaSuccess) return e;
  if (pl.tile_blocks.size() != pl.groups.size()) pl.tile_blocks.assign(pl.groups.size(), 1);
  // items: per mesh, tiles of tile_blocks x EPB elements; larger orders first
  // (longer items), meshes in batch order within an order
  std::vector<AxItem> items;
  std::vector<int> need(pl.B, 0);
  std::vector<int> gorder(pl.groups.size());
  for (size_t g = 0; g < gorder.size(); ++g) gorder[g] = (int)g;
  std::stable_sort(gorder.begin(), gorder.end(), [&](int a, int b) { return pl.groups[a].N1 > pl.groups[b].N1; });
  for (int g : gorder) {
    const int64_t tile = (int64_t)pl.tile_blocks[g] * epb_of(pl.groups[g].N1);
    for (int m = 0; m < pl.B; ++m) {
      if (pl.mesh_group[m] != g) continue;
      for (int64_t a = 0; a < pl.mesh_E[m]; a += tile) {
        AxItem it;
        it.group = g;
        it.mesh = m;
        it.e0 = pl.mesh_e0[m] + a;
        it.cnt = (int)std::min<int64_t>(tile, pl.mesh_E[m] - a);
        items.push_back(it);
        ++need[m];
      }
    }
  }
  // vector chunks of the CG phases: kChunk global nodes, never across meshes
  std::vector<int> cm, pb(pl.B + 1, 0);
  std::vector<int64_t> lo, hi;
  for (int m = 0; m < pl.B; ++m) {
    pb[m] = (int)cm.size();
    for (int64_t g = pl.glob_off[m]; g < pl.glob_off[m + 1]; g += kChunk) {
      cm.push_back(m);
      lo.push_back(g);
      hi.push_back(std::min<int64_t>(g + kChunk, pl.glob_off[m + 1]));
    }
  }
  pb[pl.B] = (int)cm.size();
  plan_free(pl);
  e = cudaMalloc(&pl.groups_d, sizeof(Group) * pl.groups.size());
  if (e == cudaSuccess) e = cudaMalloc(&pl.cmesh_d, sizeof(int) * std::max<size_t>(1, cm.size()));
  if (e == cudaSuccess) e = cudaMalloc(&pl.clo_d, sizeof(int64_t) * std::max<size_t>(1, lo.size()));
  if (e == cudaSuccess) e = cudaMalloc(&pl.chi_d, sizeof(int64_t) * std::max<size_t>(1, hi.size()));
  if (e == cudaSuccess) e = cudaMalloc(&pl.pbeg_d, sizeof(int) * pb.size());
  if (e == cudaSuccess && !cm.empty()) {
    e = cudaMemcpyAsync(pl.cmesh_d, cm.data(), sizeof(int) * cm.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pl.clo_d, lo.data(), sizeof(int64_t) * lo.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pl.chi_d, hi.data(), sizeof(int64_t) * hi.size(), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.pbeg_d, pb.data(), sizeof(int) * pb.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMalloc(&pl.ax_d, sizeof(AxItem) * std::max<size_t>(1, items.size()));
  if (e == cudaSuccess) e = cudaMalloc(&pl.ax_need_d, sizeof(int) * pl.B);
  if (e == cudaSuccess) e = cudaMalloc(&pl.ctl_d, sizeof(int) * (4 + 3 * pl.B));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl.groups_d, pl.groups.data(), sizeof(Group) * pl.groups.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(pl.ax_d, items.data(), sizeof(AxItem) * items.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pl.ax_need_d, need.data(), sizeof(int) * pl.B, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl.ctl_d, 0, sizeof(int) * (4 + 3 * pl.B), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
  if (e != cudaSuccess) return e;
  pl.sc.B = pl.B;
  pl.sc.n_chunks = (int)cm.size();
  pl.sc.cmesh = pl.cmesh_d;
  pl.sc.clo = pl.clo_d;
  pl.sc.chi = pl.chi_d;
  pl.sc.pbeg = pl.pbeg_d;
  pl.sc.groups = pl.groups_d;
  pl.sc.ax = pl.ax_d;
  pl.sc.n_ax = (int)items.size();
  pl.sc.ax_need = pl.ax_need_d;
  pl.sc.ticket = pl.ctl_d;
  pl.sc.exitc = pl.ctl_d + 1;
  pl.sc.status = pl.ctl_d + 2;
  pl.sc.abortf = pl.ctl_d + 3;
  pl.sc.cnt = pl.ctl_d + 4;
  return cudaSuccess;
}

cudaError_t plan_reset(Plan &pl, cudaStream_t s) { return cudaMemsetAsync(pl.ctl_d + 2, 0, 2 * sizeof(int), s); }

cudaError_t launch_local(const Plan &pl, const float *X, float *Y, cudaStream_t s) {
  if (pl.sc.n_ax == 0) return cudaSuccess;
  const int grid = std::min(plan_grid(pl), pl.sc.n_ax);
  Vecs v;
  switch (pl.kind) {
#define PL_CASE(K) \
  case K: persist_kernel<K, false><<<grid, kThreads, pl.smem, s>>>(pl.sc, v, X, Y); break;
    PL_CASE(AX_GEOM_STORED) PL_CASE(AX_GEOM_TRILINEAR) PL_CASE(AX_GEOM_PARALLELEPIPED)
    PL_CASE(AX_GEOM_TRILINEAR_PARTIAL)
#undef PL_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_iteration(const Plan &pl, const Vecs &v, cudaStream_t s) {
  const int total = pl.sc.n_ax + 3 * pl.sc.n_chunks;
  if (total == 0) return cudaSuccess;
  const int grid = std::min(plan_grid(pl), total);
  switch (pl.kind) {
#define PL_CASE(K) \
  case K: persist_kernel<K, true><<<grid, kThreads, pl.smem, s>>>(pl.sc, v, nullptr, nullptr); break;
    PL_CASE(AX_GEOM_STORED) PL_CASE(AX_GEOM_TRILINEAR) PL_CASE(AX_GEOM_PARALLELEPIPED)
    PL_CASE(AX_GEOM_TRILINEAR_PARTIAL)
#undef PL_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace persist
}  // namespace ax
