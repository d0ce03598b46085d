// Gather-scatter (Eq. 1: Q and Q^T) and the (P)CG driver around AxLocal.
//
// Q is stored as a CSR from global node to its local copies, built once on
// the host in increasing local order, so every sum below has a fixed order
// and the results are deterministic (no atomics).  Dirichlet nodes are
// masked: their rows and columns are dropped from the assembled operator.
//
// CG is the textbook preconditioned conjugate gradient method (Jacobi
// preconditioner = the assembled diagonal of the operator).  Scalars live
// on the device; dot products are two-stage reductions with a fixed grid
// (deterministic).  The host reads one scalar per iteration (||r||^2) for
// the convergence test.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "ax_internal.h"
#include "reduce.cuh"

namespace ax {
namespace gs {

// stage-1 blocks of every reduction: fixed, so that every sum has one order
// (determinism); four per SM of a 152-SM GB300, all resident in one wave
constexpr int kRedBlocks = 608;
constexpr int kRedThreads = 256;

template <typename T>
__global__ void scatter_kernel(int64_t n_local, const gidx *__restrict__ gid, const T *__restrict__ u,
                               T *__restrict__ U) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n_local; m += (int64_t)gridDim.x * blockDim.x)
    U[m] = u[gid[m]];
}

// y[g] = sum of the local copies of g (0 on masked nodes)
template <typename T>
__global__ void gather_kernel(int64_t n_global, const gidx *__restrict__ off, const gidx *__restrict__ idx,
                              const T *__restrict__ Y, T *__restrict__ y, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_global; g += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
    y[g] = (mask && mask[g]) ? T(0) : s;
  }
}

// Y <- Q Q^T Y in place
template <typename T>
__global__ void assemble_kernel(int64_t n_global, const gidx *__restrict__ off, const gidx *__restrict__ idx,
                                T *__restrict__ Y) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_global; g += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
    for (gidx q = off[g]; q < off[g + 1]; ++q) Y[idx[q]] = s;
  }
}

// partial[b] = sum over this block's slice of a*b
template <typename T>
__global__ void __launch_bounds__(kRedThreads) dot_kernel(int64_t n, const T *__restrict__ a, const T *__restrict__ b,
                                                          double *__restrict__ partial) {
  double s = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    s += (double)a[g] * (double)b[g];
  red::block_reduce_store(s, partial + blockIdx.x);
}

// final stage: out = sum(partial[0..nb)) (one block)
__global__ void __launch_bounds__(kRedThreads) finish_kernel(const double *__restrict__ partial, int nb,
                                                             double *__restrict__ out) {
  double s = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) s += partial[q];
  red::block_reduce_store(s, out);
}

// Scalars S: [0] rz, [1] pw, [2] rr, [3] bb, [4] rz_new, [5] sigma (mixed
// precision), [6] done flag, [7] iteration at which the test was met
// (negative: NaN), [8] tol^2 = rtol^2 bb, [9] iterations issued,
// [10] alpha, [11] beta.  alpha and beta are divided once per iteration by
// one thread: FP64 division is a long sequence on GB300's slow FP64 pipe.
// Vector kernels accumulate their partial dot products in their own type T
// (no float -> double conversions per element on the FP64 pipe).
// Once done is set, the kernels of an iteration return at once, so
// iterations queued after convergence leave x unchanged (the host checks
// every few iterations).
//
// One CG iteration is four launches:
//   direction_scatter  p = z + beta p;  U = Q p              (global -> local)
//   AxLocal            W = A_e U                             (per element)
//   gather_dot_alpha   w = mask(Q^T W);  alpha = rz / (p.w)  (last block)
//   update_check       x += alpha p; r -= alpha w; z = M^-1 r;
//                      rz_new, rr; test; beta = rz_new / rz  (last block)
constexpr int kScalars = 16;

// The vector kernels take four nodes per thread and pass (g, g + stride,
// g + 2 stride, g + 3 stride: each access coalesced across the warp) and
// issue all their loads before the first store, so that a thread has four
// independent memory round trips in flight instead of one; the nodes are
// summed in the same order as one node per pass would.  Two nodes in
// float64 (the update kernel's five vectors of four doubles spill at the
// 64 registers that four resident blocks per SM allow).
template <typename T>
constexpr int kUnroll = sizeof(T) == 8 ? 2 : 4;

template <typename T>
__global__ void direction_scatter_kernel(int64_t n_global, const double *__restrict__ S, const T *__restrict__ z,
                                         T *__restrict__ p, const gidx *__restrict__ off,
                                         const gidx *__restrict__ idx, T *__restrict__ U) {
  if (S[6] != 0.0) return;
  constexpr int kU = kUnroll<T>;
  const T beta = (T)S[11];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + (kU - 1) * stride < n_global; g += kU * stride) {
    T zv[kU], pv[kU];
    gidx b[kU], e[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t q = g + u * stride;
      zv[u] = z[q];
      pv[u] = p[q];
      b[u] = off[q];
      e[u] = off[q + 1];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const T pg = zv[u] + beta * pv[u];
      p[g + u * stride] = pg;
      for (gidx q = b[u]; q < e[u]; ++q) U[idx[q]] = pg;
    }
  }
  for (; g < n_global; g += stride) {
    const T pg = z[g] + beta * p[g];
    p[g] = pg;
    for (gidx q = off[g]; q < off[g + 1]; ++q) U[idx[q]] = pg;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads, kRedBlocks / 152)
    gather_dot_alpha_kernel(int64_t n_global, const gidx *__restrict__ off, const gidx *__restrict__ idx,
                            const T *__restrict__ Y, T *__restrict__ w, const uint8_t *__restrict__ mask,
                            const T *__restrict__ p, double *__restrict__ partial, unsigned *__restrict__ cnt,
                            double *__restrict__ S) {
  if (S[6] != 0.0) return;
  constexpr int kU = kUnroll<T>;
  T d = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + (kU - 1) * stride < n_global; g += kU * stride) {
    T s[kU], pv[kU];
    gidx b[kU], e[kU];
    bool mv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t q = g + u * stride;
      b[u] = off[q];
      e[u] = off[q + 1];
      pv[u] = p[q];
      mv[u] = mask && mask[q];
    }
    // the first local copy of the four nodes at once (a node without any
    // copy sums to zero), then the rest
#pragma unroll
    for (int u = 0; u < kU; ++u) s[u] = b[u] < e[u] ? T(0) + Y[idx[b[u]]] : T(0);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      for (gidx q = b[u] + 1; q < e[u]; ++q) s[u] += Y[idx[q]];
      if (mv[u]) s[u] = T(0);
      w[g + u * stride] = s[u];
      d += pv[u] * s[u];
    }
  }
  for (; g < n_global; g += stride) {
    T s = T(0);
    for (gidx q = off[g]; q < off[g + 1]; ++q) s += Y[idx[q]];
    if (mask && mask[g]) s = T(0);
    w[g] = s;
    d += p[g] * s;
  }
  red::block_reduce2_store<T>(d, T(0), partial + blockIdx.x, nullptr);
  if (!red::arrive_last(cnt)) return;
  const double pw = red::sum_partials(partial, gridDim.x);
  if (threadIdx.x == 0) {
    S[1] = pw;
    S[10] = pw != 0.0 ? S[0] / pw : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads, kRedBlocks / 152)
    update_check_kernel(int64_t n, double *__restrict__ S, const T *__restrict__ p, const T *__restrict__ w,
                        T *__restrict__ x, T *__restrict__ r, T *__restrict__ z, const T *__restrict__ inv_diag,
                        const uint8_t *__restrict__ mask, double *__restrict__ part_rz, double *__restrict__ part_rr,
                        unsigned *__restrict__ cnt) {
  if (S[6] != 0.0) return;
  constexpr int kU = kUnroll<T>;
  const T alpha = (T)S[10];
  T rz = T(0), rr = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + (kU - 1) * stride < n; g += kU * stride) {
    T xv[kU], pv[kU], rv[kU], wv[kU], iv[kU];
    bool mv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t q = g + u * stride;
      xv[u] = x[q];
      pv[u] = p[q];
      rv[u] = r[q];
      wv[u] = w[q];
      iv[u] = inv_diag ? inv_diag[q] : T(1);
      mv[u] = mask && mask[q];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t q = g + u * stride;
      const T rg = rv[u] - alpha * wv[u];
      T zg = inv_diag ? rg * iv[u] : rg;
      if (mv[u]) zg = T(0);
      x[q] = xv[u] + alpha * pv[u];
      r[q] = rg;
      z[q] = zg;
      rz += rg * zg;
      rr += rg * rg;
    }
  }
  for (; g < n; g += stride) {
    const T xg = x[g] + alpha * p[g];
    const T rg = r[g] - alpha * w[g];
    T zg = inv_diag ? rg * inv_diag[g] : rg;
    if (mask && mask[g]) zg = T(0);
    x[g] = xg;
    r[g] = rg;
    z[g] = zg;
    rz += rg * zg;
    rr += rg * rg;
  }
  red::block_reduce2_store<T>(rz, rr, part_rz + blockIdx.x, part_rr + blockIdx.x);
  if (!red::arrive_last(cnt)) return;
  double rz_new, rr_new;
  red::sum_partials2(part_rz, part_rr, gridDim.x, rz_new, rr_new);
  if (threadIdx.x == 0) {
    S[4] = rz_new;
    S[2] = rr_new;
    S[11] = S[0] != 0.0 ? rz_new / S[0] : 0.0;
    S[0] = rz_new;
    const double it = S[9] + 1.0;
    S[9] = it;
    if (rr_new <= S[8]) {
      S[6] = 1.0;
      S[7] = it;
    } else if (!(rr_new == rr_new)) {
      S[6] = 1.0;
      S[7] = -it;
    }
  }
}

__global__ void set_kernel(double *S, int idx, double v) { S[idx] = v; }

// initial: r = b - w (masked), z = r * inv_diag, p = z; partials of r.z, r.r, b.b
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    init_kernel(int64_t n, const T *__restrict__ b, const T *__restrict__ w, T *__restrict__ r, T *__restrict__ z,
                T *__restrict__ p, const T *__restrict__ inv_diag, const uint8_t *__restrict__ mask,
                double *__restrict__ part_rz, double *__restrict__ part_rr, double *__restrict__ part_bb) {
  T rz = T(0), rr = T(0), bb = T(0);
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const bool m = mask && mask[g];
    const T bg = m ? T(0) : b[g];
    const T rg = m ? T(0) : bg - w[g];
    const T zg = m ? T(0) : (inv_diag ? rg * inv_diag[g] : rg);
    r[g] = rg;
    z[g] = zg;
    p[g] = zg;
    rz += rg * zg;
    rr += rg * rg;
    bb += bg * bg;
  }
  red::block_reduce_store((double)rz, part_rz + blockIdx.x);
  __syncthreads();
  red::block_reduce_store((double)rr, part_rr + blockIdx.x);
  __syncthreads();
  red::block_reduce_store((double)bb, part_bb + blockIdx.x);
}

template <typename T>
__global__ void mask_zero_kernel(int64_t n, T *__restrict__ x, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (mask[g]) x[g] = T(0);
}

template <typename T>
__global__ void invert_kernel(int64_t n, const T *__restrict__ d, T *__restrict__ inv, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    inv[g] = (mask && mask[g]) ? T(0) : T(1) / d[g];
}

inline unsigned grid_for(int64_t n, int block = 256) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 65535 * 16) g = 65535 * 16;
  return (unsigned)g;
}

}  // namespace gs

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

cudaError_t gs_build(GsPlan &plan, const int64_t *gid_dev, int64_t n_local, int64_t n_global, const uint8_t *mask_dev,
                     cudaStream_t s, int64_t *bad_ids) {
  *bad_ids = 0;
  std::vector<int64_t> gid((size_t)n_local);
  cudaError_t e = cudaMemcpyAsync(gid.data(), gid_dev, sizeof(int64_t) * n_local, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  std::vector<gidx> off((size_t)n_global + 1, 0);
  for (int64_t m = 0; m < n_local; ++m) {
    const int64_t g = gid[m];
    if (g < 0 || g >= n_global) {
      ++*bad_ids;
      continue;
    }
    ++off[g + 1];
  }
  if (*bad_ids) return cudaSuccess;
  for (int64_t g = 0; g < n_global; ++g) off[g + 1] += off[g];
  std::vector<gidx> idx((size_t)n_local), gid32((size_t)n_local), fill(off.begin(), off.end() - 1);
  for (int64_t m = 0; m < n_local; ++m) {
    gid32[m] = (gidx)gid[m];
    idx[fill[gid[m]]++] = (gidx)m;  // increasing local order per global node
  }
  plan.n_global = n_global;
  plan.n_local = n_local;
  const size_t nl1 = n_local > 0 ? (size_t)n_local : 1;
  e = cudaMalloc(&plan.off, sizeof(gidx) * (n_global + 1));
  if (e == cudaSuccess) e = cudaMalloc(&plan.idx, sizeof(gidx) * nl1);
  if (e == cudaSuccess) e = cudaMalloc(&plan.gid, sizeof(gidx) * nl1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(plan.off, off.data(), sizeof(gidx) * (n_global + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_local)
    e = cudaMemcpyAsync(plan.idx, idx.data(), sizeof(gidx) * n_local, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_local)
    e = cudaMemcpyAsync(plan.gid, gid32.data(), sizeof(gidx) * n_local, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && mask_dev) {
    e = cudaMalloc(&plan.mask, n_global > 0 ? n_global : 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan.mask, mask_dev, n_global, cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors die with this scope
  return e;
}

void gs_free(GsPlan &plan) {
  cudaFree(plan.off);
  cudaFree(plan.idx);
  cudaFree(plan.gid);
  cudaFree(plan.mask);
  plan = GsPlan();
}

template <typename T>
static cudaError_t gs_assemble_t(const GsPlan &p, void *Y, cudaStream_t s) {
  if (p.n_global == 0) return cudaSuccess;
  gs::assemble_kernel<T><<<gs::grid_for(p.n_global), 256, 0, s>>>(p.n_global, p.off, p.idx, (T *)Y);
  return cudaGetLastError();
}
template <typename T>
static cudaError_t gs_gather_t(const GsPlan &p, const void *Y, void *y, cudaStream_t s) {
  if (p.n_global == 0) return cudaSuccess;
  gs::gather_kernel<T><<<gs::grid_for(p.n_global), 256, 0, s>>>(p.n_global, p.off, p.idx, (const T *)Y, (T *)y,
                                                                 p.mask);
  return cudaGetLastError();
}
template <typename T>
static cudaError_t gs_scatter_t(const GsPlan &p, const void *u, void *U, cudaStream_t s) {
  if (p.n_local == 0) return cudaSuccess;
  gs::scatter_kernel<T><<<gs::grid_for(p.n_local), 256, 0, s>>>(p.n_local, p.gid, (const T *)u, (T *)U);
  return cudaGetLastError();
}

cudaError_t gs_assemble_run(const GsPlan &p, bool f64, void *Y, cudaStream_t s) {
  return f64 ? gs_assemble_t<double>(p, Y, s) : gs_assemble_t<float>(p, Y, s);
}
cudaError_t gs_gather_run(const GsPlan &p, bool f64, const void *Y, void *y, cudaStream_t s) {
  return f64 ? gs_gather_t<double>(p, Y, y, s) : gs_gather_t<float>(p, Y, y, s);
}
cudaError_t gs_scatter_run(const GsPlan &p, bool f64, const void *u, void *U, cudaStream_t s) {
  return f64 ? gs_scatter_t<double>(p, u, U, s) : gs_scatter_t<float>(p, u, U, s);
}

// Work vectors of one CG solve (allocated once per solve, reused across the
// inner solves of the mixed-precision driver), with the private stream and
// the instantiated graph of kCheck iterations.
constexpr int kCheck = 16;  // iterations per graph launch (between host checks)

template <typename T>
struct PcgWork {
  int64_t n = 0, nl = 0;
  T *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr, *Ul = nullptr, *Yl = nullptr, *inv = nullptr;
  double *S = nullptr, *part = nullptr, *hS = nullptr;
  unsigned *cnt = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void *graph_b = nullptr;  // the (b, x, preconditioner, operator) the graph was captured for
  void *graph_x = nullptr;
  bool graph_jac = false;
  const void *graph_op = nullptr;
  bool jac = false;  // Jacobi on: inv holds the inverted diagonal
  T *inv_or_null() const { return jac ? inv : nullptr; }
  cudaError_t alloc(int64_t n_, int64_t nl_, bool jacobi) {
    n = n_;
    nl = nl_;
    cudaError_t e = cudaMalloc(&r, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Ul, sizeof(T) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&Yl, sizeof(T) * nl);
    (void)jacobi;
    if (e == cudaSuccess) e = cudaMalloc(&inv, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(double) * gs::kScalars);
    if (e == cudaSuccess) e = cudaMemset(S, 0, sizeof(double) * gs::kScalars);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 3 * gs::kRedBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(unsigned) * 2);
    if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(unsigned) * 2);
    if (e == cudaSuccess) e = cudaMallocHost(&hS, sizeof(double) * gs::kScalars);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    return e;
  }
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    cudaFree(r); cudaFree(z); cudaFree(p); cudaFree(w); cudaFree(Ul); cudaFree(Yl); cudaFree(inv);
    cudaFree(S); cudaFree(part); cudaFree(cnt); cudaFreeHost(hS);
    *this = PcgWork();
  }
};

// One CG iteration (four launches) on stream s.
template <typename T>
static cudaError_t pcg_iteration(const GsPlan &P, const AxArgs &a, cudaError_t (*launch)(const AxArgs &),
                                 PcgWork<T> &W, T *x, cudaStream_t s) {
  const int64_t n = P.n_global;
  const int RB = gs::kRedBlocks, RT = gs::kRedThreads;
  gs::direction_scatter_kernel<T><<<gs::grid_for(n), 256, 0, s>>>(n, W.S, W.z, W.p, P.off, P.idx, W.Ul);
  cudaError_t e = launch(a);
  if (e != cudaSuccess) return e;
  gs::gather_dot_alpha_kernel<T><<<RB, RT, 0, s>>>(n, P.off, P.idx, W.Yl, W.w, P.mask, W.p, W.part + 2 * RB, W.cnt,
                                                   W.S);
  gs::update_check_kernel<T><<<RB, RT, 0, s>>>(n, W.S, W.p, W.w, x, W.r, W.z, W.inv_or_null(), P.mask, W.part, W.part + RB,
                                               W.cnt + 1);
  return cudaGetLastError();
}

// (P)CG on the assembled masked system with work W (W.inv already holds the
// inverted diagonal when Jacobi is on).  launch() runs AxLocal on W.Ul -> W.Yl.
// Setup runs on the caller's stream s; the iterations run as graph launches
// of kCheck iterations on the work's private stream (ordered after s by an
// event, and s after it on return); the host reads the scalars after each.
template <typename T>
static cudaError_t pcg_core(const GsPlan &P, const AxArgs &base, cudaError_t (*launch)(const AxArgs &), PcgWork<T> &W,
                            const T *b, T *x, double rtol, int maxit, int *iters, double *relres, int *converged,
                            cudaStream_t s) {
  const int64_t n = P.n_global, nl = P.n_local;
  const int RB = gs::kRedBlocks, RT = gs::kRedThreads;
  AxArgs a = base;
  a.X = W.Ul;
  a.Y = W.Yl;
  a.stream = s;
  *iters = 0;
  *relres = 0.0;
  *converged = 0;
  double *S = W.S, *part = W.part, *hS = W.hS;
  if (P.mask) gs::mask_zero_kernel<T><<<gs::grid_for(n), 256, 0, s>>>(n, x, P.mask);
  gs::scatter_kernel<T><<<gs::grid_for(nl), 256, 0, s>>>(nl, P.gid, x, W.Ul);
  cudaError_t e = launch(a);
  if (e != cudaSuccess) return e;
  gs::gather_kernel<T><<<gs::grid_for(n), 256, 0, s>>>(n, P.off, P.idx, W.Yl, W.w, P.mask);
  gs::init_kernel<T><<<RB, RT, 0, s>>>(n, b, W.w, W.r, W.z, W.p, W.inv_or_null(), P.mask, part, part + RB,
                                       part + 2 * RB);
  gs::finish_kernel<<<1, RT, 0, s>>>(part, RB, S + 0);
  gs::finish_kernel<<<1, RT, 0, s>>>(part + RB, RB, S + 2);
  gs::finish_kernel<<<1, RT, 0, s>>>(part + 2 * RB, RB, S + 3);
  e = cudaMemcpyAsync(hS, S, sizeof(double) * gs::kScalars, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const double bnorm = std::sqrt(hS[3]);
  double rnorm = std::sqrt(hS[2]);
  int it = 0;
  if (bnorm == 0.0 || rnorm <= rtol * bnorm) {
    *converged = 1;
  } else {
    gs::set_kernel<<<1, 1, 0, s>>>(S, 8, rtol * rtol * hS[3]);
    gs::set_kernel<<<1, 1, 0, s>>>(S, 6, 0.0);
    gs::set_kernel<<<1, 1, 0, s>>>(S, 9, 0.0);
    gs::set_kernel<<<1, 1, 0, s>>>(S, 11, 0.0);  // first direction: p = z
    cudaStream_t cs = W.cs;
    e = cudaEventRecord(W.ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, W.ev, 0);
    a.stream = cs;
    if (e == cudaSuccess && maxit >= kCheck &&
        (!W.exec || W.graph_b != (const void *)b || W.graph_x != (void *)x || W.graph_jac != W.jac ||
         W.graph_op != base.geo)) {
      if (W.exec) cudaGraphExecDestroy(W.exec);
      W.exec = nullptr;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      for (int q = 0; q < kCheck && e == cudaSuccess; ++q) e = pcg_iteration<T>(P, a, launch, W, x, cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = ec;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&W.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) {
        W.graph_b = b;
        W.graph_x = x;
        W.graph_jac = W.jac;
        W.graph_op = base.geo;
      }
    }
    int issued = 0;
    while (e == cudaSuccess && issued < maxit) {
      const int block = (maxit - issued) < kCheck ? (maxit - issued) : kCheck;
      if (block == kCheck) {
        e = cudaGraphLaunch(W.exec, cs);
      } else {
        for (int q = 0; q < block && e == cudaSuccess; ++q) e = pcg_iteration<T>(P, a, launch, W, x, cs);
      }
      issued += block;
      if (e == cudaSuccess) e = cudaMemcpyAsync(hS, S, sizeof(double) * gs::kScalars, cudaMemcpyDeviceToHost, cs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
      if (e != cudaSuccess) break;
      rnorm = std::sqrt(hS[2]);
      if (hS[6] != 0.0) {
        if (hS[7] > 0.0) {
          *converged = 1;
          it = (int)hS[7];
        } else {
          it = (int)(-hS[7]);
        }
        break;
      }
      it = issued;
    }
    const cudaError_t e2 = cudaEventRecord(W.ev, cs);
    if (e2 == cudaSuccess) cudaStreamWaitEvent(s, W.ev, 0);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e;
  }
  *iters = it;
  *relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

template <typename T>
static void delete_work(void *p) {
  PcgWork<T> *W = static_cast<PcgWork<T> *>(p);
  W->release();
  delete W;
}

// The context's cached work of type T (allocated on first use).
template <typename T>
static cudaError_t cached_work(Ctx &ctx, int slot, PcgWork<T> **out) {
  PcgWork<T> *W = static_cast<PcgWork<T> *>(ctx.ws[slot]);
  if (W && (W->n != ctx.gs.n_global || W->nl != ctx.gs.n_local)) {
    ctx.ws_del[slot](W);
    ctx.ws[slot] = nullptr;
    W = nullptr;
  }
  if (!W) {
    W = new (std::nothrow) PcgWork<T>;
    if (!W) return cudaErrorMemoryAllocation;
    cudaError_t e = W->alloc(ctx.gs.n_global, ctx.gs.n_local, true);
    if (e != cudaSuccess) {
      delete_work<T>(W);
      return e;
    }
    ctx.ws[slot] = W;
    ctx.ws_del[slot] = delete_work<T>;
  }
  *out = W;
  return cudaSuccess;
}

template <typename T>
static cudaError_t pcg_t(Ctx &ctx, int slot, const AxArgs &base, cudaError_t (*launch)(const AxArgs &), const T *b,
                         T *x, const T *diag_global, double rtol, int maxit, int *iters, double *relres,
                         int *converged, cudaStream_t s) {
  const GsPlan &P = ctx.gs;
  PcgWork<T> *W = nullptr;
  cudaError_t e = cached_work<T>(ctx, slot, &W);
  if (e != cudaSuccess) return e;
  W->jac = diag_global != nullptr;
  if (W->jac) gs::invert_kernel<T><<<gs::grid_for(P.n_global), 256, 0, s>>>(P.n_global, diag_global, W->inv, P.mask);
  return pcg_core<T>(P, base, launch, *W, b, x, rtol, maxit, iters, relres, converged, s);
}

cudaError_t pcg_run(Ctx &ctx, bool f64, const AxArgs &base, cudaError_t (*launch)(const AxArgs &), const void *b,
                    void *x, const void *diag_global, double rtol, int maxit, int *iters, double *relres,
                    int *converged, cudaStream_t s) {
  if (f64)
    return pcg_t<double>(ctx, Ctx::kWsCg64, base, launch, (const double *)b, (double *)x, (const double *)diag_global,
                         rtol, maxit, iters, relres, converged, s);
  return pcg_t<float>(ctx, Ctx::kWsCg32, base, launch, (const float *)b, (float *)x, (const float *)diag_global, rtol,
                      maxit, iters, relres, converged, s);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP64 iterative refinement around an inner FP32 solve.
//   r = b - A x            (hi context: FP64-accurate AxLocal, float64 vectors)
//   A d = r / sigma        (lo context: inner Jacobi-PCG in float32 to inner_rtol)
//   x = x + sigma d        (sigma = ||r||_inf keeps the float32 data near 1)
// until ||r||_2 <= rtol ||b||_2.
// ---------------------------------------------------------------------------
namespace gs {
__global__ void residual_kernel(int64_t n, const double *__restrict__ b, const double *__restrict__ w,
                                double *__restrict__ r, const uint8_t *__restrict__ mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    r[g] = (mask && mask[g]) ? 0.0 : b[g] - w[g];
}
__global__ void __launch_bounds__(kRedThreads) norms_kernel(int64_t n, const double *__restrict__ r,
                                                            double *__restrict__ part2, double *__restrict__ partinf) {
  double s = 0.0, m = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    s += r[g] * r[g];
    m = fmax(m, fabs(r[g]));
  }
  red::block_reduce_store(s, part2 + blockIdx.x);
  __syncthreads();
  // max: fixed-order warp/block max
  __shared__ double sh[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = m;
  __syncthreads();
  if (wid == 0) {
    m = lane < kRedThreads / 32 ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) partinf[blockIdx.x] = m;
  }
}
__global__ void __launch_bounds__(kRedThreads) finish_max_kernel(const double *__restrict__ part, int nb,
                                                                 double *__restrict__ out) {
  __shared__ double sh[kRedThreads];
  double m = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) m = fmax(m, part[q]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}
__global__ void scale_down_kernel(int64_t n, const double *__restrict__ r, const double *__restrict__ sig,
                                  float *__restrict__ r32, float *__restrict__ d32) {
  const double inv = *sig > 0.0 ? 1.0 / *sig : 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    r32[g] = (float)(r[g] * inv);
    d32[g] = 0.0f;
  }
}
__global__ void correct_kernel(int64_t n, const float *__restrict__ d32, const double *__restrict__ sig,
                               double *__restrict__ x) {
  const double sg = *sig;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] += sg * (double)d32[g];
}
}  // namespace gs

// Work of the mixed-precision driver: the inner float32 CG work plus the
// outer float64 vectors (kept in the high-precision context between calls).
struct MixedWork {
  PcgWork<float> W;
  double *r = nullptr, *w = nullptr, *Ul = nullptr, *Yl = nullptr, *S = nullptr, *part = nullptr, *hS = nullptr;
  float *r32 = nullptr, *d32 = nullptr;
  cudaError_t alloc(int64_t n, int64_t nl) {
    cudaError_t e = W.alloc(n, nl, true);
    if (e == cudaSuccess) e = cudaMalloc(&r, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Ul, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&Yl, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&r32, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d32, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(double) * gs::kScalars);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * 2 * gs::kRedBlocks);
    if (e == cudaSuccess) e = cudaMallocHost(&hS, sizeof(double) * gs::kScalars);
    return e;
  }
  void release() {
    W.release();
    cudaFree(r); cudaFree(w); cudaFree(Ul); cudaFree(Yl); cudaFree(r32); cudaFree(d32);
    cudaFree(S); cudaFree(part); cudaFreeHost(hS);
  }
};
static void delete_mixed(void *p) {
  MixedWork *M = static_cast<MixedWork *>(p);
  M->release();
  delete M;
}

cudaError_t pcg_mixed_run(Ctx &ctx, const AxArgs &hi, cudaError_t (*launch_hi)(const AxArgs &), const AxArgs &lo,
                          cudaError_t (*launch_lo)(const AxArgs &), const double *b, double *x, const float *diag_lo,
                          double rtol, double inner_rtol, int max_outer, int max_inner, int *outer, int *inner_total,
                          double *relres, int *converged, cudaStream_t s) {
  const GsPlan &P = ctx.gs;
  const int64_t n = P.n_global, nl = P.n_local;
  const int RB = gs::kRedBlocks, RT = gs::kRedThreads;
  *outer = 0;
  *inner_total = 0;
  *relres = 0.0;
  *converged = 0;
  MixedWork *MW = static_cast<MixedWork *>(ctx.ws[Ctx::kWsMixed]);
  cudaError_t e = cudaSuccess;
  if (MW && (MW->W.n != n || MW->W.nl != nl)) {
    delete_mixed(MW);
    ctx.ws[Ctx::kWsMixed] = nullptr;
    MW = nullptr;
  }
  if (!MW) {
    MW = new (std::nothrow) MixedWork;
    if (!MW) return cudaErrorMemoryAllocation;
    e = MW->alloc(n, nl);
    if (e != cudaSuccess) {
      delete_mixed(MW);
      return e;
    }
    ctx.ws[Ctx::kWsMixed] = MW;
    ctx.ws_del[Ctx::kWsMixed] = delete_mixed;
  }
  PcgWork<float> &W = MW->W;
  double *r = MW->r, *w = MW->w, *Ul = MW->Ul, *Yl = MW->Yl, *S = MW->S, *part = MW->part, *hS = MW->hS;
  float *r32 = MW->r32, *d32 = MW->d32;
  W.jac = diag_lo != nullptr;
  if (W.jac) gs::invert_kernel<float><<<gs::grid_for(n), 256, 0, s>>>(n, diag_lo, W.inv, P.mask);
  AxArgs ah = hi;
  ah.X = Ul;
  ah.Y = Yl;
  ah.stream = s;
  double bnorm = 0.0;
  {
    // ||b|| over the unmasked nodes: r = b - 0 (masked)
    gs::mask_zero_kernel<double><<<gs::grid_for(n), 256, 0, s>>>(n, x, P.mask);
    e = cudaMemsetAsync(w, 0, sizeof(double) * n, s);
    gs::residual_kernel<<<gs::grid_for(n), 256, 0, s>>>(n, b, w, r, P.mask);
    gs::norms_kernel<<<RB, RT, 0, s>>>(n, r, part, part + RB);
    gs::finish_kernel<<<1, RT, 0, s>>>(part, RB, S + 3);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hS, S, sizeof(double) * gs::kScalars, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    bnorm = std::sqrt(hS[3]);
  }
  while (e == cudaSuccess) {
    // r = b - A x in FP64-accurate arithmetic
    gs::scatter_kernel<double><<<gs::grid_for(nl), 256, 0, s>>>(nl, P.gid, x, Ul);
    e = launch_hi(ah);
    if (e != cudaSuccess) break;
    gs::gather_kernel<double><<<gs::grid_for(n), 256, 0, s>>>(n, P.off, P.idx, Yl, w, P.mask);
    gs::residual_kernel<<<gs::grid_for(n), 256, 0, s>>>(n, b, w, r, P.mask);
    gs::norms_kernel<<<RB, RT, 0, s>>>(n, r, part, part + RB);
    gs::finish_kernel<<<1, RT, 0, s>>>(part, RB, S + 2);
    gs::finish_max_kernel<<<1, RT, 0, s>>>(part + RB, RB, S + 5);
    e = cudaMemcpyAsync(hS + 2, S + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    const double rn = std::sqrt(hS[2]);
    *relres = bnorm > 0.0 ? rn / bnorm : 0.0;
    if (bnorm == 0.0 || rn <= rtol * bnorm) {
      *converged = 1;
      break;
    }
    if (!(rn == rn) || *outer >= max_outer) break;
    // inner solve A d = r / sigma in float32
    gs::scale_down_kernel<<<gs::grid_for(n), 256, 0, s>>>(n, r, S + 5, r32, d32);
    int it = 0, conv = 0;
    double rr = 0.0;
    e = pcg_core<float>(P, lo, launch_lo, W, r32, d32, inner_rtol, max_inner, &it, &rr, &conv, s);
    if (e != cudaSuccess) break;
    *inner_total += it;
    gs::correct_kernel<<<gs::grid_for(n), 256, 0, s>>>(n, d32, S + 5, x);
    ++*outer;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace ax
