// Deterministic block and grid reductions shared by the solver kernels.
// Every sum has a fixed order (a fixed grid, a fixed tree), so results do not
// depend on scheduling.  The grid-level sum is finished inside the producing
// kernel by the block that arrives last (a release fence and an atomic count).
#pragma once

#include <cuda_runtime.h>

namespace ax {
namespace red {

constexpr int kThreads = 256;  // block size of every kernel that uses these helpers

// Fixed-order block reduction of v into out[blockIdx.x] (double accumulation).
__device__ __forceinline__ void block_reduce_store(double v, double *out) {
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
}

// Fixed-order block reduction of two values at once, out_a[blockIdx.x] and
// out_b[blockIdx.x]: the warp-level tree in the values' own type T (float
// sums stay on the FP32 pipe; GB300's FP64 rate is 1/64 of it), the eight
// warp results in double.  One CTA barrier.
template <typename T>
__device__ __forceinline__ void block_reduce2_store(T a, T b, double *out_a, double *out_b) {
  __shared__ double sh[2][kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = (double)a;
    sh[1][wid] = (double)b;
  }
  __syncthreads();
  if (wid == 0) {
    double va = lane < kThreads / 32 ? sh[0][lane] : 0.0, vb = lane < kThreads / 32 ? sh[1][lane] : 0.0;
    for (int o = kThreads / 64; o > 0; o >>= 1) {
      va += __shfl_down_sync(0xffffffffu, va, o);
      vb += __shfl_down_sync(0xffffffffu, vb, o);
    }
    if (lane == 0) {
      *out_a = va;
      if (out_b) *out_b = vb;
    }
  }
}

// Returns true in the block that arrives last at *cnt (after every block has
// written its partial: a release fence before the count) and resets *cnt.
__device__ __forceinline__ bool arrive_last(unsigned *cnt) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    if (last) *cnt = 0u;
  }
  __syncthreads();
  return last;
}

// Fixed-order sum of partial[0..nb) by one block (the last to arrive), read
// past L1: the partials were written by other SMs in this launch.
__device__ __forceinline__ double sum_partials(const double *partial, int nb) {
  __shared__ double total;
  double s = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) s += __ldcg(partial + q);
  block_reduce_store(s, &total);
  __syncthreads();
  return total;
}

// Fixed-order sums of two partial arrays a[0..nb), b[0..nb) by one block
// (the last to arrive), read past L1.
__device__ __forceinline__ void sum_partials2(const double *pa, const double *pb, int nb, double &ta, double &tb) {
  __shared__ double total[2];
  double sa = 0.0, sb = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) {
    sa += __ldcg(pa + q);
    sb += __ldcg(pb + q);
  }
  block_reduce2_store<double>(sa, sb, &total[0], &total[1]);
  __syncthreads();
  ta = total[0];
  tb = total[1];
}

}  // namespace red
}  // namespace ax
