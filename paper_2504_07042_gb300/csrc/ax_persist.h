// Persistent batched AxLocal and batched CG iteration (ax_persist.cu):
// internal interface used by the batch layer (ax_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ax_internal.h"

namespace ax {
namespace persist {

constexpr int kThreads = 128;  // CTA of the persistent kernel: the widest order shape for N1 <= 10
constexpr int kMaxOrder = 9;   // orders the persistent kernel carries (N1 = 2..10)
constexpr long long kDefaultBudgetNs = 2000000000LL;  // bound of one dependency wait: 2 s
// global nodes per vector item of the CG phases (32 per thread): few enough
// items that the dequeue, wait and arrival cost stays small per node
constexpr int64_t kChunk = 4096;

// One order group of the batch: a context over the union of its meshes'
// elements (float32 geometry records), its elements at loc in the batch's
// local vector.
struct Group {
  int N1 = 0;
  int64_t E = 0, loc = 0;
  const void *geo = nullptr, *lam = nullptr;
};

// An AxLocal item: elements [e0, e0 + cnt) of group `group`, all of mesh `mesh`.
struct AxItem {
  int group = 0, mesh = 0;
  int64_t e0 = 0;
  int cnt = 0;
};

// Device view of the queue (kernel argument).
struct Sched {
  int B = 0;
  const Group *groups = nullptr;
  const AxItem *ax = nullptr;
  int n_ax = 0;
  const int *ax_need = nullptr;  // [B] AxLocal items per mesh
  // vector chunks (kChunk global nodes, never across meshes): chunk c covers
  // global nodes [clo[c], chi[c]) of mesh cmesh[c]; mesh m owns chunks [pbeg[m], pbeg[m+1])
  int n_chunks = 0;
  const int *cmesh = nullptr;
  const int64_t *clo = nullptr, *chi = nullptr;
  const int *pbeg = nullptr;
  // control words (device, zero at rest): ticket, exit count, status, abort flag, then cnt[3][B]
  int *ticket = nullptr, *exitc = nullptr, *status = nullptr, *abortf = nullptr, *cnt = nullptr;
  long long budget_ns = kDefaultBudgetNs;
  int stuck_mesh = -1;  // test hook: this mesh's chunks wait for one AxLocal item too many
};

// The CG state of the batch (float32 vectors; per-mesh scalars in S[m][16]).
struct Vecs {
  float *p = nullptr, *z = nullptr, *r = nullptr, *x = nullptr, *w = nullptr, *Yl = nullptr;
  const float *inv = nullptr;
  const gidx *gid = nullptr, *off = nullptr, *idx = nullptr;
  const uint8_t *mask = nullptr;
  double *S = nullptr, *part = nullptr;  // part: [3][n_chunks]
};

// Host-side plan of one batch.
struct Plan {
  int kind = 0, B = 0;
  std::vector<Group> groups;             // per order group
  std::vector<int> tile_blocks;          // per group: element blocks per AxLocal item (autotuned)
  std::vector<int> mesh_group;           // per mesh
  std::vector<int64_t> mesh_e0, mesh_E;  // per mesh: first element within its group, element count
  std::vector<int64_t> glob_off;         // [B + 1] offsets of the meshes in the batch's global vector
  int grid_mult = 0;                     // CTAs = grid_mult x SMs (0: the occupancy limit)
  int sms = 0, occ = 0;
  size_t smem = 0;
  Sched sc;                              // device pointers (owned)
  Group *groups_d = nullptr;
  AxItem *ax_d = nullptr;
  int *ax_need_d = nullptr, *ctl_d = nullptr;
  int *cmesh_d = nullptr, *pbeg_d = nullptr;
  int64_t *clo_d = nullptr, *chi_d = nullptr;
};

// Whether a batch of these orders and this precision runs on the persistent kernel.
bool supported(ax_precision prec, const std::vector<int> &orders);
// Build (or rebuild, after tile_blocks changed) the device queue.
cudaError_t plan_build(Plan &pl, cudaStream_t s);
void plan_free(Plan &pl);
// Clear the status and abort words (before a solve).
cudaError_t plan_reset(Plan &pl, cudaStream_t s);
int plan_grid(const Plan &pl);
// AxLocal of the whole batch: one launch.
cudaError_t launch_local(const Plan &pl, const float *X, float *Y, cudaStream_t s);
// One CG iteration of every mesh: one launch.
cudaError_t launch_iteration(const Plan &pl, const Vecs &v, cudaStream_t s);
// Elements per block of an order (the persistent CTA's shape).
int epb_of(int N1);

}  // namespace persist
}  // namespace ax
