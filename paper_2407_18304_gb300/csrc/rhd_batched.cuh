// rhd_batched.cuh -- many uneven grids in persistent launches.
//
// A work item is (grid j, tile t): cells [t*cpi, (t+1)*cpi) of grid j.  The
// items of a set of grids are numbered consecutively (item_off[k] is grid
// sel[k]'s first item), and a CTA takes the next item from a device counter
// (atomicAdd; no waiting, so nothing can spin).  The queue balances the
// uneven grids and the uneven per-cell iteration counts across the CTAs.
// Each CTA keeps the group table of its current grid in shared memory and
// reloads it only when the grid changes.
//
// The grids fall into buckets by group count (up to 16, 17..32, 33..64); each
// bucket has its own mapping of cells to lanes -- one cell per thread, or L
// lanes per cell with GPL groups each -- for the passes and for the
// correction step, chosen per bucket (rhd_context_autotune times them).  The
// FP64 form is one launch of FP64 passes per bucket; the mixed form runs a
// grid's phases as the one-grid call runs them (FP32 passes, the correction
// step's float-float first step and its FP64 steps, FP64 passes for the cells
// it did not finish), each phase one launch per bucket, handing over through
// the grid's own workspace.
// Per cell the algorithm is the one-grid call's (the same device functions).
#pragma once
#include "rhd_correct.cuh"
#include "rhd_fp64.cuh"
#include "rhd_mixed.cuh"
#include "rhd_refine.cuh"
#include "rhd_warp.cuh"
#include "rhd_warp32.cuh"

namespace rhd {

constexpr int kMaxGB = RHD_MAX_GROUPS_BATCHED;
// shared memory of a batched CTA: the Planck polynomials and the largest table
constexpr size_t kBatchTableBytes = ((sizeof(double) * kPlanckWords +
                                      sizeof(double) * (kTableArrays * kMaxGB + 1) +
                                      sizeof(float) * (4 * kMaxGB + 1) + 64) + 15) & ~(size_t)15;

// The group-table arrays of build_table for G groups starting at sm, with
// the Planck polynomials at pc.
__device__ __forceinline__ GroupTable table_view(const double *sm, int G, const double *pc) {
  const double *xe = sm, *kbar = sm + G + 1, *ikbar = kbar + G, *rm = ikbar + G, *rp = rm + G,
               *alp = rp + G;
  const float *xef = reinterpret_cast<const float *>(alp + G), *rmf = xef + G + 1, *rpf = rmf + G,
              *alf = rpf + G;
  return GroupTable{xe, kbar, ikbar, rm, rp, alp, xef, rmf, rpf, alf, pc};
}

__host__ __device__ __forceinline__ int group_table_words(int G) {
  return (int)(group_table_bytes(G) / sizeof(double)) + 1;
}

// One CTA per grid: build its group table and write it to tables + j * stride.
__global__ void tables_kernel(const KParams *__restrict__ grids, double *tables, int64_t stride) {
  extern __shared__ double sm[];
  const KParams &P = grids[blockIdx.x];
  build_table(P, sm);
  const int words = group_table_words(P.G);
  double *dst = tables + (int64_t)blockIdx.x * stride;
  for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = sm[kPlanckWords + k];
}

// The work of one launch: the grids sel[0 .. n_sel) with their items, the
// queue head, and (mixed form) each grid's workspace view, by grid index.
struct BatchArgs {
  const KParams *__restrict__ grids;
  const double *__restrict__ tables;
  int64_t table_stride;
  const WarmOut *__restrict__ warm;  // [grid], or null (FP64 form: cold start)
  const int *__restrict__ sel;
  const int64_t *__restrict__ item_off;
  int n_sel, cpi;
  unsigned long long *head;
};

// The FP64 passes' start for grid j: the workspace after the correction step
// (mixed form), or the cold start.
__device__ __forceinline__ WarmStart batch_start(const BatchArgs &A, int j) {
  if (!A.warm) return WarmStart{nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                                nullptr, nullptr, nullptr};
  const WarmOut &w = A.warm[j];
  return WarmStart{w.eint, w.mom, w.r, w.f, w.nit, 1, w.ur, w.uf, w.done};
}

__device__ __forceinline__ WarmStart no_start() {
  return WarmStart{nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
}

// Take items until the queue is empty; for each, make sure the CTA holds its
// grid's table and call body(P, tab, j, c0, c1) with every thread of the CTA.
// Thread 0 takes the item and finds its grid by binary search; the CTA then
// shares it.  The Planck polynomials must already be at sm (made visible by
// the first barrier here).
template <class Body>
__device__ __forceinline__ void for_items(const BatchArgs &A, double *sm, Body &&body) {
  __shared__ long long s_item;
  __shared__ int s_k;
  const int64_t total = A.item_off[A.n_sel];
  int cur = -1;
  GroupTable tab;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(A.head, 1ULL);
      int lo = 0, hi = A.n_sel;  // k with item_off[k] <= it < item_off[k+1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.item_off[mid] <= it) lo = mid;
        else hi = mid;
      }
      s_item = it;
      s_k = lo;
    }
    __syncthreads();
    const long long item = s_item;
    const int k = s_k;
    if (item >= total) break;
    const int j = A.sel[k];
    const KParams &P = A.grids[j];
    if (j != cur) {
      const int words = group_table_words(P.G);
      const double *src = A.tables + (int64_t)j * A.table_stride;
      for (int t = threadIdx.x; t < words; t += blockDim.x) sm[kPlanckWords + t] = src[t];
      cur = j;
      tab = table_view(sm + kPlanckWords, P.G, sm);
    }
    __syncthreads();
    const int64_t c0 = (item - A.item_off[k]) * (int64_t)A.cpi;
    const int64_t c1 = c0 + A.cpi < P.n ? c0 + A.cpi : P.n;
    body(P, tab, j, c0, c1);
    __syncthreads();  // s_item, s_k and the table are reused by the next item
  }
}

// ---- FP32 passes (mixed form) ----------------------------------------------

// One cell per thread, lane-persistent within an item.
template <int MAXG>
__global__ void batched_fp32_kernel(const BatchArgs A) {
  extern __shared__ double sm[];
  load_planck(sm);
  for_items(A, sm, [&](const KParams &P, const GroupTable &tab, int j, int64_t c0, int64_t c1) {
    fp32_cells<MAXG>(P, tab, A.warm[j], no_start(), c0 + threadIdx.x, c1, blockDim.x);
  });
}

// L lanes per cell, GPL groups per lane.
template <int L, int GPL>
__global__ void __launch_bounds__(128) batched_w32_kernel(const BatchArgs A) {
  extern __shared__ double sm[];
  __shared__ float pf[kPlanckF];
  load_planck(sm);
  __syncthreads();
  load_planck32(sm, pf);  // visible after the first barrier of for_items
  const int lane = threadIdx.x & 31, seg = lane / L, l = lane % L, lane0 = seg * L;
  const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << lane0);
  constexpr int CPW = 32 / L;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  WCell32<L, GPL> C;
  for_items(A, sm, [&](const KParams &P, const GroupTable &tab, int j, int64_t c0, int64_t c1) {
    for (int64_t i = c0 + wid * CPW + seg; i < c1; i += nw * CPW)
      w32_cell<L, GPL>(P, tab, pf, A.warm[j], no_start(), i, l, lane0, mask, C);
  });
}

// ---- correction step (mixed form) ------------------------------------------

__device__ __forceinline__ float *batch_blocks(double *sm) {
  return reinterpret_cast<float *>(reinterpret_cast<char *>(sm) + kBatchTableBytes);
}
__host__ __device__ __forceinline__ size_t batch_correct_smem(int GPL) {
  return kBatchTableBytes + sizeof(float) * 20 * GPL * 128;
}

template <int L, int GPL>
__global__ void __launch_bounds__(128) batched_correct_kernel(const BatchArgs A) {
  extern __shared__ double sm[];
  load_planck(sm);
  const int lane = threadIdx.x & 31, seg = lane / L;
  constexpr int CPW = 32 / L;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float *gb = warp_blocks<GPL>(batch_blocks(sm), wid);
  CCell<GPL> C;
  for_items(A, sm, [&](const KParams &P, const GroupTable &tab, int j, int64_t c0, int64_t c1) {
    const WarmOut &w = A.warm[j];
    const CorrOut U{w.ur, w.uf, w.done, 1};
    for (int64_t i = c0 + wid * CPW + seg; i < c1; i += nw * CPW)
      correct_cell<L, GPL>(P, tab, w, U, gb, i, lane, C);
  });
}

// The correction's first step with a float-float residual (rhd_refine.cuh),
// on the correction's mapping and items; the float-float group table after
// the FP64 one, rebuilt when the CTA's grid changes.
__host__ __device__ __forceinline__ size_t batch_refine_smem(int GPL) {
  return kBatchTableBytes + refine_planck_bytes() + refine_df_bytes(kMaxGB) +
         sizeof(float) * 20 * GPL * 128;
}

template <int L, int GPL>
__global__ void __launch_bounds__(128) batched_refine_kernel(const BatchArgs A) {
  extern __shared__ double sm[];
  load_planck(sm);
  __syncthreads();
  const int lane = threadIdx.x & 31, seg = lane / L;
  constexpr int CPW = 32 / L;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  char *base = reinterpret_cast<char *>(batch_blocks(sm));
  // visible after the first barrier of for_items
  const DfPlanck pl = build_df_planck(sm, reinterpret_cast<float *>(base));
  float2 *dfs = reinterpret_cast<float2 *>(base + refine_planck_bytes());
  float *gb = warp_blocks<GPL>(reinterpret_cast<float *>(dfs + 6 * kMaxGB + 1), wid);
  int cur = -1;
  DfTable dt;
  for_items(A, sm, [&](const KParams &P, const GroupTable &tab, int j, int64_t c0, int64_t c1) {
    if (j != cur) {  // every thread of the CTA takes the same branch
      __syncthreads();
      dt = build_df_table(tab, dfs, P.G);
      cur = j;
    }
    const WarmOut &w = A.warm[j];
    const CorrOut U{w.ur, w.uf, w.done, 1};
    for (int64_t i = c0 + wid * CPW + seg; i < c1; i += nw * CPW)
      refine_cell<L, GPL>(P, tab, dt, pl, w, U, gb, i, lane);
  });
}

// ---- FP64 passes (FP64 form; the mixed form's cells left by the correction)

template <int MAXG>
__global__ void batched_fp64_kernel(const BatchArgs A) {
  extern __shared__ double sm[];
  load_planck(sm);
  Arr64<MAXG> R;
  Cell C;
  for_items(A, sm, [&](const KParams &P, const GroupTable &tab, int j, int64_t c0, int64_t c1) {
    const WarmStart W = batch_start(A, j);
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
      fp64_cell<MAXG>(P, tab, W, i, C, R);
  });
}

template <int L, int GPL>
__global__ void __launch_bounds__(128) batched_w64_kernel(const BatchArgs A) {
  extern __shared__ double sm[];
  load_planck(sm);
  const int lane = threadIdx.x & 31, seg = lane / L, l = lane % L, lane0 = seg * L;
  const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << lane0);
  constexpr int CPW = 32 / L;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  WCell<L, GPL> C;
  for_items(A, sm, [&](const KParams &P, const GroupTable &tab, int j, int64_t c0, int64_t c1) {
    const WarmStart W = batch_start(A, j);
    for (int64_t i = c0 + wid * CPW + seg; i < c1; i += nw * CPW)
      warp_cell<L, GPL>(P, tab, W, i, l, lane0, mask, C);
  });
}

}  // namespace rhd
