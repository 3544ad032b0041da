// rhd_batched.cuh -- many uneven grids in one persistent launch.
//
// A work item is (grid j, tile t): cells [t*cpi, (t+1)*cpi) of grid j.  The
// items of all grids are numbered consecutively (item_off[j] is grid j's
// first item), and a CTA takes the next item from a device counter
// (atomicAdd; no waiting, so nothing can spin).  Converged cells retire as
// soon as they are stored; the queue balances the uneven grids and the
// uneven per-cell iteration counts across the CTAs.  Each CTA keeps the group
// table of its current grid in shared memory and reloads it only when the
// grid changes.  Per cell the algorithm is the single-grid one
// (rhd_fp64.cuh, rhd_mixed.cuh).
#pragma once
#include "rhd_fp64.cuh"
#include "rhd_mixed.cuh"
#include "rhd_warp.cuh"
#include "rhd_warp32.cuh"

namespace rhd {

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

// One cell, start to finish.  MIXED: the FP32 pass runs first and its
// result is handed to the FP64 passes exactly as the two-launch form hands it
// over through the workspace (same rounding of R and F to FP32), so both forms
// give identical results.
template <int MAXG, bool MIXED>
__device__ __forceinline__ void solve_cell(const KParams &P, const GroupTable &tab, int64_t i,
                                           Cell &C, Arr64<MAXG> &A, Arr32<MAXG> &B, Cell32 &D) {
  bool warm = false;
  double eint = 0.0, m[3] = {0.0, 0.0, 0.0};
  int nit = 0;
  if (MIXED && load_cell32(P, tab, i, C, D, B)) {
    outer_begin32(P, C, D, B);
    for (;;) {
      const int r = inner_step32(P, tab, C, D, B);
      if (r != 0 && outer_end32(P, tab, C, D, B)) break;
    }
    warm = true;
    eint = C.Eint;
    m[0] = C.m[0];
    m[1] = C.m[1];
    m[2] = C.m[2];
    nit = C.nit > 255 ? 255 : C.nit;
  }
  if (!load_cell(P, i, C, A)) return;
  for (int attempt = 0; attempt < 2; ++attempt) {  // as solve_fp64_kernel (fallback)
    int nit0 = 0;
    if (attempt == 1) {
      if (!(warm && C.stat != RHD_STATUS_OK)) break;
      nit0 = C.nit;
      load_cell(P, i, C, A);
    }
    set_tau(P, tab, C, A, C.chi0s);
    if (warm && attempt == 0) {
      C.Eint = eint;
      C.m[0] = m[0];
      C.m[1] = m[1];
      C.m[2] = m[2];
      C.nit = nit;
      const double fs = P.c * C.Etot;
      for (int g = 0; g < P.G; ++g) {
        A.R[g] = (double)B.R[g] * C.Etot;
        A.Fk[3 * g] = (double)B.f[3 * g] * fs;
        A.Fk[3 * g + 1] = (double)B.f[3 * g + 1] * fs;
        A.Fk[3 * g + 2] = (double)B.f[3 * g + 2] * fs;
      }
    }
    outer_begin(P, C, A);
    for (;;) {
      const int r = inner_step(P, tab, C, A);
      if (r == 0) continue;
      if (r == 2) C.stat = RHD_STATUS_MAXITER;
      if (outer_end(P, tab, C, A)) break;
    }
    if (attempt == 1) {
      C.nit += nit0;
      if (C.stat == RHD_STATUS_OK) C.stat = RHD_STATUS_FALLBACK;
    }
  }
  store_cell(P, C, A);
}

// Work items over the grids sel[0 .. n_sel): item_off[k] is grid sel[k]'s
// first item, item_off[n_sel] the total.  Thread 0 takes the next item from
// *head and finds its grid by binary search; the CTA then shares it.
__device__ __forceinline__ bool next_item(const int64_t *item_off, int n_sel,
                                          unsigned long long *head, long long &s_item,
                                          int &s_k) {
  if (threadIdx.x == 0) {
    const long long it = (long long)atomicAdd(head, 1ULL);
    int lo = 0, hi = n_sel;  // k with item_off[k] <= it < item_off[k+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (item_off[mid] <= it) lo = mid;
      else hi = mid;
    }
    s_item = it;
    s_k = lo;
  }
  __syncthreads();
  return s_item < item_off[n_sel];
}

// One cell per thread (grids of up to 32 groups, or that ask for it).
template <int MAXG, bool MIXED>
__global__ void batched_kernel(const KParams *__restrict__ grids, const double *__restrict__ tables,
                               int64_t table_stride, const int *__restrict__ sel,
                               const int64_t *__restrict__ item_off, int n_sel, int cpi,
                               unsigned long long *head) {
  extern __shared__ double sm[];
  __shared__ long long s_item;
  __shared__ int s_grid;
  const long long total = item_off[n_sel];
  int cur = -1;
  GroupTable tab;
  Arr64<MAXG> A;
  Arr32<MAXG> B;
  Cell C;
  Cell32 D;
  load_planck(sm);  // visible after the first __syncthreads below
  for (;;) {
    if (!next_item(item_off, n_sel, head, s_item, s_grid)) break;
    const long long item = s_item;
    const int k = s_grid, j = sel[k];
    if (item >= total) break;
    const KParams &P = grids[j];
    if (j != cur) {
      const int words = group_table_words(P.G);
      const double *src = tables + (int64_t)j * table_stride;
      for (int k = threadIdx.x; k < words; k += blockDim.x) sm[kPlanckWords + k] = src[k];
      cur = j;
      tab = table_view(sm + kPlanckWords, P.G, sm);
    }
    __syncthreads();
    const int64_t c0 = (item - item_off[k]) * (int64_t)cpi;
    const int64_t c1 = c0 + cpi < P.n ? c0 + cpi : P.n;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
      solve_cell<MAXG, MIXED>(P, tab, i, C, A, B, D);
    __syncthreads();  // s_item, s_grid and the table are reused by the next item
  }
}

// One cell per warp (grids of 33..64 groups): the mixed form's FP32 passes
// (rhd_warp32.cuh) and FP64 passes (rhd_warp.cuh) of a cell run in the same
// warp; the FP32 result is handed over rounded exactly as the two-launch
// form's workspace rounds it (R_g / E_tot and F_g / (c E_tot) in FP32, E_int
// and rho v in FP64), then the FP64 passes with the cold restart on failure.
template <bool MIXED>
__device__ __forceinline__ void solve_cell_warp(const KParams &P, const GroupTable &tab,
                                                const float *pf, int64_t i, int l,
                                                WCell<32, 2> &C, WCell32<32, 2> &D) {
  constexpr unsigned mask = 0xffffffffu;
  bool warm = false;
  double eint = 0.0, m[3] = {0.0, 0.0, 0.0};
  int nit = 0;
  float r32[2] = {0.0f, 0.0f}, f32[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
  if (MIXED && w32_load(P, tab, i, l, mask, D)) {
    w32_outer_begin(P, D);
    for (;;) {
      const int r = w32_inner_step(P, tab, pf, l, 0, mask, D);
      if (r != 0 && w32_outer_end(P, tab, l, mask, D)) break;
    }
    warm = D.Eint > 0.0;
    eint = D.Eint;
    m[0] = D.m[0];
    m[1] = D.m[1];
    m[2] = D.m[2];
    nit = D.nit > 255 ? 255 : D.nit;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      r32[j] = D.R[j];
      for (int d = 0; d < 3; ++d) f32[j][d] = D.f[j][d];
    }
  }
  if (!wload(P, i, l, mask, C)) return;
  for (int attempt = 0; attempt < 2; ++attempt) {
    int nit0 = 0;
    if (attempt == 1) {
      if (!(warm && C.stat != RHD_STATUS_OK)) break;
      nit0 = C.nit;
      wload(P, i, l, mask, C);
    }
    wset_tau(P, tab, l, C, C.chi0s);
    if (warm && attempt == 0) {
      C.Eint = eint;
      C.m[0] = m[0];
      C.m[1] = m[1];
      C.m[2] = m[2];
      C.nit = nit;
      const double fs = P.c * C.Etot;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (l + 32 * j >= P.G) continue;
        C.R[j] = (double)r32[j] * C.Etot;
        for (int d = 0; d < 3; ++d) C.Fk[j][d] = (double)f32[j][d] * fs;
      }
    }
    wouter_begin(P, C);
    for (;;) {
      const int r = winner_step(P, tab, l, 0, mask, C);
      if (r == 0) continue;
      if (r == 2) C.stat = RHD_STATUS_MAXITER;
      if (wouter_end(P, tab, l, mask, C)) break;
    }
    if (attempt == 1) {
      C.nit += nit0;
      if (C.stat == RHD_STATUS_OK) C.stat = RHD_STATUS_FALLBACK;
    }
  }
  wstore(P, l, C);
}

template <bool MIXED>
__global__ void __launch_bounds__(128) batched_warp_kernel(
    const KParams *__restrict__ grids, const double *__restrict__ tables, int64_t table_stride,
    const int *__restrict__ sel, const int64_t *__restrict__ item_off, int n_sel, int cpi,
    unsigned long long *head) {
  extern __shared__ double sm[];
  __shared__ float pf[kPlanckF];
  __shared__ long long s_item;
  __shared__ int s_k;
  load_planck(sm);
  __syncthreads();
  {
    using namespace planck_table;
    for (int t = threadIdx.x; t < kPlanckF; t += blockDim.x) {
      const int k = t / kSeg, sg = t % kSeg;
      const int src = k <= kDeg32 ? k * kSeg + sg : (kDeg + 1 + (k - kDeg32 - 1)) * kSeg + sg;
      pf[t] = (float)sm[src];
    }
  }
  const int l = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int cur = -1;
  GroupTable tab;
  WCell<32, 2> C;
  WCell32<32, 2> D;
  for (;;) {
    if (!next_item(item_off, n_sel, head, s_item, s_k)) break;
    const long long item = s_item;
    const int k = s_k, j = sel[k];
    const KParams &P = grids[j];
    if (j != cur) {
      const int words = group_table_words(P.G);
      const double *src = tables + (int64_t)j * table_stride;
      for (int t = threadIdx.x; t < words; t += blockDim.x) sm[kPlanckWords + t] = src[t];
      cur = j;
      tab = table_view(sm + kPlanckWords, P.G, sm);
    }
    __syncthreads();
    const int64_t c0 = (item - item_off[k]) * (int64_t)cpi;
    const int64_t c1 = c0 + cpi < P.n ? c0 + cpi : P.n;
    for (int64_t i = c0 + wid; i < c1; i += nw) solve_cell_warp<MIXED>(P, tab, pf, i, l, C, D);
    __syncthreads();  // s_item, s_k and the table are reused by the next item
  }
}

}  // namespace rhd
