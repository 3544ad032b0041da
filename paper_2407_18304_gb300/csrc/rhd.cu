// rhd.cu -- host side of the C ABI in include/rhd.h: argument checks, the
// once-per-device constant tables, and the kernel launches.  The kernels are
// in rhd_fp64.cuh (FP64 passes), rhd_mixed.cuh (FP32 warm-start pass) and
// rhd_batched.cuh (many grids, one persistent launch); this is the only
// translation unit.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "rhd_common.cuh"
#include "rhd_fp64.cuh"
#include "rhd_pplfree.cuh"
#include "rhd_mixed.cuh"
#include "rhd_batched.cuh"
#include "rhd_warp.cuh"
#include "rhd_warp32.cuh"
#include "rhd_correct.cuh"
#include "rhd_refine.cuh"

namespace rhd {
namespace {

std::mutex g_mu;
constexpr int kMaxDevices = 64;
bool g_ready[kMaxDevices];
int g_sms[kMaxDevices];
// Per-device workspace of the mixed form's warm start, grown on demand (the
// first call at a new largest size allocates; later calls reuse it).
void *g_ws[kMaxDevices];
size_t g_ws_bytes[kMaxDevices];

size_t warm_bytes(int64_t n, int G) {
  return (size_t)n * (4 * sizeof(double) + 2) + (size_t)n * G * 8 * sizeof(float) + 1024;
}

// Carve the warm-start arrays out of a workspace starting at p: E_int and
// momentum (FP64), the FP32 iterate R_g / E_tot and F_g / (c E_tot), the
// correction step in the same layout, the FP32 iteration counts.  The
// WarmStart leaves the step out (ur = uf = null) until a correction has run.
void carve(char *p, int64_t n, int G, WarmOut *w, WarmStart *r) {
  w->eint = reinterpret_cast<double *>(p);
  w->mom = w->eint + n;
  w->r = reinterpret_cast<float *>(w->mom + 3 * n);
  w->f = w->r + (size_t)G * n;
  w->ur = w->f + (size_t)3 * G * n;
  w->uf = w->ur + (size_t)G * n;
  w->nit = reinterpret_cast<uint8_t *>(w->uf + (size_t)3 * G * n);
  w->done = w->nit + n;
  *r = WarmStart{w->eint, w->mom, w->r, w->f, w->nit, 1, nullptr, nullptr, nullptr};
}

int workspace(int64_t n, int G, WarmOut *w, WarmStart *r) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RHD_ECUDA;
  const size_t need = warm_bytes(n, G);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ws_bytes[dev] < need) {
    if (g_ws[dev]) cudaFree(g_ws[dev]);
    g_ws[dev] = nullptr;
    g_ws_bytes[dev] = 0;
    if (cudaMalloc(&g_ws[dev], need) != cudaSuccess) return RHD_ENOMEM;
    g_ws_bytes[dev] = need;
  }
  carve(static_cast<char *>(g_ws[dev]), n, G, w, r);
  return RHD_OK;
}

// Workspace of rhd_source_update_noalloc: a file-scope device array (every
// device that loads the library holds it).  Host code must not use the symbol
// as an address: noalloc_base() looks the device address up once per device.
__device__ __align__(256) unsigned char g_noalloc_ws[RHD_NOALLOC_BYTES];
char *g_noalloc_ptr[kMaxDevices];

int noalloc_base(char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RHD_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_ws) != cudaSuccess || !ptr) return RHD_ECUDA;
    g_noalloc_ptr[dev] = static_cast<char *>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return RHD_OK;
}

// B_2j/(2j)! = (-1)^(j+1) 2 zeta(2j) / (2 pi)^(2j).  zeta(2j) in closed form for
// j <= 4 and from the Euler product over the primes below 2000 for j >= 5
// (the neglected factors differ from 1 by less than 2000^-10).
void series_tables(double *b, double *b3, double *invn) {
  const double pi = 3.14159265358979323846;
  std::vector<int> primes;
  std::vector<char> sieve(2000, 1);
  for (int p = 2; p < 2000; ++p) {
    if (!sieve[p]) continue;
    primes.push_back(p);
    for (int q = 2 * p; q < 2000; q += p) sieve[q] = 0;
  }
  for (int j = 1; j <= kNB; ++j) {
    double zeta;
    switch (j) {
      case 1: zeta = std::pow(pi, 2) / 6.0; break;
      case 2: zeta = std::pow(pi, 4) / 90.0; break;
      case 3: zeta = std::pow(pi, 6) / 945.0; break;
      case 4: zeta = std::pow(pi, 8) / 9450.0; break;
      default: {
        zeta = 1.0;
        for (int p : primes) zeta /= (1.0 - std::pow((double)p, -2.0 * j));
      }
    }
    const double sign = (j % 2 == 1) ? 1.0 : -1.0;
    b[j - 1] = sign * 2.0 * zeta / std::pow(2.0 * pi, 2.0 * j);
    b3[j - 1] = b[j - 1] / (2.0 * j + 3.0);
  }
  invn[0] = 0.0;
  for (int n = 1; n <= kNQ; ++n) invn[n] = 1.0 / n;
}

int ensure_device(int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RHD_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ready[dev]) {
    double b[kNB], b3[kNB], invn[kNQ + 1];
    series_tables(b, b3, invn);
    {
      using namespace planck_table;
      static double pt[kPlanckWords];
      for (int k = 0; k <= kDeg; ++k)
        for (int j = 0; j < kSeg; ++j) pt[k * kSeg + j] = kCoef[k][j];
      for (int j = 0; j < kSeg; ++j) {
        pt[(kDeg + 1) * kSeg + j] = kCentre[j];
        pt[(kDeg + 2) * kSeg + j] = kInvHalf[j];
      }
      if (cudaMemcpyToSymbol(c_planck, pt, sizeof(pt)) != cudaSuccess) return RHD_ECUDA;
    }
    float bf[kNB32], b3f[kNB32], invnf[kNQ32 + 1];
    for (int j = 0; j < kNB32; ++j) {
      bf[j] = (float)b[j];
      b3f[j] = (float)b3[j];
    }
    for (int n = 0; n <= kNQ32; ++n) invnf[n] = (float)invn[n];
    if (cudaMemcpyToSymbol(c_bern_f, bf, sizeof(bf)) != cudaSuccess) return RHD_ECUDA;
    if (cudaMemcpyToSymbol(c_bern3_f, b3f, sizeof(b3f)) != cudaSuccess) return RHD_ECUDA;
    if (cudaMemcpyToSymbol(c_invn_f, invnf, sizeof(invnf)) != cudaSuccess) return RHD_ECUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return RHD_ECUDA;
    g_sms[dev] = n;
    g_ready[dev] = true;
  }
  *sms = g_sms[dev];
  return RHD_OK;
}

bool pos_finite(double x) { return std::isfinite(x) && x > 0.0; }

// rhd_events_start/stop: the update calls of this thread add their events to
// g_events (pack sets KParams::count); the inference's cells are counted here.
thread_local bool t_counting = false;
thread_local unsigned long long t_infer_cells = 0;

// rhd_profile_start/stop: event pairs around the launches of this thread, by kind.
thread_local bool t_profiling = false;
thread_local std::vector<std::pair<cudaEvent_t, cudaEvent_t>> t_events[RHD_KERNELS];
thread_local int32_t t_prof_n[RHD_KERNELS];
thread_local double t_prof_ms[RHD_KERNELS];

// Run launch() between two events on st when profiling (kind: RHD_KERNEL_*).
template <typename F>
void timed_launch(int kind, cudaStream_t st, F &&launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (t_profiling && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    t_events[kind].emplace_back(a, b);
    return;
  }
  launch();
}

// Fill the launch parameters from the public structs; RHD_OK or an error.
int pack(const rhd_state_t *s, const rhd_groups_t *gr, const rhd_opacity_law_t *law, double dt,
         int64_t n, KParams *kp) {
  if (!s || !gr || !law || n < 0) return RHD_EINVAL;
  if (gr->n_groups < 1) return RHD_EINVAL;
  if (gr->n_groups > kMaxG) return RHD_ESIZE;
  if (!gr->edges) return RHD_EINVAL;
  const int G = gr->n_groups;
  if (n > 0 && (!s->rho || !s->mom[0] || !s->mom[1] || !s->mom[2] || !s->egas || !s->erad ||
                !s->frad[0] || !s->frad[1] || !s->frad[2]))
    return RHD_EINVAL;
  const int64_t gs = s->group_stride == 0 ? n : s->group_stride;
  if (gs < n) return RHD_EINVAL;
  if (!pos_finite(s->c_v) || !pos_finite(s->theta) || !pos_finite(s->c) || !pos_finite(s->c_hat) ||
      !pos_finite(s->a_rad) || !pos_finite(s->h) || !pos_finite(s->k_B))
    return RHD_EINVAL;
  if (!std::isfinite(dt) || dt < 0.0) return RHD_EINVAL;
  if (s->precision != RHD_FP64 && s->precision != RHD_MIXED) return RHD_EINVAL;
  if (s->closure != RHD_M1 && s->closure != RHD_EDDINGTON) return RHD_EINVAL;
  if (s->flags & ~(RHD_GROUP_TEST | RHD_FLUX_TEST | RHD_CELL_PER_THREAD | RHD_LANES_16))
    return RHD_EINVAL;
  if (law->mode != RHD_PPL_FIXED && law->mode != RHD_PC && law->mode != RHD_PPL_FREE)
    return RHD_ELAW;
  // edges: strictly increasing; PPL needs finite positive edges
  for (int e = 0; e <= G; ++e) {
    const double x = gr->edges[e];
    if (std::isnan(x) || x < 0.0) return RHD_EEDGES;
    if (e > 0 && !(x > gr->edges[e - 1])) return RHD_EEDGES;
    if (law->mode != RHD_PC && !pos_finite(x)) return RHD_EEDGES;
    if (law->mode == RHD_PC && std::isinf(x) && e != G) return RHD_EEDGES;
  }
  std::memset(kp, 0, sizeof(KParams));
  kp->has_table = law->khat_gminus != nullptr;
  if (kp->has_table) {
    for (int g = 0; g < G; ++g) {
      if (!pos_finite(law->khat_gminus[g])) return RHD_ELAW;
      kp->khat_g[g] = law->khat_gminus[g];
      if (law->mode != RHD_PC) {
        if (!law->alpha_g || !std::isfinite(law->alpha_g[g])) return RHD_ELAW;
        kp->alpha_g[g] = law->alpha_g[g];
      }
    }
    kp->n_seg = 1;
    kp->nu_ref = 1.0;
  } else {
    if (law->n_seg < 1) return RHD_ELAW;
    if (law->n_seg > kMaxSeg) return RHD_ESIZE;
    if (!law->seg_logk || !law->seg_beta || (law->n_seg > 1 && !law->nu_break)) return RHD_ELAW;
    if (!pos_finite(law->nu_ref)) return RHD_ELAW;
    for (int k = 0; k < law->n_seg; ++k) {
      if (!std::isfinite(law->seg_logk[k]) || !std::isfinite(law->seg_beta[k])) return RHD_ELAW;
      kp->seg_logk[k] = law->seg_logk[k];
      kp->seg_beta[k] = law->seg_beta[k];
    }
    for (int k = 0; k + 1 < law->n_seg; ++k) {
      if (!pos_finite(law->nu_break[k])) return RHD_ELAW;
      if (k > 0 && !(law->nu_break[k] > law->nu_break[k - 1])) return RHD_ELAW;
      kp->nu_break[k] = law->nu_break[k];
    }
    kp->n_seg = law->n_seg;
    kp->nu_ref = law->nu_ref;
  }
  if (!std::isfinite(law->temp_exponent)) return RHD_ELAW;
  if (law->temp_exponent != 0.0 && !pos_finite(law->T_ref)) return RHD_ELAW;
  kp->temp_exp = law->temp_exponent;
  kp->T_ref = law->temp_exponent != 0.0 ? law->T_ref : 1.0;
  for (int e = 0; e <= G; ++e) kp->edges[e] = gr->edges[e];

  kp->rho = s->rho;
  for (int d = 0; d < 3; ++d) {
    kp->mom[d] = s->mom[d];
    kp->frad[d] = s->frad[d];
  }
  kp->egas = s->egas;
  kp->kappa0 = s->kappa0;
  kp->erad = s->erad;
  kp->src = s->src;
  kp->status = s->status;
  kp->iters = s->iters;
  kp->n = n;
  kp->gs = gs;
  kp->c_v = s->c_v;
  kp->theta = s->theta;
  kp->dt = dt;
  kp->c = s->c;
  kp->c_hat = s->c_hat;
  kp->cr = s->c / s->c_hat;
  kp->ic = 1.0 / s->c;
  kp->inv_c2 = 1.0 / (s->c * s->c);
  kp->icc = 1.0 / (s->c * s->c_hat);
  kp->a_rad = s->a_rad;
  kp->h_over_k = s->h / s->k_B;
  kp->tol = s->tol > 0.0 ? s->tol : 1e-11;
  kp->tol_outer = s->tol_outer > 0.0 ? s->tol_outer : 1e-13;
  kp->max_newton = s->max_newton > 0 ? s->max_newton : 64;
  kp->max_outer = s->max_outer > 0 ? s->max_outer : 16;
  kp->closure = s->closure;
  kp->flags = s->flags;
  kp->G = G;
  kp->mode = law->mode;
  kp->count = t_counting ? 1 : 0;
  return RHD_OK;
}

// Grid of a lane-persistent kernel: the CTAs that are resident at once (so
// every lane walks its share of cells in one wave), fewer for small grids.
template <typename K>
int persistent_blocks(K kernel, size_t smem, int sms, int64_t n, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t want = (n + threads - 1) / threads;
  const int64_t full = (int64_t)sms * per_sm;
  return (int)(want < full ? want : full);
}

template <int L, int GPL>
void launch_warp(const KParams &kp, const WarmStart &W, int sms, cudaStream_t st) {
  const int threads = 128;
  const size_t smem = table_bytes(kp.G);
  const int b = persistent_blocks(solve_warp_kernel<L, GPL>, smem, sms, kp.n * L, threads);
  solve_warp_kernel<L, GPL><<<b, threads, smem, st>>>(kp, W);
}

template <int MAXG>
void launch_free(const KParams &kp, const WarmStart &W, int sms, cudaStream_t st) {
  const int threads = 128;
  const size_t smem = free_table_bytes(kp.G);
  const int b = persistent_blocks(solve_free_kernel<MAXG>, smem, sms, kp.n, threads);
  solve_free_kernel<MAXG><<<b, threads, smem, st>>>(kp, W);
}

template <int MAXG, bool CACHE = false>
void launch_thread(const KParams &kp, const WarmStart &W, int sms, cudaStream_t st) {
  const int threads = 128;
  const size_t smem = table_bytes(kp.G);
  const int b = persistent_blocks(solve_fp64_kernel<MAXG, CACHE>, smem, sms, kp.n, threads);
  solve_fp64_kernel<MAXG, CACHE><<<b, threads, smem, st>>>(kp, W);
}

// Lanes per cell of the FP32 passes up to 16 and from 17 to 32 groups, 2
// groups per lane (measured on GB300, 2M cells: 8 lanes at 16 groups 12.3 ms
// against 23.9 ms one cell per thread; 16 lanes at 32 groups 23.2 ms against
// 50.5 ms, 24.8 ms with 32 lanes of one group, 29.3 ms with 8 lanes of four).
constexpr int kFp32LanesLe16 = 8, kFp32LanesLe32 = 16;

void launch_fp64_passes_impl(const KParams &kp, const WarmStart &W, int sms, cudaStream_t st);

void launch_fp64_passes(const KParams &kp, const WarmStart &W, int sms, cudaStream_t st) {
  timed_launch(RHD_KERNEL_FP64, st, [&] { launch_fp64_passes_impl(kp, W, sms, st); });
}

// The FP64 passes (cold, or from the warm start in W): one cell per thread
// up to 32 groups, a whole warp per cell from 33 to 128 groups
// (rhd_warp.cuh; the split measured on GB300), one cell per thread again past
// 128 groups, where a lane's share of the groups no longer fits in registers.
void launch_fp64_passes_impl(const KParams &kp, const WarmStart &W, int sms, cudaStream_t st) {
  if (kp.mode == RHD_PPL_FREE) {  // free slopes: one cell per thread (rhd_pplfree.cuh)
    if (kp.G <= 16) launch_free<16>(kp, W, sms, st);
    else if (kp.G <= 64) launch_free<64>(kp, W, sms, st);
    else launch_free<kMaxG>(kp, W, sms, st);
    return;
  }
  if (kp.flags & RHD_CELL_PER_THREAD) {  // with the warp mapping's cached iterations
    if (kp.G <= 16) launch_thread<16, true>(kp, W, sms, st);
    else if (kp.G <= 64) launch_thread<64, true>(kp, W, sms, st);
    else launch_thread<kMaxG, true>(kp, W, sms, st);
    return;
  }
  if (W.done && kp.G <= 32) {  // the mixed form's cells the correction left: its FP32 passes' lanes
    if (kp.G <= 16) launch_warp<kFp32LanesLe16, 2>(kp, W, sms, st);
    else launch_warp<kFp32LanesLe32, 2>(kp, W, sms, st);
    return;
  }
  if (kp.G <= 16) launch_thread<16>(kp, W, sms, st);
  else if (kp.G <= 32) launch_thread<32>(kp, W, sms, st);
  else if (kp.G <= 64 && (kp.flags & RHD_LANES_16)) launch_warp<16, 4>(kp, W, sms, st);
  else if (kp.G <= 64) launch_warp<32, 2>(kp, W, sms, st);
  else if (kp.G <= 128) launch_warp<32, 4>(kp, W, sms, st);
  else launch_thread<kMaxG>(kp, W, sms, st);
}

template <int L, int GPL>
void launch_w32(const KParams &kp, const WarmOut &wo, const WarmStart &S, int sms,
                cudaStream_t st) {
  const int threads = 128;
  const size_t smem = table_bytes(kp.G);
  const int b = persistent_blocks(warm_warp32_kernel<L, GPL>, smem, sms, kp.n * L, threads);
  warm_warp32_kernel<L, GPL><<<b, threads, smem, st>>>(kp, wo, S);
}


// The FP32 passes of the mixed form (writing the warm start wo; starting
// from S where S.r is set): a warp per cell from 33 to 64 groups (two with
// RHD_LANES_16), the lanes above at 1..32 groups (four or two cells per
// warp), one cell per thread past 64 groups and with RHD_CELL_PER_THREAD
// (rhd_warp32.cuh, rhd_mixed.cuh).
template <int MAXG>
void launch_fp32_passes_impl(const KParams &kp, const WarmOut &wo, const WarmStart &S, int sms,
                             cudaStream_t st) {
  if (!(kp.flags & RHD_CELL_PER_THREAD)) {
    const int lanes = kp.G <= 16 ? kFp32LanesLe16
                      : kp.G <= 32 ? kFp32LanesLe32
                      : kp.G <= 64 ? ((kp.flags & RHD_LANES_16) ? 16 : 32) : 0;
    switch (kp.G <= 16 ? 100 + lanes : kp.G <= 32 ? 200 + lanes : 300 + lanes) {
      case 108: launch_w32<8, 2>(kp, wo, S, sms, st); return;
      case 216: launch_w32<16, 2>(kp, wo, S, sms, st); return;
      case 316: launch_w32<16, 4>(kp, wo, S, sms, st); return;
      case 332: launch_w32<32, 2>(kp, wo, S, sms, st); return;
      default: break;
    }
  }
  const int threads = 128;
  const size_t smem = table_bytes(kp.G);
  const int ba = persistent_blocks(warm_fp32_kernel<MAXG>, smem, sms, kp.n, threads);
  warm_fp32_kernel<MAXG><<<ba, threads, smem, st>>>(kp, wo, S);
}

template <int MAXG>
void launch_fp32_passes(const KParams &kp, const WarmOut &wo, const WarmStart &S, int sms,
                        cudaStream_t st) {
  timed_launch(RHD_KERNEL_FP32, st, [&] { launch_fp32_passes_impl<MAXG>(kp, wo, S, sms, st); });
}

template <int L, int GPL>
void launch_correct_k(const KParams &kp, const WarmOut &wo, int sms, cudaStream_t st) {
  const int threads = 128;
  const size_t smem = correct_smem_bytes(kp.G, GPL, threads);
  if (smem > 48 * 1024) allow_smem<correct_warp_kernel<L, GPL>>(smem);
  const int b = persistent_blocks(correct_warp_kernel<L, GPL>, smem, sms, kp.n * L, threads);
  correct_warp_kernel<L, GPL><<<b, threads, smem, st>>>(kp, wo,
                                                        CorrOut{wo.ur, wo.uf, wo.done, 1});
}

template <int L, int GPL>
void launch_refine_k(const KParams &kp, const WarmOut &wo, int sms, cudaStream_t st) {
  const int threads = 128;
  const size_t smem = refine_smem_bytes(kp.G, GPL, threads);
  if (smem > 48 * 1024) allow_smem<refine_warp_kernel<L, GPL>>(smem);
  const int b = persistent_blocks(refine_warp_kernel<L, GPL>, smem, sms, kp.n * L, threads);
  refine_warp_kernel<L, GPL><<<b, threads, smem, st>>>(kp, wo, CorrOut{wo.ur, wo.uf, wo.done, 1});
}

// The correction step after the FP32 passes (rhd_correct.cuh): L lanes per
// cell with GPL groups each (up to 128 groups); it finishes most cells and
// returns the warm start of the FP64 passes for the rest.
WarmStart launch_correct(const KParams &kp, const WarmOut &wo, const WarmStart &wi, int sms,
                         cudaStream_t st) {
  WarmStart w = wi;
  if (kp.G > 128) return w;
  const bool l16 = (kp.flags & RHD_LANES_16) != 0;
  timed_launch(RHD_KERNEL_REFINE, st, [&] {
    if (kp.G <= 16) launch_refine_k<8, 2>(kp, wo, sms, st);
    else if (kp.G <= 32) launch_refine_k<16, 2>(kp, wo, sms, st);
    else if (kp.G <= 64 && l16) launch_refine_k<16, 4>(kp, wo, sms, st);
    else if (kp.G <= 64) launch_refine_k<32, 2>(kp, wo, sms, st);
    else launch_refine_k<32, 4>(kp, wo, sms, st);
  });
  timed_launch(RHD_KERNEL_CORRECTION, st, [&] {
    if (kp.G <= 16) launch_correct_k<8, 2>(kp, wo, sms, st);
    else if (kp.G <= 32) launch_correct_k<16, 2>(kp, wo, sms, st);
    else if (kp.G <= 64 && l16) launch_correct_k<16, 4>(kp, wo, sms, st);
    else if (kp.G <= 64) launch_correct_k<32, 2>(kp, wo, sms, st);
    else launch_correct_k<32, 4>(kp, wo, sms, st);
  });
  w.ur = wo.ur;
  w.uf = wo.uf;
  w.done = wo.done;
  return w;
}

template <int MAXG>
int launch_mixed(const KParams &kp, const WarmOut &wo, const WarmStart &wi, int sms,
                 cudaStream_t st) {
  const WarmStart none{nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
  if (kp.mode == RHD_PPL_FREE) {  // no FP32 passes for free slopes: FP64 from the cold start
    launch_fp64_passes(kp, none, sms, st);
    return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
  }
  launch_fp32_passes<MAXG>(kp, wo, none, sms, st);
  launch_fp64_passes(kp, launch_correct(kp, wo, wi, sms, st), sms, st);
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

// Solve from a warm start already in the workspace (wo/wi view the same
// arrays): FP64 form directly from it; mixed form FP32 passes from it (in
// place), the correction step, then the FP64 passes from their result.  Cold
// restart on failure.
template <int MAXG>
int launch_warm_g(const KParams &kp, int precision, const WarmOut &wo, const WarmStart &wi,
                  int sms, cudaStream_t st) {
  if (precision == RHD_MIXED && kp.mode != RHD_PPL_FREE) {
    launch_fp32_passes<MAXG>(kp, wo, wi, sms, st);
    launch_fp64_passes(kp, launch_correct(kp, wo, wi, sms, st), sms, st);
  } else {
    launch_fp64_passes(kp, wi, sms, st);
  }
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

int launch_warm(const KParams &kp, int precision, const WarmOut &wo, const WarmStart &wi, int sms,
                cudaStream_t st) {
  if (kp.G <= 16) return launch_warm_g<16>(kp, precision, wo, wi, sms, st);
  return launch_warm_g<64>(kp, precision, wo, wi, sms, st);
}

template <int MAXG>
int launch_g(const KParams &kp, int precision, int sms, cudaStream_t st) {
  if (precision == RHD_FP64) {
    const WarmStart cold{nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
    launch_fp64_passes(kp, cold, sms, st);
  } else {
    WarmOut wo;
    WarmStart wi;
    const int rc = workspace(kp.n, kp.G, &wo, &wi);
    if (rc != RHD_OK) return rc;
    return launch_mixed<MAXG>(kp, wo, wi, sms, st);
  }
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

int launch(const KParams &kp, int precision, int sms, cudaStream_t st) {
  if (kp.G <= 16) return launch_g<16>(kp, precision, sms, st);
  if (kp.G <= 64) return launch_g<64>(kp, precision, sms, st);
  return launch_g<kMaxG>(kp, precision, sms, st);
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_source_update(rhd_state_t *state, const rhd_groups_t *groups,
                                 const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                                 void *stream) {
  static thread_local rhd::KParams kp;
  int rc = rhd::pack(state, groups, opacity_law, dt, n_cells, &kp);
  if (rc != RHD_OK) return rc;
  if (n_cells == 0) return RHD_OK;
  int sms = 0;
  rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  return rhd::launch(kp, state->precision, sms, (cudaStream_t)stream);
}

extern "C" int rhd_source_update_noalloc(rhd_state_t *state, const rhd_groups_t *groups,
                                         const rhd_opacity_law_t *opacity_law, double dt,
                                         int64_t n_cells, void *stream) {
  static thread_local rhd::KParams kp;
  int rc = rhd::pack(state, groups, opacity_law, dt, n_cells, &kp);
  if (rc != RHD_OK) return rc;
  if ((int64_t)rhd::warm_bytes(n_cells, kp.G) > RHD_NOALLOC_BYTES) return RHD_ESIZE;
  if (n_cells == 0) return RHD_OK;
  int sms = 0;
  rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  char *base = nullptr;
  rc = rhd::noalloc_base(&base);
  if (rc != RHD_OK) return rc;
  rhd::WarmOut wo;
  rhd::WarmStart wi;
  rhd::carve(base, n_cells, kp.G, &wo, &wi);
  cudaStream_t st = (cudaStream_t)stream;
  if (kp.G <= 16) return rhd::launch_mixed<16>(kp, wo, wi, sms, st);
  if (kp.G <= 64) return rhd::launch_mixed<64>(kp, wo, wi, sms, st);
  return rhd::launch_mixed<rhd::kMaxG>(kp, wo, wi, sms, st);
}

// ---------------------------------------------------------------------------
// The two-stage IMEX step without transport
// ---------------------------------------------------------------------------
namespace rhd {
namespace {

void *g_imex_ws[kMaxDevices];
size_t g_imex_bytes[kMaxDevices];

// mode 0: U^(n) -> ws; 1: U = (U + ws)/2 and stage-1 status/iters -> ws;
// 2: status = max(status, ws status), iters = min(255, iters + ws iters).
__global__ void imex_kernel(const __grid_constant__ KParams P, double *ws, uint8_t *ws_st,
                            int mode) {
  const int64_t n = P.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mode == 2) {
      if (P.status) P.status[i] = P.status[i] > ws_st[i] ? P.status[i] : ws_st[i];
      if (P.iters) {
        const int it = (int)P.iters[i] + (int)ws_st[n + i];
        P.iters[i] = (uint8_t)(it > 255 ? 255 : it);
      }
      continue;
    }
    double *w = ws;
    double *u[4] = {P.egas, P.mom[0], P.mom[1], P.mom[2]};
    for (int k = 0; k < 4; ++k) {
      if (mode == 0) w[(int64_t)k * n + i] = u[k][i];
      else u[k][i] = 0.5 * (u[k][i] + w[(int64_t)k * n + i]);
    }
    w += 4 * n;
    for (int g = 0; g < P.G; ++g) {
      const int64_t o = (int64_t)g * P.gs + i;
      double *a[4] = {P.erad, P.frad[0], P.frad[1], P.frad[2]};
      for (int k = 0; k < 4; ++k) {
        const int64_t q = ((int64_t)k * P.G + g) * n + i;
        if (mode == 0) w[q] = a[k][o];
        else a[k][o] = 0.5 * (a[k][o] + w[q]);
      }
    }
    if (mode == 1) {
      ws_st[i] = P.status ? P.status[i] : 0;
      ws_st[n + i] = P.iters ? P.iters[i] : 0;
    }
  }
}

int imex_workspace(int64_t n, int G, double **ws, uint8_t **st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RHD_ECUDA;
  const size_t words = (size_t)n * (4 + 4 * (size_t)G);
  const size_t bytes = words * sizeof(double) + 2 * (size_t)n + 256;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_imex_bytes[dev] < bytes) {
    if (g_imex_ws[dev]) cudaFree(g_imex_ws[dev]);
    g_imex_ws[dev] = nullptr;
    g_imex_bytes[dev] = 0;
    if (cudaMalloc(&g_imex_ws[dev], bytes) != cudaSuccess) return RHD_ENOMEM;
    g_imex_bytes[dev] = bytes;
  }
  *ws = (double *)g_imex_ws[dev];
  *st = (uint8_t *)(*ws + words);
  return RHD_OK;
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_imex_step(rhd_state_t *state, const rhd_groups_t *groups,
                             const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                             void *stream) {
  if (!state) return RHD_EINVAL;
  if (state->src) return RHD_EINVAL;
  static thread_local rhd::KParams kp;
  rhd_state_t s1 = *state;
  s1.theta = 1.0;
  int rc = rhd::pack(&s1, groups, opacity_law, dt, n_cells, &kp);
  if (rc != RHD_OK) return rc;
  if (n_cells == 0) return RHD_OK;
  int sms = 0;
  rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  double *ws = nullptr;
  uint8_t *wst = nullptr;
  rc = rhd::imex_workspace(kp.n, kp.G, &ws, &wst);
  if (rc != RHD_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (int)((n_cells + 255) / 256 < 65535 ? (n_cells + 255) / 256 : 65535);
  rhd::imex_kernel<<<blocks, 256, 0, st>>>(kp, ws, wst, 0);           // keep U^(n)
  rc = rhd::launch(kp, state->precision, sms, st);                     // stage 1, theta = 1
  if (rc != RHD_OK) return rc;
  rhd::imex_kernel<<<blocks, 256, 0, st>>>(kp, ws, wst, 1);           // (U^(n) + U^(n+1/2))/2
  kp.theta = 0.5;
  rc = rhd::launch(kp, state->precision, sms, st);                     // stage 2, theta = 1/2
  if (rc != RHD_OK) return rc;
  rhd::imex_kernel<<<blocks, 256, 0, st>>>(kp, ws, wst, 2);           // status, iters
  return cudaGetLastError() == cudaSuccess ? RHD_OK : RHD_ECUDA;
}

// ---------------------------------------------------------------------------
// Batched uneven grids
// ---------------------------------------------------------------------------
// The grids fall into RHD_BATCH_BUCKETS buckets by group count, each with its
// own mapping of cells to lanes and its own queues (rhd_batched.cuh).
// Staging layout: offsets [2 * buckets][cap + 1] (bucket b's pass items at
// 2b, its correction items at 2b + 1), selections [buckets][cap], queue heads
// [3 * buckets] (FP32 passes, correction, FP64 passes of each bucket).
namespace rhd {
namespace {
constexpr int kBuckets = RHD_BATCH_BUCKETS;
constexpr int kCpiWarp = 64;  // cells per work item of a lane-segment mapping
constexpr int kCpiCorr = 64;  // cells per work item of the correction step
constexpr int kSigWords = 5 + 2 * kBuckets + 3 * kBuckets;

int bucket_of(int G) { return G <= 16 ? 0 : G <= 32 ? 1 : 2; }

// The mappings each bucket offers (lanes per cell; 1 = one cell per thread).
// The groups per lane follow: the bucket's largest group count / lanes.
// 0: the one-grid call's mapping for the call's precision (pass_lanes)
bool pass_mapping_ok(int b, int m) {
  switch (b) {
    case 0: return m == 0 || m == 1 || m == 8;
    case 1: return m == 0 || m == 1 || m == 8 || m == 16 || m == 32;
    case 2: return m == 0 || m == 1 || m == 16 || m == 32;
  }
  return false;
}
bool corr_mapping_ok(int b, int m) {
  switch (b) {
    case 0: return m == 8;
    case 1: return m == 8 || m == 16;
    case 2: return m == 16 || m == 32;
  }
  return false;
}
}  // namespace
}  // namespace rhd

struct rhd_context {
  int device = -1;
  int threads = 128, cpi = 512;                // shape of the cell-per-thread mapping (autotuned)
  int pass_map[RHD_BATCH_BUCKETS] = {0, 0, 0};   // lanes per cell of each bucket's passes (0: as one grid)
  int corr_map[RHD_BATCH_BUCKETS] = {8, 16, 32}; // lanes per cell of its correction step
  int cap_grids = 0;
  rhd::KParams *h_grids = nullptr, *d_grids = nullptr;
  rhd::WarmOut *h_warm = nullptr, *d_warm = nullptr;
  int64_t *h_off = nullptr, *d_off = nullptr;
  int *h_sel = nullptr, *d_sel = nullptr;
  int n_sel[RHD_BATCH_BUCKETS] = {0, 0, 0};
  double *d_tables = nullptr;
  unsigned long long *d_head = nullptr;
  char *d_ws = nullptr;  // the mixed form's per-grid workspaces
  size_t ws_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaStream_t side[RHD_BATCH_BUCKETS - 1] = {};  // buckets 1.. run here, forked from the main stream
  cudaEvent_t fork = nullptr, join[RHD_BATCH_BUCKETS - 1] = {};
  cudaGraphExec_t exec = nullptr;
  int64_t sig[rhd::kSigWords] = {};
  bool has_sig = false;
  cudaEvent_t done = nullptr;
  bool pending = false;
};

namespace rhd {
namespace {

const int64_t kTableWords = group_table_words(kMaxGB) + 1;

// Lanes per cell of bucket b's passes: the mapping set, else the one-grid
// call's for the precision (mixed form: the FP32 passes' 8, 16, 32 lanes,
// which its FP64 passes follow; FP64 form: one cell per thread up to 32
// groups, 32 lanes above).
int pass_lanes(const rhd_context *c, int b, int prec) {
  if (c->pass_map[b] != 0) return c->pass_map[b];
  static const int mixed[kBuckets] = {kFp32LanesLe16, kFp32LanesLe32, 32};
  static const int fp64[kBuckets] = {1, 1, 32};
  return prec == RHD_MIXED ? mixed[b] : fp64[b];
}

void ctx_free(rhd_context *c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->h_grids) cudaFreeHost(c->h_grids);
  if (c->h_warm) cudaFreeHost(c->h_warm);
  if (c->h_off) cudaFreeHost(c->h_off);
  if (c->h_sel) cudaFreeHost(c->h_sel);
  if (c->d_grids) cudaFree(c->d_grids);
  if (c->d_warm) cudaFree(c->d_warm);
  if (c->d_off) cudaFree(c->d_off);
  if (c->d_sel) cudaFree(c->d_sel);
  if (c->d_tables) cudaFree(c->d_tables);
  if (c->d_head) cudaFree(c->d_head);
  c->exec = nullptr;
  c->has_sig = false;
  c->h_grids = c->d_grids = nullptr;
  c->h_warm = c->d_warm = nullptr;
  c->h_off = c->d_off = nullptr;
  c->h_sel = c->d_sel = nullptr;
  c->d_tables = nullptr;
  c->d_head = nullptr;
  c->cap_grids = 0;
}

int ctx_reserve(rhd_context *c, int n_grids) {
  if (n_grids <= c->cap_grids) return RHD_OK;
  if (c->pending) cudaEventSynchronize(c->done);
  c->pending = false;
  ctx_free(c);
  int cap = 64;
  while (cap < n_grids) cap *= 2;
  const size_t noff = sizeof(int64_t) * 2 * kBuckets * (cap + 1), nsel = sizeof(int) * kBuckets * cap;
  if (cudaHostAlloc(&c->h_grids, sizeof(KParams) * cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&c->h_warm, sizeof(WarmOut) * cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&c->h_off, noff, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&c->h_sel, nsel, cudaHostAllocDefault) != cudaSuccess ||
      cudaMalloc(&c->d_grids, sizeof(KParams) * cap) != cudaSuccess ||
      cudaMalloc(&c->d_warm, sizeof(WarmOut) * cap) != cudaSuccess ||
      cudaMalloc(&c->d_off, noff) != cudaSuccess || cudaMalloc(&c->d_sel, nsel) != cudaSuccess ||
      cudaMalloc(&c->d_tables, sizeof(double) * kTableWords * cap) != cudaSuccess ||
      cudaMalloc(&c->d_head, 4 * kBuckets * sizeof(unsigned long long)) != cudaSuccess) {
    ctx_free(c);
    return RHD_ENOMEM;
  }
  c->cap_grids = cap;
  return RHD_OK;
}

int64_t *off_of(int64_t *base, const rhd_context *c, int set) {
  return base + (int64_t)set * (c->cap_grids + 1);
}

// Pack the grids into the pinned staging buffers and split them into the
// buckets; work items per set out (items[2b] bucket b's passes, items[2b+1]
// its correction step).  Mixed form: each grid's workspace is carved out of
// the context's (grown here, before anything is enqueued).
int pack_batch(rhd_context *c, const rhd_grid_t *grids, int n_grids, int cpi, int *prec,
               int64_t items[2 * kBuckets]) {
  int64_t acc[2 * kBuckets] = {};
  int ns[kBuckets] = {};
  *prec = -1;
  size_t ws = 0;
  for (int j = 0; j < n_grids; ++j) {
    const rhd_grid_t &g = grids[j];
    const int rc = pack(&g.state, &g.groups, &g.opacity_law, g.dt, g.n_cells, &c->h_grids[j]);
    if (rc != RHD_OK) return rc;
    if (g.opacity_law.mode == RHD_PPL_FREE) return RHD_ELAW;  // per-cell solve only
    if (g.groups.n_groups > kMaxGB) return RHD_ESIZE;
    if (*prec < 0) *prec = g.state.precision;
    if (g.state.precision != *prec) return RHD_EINVAL;
    ws += (warm_bytes(g.n_cells, g.groups.n_groups) + 255) & ~(size_t)255;
  }
  if (*prec == RHD_MIXED && ws > c->ws_bytes) {
    if (c->pending) cudaEventSynchronize(c->done);
    c->pending = false;
    if (c->d_ws) cudaFree(c->d_ws);
    c->d_ws = nullptr;
    c->ws_bytes = 0;
    if (cudaMalloc(&c->d_ws, ws) != cudaSuccess) return RHD_ENOMEM;
    c->ws_bytes = ws;
  }
  size_t at = 0;
  for (int j = 0; j < n_grids; ++j) {
    const rhd_grid_t &g = grids[j];
    const int G = g.groups.n_groups, b = bucket_of(G);
    if (*prec == RHD_MIXED) {
      WarmStart unused;
      carve(c->d_ws + at, g.n_cells, G, &c->h_warm[j], &unused);
      at += (warm_bytes(g.n_cells, G) + 255) & ~(size_t)255;
    }
    const int per = pass_lanes(c, b, *prec) == 1 ? cpi : kCpiWarp;
    off_of(c->h_off, c, 2 * b)[ns[b]] = acc[2 * b];
    off_of(c->h_off, c, 2 * b + 1)[ns[b]] = acc[2 * b + 1];
    c->h_sel[(int64_t)b * c->cap_grids + ns[b]] = j;
    ++ns[b];
    acc[2 * b] += (g.n_cells + per - 1) / per;
    acc[2 * b + 1] += (g.n_cells + kCpiCorr - 1) / kCpiCorr;
  }
  for (int b = 0; b < kBuckets; ++b) {
    for (int s = 2 * b; s <= 2 * b + 1; ++s) {
      off_of(c->h_off, c, s)[ns[b]] = acc[s];
      items[s] = acc[s];
    }
    c->n_sel[b] = ns[b];
  }
  return RHD_OK;
}

// A persistent launch over a queue of `items` work items: the CTAs resident
// at once, fewer when there are fewer items.
template <typename K>
void launch_queue(K kernel, int threads, size_t smem, int sms, int64_t items, const BatchArgs &A,
                  cudaStream_t s) {
  if (items <= 0) return;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t full = (int64_t)sms * per_sm;
  kernel<<<(int)(items < full ? items : full), threads, smem, s>>>(A);
}

template <int L, int GPL>
void launch_segments(int phase, int sms, int64_t items, const BatchArgs &A, cudaStream_t s) {
  if (phase == 0) launch_queue(batched_w32_kernel<L, GPL>, 128, kBatchTableBytes, sms, items, A, s);
  else launch_queue(batched_w64_kernel<L, GPL>, 128, kBatchTableBytes, sms, items, A, s);
}

// Bucket b's FP32 (phase 0) or FP64 (phase 2) passes with mapping m.
void launch_passes(int phase, int b, int m, int threads, int sms, int64_t items,
                   const BatchArgs &A, cudaStream_t s) {
  if (m == 1) {
    if (phase == 0) launch_queue(batched_fp32_kernel<kMaxGB>, threads, kBatchTableBytes, sms, items, A, s);
    else launch_queue(batched_fp64_kernel<kMaxGB>, threads, kBatchTableBytes, sms, items, A, s);
    return;
  }
  switch (100 * b + m) {  // groups per lane = the bucket's largest group count / lanes
    case 8: launch_segments<8, 2>(phase, sms, items, A, s); break;
    case 108: launch_segments<8, 4>(phase, sms, items, A, s); break;
    case 116: launch_segments<16, 2>(phase, sms, items, A, s); break;
    case 132: launch_segments<32, 1>(phase, sms, items, A, s); break;
    case 216: launch_segments<16, 4>(phase, sms, items, A, s); break;
    case 232: launch_segments<32, 2>(phase, sms, items, A, s); break;
  }
}

template <int L, int GPL>
void launch_corr(bool refine, int sms, int64_t items, const BatchArgs &A, cudaStream_t s) {
  if (refine)
    launch_queue(batched_refine_kernel<L, GPL>, 128, batch_refine_smem(GPL), sms, items, A, s);
  else
    launch_queue(batched_correct_kernel<L, GPL>, 128, batch_correct_smem(GPL), sms, items, A, s);
}

// Bucket b's correction with mapping m: its float-float first step (refine)
// or its FP64 steps.
void launch_correction(int b, int m, bool refine, int sms, int64_t items, const BatchArgs &A,
                       cudaStream_t s) {
  switch (100 * b + m) {
    case 8: launch_corr<8, 2>(refine, sms, items, A, s); break;
    case 108: launch_corr<8, 4>(refine, sms, items, A, s); break;
    case 116: launch_corr<16, 2>(refine, sms, items, A, s); break;
    case 216: launch_corr<16, 4>(refine, sms, items, A, s); break;
    case 232: launch_corr<32, 2>(refine, sms, items, A, s); break;
  }
}

// The shared-memory opt-in of the correction kernels above 48 KB; made once
// per device, before any capture.
cudaError_t batch_prepare() {
  cudaError_t e = cudaSuccess;
  if (batch_correct_smem(4) > 48 * 1024) {
    if ((e = allow_smem<batched_correct_kernel<8, 4>>(batch_correct_smem(4))) != cudaSuccess) return e;
    if ((e = allow_smem<batched_correct_kernel<16, 4>>(batch_correct_smem(4))) != cudaSuccess) return e;
  }
  if (batch_correct_smem(2) > 48 * 1024) {
    if ((e = allow_smem<batched_correct_kernel<8, 2>>(batch_correct_smem(2))) != cudaSuccess) return e;
    if ((e = allow_smem<batched_correct_kernel<16, 2>>(batch_correct_smem(2))) != cudaSuccess) return e;
    if ((e = allow_smem<batched_correct_kernel<32, 2>>(batch_correct_smem(2))) != cudaSuccess) return e;
  }
  if (batch_refine_smem(4) > 48 * 1024) {
    if ((e = allow_smem<batched_refine_kernel<8, 4>>(batch_refine_smem(4))) != cudaSuccess) return e;
    if ((e = allow_smem<batched_refine_kernel<16, 4>>(batch_refine_smem(4))) != cudaSuccess) return e;
  }
  if (batch_refine_smem(2) > 48 * 1024) {
    if ((e = allow_smem<batched_refine_kernel<8, 2>>(batch_refine_smem(2))) != cudaSuccess) return e;
    if ((e = allow_smem<batched_refine_kernel<16, 2>>(batch_refine_smem(2))) != cudaSuccess) return e;
    if ((e = allow_smem<batched_refine_kernel<32, 2>>(batch_refine_smem(2))) != cudaSuccess) return e;
  }
  return e;
}

// Everything one batched call enqueues: descriptors, queue reset, tables,
// then each bucket's phases on its own stream (bucket 0 on st).
cudaError_t enqueue_batch(rhd_context *c, int prec, int n_grids, int threads, int cpi, int sms,
                          const int64_t items[2 * kBuckets], cudaStream_t st) {
  const int cap = c->cap_grids;
  const bool mixed = prec == RHD_MIXED;
  cudaMemcpyAsync(c->d_grids, c->h_grids, sizeof(KParams) * n_grids, cudaMemcpyHostToDevice, st);
  if (mixed)
    cudaMemcpyAsync(c->d_warm, c->h_warm, sizeof(WarmOut) * n_grids, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->d_off, c->h_off, sizeof(int64_t) * 2 * kBuckets * (cap + 1),
                  cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->d_sel, c->h_sel, sizeof(int) * kBuckets * cap, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(c->d_head, 0, 4 * kBuckets * sizeof(unsigned long long), st);
  tables_kernel<<<n_grids, 128, table_bytes(kMaxGB) + 64, st>>>(c->d_grids, c->d_tables,
                                                                   kTableWords);
  bool forked = false;
  for (int b = 0; b < kBuckets; ++b) {
    if (c->n_sel[b] == 0 || items[2 * b] == 0) continue;
    cudaStream_t s = st;
    if (b > 0) {
      if (!forked) cudaEventRecord(c->fork, st);
      forked = true;
      s = c->side[b - 1];
      cudaStreamWaitEvent(s, c->fork, 0);
    }
    const int pm = pass_lanes(c, b, prec);
    BatchArgs A{c->d_grids, c->d_tables, kTableWords, mixed ? c->d_warm : nullptr,
                c->d_sel + (int64_t)b * cap, off_of(c->d_off, c, 2 * b), c->n_sel[b],
                pm == 1 ? cpi : kCpiWarp, nullptr};
    const int th = pm == 1 ? threads : 128;
    if (mixed) {
      A.head = c->d_head + 4 * b;
      launch_passes(0, b, pm, th, sms, items[2 * b], A, s);
      BatchArgs Ac = A;
      Ac.item_off = off_of(c->d_off, c, 2 * b + 1);
      Ac.cpi = kCpiCorr;
      Ac.head = c->d_head + 4 * b + 1;
      launch_correction(b, c->corr_map[b], true, sms, items[2 * b + 1], Ac, s);
      Ac.head = c->d_head + 4 * b + 2;
      launch_correction(b, c->corr_map[b], false, sms, items[2 * b + 1], Ac, s);
    }
    A.head = c->d_head + 4 * b + 3;
    launch_passes(2, b, pm, th, sms, items[2 * b], A, s);
    if (s != st) {
      cudaEventRecord(c->join[b - 1], s);
      cudaStreamWaitEvent(st, c->join[b - 1], 0);
    }
  }
  return cudaGetLastError();
}

void signature(const rhd_context *c, int prec, int n_grids, const int64_t items[2 * kBuckets],
               int64_t out[kSigWords]) {
  int k = 0;
  out[k++] = n_grids;
  out[k++] = prec;
  out[k++] = c->threads;
  out[k++] = c->cpi;
  out[k++] = c->cap_grids;
  for (int s = 0; s < 2 * kBuckets; ++s) out[k++] = items[s];
  for (int b = 0; b < kBuckets; ++b) out[k++] = c->n_sel[b];
  for (int b = 0; b < kBuckets; ++b) out[k++] = c->pass_map[b];
  for (int b = 0; b < kBuckets; ++b) out[k++] = c->corr_map[b];
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_context_create(rhd_context_t **ctx) {
  if (!ctx) return RHD_EINVAL;
  rhd_context *c = new (std::nothrow) rhd_context();
  if (!c) return RHD_ENOMEM;
  bool ok = cudaGetDevice(&c->device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < rhd::kBuckets - 1; ++k)
    ok = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->done) cudaEventDestroy(c->done);
    for (int k = 0; k < rhd::kBuckets - 1; ++k) {
      if (c->side[k]) cudaStreamDestroy(c->side[k]);
      if (c->join[k]) cudaEventDestroy(c->join[k]);
    }
    delete c;
    return RHD_ECUDA;
  }
  *ctx = c;
  return RHD_OK;
}

extern "C" int rhd_context_destroy(rhd_context_t *ctx) {
  if (!ctx) return RHD_EINVAL;
  if (ctx->pending) cudaEventSynchronize(ctx->done);
  rhd::ctx_free(ctx);
  if (ctx->d_ws) cudaFree(ctx->d_ws);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->done) cudaEventDestroy(ctx->done);
  for (int k = 0; k < rhd::kBuckets - 1; ++k) {
    if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
    if (ctx->join[k]) cudaEventDestroy(ctx->join[k]);
  }
  delete ctx;
  return RHD_OK;
}

extern "C" int rhd_context_shape(const rhd_context_t *ctx, int32_t *threads,
                                 int32_t *cells_per_item) {
  if (!ctx || !threads || !cells_per_item) return RHD_EINVAL;
  *threads = ctx->threads;
  *cells_per_item = ctx->cpi;
  return RHD_OK;
}

extern "C" int rhd_context_mapping(const rhd_context_t *ctx, int32_t bucket, int32_t *passes,
                                   int32_t *correction) {
  if (!ctx || !passes || !correction || bucket < 0 || bucket >= rhd::kBuckets) return RHD_EINVAL;
  *passes = ctx->pass_map[bucket];
  *correction = ctx->corr_map[bucket];
  return RHD_OK;
}

extern "C" int rhd_context_set_mapping(rhd_context_t *ctx, int32_t bucket, int32_t passes,
                                       int32_t correction) {
  if (!ctx || bucket < 0 || bucket >= rhd::kBuckets) return RHD_EINVAL;
  if (!rhd::pass_mapping_ok(bucket, passes) || !rhd::corr_mapping_ok(bucket, correction))
    return RHD_EINVAL;
  ctx->pass_map[bucket] = passes;
  ctx->corr_map[bucket] = correction;
  return RHD_OK;
}

extern "C" int rhd_source_update_batched(rhd_context_t *ctx, const rhd_grid_t *grids,
                                         int32_t n_grids, void *stream) {
  if (!ctx || !grids || n_grids < 1) return RHD_EINVAL;
  if (n_grids > RHD_MAX_GRIDS) return RHD_ESIZE;
  int sms = 0;
  int rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  if (rhd::batch_prepare() != cudaSuccess) return RHD_ECUDA;
  // the previous call of this context may still read the staging buffers
  if (ctx->pending) {
    cudaEventSynchronize(ctx->done);
    ctx->pending = false;
  }
  rc = rhd::ctx_reserve(ctx, n_grids);
  if (rc != RHD_OK) return rc;
  int prec = 0;
  int64_t items[2 * rhd::kBuckets] = {};
  rc = rhd::pack_batch(ctx, grids, n_grids, ctx->cpi, &prec, items);
  if (rc != RHD_OK) return rc;
  int64_t any = 0;
  for (int b = 0; b < rhd::kBuckets; ++b) any += items[2 * b];
  if (any == 0) return RHD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t sig[rhd::kSigWords];
  rhd::signature(ctx, prec, n_grids, items, sig);
  const bool same = ctx->exec && ctx->has_sig && std::memcmp(sig, ctx->sig, sizeof(sig)) == 0;
  if (!same) {
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    ctx->exec = nullptr;
    ctx->has_sig = false;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return RHD_ECUDA;
    const cudaError_t le =
        rhd::enqueue_batch(ctx, prec, n_grids, ctx->threads, ctx->cpi, sms, items, ctx->cap);
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &graph);
    if (le != cudaSuccess || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return RHD_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&ctx->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      ctx->exec = nullptr;
      return RHD_ECUDA;
    }
    std::memcpy(ctx->sig, sig, sizeof(sig));
    ctx->has_sig = true;
  }
  if (cudaGraphLaunch(ctx->exec, st) != cudaSuccess) return RHD_ECUDA;
  if (cudaEventRecord(ctx->done, st) != cudaSuccess) return RHD_ECUDA;
  ctx->pending = true;
  return RHD_OK;
}

namespace rhd {
namespace {

// The device copy of every grid's in/out arrays, restored after each
// candidate the autotuner times.
struct StateSave {
  struct Buf {
    void *dst;
    const void *src;
    size_t bytes;
  };
  std::vector<Buf> bufs;
  char *save = nullptr;

  int take(const rhd_grid_t *grids, int n_grids, cudaStream_t st) {
    size_t total = 0;
    for (int j = 0; j < n_grids; ++j) {
      const rhd_grid_t &g = grids[j];
      if (g.n_cells <= 0) continue;
      const int64_t gs = g.state.group_stride ? g.state.group_stride : g.n_cells;
      const size_t per = sizeof(double) * g.n_cells;
      const size_t pg = sizeof(double) * ((int64_t)(g.groups.n_groups - 1) * gs + g.n_cells);
      if (!g.state.egas || !g.state.erad) return RHD_EINVAL;
      bufs.push_back({nullptr, g.state.egas, per});
      for (int d = 0; d < 3; ++d) bufs.push_back({nullptr, g.state.mom[d], per});
      bufs.push_back({nullptr, g.state.erad, pg});
      for (int d = 0; d < 3; ++d) bufs.push_back({nullptr, g.state.frad[d], pg});
    }
    for (auto &b : bufs) total += (b.bytes + 255) & ~size_t(255);
    if (total && cudaMalloc(&save, total) != cudaSuccess) return RHD_ENOMEM;
    size_t off = 0;
    for (auto &b : bufs) {
      b.dst = save + off;
      off += (b.bytes + 255) & ~size_t(255);
      cudaMemcpyAsync(b.dst, b.src, b.bytes, cudaMemcpyDeviceToDevice, st);
    }
    return RHD_OK;
  }
  void restore(cudaStream_t st) const {
    for (auto &b : bufs)
      cudaMemcpyAsync(const_cast<void *>(b.src), b.dst, b.bytes, cudaMemcpyDeviceToDevice, st);
  }
  ~StateSave() {
    if (save) cudaFree(save);
  }
};

// Time one candidate: the batched call (not captured) on these grids with the
// context's current mappings and the given shape, then the state restored.
// The best of two runs (the first also loads the kernels).
int time_candidate(rhd_context *c, const rhd_grid_t *grids, int n_grids, int threads, int cpi,
                   int sms, const StateSave &sv, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st,
                   float *ms_out) {
  int prec = 0;
  int64_t items[2 * kBuckets] = {};
  int rc = pack_batch(c, grids, n_grids, cpi, &prec, items);
  if (rc != RHD_OK) return rc;
  float best = 1e30f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0, st);
    if (enqueue_batch(c, prec, n_grids, threads, cpi, sms, items, st) != cudaSuccess)
      return RHD_ECUDA;
    cudaEventRecord(e1, st);
    sv.restore(st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RHD_ECUDA;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return RHD_ECUDA;
    if (ms < best) best = ms;
  }
  *ms_out = best;
  return RHD_OK;
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_context_autotune(rhd_context_t *ctx, const rhd_grid_t *grids, int32_t n_grids,
                                    void *stream) {
  if (!ctx || !grids || n_grids < 1) return RHD_EINVAL;
  if (n_grids > RHD_MAX_GRIDS) return RHD_ESIZE;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  int rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  if (rhd::batch_prepare() != cudaSuccess) return RHD_ECUDA;
  if (ctx->pending) {
    cudaEventSynchronize(ctx->done);
    ctx->pending = false;
  }
  rc = rhd::ctx_reserve(ctx, n_grids);
  if (rc != RHD_OK) return rc;
  {  // every grid checked (and the workspace sized) before anything runs
    int prec = 0;
    int64_t items[2 * rhd::kBuckets] = {};
    rc = rhd::pack_batch(ctx, grids, n_grids, ctx->cpi, &prec, items);
    if (rc != RHD_OK) return rc;
  }
  rhd::StateSave sv;
  rc = sv.take(grids, n_grids, st);
  if (rc != RHD_OK) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RHD_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RHD_ECUDA;
  }
  const int saved_pass[rhd::kBuckets] = {ctx->pass_map[0], ctx->pass_map[1], ctx->pass_map[2]};
  const int saved_corr[rhd::kBuckets] = {ctx->corr_map[0], ctx->corr_map[1], ctx->corr_map[2]};
  // each bucket on its own grids: first the passes' mapping (cell per thread
  // or L lanes per cell), then the correction step's lanes per cell
  std::vector<rhd_grid_t> sub;
  sub.reserve(n_grids);
  for (int b = 0; b < rhd::kBuckets && rc == RHD_OK; ++b) {
    sub.clear();
    for (int j = 0; j < n_grids; ++j)
      if (rhd::bucket_of(grids[j].groups.n_groups) == b && grids[j].n_cells > 0)
        sub.push_back(grids[j]);
    if (sub.empty()) continue;
    const bool mixed = sub[0].state.precision == RHD_MIXED;
    for (int stage = 0; stage < (mixed ? 2 : 1) && rc == RHD_OK; ++stage) {
      const int cands[4] = {1, 8, 16, 32};
      float best = 1e30f;
      int pick = stage == 0 ? ctx->pass_map[b] : ctx->corr_map[b];
      for (int m : cands) {
        if (stage == 0 ? !rhd::pass_mapping_ok(b, m) : !rhd::corr_mapping_ok(b, m)) continue;
        (stage == 0 ? ctx->pass_map : ctx->corr_map)[b] = m;
        float ms = 0.0f;
        rc = rhd::time_candidate(ctx, sub.data(), (int)sub.size(), ctx->threads, ctx->cpi, sms,
                                 sv, e0, e1, st, &ms);
        if (rc != RHD_OK) break;
        if (ms < best) {
          best = ms;
          pick = m;
        }
      }
      (stage == 0 ? ctx->pass_map : ctx->corr_map)[b] = pick;
    }
  }
  // then the CTA shape of the cell-per-thread mapping, on every grid
  bool any_thread = false;
  for (int b = 0; b < rhd::kBuckets; ++b) any_thread = any_thread || ctx->pass_map[b] == 1;
  int bt = ctx->threads, bc = ctx->cpi;
  if (any_thread && rc == RHD_OK) {
    const int cand_threads[3] = {64, 128, 256};
    const int cand_mult[3] = {1, 4, 16};
    float best = 1e30f;
    for (int a = 0; a < 3 && rc == RHD_OK; ++a)
      for (int m = 0; m < 3 && rc == RHD_OK; ++m) {
        const int th = cand_threads[a], cpi = th * cand_mult[m];
        float ms = 0.0f;
        rc = rhd::time_candidate(ctx, grids, n_grids, th, cpi, sms, sv, e0, e1, st, &ms);
        if (rc == RHD_OK && ms < best) {
          best = ms;
          bt = th;
          bc = cpi;
        }
      }
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RHD_OK) {
    for (int b = 0; b < rhd::kBuckets; ++b) {
      ctx->pass_map[b] = saved_pass[b];
      ctx->corr_map[b] = saved_corr[b];
    }
    return rc;
  }
  ctx->threads = bt;
  ctx->cpi = bc;
  return RHD_OK;
}

#include "rhd_surrogate.cuh"
#include "rhd_host.cuh"

extern "C" int rhd_profile_start(void) {
  for (int k = 0; k < RHD_KERNELS; ++k) {
    for (auto &e : rhd::t_events[k]) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    rhd::t_events[k].clear();
    rhd::t_prof_n[k] = 0;
    rhd::t_prof_ms[k] = 0.0;
  }
  rhd::t_profiling = true;
  return RHD_OK;
}

extern "C" int rhd_profile_stop(int32_t *launches, double *total_ms) {
  if (!launches || !total_ms) return RHD_EINVAL;
  rhd::t_profiling = false;
  int rc = RHD_OK;
  int32_t n = 0;
  double sum = 0.0;
  for (int k = 0; k < RHD_KERNELS; ++k) {
    double s = 0.0;
    for (auto &e : rhd::t_events[k]) {
      float ms = 0.0f;
      if (cudaEventSynchronize(e.second) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e.first, e.second) != cudaSuccess)
        rc = RHD_ECUDA;
      s += ms;
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    rhd::t_prof_n[k] = (int32_t)rhd::t_events[k].size();
    rhd::t_prof_ms[k] = s;
    rhd::t_events[k].clear();
    n += rhd::t_prof_n[k];
    sum += s;
  }
  *launches = n;
  *total_ms = sum;
  return rc;
}

extern "C" int rhd_profile_kernel(int32_t kind, int32_t *launches, double *total_ms) {
  if (kind < 0 || kind >= RHD_KERNELS || !launches || !total_ms) return RHD_EINVAL;
  *launches = rhd::t_prof_n[kind];
  *total_ms = rhd::t_prof_ms[kind];
  return RHD_OK;
}

extern "C" int rhd_events_start(void) {
  int sms = 0;
  const int rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  const unsigned long long zero[RHD_EVENTS] = {};
  if (cudaMemcpyToSymbol(rhd::g_events, zero, sizeof(zero)) != cudaSuccess) return RHD_ECUDA;
  rhd::t_infer_cells = 0;
  rhd::t_counting = true;
  return RHD_OK;
}

extern "C" int rhd_events_stop(uint64_t *counts) {
  if (!counts) return RHD_EINVAL;
  rhd::t_counting = false;
  unsigned long long c[RHD_EVENTS];
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(c, rhd::g_events, sizeof(c)) != cudaSuccess)
    return RHD_ECUDA;
  for (int k = 0; k < RHD_EVENTS; ++k) counts[k] = (uint64_t)c[k];
  counts[RHD_EV_INFER] += rhd::t_infer_cells;
  return RHD_OK;
}

extern "C" const char *rhd_strerror(int code) {
  switch (code) {
    case RHD_OK: return "ok";
    case RHD_EINVAL: return "invalid argument";
    case RHD_EEDGES: return "invalid group edges";
    case RHD_ELAW: return "invalid opacity law";
    case RHD_ECUDA: return "CUDA error";
    case RHD_ENOMEM: return "out of workspace memory";
    case RHD_ESIZE: return "size exceeds a compiled limit";
    case RHD_EIO: return "file error";
    default: return "unknown error";
  }
}

extern "C" int rhd_version(void) { return 200; }
