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
  if (s->flags & ~(RHD_GROUP_TEST | RHD_FLUX_TEST | RHD_CELL_PER_THREAD)) return RHD_EINVAL;
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
  if (kp.G <= 16) launch_thread<16>(kp, W, sms, st);
  else if (kp.G <= 32) launch_thread<32>(kp, W, sms, st);
  else if (kp.G <= 64) launch_warp<32, 2>(kp, W, sms, st);
  else if (kp.G <= 128) launch_warp<32, 4>(kp, W, sms, st);
  else launch_thread<kMaxG>(kp, W, sms, st);
}

// The FP32 passes of the mixed form (writing the warm start wo; starting
// from S where S.r is set): one cell per thread up to 32 groups and past 64,
// a warp per cell in between (rhd_warp32.cuh).
template <int MAXG>
void launch_fp32_passes_impl(const KParams &kp, const WarmOut &wo, const WarmStart &S, int sms,
                             cudaStream_t st) {
  const int threads = 128;
  const size_t smem = table_bytes(kp.G);
  if (kp.G > 32 && kp.G <= 64 && !(kp.flags & RHD_CELL_PER_THREAD)) {
    const int b = persistent_blocks(warm_warp32_kernel<32, 2>, smem, sms, kp.n * 32, threads);
    warm_warp32_kernel<32, 2><<<b, threads, smem, st>>>(kp, wo, S);
    return;
  }
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
  correct_warp_kernel<L, GPL><<<b, threads, smem, st>>>(kp, wo, CorrOut{wo.ur, wo.uf, wo.done});
}

// The correction step after the FP32 passes (rhd_correct.cuh): L lanes per
// cell with GPL groups each (up to 128 groups); it finishes most cells and
// returns the warm start of the FP64 passes for the rest.
WarmStart launch_correct(const KParams &kp, const WarmOut &wo, const WarmStart &wi, int sms,
                         cudaStream_t st) {
  WarmStart w = wi;
  if (kp.G > 128) return w;
  timed_launch(RHD_KERNEL_CORRECTION, st, [&] {
    if (kp.G <= 16) launch_correct_k<8, 2>(kp, wo, sms, st);
    else if (kp.G <= 32) launch_correct_k<16, 2>(kp, wo, sms, st);
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
// Grids are split in two classes, each with its own work queue: one cell per
// thread (up to 32 groups, or RHD_CELL_PER_THREAD) and one cell per warp
// (33..64 groups).  Staging layout: offsets [2][cap + 1], selections [2][cap].
struct rhd_context {
  int device = -1;
  int threads = 128, cpi = 512;  // thread-class launch shape (autotuned)
  int cap_grids = 0;
  rhd::KParams *h_grids = nullptr, *d_grids = nullptr;
  int64_t *h_off = nullptr, *d_off = nullptr;
  int *h_sel = nullptr, *d_sel = nullptr;
  int n_sel[2] = {0, 0};
  double *d_tables = nullptr;
  unsigned long long *d_head = nullptr;  // one counter per class
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;       // the warp class runs here, forked from the main stream
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t exec = nullptr;
  int sig_grids = -1, sig_threads = 0, sig_cpi = 0, sig_prec = -1;
  int64_t sig_items[2] = {-1, -1};
  int sig_sel[2] = {-1, -1};
  cudaEvent_t done = nullptr;
  bool pending = false;
};

namespace rhd {
namespace {

constexpr int kMaxGB = RHD_MAX_GROUPS_BATCHED;
const int64_t kTableWords = group_table_words(kMaxGB) + 1;
constexpr int kCpiWarp = 64;  // cells per work item of the warp class

void ctx_free(rhd_context *c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->h_grids) cudaFreeHost(c->h_grids);
  if (c->h_off) cudaFreeHost(c->h_off);
  if (c->h_sel) cudaFreeHost(c->h_sel);
  if (c->d_grids) cudaFree(c->d_grids);
  if (c->d_off) cudaFree(c->d_off);
  if (c->d_sel) cudaFree(c->d_sel);
  if (c->d_tables) cudaFree(c->d_tables);
  if (c->d_head) cudaFree(c->d_head);
  c->exec = nullptr;
  c->h_grids = c->d_grids = nullptr;
  c->h_off = c->d_off = nullptr;
  c->h_sel = c->d_sel = nullptr;
  c->d_tables = nullptr;
  c->d_head = nullptr;
  c->cap_grids = 0;
}

int ctx_reserve(rhd_context *c, int n_grids) {
  if (n_grids <= c->cap_grids) return RHD_OK;
  if (c->pending) cudaEventSynchronize(c->done);
  ctx_free(c);
  int cap = 64;
  while (cap < n_grids) cap *= 2;
  if (cudaHostAlloc(&c->h_grids, sizeof(KParams) * cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&c->h_off, sizeof(int64_t) * 2 * (cap + 1), cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&c->h_sel, sizeof(int) * 2 * cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaMalloc(&c->d_grids, sizeof(KParams) * cap) != cudaSuccess ||
      cudaMalloc(&c->d_off, sizeof(int64_t) * 2 * (cap + 1)) != cudaSuccess ||
      cudaMalloc(&c->d_sel, sizeof(int) * 2 * cap) != cudaSuccess ||
      cudaMalloc(&c->d_tables, sizeof(double) * kTableWords * cap) != cudaSuccess ||
      cudaMalloc(&c->d_head, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    ctx_free(c);
    return RHD_ENOMEM;
  }
  c->cap_grids = cap;
  return RHD_OK;
}

// Pack the grids into the pinned staging buffers and split them into the two
// classes; work items per class out (items[0] thread class, items[1] warp class).
int pack_batch(rhd_context *c, const rhd_grid_t *grids, int n_grids, int cpi, int *prec,
               int64_t items[2]) {
  int64_t acc[2] = {0, 0};
  int ns[2] = {0, 0};
  int64_t *off[2] = {c->h_off, c->h_off + c->cap_grids + 1};
  int *sel[2] = {c->h_sel, c->h_sel + c->cap_grids};
  *prec = -1;
  for (int j = 0; j < n_grids; ++j) {
    const rhd_grid_t &g = grids[j];
    const int rc = pack(&g.state, &g.groups, &g.opacity_law, g.dt, g.n_cells, &c->h_grids[j]);
    if (rc != RHD_OK) return rc;
    if (g.opacity_law.mode == RHD_PPL_FREE) return RHD_ELAW;  // per-cell solve only
    if (g.groups.n_groups > kMaxGB) return RHD_ESIZE;
    if (*prec < 0) *prec = g.state.precision;
    if (g.state.precision != *prec) return RHD_EINVAL;
    const int cls = (g.groups.n_groups > 32 && !(g.state.flags & RHD_CELL_PER_THREAD)) ? 1 : 0;
    const int per = cls ? kCpiWarp : cpi;
    off[cls][ns[cls]] = acc[cls];
    sel[cls][ns[cls]] = j;
    ++ns[cls];
    acc[cls] += (g.n_cells + per - 1) / per;
  }
  for (int k = 0; k < 2; ++k) {
    off[k][ns[k]] = acc[k];
    items[k] = acc[k];
    c->n_sel[k] = ns[k];
  }
  return RHD_OK;
}

template <bool MIXED>
cudaError_t enqueue_batch(rhd_context *c, int n_grids, int threads, int cpi, int sms,
                          const int64_t items[2], cudaStream_t st) {
  const int cap = c->cap_grids;
  cudaMemcpyAsync(c->d_grids, c->h_grids, sizeof(KParams) * n_grids, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->d_off, c->h_off, sizeof(int64_t) * 2 * (cap + 1), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->d_sel, c->h_sel, sizeof(int) * 2 * cap, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(c->d_head, 0, 2 * sizeof(unsigned long long), st);
  tables_kernel<<<n_grids, 128, table_bytes(kMaxGB) + 64, st>>>(c->d_grids, c->d_tables,
                                                                   kTableWords);
  const size_t smem = table_bytes(kMaxGB) + 64;
  const bool both = items[0] > 0 && items[1] > 0;
  if (both) {
    cudaEventRecord(c->fork, st);
    cudaStreamWaitEvent(c->side, c->fork, 0);
  }
  if (items[0] > 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<kMaxGB, MIXED>,
                                                      threads, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    batched_kernel<kMaxGB, MIXED><<<sms * per_sm, threads, smem, st>>>(
        c->d_grids, c->d_tables, kTableWords, c->d_sel, c->d_off, c->n_sel[0], cpi, c->d_head);
  }
  if (items[1] > 0) {
    // the two classes run side by side (each one's tail overlaps the other's work)
    cudaStream_t ws = both ? c->side : st;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_warp_kernel<MIXED>, 128,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    batched_warp_kernel<MIXED><<<sms * per_sm, 128, smem, ws>>>(
        c->d_grids, c->d_tables, kTableWords, c->d_sel + cap, c->d_off + cap + 1, c->n_sel[1],
        kCpiWarp, c->d_head + 1);
    if (ws != st) {
      cudaEventRecord(c->join, ws);
      cudaStreamWaitEvent(st, c->join, 0);
    }
  }
  return cudaGetLastError();
}

cudaError_t enqueue_any(rhd_context *c, int prec, int n_grids, int threads, int cpi, int sms,
                        const int64_t items[2], cudaStream_t st) {
  return prec == RHD_MIXED ? enqueue_batch<true>(c, n_grids, threads, cpi, sms, items, st)
                           : enqueue_batch<false>(c, n_grids, threads, cpi, sms, items, st);
}

}  // namespace
}  // namespace rhd

extern "C" int rhd_context_create(rhd_context_t **ctx) {
  if (!ctx) return RHD_EINVAL;
  rhd_context *c = new (std::nothrow) rhd_context();
  if (!c) return RHD_ENOMEM;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess) {
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    if (c->done) cudaEventDestroy(c->done);
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
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->done) cudaEventDestroy(ctx->done);
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

extern "C" int rhd_source_update_batched(rhd_context_t *ctx, const rhd_grid_t *grids,
                                         int32_t n_grids, void *stream) {
  if (!ctx || !grids || n_grids < 1) return RHD_EINVAL;
  if (n_grids > RHD_MAX_GRIDS) return RHD_ESIZE;
  int sms = 0;
  int rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  // the previous call of this context may still read the staging buffers
  if (ctx->pending) {
    cudaEventSynchronize(ctx->done);
    ctx->pending = false;
  }
  rc = rhd::ctx_reserve(ctx, n_grids);
  if (rc != RHD_OK) return rc;
  int prec = 0;
  int64_t items[2] = {0, 0};
  rc = rhd::pack_batch(ctx, grids, n_grids, ctx->cpi, &prec, items);
  if (rc != RHD_OK) return rc;
  if (items[0] + items[1] == 0) return RHD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const bool same = ctx->exec && ctx->sig_grids == n_grids && ctx->sig_items[0] == items[0] &&
                    ctx->sig_items[1] == items[1] && ctx->sig_sel[0] == ctx->n_sel[0] &&
                    ctx->sig_sel[1] == ctx->n_sel[1] && ctx->sig_threads == ctx->threads &&
                    ctx->sig_cpi == ctx->cpi && ctx->sig_prec == prec;
  if (!same) {
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    ctx->exec = nullptr;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return RHD_ECUDA;
    const cudaError_t le =
        rhd::enqueue_any(ctx, prec, n_grids, ctx->threads, ctx->cpi, sms, items, ctx->cap);
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
    ctx->sig_grids = n_grids;
    ctx->sig_items[0] = items[0];
    ctx->sig_items[1] = items[1];
    ctx->sig_sel[0] = ctx->n_sel[0];
    ctx->sig_sel[1] = ctx->n_sel[1];
    ctx->sig_threads = ctx->threads;
    ctx->sig_cpi = ctx->cpi;
    ctx->sig_prec = prec;
  }
  if (cudaGraphLaunch(ctx->exec, st) != cudaSuccess) return RHD_ECUDA;
  if (cudaEventRecord(ctx->done, st) != cudaSuccess) return RHD_ECUDA;
  ctx->pending = true;
  return RHD_OK;
}

extern "C" int rhd_context_autotune(rhd_context_t *ctx, const rhd_grid_t *grids, int32_t n_grids,
                                    void *stream) {
  if (!ctx || !grids || n_grids < 1) return RHD_EINVAL;
  if (n_grids > RHD_MAX_GRIDS) return RHD_ESIZE;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  int rc = rhd::ensure_device(&sms);
  if (rc != RHD_OK) return rc;
  if (ctx->pending) {
    cudaEventSynchronize(ctx->done);
    ctx->pending = false;
  }
  rc = rhd::ctx_reserve(ctx, n_grids);
  if (rc != RHD_OK) return rc;
  // save the in/out arrays of every grid
  struct Buf {
    void *dst;
    const void *src;
    size_t bytes;
  };
  std::vector<Buf> bufs;
  size_t total_bytes = 0;
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
  for (auto &b : bufs) total_bytes += (b.bytes + 255) & ~size_t(255);
  char *save = nullptr;
  if (cudaMalloc(&save, total_bytes) != cudaSuccess) return RHD_ENOMEM;
  size_t off = 0;
  for (auto &b : bufs) {
    b.dst = save + off;
    off += (b.bytes + 255) & ~size_t(255);
    cudaMemcpyAsync(b.dst, b.src, b.bytes, cudaMemcpyDeviceToDevice, st);
  }
  auto restore = [&]() {
    for (auto &b : bufs) cudaMemcpyAsync(const_cast<void *>(b.src), b.dst, b.bytes,
                                         cudaMemcpyDeviceToDevice, st);
  };
  const int cand_threads[3] = {64, 128, 256};
  const int cand_mult[3] = {1, 4, 16};
  float best = 1e30f;
  int bt = ctx->threads, bc = ctx->cpi;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  rc = RHD_OK;
  for (int a = 0; a < 3 && rc == RHD_OK; ++a) {
    for (int b = 0; b < 3 && rc == RHD_OK; ++b) {
      const int th = cand_threads[a], cpi = th * cand_mult[b];
      int prec = 0;
      int64_t items[2] = {0, 0};
      rc = rhd::pack_batch(ctx, grids, n_grids, cpi, &prec, items);
      if (rc != RHD_OK || items[0] + items[1] == 0) break;
      cudaEventRecord(e0, st);
      if (rhd::enqueue_any(ctx, prec, n_grids, th, cpi, sms, items, st) != cudaSuccess)
        rc = RHD_ECUDA;
      cudaEventRecord(e1, st);
      restore();
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = RHD_ECUDA;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == RHD_OK && ms < best) {
        best = ms;
        bt = th;
        bc = cpi;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(save);
  if (rc != RHD_OK) return rc;
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
