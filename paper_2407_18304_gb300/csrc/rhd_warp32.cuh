// rhd_warp32.cuh -- the FP32 passes of the mixed form with the groups of a
// cell spread over the lanes of a warp (the layout of rhd_warp.cuh).
//
// The steps are those of rhd_mixed.cuh (energy-scaled variables: R~ = R /
// E_tot, f = F / (c E_tot), beta = v / c).  What changes is where FP64 is
// left: a cell's scalar work runs on every lane here, and on GB300 an FP64
// instruction costs 64 FP32 ones, so the internal energy is carried as an
// FP64 base E_int,0 (set once per outer pass, where E_gas - E_kin is formed)
// plus an FP32 offset, E_int = E_int,0 + E_tot dE~; T, a_R T^4 and the energy
// residual F_G are formed in FP32 relative to the base.  Each evaluation is
// then FP32 throughout, including the Planck edges (planck_table.h
// polynomials truncated to degree 7, whose dropped terms are below FP32
// resolution).
#pragma once
#include "rhd_mixed.cuh"
#include "rhd_warp.cuh"

namespace rhd {

constexpr int kDeg32 = 7;
constexpr int kPlanckF = (kDeg32 + 3) * planck_table::kSeg;  // coef [8][kSeg], centre, 1/half

template <int L, int GPL>
struct WCell32 {
  int64_t i;
  double rho, irho, m0[3], eg0, chi0s, Etot, irc;  // irho = 1/rho
  int shE, shV;  // E_tot = mE 2^shE, rho c = mV 2^shV (mE, mV in [0.5, 1))
  float imE, imV;  // 1 / mE, 1 / mV
  double m[3], KE, Eint;  // Eint: the FP64 base of the current pass
  double chg_prev;
  int nit, it, outer, slow;
  float eb;    // E_int,0 / E_tot
  float dlt;   // (E_int - E_int,0) / E_tot
  float FG0;   // (E_int,0 + E_kin - E_gas^t) / E_tot
  float k4;    // a_R T0^4 / E_tot
  float iT0;   // 1 / T0
  float be[3];
  float R[GPL], FR[GPL], dg[GPL], qe[GPL], itau[GPL], tau[GPL], e0[GPL], w[GPL], b[GPL],
      dnx[GPL], q[GPL];
  float f[GPL][3], ft[GPL][3];
};

// FP32 edge values from the polynomial table (float copy pf); same segments,
// outputs and conventions as edge_tab.
__device__ __forceinline__ void edge_tab32(const float *pf, float x, float &pq, float &d,
                                           float &ed, bool &low) {
  using namespace planck_table;
  if (!(x > 0.0f)) {
    pq = 0.0f;
    d = 0.0f;
    ed = 0.0f;
    low = true;
    return;
  }
  if (isinf(x)) {
    pq = 0.0f;
    d = 0.0f;
    ed = 0.0f;
    low = false;
    return;
  }
  if (x > 1.0e4f) {  // beyond FP32's range: every edge term is 0
    pq = 0.0f;
    d = 0.0f;
    ed = 0.0f;
    low = false;
    return;
  }
  const float K = (float)kPlanckNorm;
  const float em = expm1f(x);
  const float xr = isinf(em) ? 0.0f : x / em;
  const float emx = 1.0f / (em + 1.0f);
  const float x3 = x * x * x;
  d = K * x3 * xr;
  ed = d * (4.0f - xr - x);
  const int bits = __float_as_int(x);
  const int e = ((bits >> 23) & 0xFF) - 127;
  int sg = 1 + (e - kEMin) * kSub + ((bits >> 21) & 3);
  sg = e < kEMin ? 0 : (e > kEMax ? kSeg - 1 : sg);
  const float *cen = pf + (kDeg32 + 1) * kSeg, *ih = cen + kSeg;
  const float u = e > kEMax ? 0.0f : (x - cen[sg]) * ih[sg];
  float p = pf[kDeg32 * kSeg + sg];
#pragma unroll
  for (int k = kDeg32 - 1; k >= 0; --k) p = fmaf(p, u, pf[k * kSeg + sg]);
  low = x < 2.0f;
  pq = K * x3 * p * (low ? 1.0f : emx);
}

template <int L>
__device__ __forceinline__ float seg_sumf(float v, unsigned mask) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

template <int L, int GPL>
__device__ __forceinline__ void w32_set_tau(const KParams &P, const GroupTable &tab, int l,
                                            WCell32<L, GPL> &C, double cs) {
  // tau_g = c_hat theta dt cs kbar_g in FP32 from the bit patterns: with
  // c_hat theta dt cs = mt 2^et, tau_g = mt (kbar_g 2^et)
  const double tcs = P.c_hat * P.theta * P.dt * cs;
  int et = 0;
  const float mt = tcs > 0.0 ? frexp_f(tcs, et) : 0.0f;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    const float t = g < P.G ? mt * scaled_f(tab.kbar[g], -et) : 0.0f;
    C.tau[j] = t;
    C.itau[j] = t > 0.0f ? 1.0f / t : 0.0f;
    C.qe[j] = t > 0.0f ? t / (1.0f + t) : 0.0f;
  }
}

// Load (as load_cell32); false for an invalid cell (the FP64 passes write its status).
template <int L, int GPL>
__device__ __forceinline__ bool w32_load(const KParams &P, const GroupTable &tab, int64_t i, int l,
                                         unsigned mask, WCell32<L, GPL> &C) {
  const int G = P.G;
  C.i = i;
  C.rho = P.rho[i];
  C.m0[0] = P.mom[0][i];
  C.m0[1] = P.mom[1][i];
  C.m0[2] = P.mom[2][i];
  C.eg0 = P.egas[i];
  const double k0 = P.kappa0 ? P.kappa0[i] : 1.0;
  bool valid = C.rho > 0.0 && isfinite(C.rho) && isfinite(C.eg0) && isfinite(k0) && k0 >= 0.0 &&
               isfinite(C.m0[0]) && isfinite(C.m0[1]) && isfinite(C.m0[2]);
  const double KE0 = 0.5 * (C.m0[0] * C.m0[0] + C.m0[1] * C.m0[1] + C.m0[2] * C.m0[2]) / C.rho;
  valid = valid && (C.eg0 - KE0 > 0.0);
  double e[GPL], sumE0 = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    e[j] = 0.0;
    if (g < G) {
      const int64_t o = (int64_t)g * P.gs + i;
      e[j] = P.erad[o] + (P.src ? P.src[o] : 0.0);
      valid = valid && isfinite(e[j]) && isfinite(P.frad[0][o]) && isfinite(P.frad[1][o]) &&
              isfinite(P.frad[2][o]);
      sumE0 += e[j];
    }
  }
  if (!__all_sync(mask, valid)) return false;
  sumE0 = seg_sum<L>(sumE0, mask);
  C.chi0s = C.rho * k0;
  C.Etot = C.eg0 + P.cr * sumE0;
  C.irho = 1.0 / C.rho;
  C.irc = C.irho / P.c_v;
  // the energy-scaled group values are formed in FP32 from the bit patterns
  // (exact power-of-two scaling by E_tot's exponent, then one FP32 multiply):
  // no FP64 instruction per group
  C.imE = 1.0f / frexp_f(C.Etot, C.shE);
  C.imV = 1.0f / frexp_f(C.rho * P.c, C.shV);
  C.m[0] = C.m0[0];
  C.m[1] = C.m0[1];
  C.m[2] = C.m0[2];
  C.Eint = C.eg0 - KE0;
  C.nit = 0;
  C.outer = 0;
  C.chg_prev = HUGE_VAL;
  C.slow = 0;
  const float fsf = C.imE / (float)P.c;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    C.R[j] = 0.0f;
    if (g < G) {
      const int64_t o = (int64_t)g * P.gs + i;
      C.e0[j] = scaled_f(e[j], C.shE) * C.imE;
      for (int d = 0; d < 3; ++d) C.ft[j][d] = C.f[j][d] = scaled_f(P.frad[d][o], C.shE) * fsf;
    } else {
      C.e0[j] = 0.0f;
      for (int d = 0; d < 3; ++d) C.ft[j][d] = C.f[j][d] = 0.0f;
    }
  }
  w32_set_tau(P, tab, l, C, C.chi0s);
  return true;
}

// a3 for a pass, and the FP64 base of the internal energy.
template <int L, int GPL>
__device__ __forceinline__ void w32_outer_begin(const KParams &P, WCell32<L, GPL> &C) {
  C.KE = 0.5 * (C.m[0] * C.m[0] + C.m[1] * C.m[1] + C.m[2] * C.m[2]) * C.irho;
  for (int d = 0; d < 3; ++d) C.be[d] = scaled_f(C.m[d], C.shV) * C.imV;  // v / c
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    C.w[j] = C.be[0] * C.f[j][0] + C.be[1] * C.f[j][1] + C.be[2] * C.f[j][2];
  const double T0 = C.Eint * C.irc;
  C.eb = scaled_f(C.Eint, C.shE) * C.imE;
  C.dlt = 0.0f;
  C.FG0 = scaled_f(C.Eint + C.KE - C.eg0, C.shE) * C.imE;
  C.k4 = scaled_f(P.a_rad * T0 * T0 * T0 * T0, C.shE) * C.imE;
  C.iT0 = 1.0f / (float)T0;
  C.it = 0;
}

// One FP32 inner iteration (as inner_step32); 0 continue, 1 done, 2 cap.
template <int L, int GPL>
__device__ __forceinline__ int w32_inner_step(const KParams &P, const GroupTable &tab,
                                              const float *pf, int l, int lane0, unsigned mask,
                                              WCell32<L, GPL> &C) {
  constexpr int NE = GPL + 1;
  const int G = P.G;
  const float cr = (float)P.cr;
  const float tol32 = 1e-7f;  // near FP32 resolution: the correction step then needs one Newton step
  const int max_it = P.max_newton < 32 ? P.max_newton : 32;
  const float eint = C.eb + C.dlt;          // E_int / E_tot
  const float t = eint / C.eb;              // T / T0
  if (P.temp_exp != 0.0)
    w32_set_tau(P, tab, l, C, C.chi0s * pow((double)t / ((double)C.iT0 * P.T_ref), P.temp_exp));
  const float t2 = t * t;
  const float aT4s = C.k4 * t2 * t2;        // a_R T^4 / E_tot
  const float dTs = aT4s / eint;            // (a_R T^3 / E_tot) dT/dE~_int
  const float invT = C.iT0 / t;
  float pqE[NE], dE_[NE], eE[NE];
  bool lowE[NE];
#pragma unroll
  for (int jj = 0; jj < NE; ++jj) {
    const int e = l + L * jj;
    edge_tab32(pf, e <= G ? tab.xef[e] * invT : 1.0f, pqE[jj], dE_[jj], eE[jj], lowE[jj]);
  }
  float sumR = 0.0f, sFRe = 0.0f, sde = 0.0f, sabs = 0.0f;
  const int src_lane = lane0 + (l + 1) % L;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const float pa = __shfl_sync(mask, pqE[j], src_lane), pb = __shfl_sync(mask, pqE[j + 1], src_lane);
    const float da = __shfl_sync(mask, dE_[j], src_lane), db_ = __shfl_sync(mask, dE_[j + 1], src_lane);
    const float ea = __shfl_sync(mask, eE[j], src_lane), eb = __shfl_sync(mask, eE[j + 1], src_lane);
    const int la = __shfl_sync(mask, (int)lowE[j], src_lane),
              lb = __shfl_sync(mask, (int)lowE[j + 1], src_lane);
    const bool last = l == L - 1;
    const float pqU = last ? pb : pa, dU = last ? db_ : da, eU = last ? eb : ea;
    const bool lowU = (last ? lb : la) != 0;
    const int g = l + L * j;
    if (g >= G) {
      C.FR[j] = 0.0f;
      C.dg[j] = 0.0f;
      continue;
    }
    const float dP = band_fp32(pqE[j], lowE[j], pqU, lowU);
    const float dD = dU - dE_[j];
    const float b = aT4s * dP;
    const float dbs = dTs * (4.0f * dP - dD);  // d b~ / dE~_int
    const float a = tab.alphaf[g], rm = tab.rmf[g], rp = tab.rpf[g];
    float dq;
    // chiF_ratio's T-derivative, expressed per E~_int (aT3 -> dTs)
    const float q = chiF_ratio<float>(b, aT4s, dD, a, rm, rp, dE_[j], dU, dbs, dTs, eE[j], eU, dq);
    C.b[j] = b;
    C.dnx[j] = aT4s * (rp * dU - rm * dE_[j]);
    C.q[j] = q;
    const float ie = C.qe[j];
    float fr, d;
    if (ie > 0.0f) {
      const float Eg = b + (1.0f + a) * q * C.w[j] - C.R[j] * C.itau[j];
      fr = Eg - C.e0[j] - C.R[j];
      d = dbs + (1.0f + a) * dq * C.w[j];
    } else {
      fr = -C.R[j];
      d = 0.0f;
    }
    const float iee = ie > 0.0f ? ie : 1.0f;
    C.FR[j] = fr;
    C.dg[j] = d;
    sumR += C.R[j];
    sFRe -= fr * iee;
    sde -= d * iee;
    sabs += fabsf(fr);
  }
  sumR = seg_sumf<L>(sumR, mask);
  sFRe = seg_sumf<L>(sFRe, mask);
  sde = seg_sumf<L>(sde, mask);
  sabs = seg_sumf<L>(sabs, mask);
  const float FG = C.FG0 + C.dlt + cr * sumR;
  if (fabsf(FG) < tol32 && cr * sabs < tol32) return 1;
  if (C.it >= max_it) return 2;
  const float dE = (-FG + cr * sFRe) / (1.0f - cr * sde);
  float lam = 1.0f;
  for (int k = 0; k < 40 && !(eint + lam * dE > 0.0f); ++k) lam *= 0.5f;
  C.dlt += lam * dE;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const float ie = C.qe[j] > 0.0f ? C.qe[j] : 1.0f;
    C.R[j] += lam * (C.FR[j] + C.dg[j] * dE) * ie;
  }
  ++C.nit;
  ++C.it;
  return fabsf(dE) < 1e-8f ? 1 : 0;
}

// FP32 write-back, flux and momentum update, outer test (as outer_end32).
template <int L, int GPL>
__device__ __forceinline__ bool w32_outer_end(const KParams &P, const GroupTable &tab, int l,
                                              unsigned mask, WCell32<L, GPL> &C) {
  const int G = P.G;
  const double Etot = C.Etot;
  const float cr = (float)P.cr;
  float sR = 0.0f;
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    if (l + L * j < G) sR += C.R[j];
  sR = seg_sumf<L>(sR, mask);
  const double egas_new = C.eg0 - (double)cr * (double)sR * Etot;
  float df[3] = {0.0f, 0.0f, 0.0f};
  const float bmag = sqrtf(C.be[0] * C.be[0] + C.be[1] * C.be[1] + C.be[2] * C.be[2]);
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    const float En = C.e0[j] + C.R[j];
    const float t = C.tau[j], a = tab.alphaf[g];
    const float srcg = t * (C.b[j] - C.dnx[j] * (1.0f / 3.0f));
    const float inv = 1.0f / (1.0f + t * C.q[j]);
    const float base[3] = {(C.ft[j][0] + C.be[0] * srcg) * inv,
                           (C.ft[j][1] + C.be[1] * srcg) * inv,
                           (C.ft[j][2] + C.be[2] * srcg) * inv};
    const float kap = (1.0f + a) * t * inv;
    float F[3] = {C.f[j][0], C.f[j][1], C.f[j][2]};
    flux_update<float>(P.closure, 1.0f, En, kap, base, C.be, bmag, F, 1e-6f, C.slow != 0);
    for (int d = 0; d < 3; ++d) {
      df[d] += F[d] - C.ft[j][d];
      C.f[j][d] = F[d];
    }
  }
  for (int d = 0; d < 3; ++d) df[d] = seg_sumf<L>(df[d], mask);
  const double mf = Etot * P.icc * P.c;  // E_tot / c_hat
  const double mn[3] = {C.m0[0] - mf * df[0], C.m0[1] - mf * df[1], C.m0[2] - mf * df[2]};
  const double KEn = 0.5 * (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) * C.irho;
  const float bn[3] = {scaled_f(mn[0], C.shV) * C.imV, scaled_f(mn[1], C.shV) * C.imV,
                       scaled_f(mn[2], C.shV) * C.imV};
  float cg = 0.0f;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    const float wn = bn[0] * C.f[j][0] + bn[1] * C.f[j][1] + bn[2] * C.f[j][2];
    cg += fabsf((1.0f + tab.alphaf[g]) * C.q[j] * (wn - C.w[j])) * C.qe[j];
  }
  const float chg = scaled_f(fabs(KEn - C.KE), C.shE) * C.imE + seg_sumf<L>(cg, mask);
  C.m[0] = mn[0];
  C.m[1] = mn[1];
  C.m[2] = mn[2];
  if (C.outer >= 1 && chg > 0.25f * (float)C.chg_prev) C.slow = 1;
  C.chg_prev = chg;
  C.Eint = egas_new - KEn;  // the next pass's base (or the FP64 phase's start)
  if (!(C.Eint > 0.0)) C.Eint = C.eg0 - C.KE;
  ++C.outer;
  if (chg <= 3e-8f || C.outer >= P.max_outer) return true;
  w32_outer_begin(P, C);
  return false;
}

template <int L, int GPL>
__device__ __forceinline__ void w32_store(const KParams &P, const WarmOut &W, int l,
                                          const WCell32<L, GPL> &C) {
  const int64_t i = C.i, n = P.n;
  if (l == 0) {
    W.eint[i] = C.Eint;
    W.mom[i] = C.m[0];
    W.mom[n + i] = C.m[1];
    W.mom[2 * n + i] = C.m[2];
    W.nit[i] = (uint8_t)(C.nit > 255 ? 255 : C.nit);
  }
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= P.G) continue;
    const int64_t o = (int64_t)g * n + i;
    W.r[o] = C.R[j];
    W.f[o] = C.f[j][0];
    W.f[(int64_t)P.G * n + o] = C.f[j][1];
    W.f[(int64_t)2 * P.G * n + o] = C.f[j][2];
  }
}

// The FP32 passes of one cell with L lanes (lane l of the cell's segment,
// mask its lanes); writes the cell's warm start to W.  S.r non-null starts the
// cell from S (may alias W).
template <int L, int GPL>
__device__ __forceinline__ void w32_cell(const KParams &P, const GroupTable &tab, const float *pf,
                                         const WarmOut &W, const WarmStart &S, int64_t i, int l,
                                         int lane0, unsigned mask, WCell32<L, GPL> &C) {
  if (!w32_load(P, tab, i, l, mask, C)) return;
  if (S.r && S.eint[i] > 0.0) {
    C.Eint = S.eint[i];
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const int g = l + L * j;
      if (g < P.G) C.R[j] = S.r[(int64_t)g * P.n + i];
    }
  }
  w32_outer_begin(P, C);
  unsigned ne = 0, no = 0;
  for (;;) {
    const int r = w32_inner_step(P, tab, pf, l, lane0, mask, C);
    ++ne;
    if (r == 0) continue;
    ++no;
    if (w32_outer_end(P, tab, l, mask, C)) break;
  }
  w32_store(P, W, l, C);
  if (l == 0) {
    count_event(P, RHD_EV_CELLS32, 1);
    count_event(P, RHD_EV_EVAL32, ne);
    count_event(P, RHD_EV_OUTER32, no);
  }
}

// The FP32 copy of the Planck polynomials the FP32 warp passes use (the
// coefficients up to kDeg32, then the segment centres and 1/half-widths),
// from the FP64 table at pc.
__device__ __forceinline__ void load_planck32(const double *pc, float *pf) {
  using namespace planck_table;
  for (int t = threadIdx.x; t < kPlanckF; t += blockDim.x) {
    const int k = t / kSeg, s = t % kSeg;
    const int src = k <= kDeg32 ? k * kSeg + s : (kDeg + 1 + (k - kDeg32 - 1)) * kSeg + s;
    pf[t] = (float)pc[src];
  }
}

// Phase A of the mixed form with L lanes per cell (warm_fp32_kernel's job):
// writes the warm start W; S.r non-null starts each cell from S (may alias W).
template <int L, int GPL>
__global__ void __launch_bounds__(128) warm_warp32_kernel(const __grid_constant__ KParams P,
                                                          const WarmOut W, const WarmStart S) {
  extern __shared__ double sm[];
  __shared__ float pf[kPlanckF];
  const GroupTable tab = build_table(P, sm);
  load_planck32(tab.pc, pf);
  __syncthreads();
  const int lane = threadIdx.x & 31, seg = lane / L, l = lane % L, lane0 = seg * L;
  const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << lane0);
  constexpr int CPW = 32 / L;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  WCell32<L, GPL> C;
  for (int64_t i = warp * CPW + seg; i < P.n; i += nwarps * CPW)
    w32_cell<L, GPL>(P, tab, pf, W, S, i, l, lane0, mask, C);
}

}  // namespace rhd
