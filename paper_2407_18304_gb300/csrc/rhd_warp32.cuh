// rhd_warp32.cuh -- the FP32 passes of the mixed form with the groups of a
// cell spread over the lanes of a warp (the layout of rhd_warp.cuh).
//
// The steps are those of rhd_mixed.cuh (energy-scaled variables: R~ = R /
// E_tot, f = F / (c E_tot), beta = v / c).  What changes is where FP64 is
// left: a cell's scalar work runs on every lane here, and on GB300 an FP64
// instruction costs 64 FP32 ones (a warp-wide one holds the FP64 pipe of its
// SM sub-partition for 64 cycles), so nothing of the iteration is FP64: the
// quantities that cancel -- the internal energy E_int = E_gas - E_kin and the
// momentum -- are carried in float-float arithmetic (rhd_df.cuh, ~48 bits) in
// units of E_tot and rho c, the internal energy as a base E_int,0 (set once
// per outer pass, where E_gas - E_kin is formed) plus an FP32 offset,
// E_int = E_int,0 + E_tot dE~; T, a_R T^4 and the energy residual F_G are
// formed in FP32 relative to the base.  Each evaluation is FP32 throughout,
// including the Planck edges (planck_table.h polynomials truncated to degree
// 7, whose dropped terms are below FP32 resolution).  FP64 is left to loading
// a cell (its validity and E_tot, tested as the FP64 passes test them) and to
// storing its iterate.
#pragma once
#include "rhd_df.cuh"
#include "rhd_mixed.cuh"
#include "rhd_warp.cuh"

namespace rhd {

constexpr int kDeg32 = 7;
constexpr int kPlanckF = (kDeg32 + 3) * planck_table::kSeg;  // coef [8][kSeg], centre, 1/half

template <int L, int GPL>
struct WCell32 {
  int64_t i;
  double chi0s, Etot, rhoc;  // rho kappa0, E_tot, rho c (loading and storing only)
  int shE;     // E_tot = mE 2^shE (mE in [0.5, 1))
  float imE;   // 1 / mE
  float irc;   // E_tot / (rho c_v): T = (E_int / E_tot) irc
  dflt egs;    // E_gas^t / E_tot
  dflt bm0[3], bm[3];  // (rho v)^t and rho v in units of rho c: beta^t, beta
  dflt kmu;    // E_tot / (rho c c_hat): beta = beta^t - kmu sum_g (f_g - f_g^t), eq. vupdate
  dflt kke;    // rho c^2 / E_tot: E_kin / E_tot = kke |beta|^2 / 2
  dflt ke, ei; // E_kin / E_tot and E_int,0 / E_tot (the base of the current pass)
  float chg_prev;
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

// x 2^k for a float x and |k| up to ~250, in two exact power-of-two steps.
__device__ __forceinline__ float times_pow2(float x, int k) {
  const int k1 = k / 2, k2 = k - k1;
  return x * __int_as_float((127 + k1) << 23) * __int_as_float((127 + k2) << 23);
}

// Load (as load_cell32); false for an invalid cell (the FP64 passes write its
// status).  S.r non-null starts the cell from S's internal energy and R_g.
template <int L, int GPL>
__device__ __forceinline__ bool w32_load(const KParams &P, const GroupTable &tab, int64_t i, int l,
                                         unsigned mask, const WarmStart &S, WCell32<L, GPL> &C) {
  const int G = P.G;
  C.i = i;
  const double rho = P.rho[i];
  const double m0[3] = {P.mom[0][i], P.mom[1][i], P.mom[2][i]};
  const double eg0 = P.egas[i];
  const double k0 = P.kappa0 ? P.kappa0[i] : 1.0;
  bool valid = rho > 0.0 && isfinite(rho) && isfinite(eg0) && isfinite(k0) && k0 >= 0.0 &&
               isfinite(m0[0]) && isfinite(m0[1]) && isfinite(m0[2]);
  const double KE0 = 0.5 * (m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2]) / rho;
  valid = valid && (eg0 - KE0 > 0.0);  // the FP64 passes' test, to the bit
  double e[GPL], sumE0 = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    e[j] = 0.0;
    if (g < G) {
      const int64_t o = (int64_t)g * P.gs + i;
      e[j] = P.src ? P.erad[o] + P.src[o] : P.erad[o];
      valid = valid && isfinite(e[j]) && isfinite(P.frad[0][o]) && isfinite(P.frad[1][o]) &&
              isfinite(P.frad[2][o]);
      sumE0 += e[j];
    }
  }
  if (!__all_sync(mask, valid)) return false;
  sumE0 = seg_sum<L>(sumE0, mask);
  C.chi0s = rho * k0;
  C.Etot = eg0 + P.cr * sumE0;
  C.rhoc = rho * P.c;
  // the energy-scaled group values are formed in FP32 from the bit patterns
  // (exact power-of-two scaling by E_tot's exponent, then one FP32 multiply):
  // no FP64 instruction per group
  const float mE = frexp_f(C.Etot, C.shE);
  C.imE = 1.0f / mE;
  int shV, shR;
  frexp_f(C.rhoc, shV);
  const float mR = frexp_f(rho * P.c_v, shR);
  C.irc = times_pow2(mE / mR, C.shE - shR);
  // the per-cell scalars in float-float, in units of E_tot and rho c
  const dflt mEd = df_from_double(C.Etot, C.shE), imEd = df_rcp(mEd);
  const dflt imVd = df_rcp(df_from_double(C.rhoc, shV));
  C.egs = df_from_double(eg0, C.shE) * imEd;
#pragma unroll
  for (int d = 0; d < 3; ++d) C.bm0[d] = C.bm[d] = df_from_double(m0[d], shV) * imVd;
  C.kmu = mEd / df_from_double(C.rhoc * P.c_hat, C.shE);
  C.kke = df_from_double(C.rhoc * P.c, C.shE) * imEd;
  C.ke = df_scale(C.kke * (C.bm0[0] * C.bm0[0] + C.bm0[1] * C.bm0[1] + C.bm0[2] * C.bm0[2]), 0.5f);
  C.ei = C.egs - C.ke;
  const bool warm = S.r && S.eint[i] > 0.0;
  if (warm) C.ei = df_from_double(S.eint[i], C.shE) * imEd;
  C.nit = 0;
  C.outer = 0;
  C.chg_prev = __int_as_float(0x7F800000);
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
      if (warm) C.R[j] = S.r[(int64_t)g * P.n + i];
    } else {
      C.e0[j] = 0.0f;
      for (int d = 0; d < 3; ++d) C.ft[j][d] = C.f[j][d] = 0.0f;
    }
  }
  w32_set_tau(P, tab, l, C, C.chi0s);
  return true;
}

// a3 for a pass, and the base of the internal energy.
template <int L, int GPL>
__device__ __forceinline__ void w32_outer_begin(const KParams &P, WCell32<L, GPL> &C) {
  for (int d = 0; d < 3; ++d) C.be[d] = C.bm[d].hi;  // v / c
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    C.w[j] = C.be[0] * C.f[j][0] + C.be[1] * C.f[j][1] + C.be[2] * C.f[j][2];
  C.eb = C.ei.hi;
  C.dlt = 0.0f;
  C.FG0 = ((C.ei + C.ke) - C.egs).hi;
  // T0 = mT 2^eT; a_R T0^4 / E_tot = mT^4 (a_R 2^(4 eT - shE)) / mE, each factor
  // inside FP32's range
  const float T0 = C.eb * C.irc;
  const int eT = ((__float_as_int(T0) >> 23) & 0xFF) - 126;
  const float mT = __int_as_float((__float_as_int(T0) & 0x807FFFFF) | (126 << 23));
  const float mT2 = mT * mT;
  C.k4 = mT2 * mT2 * (scaled_f(P.a_rad, C.shE - 4 * eT) * C.imE);
  C.iT0 = 1.0f / T0;
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

// FP32 write-back, flux and momentum update, outer test (as outer_end32);
// the gas energy, momentum and kinetic energy in float-float.
template <int L, int GPL>
__device__ __forceinline__ bool w32_outer_end(const KParams &P, const GroupTable &tab, int l,
                                              unsigned mask, WCell32<L, GPL> &C) {
  const int G = P.G;
  const float cr = (float)P.cr;
  float sR = 0.0f;
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    if (l + L * j < G) sR += C.R[j];
  sR = seg_sumf<L>(sR, mask);
  const dflt egas_new = C.egs - two_prod(cr, sR);  // E_gas / E_tot after the write-back
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
  // eq. vupdate in units of rho c, and the kinetic energy of the new momentum
  dflt bn[3];
  for (int d = 0; d < 3; ++d) bn[d] = C.bm0[d] - C.kmu * df[d];
  const dflt KEn = df_scale(C.kke * (bn[0] * bn[0] + bn[1] * bn[1] + bn[2] * bn[2]), 0.5f);
  const float bnf[3] = {bn[0].hi, bn[1].hi, bn[2].hi};
  float cg = 0.0f;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    const float wn = bnf[0] * C.f[j][0] + bnf[1] * C.f[j][1] + bnf[2] * C.f[j][2];
    cg += fabsf((1.0f + tab.alphaf[g]) * C.q[j] * (wn - C.w[j])) * C.qe[j];
  }
  const float chg = fabsf((KEn - C.ke).hi) + seg_sumf<L>(cg, mask);
  for (int d = 0; d < 3; ++d) C.bm[d] = bn[d];
  if (C.outer >= 1 && chg > 0.25f * C.chg_prev) C.slow = 1;
  C.chg_prev = chg;
  dflt ein = egas_new - KEn;  // the next pass's base (or the correction's start)
  if (!(ein.hi > 0.0f)) ein = C.egs - C.ke;
  C.ei = ein;
  C.ke = KEn;
  ++C.outer;
  if (chg <= 3e-8f || C.outer >= P.max_outer) return true;
  w32_outer_begin(P, C);
  return false;
}

// A float-float value in units of u (a double) as a double: two widenings
// from the bit patterns (no FP64 instruction), one addition, one product.
__device__ __forceinline__ double df_to_double(dflt v, double u) {
  return (f2d(v.hi) + f2d(v.lo)) * u;
}

template <int L, int GPL>
__device__ __forceinline__ void w32_store(const KParams &P, const WarmOut &W, int l,
                                          const WCell32<L, GPL> &C) {
  const int64_t i = C.i, n = P.n;
  if (l == 0) {
    W.eint[i] = df_to_double(C.ei, C.Etot);
    W.mom[i] = df_to_double(C.bm[0], C.rhoc);
    W.mom[n + i] = df_to_double(C.bm[1], C.rhoc);
    W.mom[2 * n + i] = df_to_double(C.bm[2], C.rhoc);
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
  if (!w32_load(P, tab, i, l, mask, S, C)) return;
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
