// rhd_refine.cuh -- the first Newton step of the mixed form's correction,
// with the residual of the coupled per-cell system evaluated in float-float
// arithmetic (rhd_df.cuh) instead of FP64.
//
// The correction step (rhd_correct.cuh) takes the FP32 passes' iterate to the
// root of the coupled system (eqs. FGFR, Rnew, fupdate with the momentum of
// eq. vupdate) by Newton steps whose residual is accurate to FP64 and whose
// Jacobian is FP32; it needs two FP64 residuals per cell, one to take the
// step and one to see that the paper's tests hold after it.  The step only
// needs a residual accurate to a few units of 1e-14 of the cell's energy
// scale, which float-float arithmetic gives at a fraction of FP64's cost on
// GB300.  So this kernel evaluates the residual at the FP32 iterate with the
// edge Planck terms in FP64 (the Planck differences stay FP64) and everything
// after them in float-float, takes the FP32 Newton step of the correction and
// leaves it in the correction's step arrays; the correction then starts from
// the stepped iterate, evaluates the FP64 residual there, applies the paper's
// tests and finishes the cell (or steps again).  Nothing here decides
// convergence: a cell this kernel moves badly costs the correction one more
// FP64 step, and its result is still judged on the FP64 residual.
//
// Variables as in rhd_correct.cuh: energies in units of E_tot, fluxes in
// units of c E_tot, velocities in units of c.
#pragma once
#include "rhd_correct.cuh"
#include "rhd_df.cuh"

namespace rhd {

constexpr dflt kThirdDF = {0x1.555556p-2f, -0x1.555556p-27f};  // 1/3

// Float-float copies of a grid's group table (kbar, 1/kbar, alpha, rm, rp as
// hi/lo pairs), built in shared memory after the FP64 table.
struct DfTable {
  const float2 *kbar, *ikbar, *alpha, *rm, *rp;
  const float2 *xe;  // [G + 1] h nu_e / k_B (x_e = xe / T)
};

__host__ __device__ __forceinline__ size_t refine_df_bytes(int G) {
  return sizeof(float2) * (6 * G + 1);
}
// Shared memory of the refine kernel: the FP64 tables (build_table), the
// float-float Planck polynomials, the float-float group table, then the group
// blocks (20 floats per group slot per thread).
__host__ __device__ __forceinline__ size_t refine_planck_bytes() {
  return ((sizeof(float) * 2 * (8 + 1) * planck_table::kSeg +
           sizeof(float) * (planck_table::kDeg - 8 + 2) * planck_table::kSeg) + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t refine_smem_bytes(int G, int GPL, int threads) {
  return ((table_bytes(G) + 15) & ~(size_t)15) + refine_planck_bytes() + refine_df_bytes(G) +
         sizeof(float) * 20 * GPL * threads;
}

__device__ __forceinline__ dflt df_of(float2 v) { return dflt{v.x, v.y}; }

// Build the float-float table of G groups at d (all threads of the CTA; ends
// with __syncthreads()).
__device__ __forceinline__ DfTable build_df_table(const GroupTable &tab, float2 *d, int G) {
  for (int t = threadIdx.x; t <= G; t += blockDim.x) {
    const dflt xe = isinf(tab.xe[t]) ? dflt{__int_as_float(0x7F800000), 0.0f}
                                     : df_from_double(tab.xe[t], 0);
    d[5 * G + t] = make_float2(xe.hi, xe.lo);
    if (t == G) continue;
    const double v[5] = {tab.kbar[t], tab.ikbar[t], tab.alpha[t], tab.rm[t], tab.rp[t]};
    for (int k = 0; k < 5; ++k) {
      const dflt x = df_from_double(v[k], 0);
      d[k * G + t] = make_float2(x.hi, x.lo);
    }
  }
  __syncthreads();
  return DfTable{d, d + G, d + 2 * G, d + 3 * G, d + 4 * G, d + 5 * G};
}

// ---- Planck edge terms in float-float ---------------------------------------
//
// The same functions as edge_tab (P(x) below x = 2, else Q(x) = 1 - P(x);
// D(x) = (15/pi^4) x^4/(e^x - 1); x dD/dx), from the same planck_table.h
// polynomials: coefficients 0..8 of each segment in float-float, 9..13 (below
// 3e-7 of the leading one) in FP32, centres and inverse half-widths exact in
// FP32.  e^x enters through one exponential of s = x (x < 2: x/(e^x - 1) from
// expm1(x)) or s = -x (x >= 2: e^-x and x e^-x/(1 - e^-x)): s = k ln 2 + r with
// ln 2 split in three (Cody & Waite: k ln2_a and k ln2_b exact), expm1(r) from
// its Taylor series to r^13/13! (|r| <= ln2/2: the next term is below 4e-18).
// Beyond x = 80, e^-x is below FP32's normal range and every edge term is
// taken as 0 (Q(80) ~ 1e-30).
constexpr int kDfDeg = 8;  // float-float coefficients 0..kDfDeg
constexpr int kDfPlanckFloats =
    2 * (kDfDeg + 1) * planck_table::kSeg + (planck_table::kDeg - kDfDeg + 2) * planck_table::kSeg;
constexpr dflt kPlanckNormDF = {0x1.3b5ef8p-3f, 0x1.ab60cep-30f};  // 15/pi^4
constexpr float kLn2a = 0x1.62ep-1f, kLn2b = 0x1.0bep-15f, kLn2c = 0x1.be8e7cp-27f;
constexpr float kLog2e = 0x1.715476p+0f;
struct DfPlanck {
  const float2 *c;  // [kDfDeg + 1][kSeg]
  const float *ct;  // [kDeg - kDfDeg][kSeg], coefficients kDfDeg + 1 .. kDeg
  const float *cen, *ih;
};

// Convert the CTA's FP64 polynomial table (pc, planck_table.h layout) to dst
// (all threads; the caller synchronises).
__device__ __forceinline__ DfPlanck build_df_planck(const double *pc, float *dst) {
  using namespace planck_table;
  float2 *c = reinterpret_cast<float2 *>(dst);
  float *ct = dst + 2 * (kDfDeg + 1) * kSeg, *cen = ct + (kDeg - kDfDeg) * kSeg, *ih = cen + kSeg;
  for (int t = threadIdx.x; t < (kDeg + 1) * kSeg; t += blockDim.x) {
    const int k = t / kSeg;
    if (k <= kDfDeg) {
      const dflt v = df_from_double(pc[t], 0);
      c[t] = make_float2(v.hi, v.lo);
    } else {
      ct[t - (kDfDeg + 1) * kSeg] = (float)pc[t];
    }
  }
  for (int t = threadIdx.x; t < kSeg; t += blockDim.x) {
    cen[t] = (float)pc[(kDeg + 1) * kSeg + t];  // exact: a few significant bits
    ih[t] = (float)pc[(kDeg + 2) * kSeg + t];   // powers of two
  }
  return DfPlanck{c, ct, cen, ih};
}

// expm1(r) for |r| <= ln2/2: r + r^2 S(r), S = sum_k r^(k-2)/k!, the terms
// k >= 8 (below 5e-8 of S) in FP32, k = 2..7 with float-float coefficients.
__device__ __forceinline__ dflt expm1_small_df(dflt r) {
  float t = 0x1.612462p-33f;             // 1/13!
  t = fmaf(t, r.hi, 0x1.1eed8ep-29f);    // 1/12!
  t = fmaf(t, r.hi, 0x1.ae6456p-26f);    // 1/11!
  t = fmaf(t, r.hi, 0x1.27e4fcp-22f);    // 1/10!
  t = fmaf(t, r.hi, 0x1.71de3ap-19f);    // 1/9!
  t = fmaf(t, r.hi, 0x1.a01a02p-16f);    // 1/8!
  dflt S = {t, 0.0f};
  S = S * r + dflt{0x1.a01a02p-13f, -0x1.7f97fap-39f};   // 1/7!
  S = S * r + dflt{0x1.6c16c2p-10f, -0x1.27d27ep-35f};   // 1/6!
  S = S * r + dflt{0x1.111112p-7f, -0x1.dddddep-32f};    // 1/5!
  S = S * r + dflt{0x1.555556p-5f, -0x1.555556p-30f};    // 1/4!
  S = S * r + dflt{0x1.555556p-3f, -0x1.555556p-28f};    // 1/3!
  S = S * r + dflt{0x1p-1f, 0.0f};                       // 1/2!
  return r + (r * r) * S;
}

// Edge values at x (float-float): pq = P(x) (low, x < 2) or Q(x), d = D(x),
// ed = x dD/dx (FP32, for the Jacobian).
__device__ __forceinline__ void edge_df(const DfPlanck &T, dflt x, dflt &pq, dflt &d, float &ed,
                                        bool &low) {
  using namespace planck_table;
  low = !(x.hi > 0.0f);
  if (low || !(x.hi < 80.0f)) {
    pq = d = dflt{0.0f, 0.0f};
    ed = 0.0f;
    return;
  }
  low = x.hi < 2.0f;
  const dflt s = low ? x : -x;
  const float k = rintf(s.hi * kLog2e);
  const dflt r = ((s - k * kLn2a) - k * kLn2b) - two_prod(k, kLn2c);
  const dflt em = expm1_small_df(r);
  const float p2 = __int_as_float((127 + (int)k) << 23);  // 2^k, k in [-116, 3]
  const dflt ex = df_scale(em + 1.0f, p2);                  // e^s (e^-x on the Wien side)
  const dflt e1 = df_scale(em, p2) + (p2 - 1.0f);           // expm1(s)
  // x/(e^x - 1): x / expm1(x) below 2, x e^-x / (1 - e^-x) above
  const dflt B = (low ? x : x * ex) / (low ? e1 : 1.0f - ex);
  const int bits = __float_as_int(x.hi);
  const int e = ((bits >> 23) & 0xFF) - 127;
  int sg = 1 + (e - kEMin) * kSub + ((bits >> 21) & 3);
  sg = e < kEMin ? 0 : (e > kEMax ? kSeg - 1 : sg);
  const dflt u = df_scale(x - T.cen[sg], T.ih[sg]);
  float pt = T.ct[(kDeg - kDfDeg - 1) * kSeg + sg];
#pragma unroll
  for (int c = kDeg - 1; c > kDfDeg; --c) pt = fmaf(pt, u.hi, T.ct[(c - kDfDeg - 1) * kSeg + sg]);
  dflt p = {pt, 0.0f};
#pragma unroll
  for (int c = kDfDeg; c >= 0; --c) p = p * u + df_of(T.c[c * kSeg + sg]);
  const dflt kx3 = kPlanckNormDF * (x * x * x);
  pq = kx3 * (low ? p : p * ex);
  d = kx3 * B;
  ed = d.hi * (4.0f - B.hi - x.hi);
}

template <int L>
__device__ __forceinline__ dflt seg_sum_df(dflt v, unsigned mask) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) {
    const dflt w = {__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o)};
    v = v + w;  // float-float addition is commutative bit for bit: every lane gets the same sum
  }
  return v;
}

// Planck fraction of a band (band_fp64 in float-float).
__device__ __forceinline__ dflt band_df(dflt pqL, bool lowL, dflt pqU, bool lowU) {
  if (!lowL) return pqL - pqU;
  if (lowU) return pqU - pqL;
  return (1.0f - pqU) - pqL;
}

// The refinement step of cell i with L lanes (the layout of correct_cell).
template <int L, int GPL>
__device__ __forceinline__ void refine_cell(const KParams &P, const GroupTable &tab,
                                            const DfTable &dt, const DfPlanck &pl,
                                            const WarmOut &W, const CorrOut &U, float *gb,
                                            int64_t i, int lane) {
  constexpr int NE = GPL + 1;
  const int seg = lane / L, l = lane % L, lane0 = seg * L;
  const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << lane0);
  const int G = P.G;
  const int64_t n = P.n;
  const double c = P.c, tdt = P.c_hat * P.theta * P.dt;
  const int src_lane = lane0 + (l + 1) % L;
  const float crf = (float)P.cr;
  // ---- the cell, validated as the correction validates it
  const double Eint = W.eint[i];
  const double rho = P.rho[i];
  const double k0 = P.kappa0 ? P.kappa0[i] : 1.0;
  const double m0[3] = {P.mom[0][i], P.mom[1][i], P.mom[2][i]};
  const double eg0 = P.egas[i];
  bool valid = Eint > 0.0 && rho > 0.0 && isfinite(rho) && isfinite(eg0) && isfinite(k0) &&
               k0 >= 0.0 && isfinite(m0[0]) && isfinite(m0[1]) && isfinite(m0[2]);
  const double eint0 = eg0 - 0.5 * (m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2]) / rho;
  valid = valid && eint0 > 0.0;
  double E0[GPL], ft[GPL][3];
  float rw[GPL], fw[GPL][3];
  double sumE0 = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    E0[j] = 0.0;
    rw[j] = 0.0f;
    for (int d = 0; d < 3; ++d) {
      fw[j][d] = 0.0f;
      ft[j][d] = 0.0;
    }
    if (g < G && valid) {
      const int64_t o = (int64_t)g * P.gs + i;
      const double e = P.erad[o], sg = P.src ? P.src[o] : 0.0;
      E0[j] = e + sg;
      valid = valid && isfinite(e) && isfinite(sg);
      sumE0 += E0[j];
      const int64_t ow = (int64_t)g * n + i;
      rw[j] = W.r[ow];
      for (int d = 0; d < 3; ++d) {
        ft[j][d] = P.frad[d][o];
        valid = valid && isfinite(ft[j][d]);
        fw[j][d] = W.f[(int64_t)d * G * n + ow];
      }
    }
  }
  bool stepped = false;
  float x = 0.0f, u[GPL][4];
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    for (int t = 0; t < 4; ++t) u[j][t] = 0.0f;
  if (__all_sync(mask, valid)) {
    sumE0 = seg_sum<L>(sumE0, mask);
    const double Et = eg0 + P.cr * sumE0;
    // units: E_tot = mE 2^shE, c E_tot = mF 2^shF, rho c = mV 2^shV
    int shE, shF, shV;
    frexp_f(Et, shE);
    frexp_f(c * Et, shF);
    frexp_f(rho * c, shV);
    // 1 / mantissa of each, in float-float
    const dflt mEd = df_from_double(Et, shE);
    const dflt imE = df_rcp(mEd), imF = df_rcp(df_from_double(c * Et, shF)),
               imV = df_rcp(df_from_double(rho * c, shV));
    // the iterate's momentum (eq. vupdate) from its fluxes, in units of rho c
    dflt e0[GPL], ftd[GPL][3], sdf[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    dflt sr = {0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      e0[j] = df_from_double(E0[j], shE) * imE;
      sr = sr + rw[j];
      for (int d = 0; d < 3; ++d) {
        ftd[j][d] = df_from_double(ft[j][d], shF) * imF;
        sdf[d] = sdf[d] + (fw[j][d] - ftd[j][d]);
      }
    }
    sr = seg_sum_df<L>(sr, mask);
    for (int d = 0; d < 3; ++d) sdf[d] = seg_sum_df<L>(sdf[d], mask);
    const dflt mu = mEd / df_from_double(rho * c * P.c_hat, shE);  // E_tot / (rho c c_hat)
    dflt be[3], dbe[3], b0[3];
    for (int d = 0; d < 3; ++d) {
      b0[d] = df_from_double(m0[d], shV) * imV;
      dbe[d] = -(mu * sdf[d]);
      be[d] = b0[d] + dbe[d];
    }
    const dflt kE = df_from_double(rho * c * c, shE) * imE;  // rho c^2 / E_tot
    // F_G = E_int - E_int^t + (E_kin - E_kin^t) + (c/c_hat) sum_g R_g: the
    // kinetic energy enters through its change, (1/2) rho c^2 dbeta.(beta + beta^t),
    // so a cell whose gas energy is mostly kinetic loses nothing to cancellation
    const dflt dke = dbe[0] * (be[0] + b0[0]) + dbe[1] * (be[1] + b0[1]) + dbe[2] * (be[2] + b0[2]);
    const dflt FG = df_from_double(Eint - eint0, shE) * imE + df_scale(kE * dke, 0.5f) +
                    df_from_double(P.cr, 0) * sr;
    // T, the opacity scale and the edge terms, all in float-float
    double cs = rho * k0;
    if (P.temp_exp != 0.0) cs *= pow(Eint / (rho * P.c_v * P.T_ref), P.temp_exp);
    const dflt tcs = df_from_double(tdt * cs, 0), its = df_rcp(tcs);
    int et = 0;
    const float mt = tdt * cs > 0.0 ? frexp_f(tdt * cs, et) : 0.0f;
    const dflt T = df_from_double(Eint, 0) / df_from_double(rho * P.c_v, 0);
    const dflt invT = df_rcp(T);
    // a_R T^4 / E_tot as (T 2^-eT)^4 (a_R 2^(4 eT - shE)) / mE: both factors of
    // order one, so neither part of a_R's float-float leaves FP32's range
    const int eT = df_exponent(T.hi);
    const dflt Tm = df_scale(T, __int_as_float((127 - eT) << 23)), T2 = Tm * Tm;
    const dflt aT4 = (T2 * T2) * (df_from_double(P.a_rad, shE - 4 * eT) * imE);
    dflt pqD[NE], dD_[NE];
    float eF[NE];
    bool lowE[NE];
#pragma unroll
    for (int jj = 0; jj < NE; ++jj) {
      const int e = l + L * jj;
      const dflt x = e <= G ? df_of(dt.xe[e]) * invT : dflt{1.0f, 0.0f};
      edge_df(pl, x, pqD[jj], dD_[jj], eF[jj], lowE[jj]);
    }
    // ---- the residual, group by group (rhd_correct.cuh's rows in float-float)
    float rR[GPL], rF[GPL][3], Eg[GPL];
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const dflt pa = {__shfl_sync(mask, pqD[j].hi, src_lane), __shfl_sync(mask, pqD[j].lo, src_lane)};
      const dflt pb = {__shfl_sync(mask, pqD[j + 1].hi, src_lane),
                       __shfl_sync(mask, pqD[j + 1].lo, src_lane)};
      const dflt da = {__shfl_sync(mask, dD_[j].hi, src_lane), __shfl_sync(mask, dD_[j].lo, src_lane)};
      const dflt db_ = {__shfl_sync(mask, dD_[j + 1].hi, src_lane),
                        __shfl_sync(mask, dD_[j + 1].lo, src_lane)};
      const int la = __shfl_sync(mask, (int)lowE[j], src_lane),
                lb = __shfl_sync(mask, (int)lowE[j + 1], src_lane);
      const bool last = l == L - 1;
      const dflt pqU = last ? pb : pa, dU = last ? db_ : da;
      const bool lowU = (last ? lb : la) != 0;
      const int g = l + L * j;
      rR[j] = 0.0f;
      rF[j][0] = rF[j][1] = rF[j][2] = 0.0f;
      Eg[j] = 0.0f;
      if (g >= G) continue;
      const dflt dP = band_df(pqD[j], lowE[j], pqU, lowU);
      const dflt dD = dU - dD_[j];
      const dflt b = aT4 * dP;
      const dflt a = df_of(dt.alpha[g]), rm = df_of(dt.rm[g]), rp = df_of(dt.rp[g]);
      const dflt X = rp * dU - rm * dD_[j];
      // eq. chiDiff as chi_F / chi_E (held to the group's range of chi_0):
      // numerator and denominator both taken times 3
      // (a_R T^4 cancels: the ratio is formed from the edge values, scaled
      // so that Wien-tail groups, far below FP32's range, keep their ratio)
      const dflt den3 = df_scale(dP, 4.0f) - dD;
      const dflt num3 = (4.0f + a) * dP - X;
      const dflt qlo = df_min(rm, rp), qhi = df_max(rm, rp);
      dflt q = {1.0f, 0.0f};
      if (df_pos(den3)) {
        q = df_div_scaled(num3, den3);
        if (!isfinite(q.hi) || !isfinite(q.lo)) q = df_pos(num3) ? qhi : qlo;
      }
      q = df_max(df_min(q, qhi), qlo);
      const dflt tau = tcs * df_of(dt.kbar[g]);
      const dflt E = e0[j] + rw[j];
      Eg[j] = E.hi;
      const dflt w = be[0] * fw[j][0] + be[1] * fw[j][1] + be[2] * fw[j][2];  // v.F / c^2
      const dflt a1 = 1.0f + a;
      const dflt FR = df_pos(tau) ? b + a1 * q * w - (its * df_of(dt.ikbar[g])) * rw[j] - E
                                  : dflt{-rw[j], 0.0f};
      // the flux row F - (eq. numF1 at the iterate), closure in units c = 1:
      // v.P = ca v + kf F.  The closure depends on F / E only, so E, F and
      // v.F are first scaled by the power of two that brings E to order one
      // (squares of a Wien-tail group's values would leave FP32's range).
      dflt ca, kf;
      const bool fz = fw[j][0] == 0.0f && fw[j][1] == 0.0f && fw[j][2] == 0.0f;
      if (P.closure == RHD_M1 && df_pos(E) && !fz) {
        const int ex = df_exponent(E.hi);
        const int e1 = ex / 2, e2 = ex - e1;
        const float s1 = __int_as_float((127 - e1) << 23), s2 = __int_as_float((127 - e2) << 23);
        const dflt Es = df_scale(df_scale(E, s1), s2), ws = df_scale(df_scale(w, s1), s2);
        const float f0 = fw[j][0] * s1 * s2, f1 = fw[j][1] * s1 * s2, f2 = fw[j][2] * s1 * s2;
        const dflt fn2 = two_prod(f0, f0) + two_prod(f1, f1) + two_prod(f2, f2);
        const dflt E2 = Es * Es;
        if (fn2 < E2) {
          const dflt S = df_sqrt(df_scale(E2, 4.0f) - fn2 * 3.0f);
          ca = (S - Es) * kThirdDF;  // scaled back below
          kf = (ws * 3.0f) / (df_scale(Es, 2.0f) + S);
        } else {
          ca = dflt{0.0f, 0.0f};
          kf = (Es * ws) / fn2;
        }
        ca = df_scale(df_scale(ca, __int_as_float((127 + e1) << 23)), __int_as_float((127 + e2) << 23));
      } else {
        ca = E * kThirdDF;
        kf = dflt{0.0f, 0.0f};
      }
      const dflt srcg = tau * (b - aT4 * X * kThirdDF);
      const dflt inv = df_rcp(1.0f + tau * q);
      const dflt kap = tau * a1 * inv;
      for (int d = 0; d < 3; ++d) {
        const dflt vp = ca * be[d] + kf * fw[j][d];
        const dflt Fn = (ftd[j][d] + be[d] * srcg) * inv + kap * vp;
        rF[j][d] = (fw[j][d] - Fn).hi;
      }
      rR[j] = FR.hi;
    }
    // ---- the FP32 Jacobian and the step (rhd_correct.cuh's, at this residual)
    const float rG = FG.hi;
    const float eint = (df_from_double(Eint, shE) * imE).hi;
    const float aT4s = aT4.hi;
    const float dTs = aT4s / eint;
    const float bef[3] = {be[0].hi, be[1].hi, be[2].hi};
    const float mc[3] = {(be[0] * kE).hi, (be[1] * kE).hi, (be[2] * kE).hi};  // m c / E_tot
    bool ok = true;
    float sums[20];
    for (int t = 0; t < 20; ++t) sums[t] = 0.0f;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const float pa = __shfl_sync(mask, pqD[j].hi, src_lane),
                  pb = __shfl_sync(mask, pqD[j + 1].hi, src_lane);
      const float da = __shfl_sync(mask, dD_[j].hi, src_lane),
                  db_ = __shfl_sync(mask, dD_[j + 1].hi, src_lane);
      const float ea = __shfl_sync(mask, eF[j], src_lane), eb = __shfl_sync(mask, eF[j + 1], src_lane);
      const int la = __shfl_sync(mask, (int)lowE[j], src_lane),
                lb = __shfl_sync(mask, (int)lowE[j + 1], src_lane);
      const bool last = l == L - 1;
      const int g = l + L * j;
      if (g >= G) {
        for (int t = 0; t < 20; ++t) gb[(j * 20 + t) * 32 + lane] = 0.0f;
        continue;
      }
      const float tau = mt * scaled_f(tab.kbar[g], -et);
      GBlock blk;
      ok = group_jac32(P.closure, tau, tab.alphaf[g], tab.rmf[g], tab.rpf[g], pqD[j].hi, lowE[j],
                       dD_[j].hi, eF[j], last ? pb : pa, (last ? lb : la) != 0, last ? db_ : da,
                       last ? eb : ea, aT4s, dTs, Eg[j], fw[j], bef, rR[j], rF[j], blk) && ok;
      sums[0] += blk.p[0];
      sums[1] += blk.q[0];
      for (int t = 0; t < 3; ++t) {
        sums[2 + t] += blk.S[t];
        sums[5 + t] += blk.p[1 + t];
        sums[8 + t] += blk.q[1 + t];
        for (int c2 = 0; c2 < 3; ++c2) sums[11 + 3 * t + c2] += blk.S[3 * (1 + t) + c2];
      }
      for (int t = 0; t < 4; ++t) {
        gb[(j * 20 + t) * 32 + lane] = blk.p[t];
        gb[(j * 20 + 4 + t) * 32 + lane] = blk.q[t];
      }
      for (int t = 0; t < 12; ++t) gb[(j * 20 + 8 + t) * 32 + lane] = blk.S[t];
    }
#pragma unroll
    for (int t = 0; t < 20; ++t) sums[t] = seg_sumf<L>(sums[t], mask);
    float beta[3] = {0.0f, 0.0f, 0.0f};
    ok = global_solve(sums, rG, crf, mc, mu.hi, x, beta) && ok;
    // a small step that keeps the internal energy well positive
    ok = ok && fabsf(x) < kMaxStep && x > -0.5f * eint;
#pragma unroll
    for (int j = 0; j < GPL; ++j)
      for (int t = 0; t < 4; ++t) {
        u[j][t] = gb[(j * 20 + t) * 32 + lane] + gb[(j * 20 + 4 + t) * 32 + lane] * x +
                  gb[(j * 20 + 8 + 3 * t) * 32 + lane] * beta[0] +
                  gb[(j * 20 + 9 + 3 * t) * 32 + lane] * beta[1] +
                  gb[(j * 20 + 10 + 3 * t) * 32 + lane] * beta[2];
        ok = ok && fabsf(u[j][t]) < kMaxStep && (l + L * j < G || u[j][t] == 0.0f);
      }
    stepped = __all_sync(mask, ok);
    if (stepped && l == 0) {
      W.eint[i] = fma(f2d(x), Et, Eint);
      const int nit = W.nit[i] + 1;
      W.nit[i] = (uint8_t)(nit > 255 ? 255 : nit);
    }
  }
  // ---- the step from the FP32 iterate (zero where none was taken)
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    const int64_t o = (int64_t)g * n + i;
    U.ur[o] = stepped ? u[j][0] : 0.0f;
    for (int d = 0; d < 3; ++d) U.uf[(int64_t)d * G * n + o] = stepped ? u[j][1 + d] : 0.0f;
  }
  if (l == 0) {
    count_event(P, RHD_EV_RESIDDF, valid ? 1 : 0);
    count_event(P, RHD_EV_STEPDF, stepped ? 1 : 0);
  }
}

template <int L, int GPL>
__global__ void __launch_bounds__(128) refine_warp_kernel(const __grid_constant__ KParams P,
                                                          const WarmOut W, const CorrOut U) {
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  char *base = reinterpret_cast<char *>(sm) + ((table_bytes(P.G) + 15) & ~(size_t)15);
  const DfPlanck pl = build_df_planck(tab.pc, reinterpret_cast<float *>(base));
  float2 *dfs = reinterpret_cast<float2 *>(base + refine_planck_bytes());
  const DfTable dt = build_df_table(tab, dfs, P.G);  // synchronises (both tables)
  float *blocks = reinterpret_cast<float *>(dfs + 6 * P.G + 1);
  const int lane = threadIdx.x & 31, seg = lane / L;
  float *gb = warp_blocks<GPL>(blocks, threadIdx.x / 32);
  constexpr int CPW = 32 / L;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t i = warp * CPW + seg; i < P.n; i += nwarps * CPW)
    refine_cell<L, GPL>(P, tab, dt, pl, W, U, gb, i, lane);
}

}  // namespace rhd
