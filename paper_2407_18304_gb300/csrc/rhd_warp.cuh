// rhd_warp.cuh -- the FP64 passes with the groups of a cell spread over lanes.
//
// L lanes (a whole warp, or an aligned segment of 16 or 8 lanes) solve one
// cell together: lane l owns the groups g = l + L j (j < GPL) and keeps all
// their per-group quantities in registers (including E_g^t + S_g, loaded once
// per cell; F_g^t is re-read from L2 by the outer step), evaluates the edges
// e = l + L j (j <= GPL) and gets
// the upper edge of each of its groups from the neighbouring lane by shuffle.
// The sums over groups of eq. matrix's elimination, of the write-back and of
// the momentum update are xor-butterflies inside the segment: every lane of
// the cell ends with the same bits, so every lane takes the same decisions.
// Iteration counts never split the lanes of a cell, which is what limits the
// one-cell-per-thread form (rhd_fp64.cuh) at large N_g.  The arithmetic of
// each step is that of rhd_fp64.cuh (same equations, same readings).
#pragma once
#include "rhd_fp64.cuh"

namespace rhd {

template <int L, int GPL>
struct WCell {
  int64_t i;
  double rho, irho, m0[3], eg0, chi0s, Etot, rcv, irc;
  double m[3], v[3], KE, Eint, egas_new, cs, its, chg_prev;
  int nit, stat, it, outer, slow;
  int fresh, cached;  // as Cell::fresh, Cell::cached
  unsigned nfn;       // group flux updates this lane solved by Newton steps
  double R[GPL], w[GPL], FR[GPL], dg[GPL], qe[GPL], bq[GPL], dnx[GPL], qF[GPL];
  double itau[GPL];   // 1/tau_E of the group (0 when uncoupled)
  double E0[GPL];     // E_g^t + S_g
  double Fk[GPL][3];  // flux of the current outer iterate (F^t is re-read from global memory)
};

template <int L>
__device__ __forceinline__ double seg_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Load and validate (a1); false = invalid (status written by lane 0).
template <int L, int GPL>
__device__ __forceinline__ bool wload(const KParams &P, int64_t i, int l, unsigned mask,
                                      WCell<L, GPL> &C) {
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
  double sumE0 = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    C.R[j] = 0.0;
    if (g < G) {
      const int64_t o = (int64_t)g * P.gs + i;
      const double e = P.erad[o], s = P.src ? P.src[o] : 0.0;
      const double f0 = P.frad[0][o], f1 = P.frad[1][o], f2 = P.frad[2][o];
      valid = valid && isfinite(e) && isfinite(s) && isfinite(f0) && isfinite(f1) && isfinite(f2);
      C.E0[j] = e + s;
      sumE0 += e + s;
      C.Fk[j][0] = f0;
      C.Fk[j][1] = f1;
      C.Fk[j][2] = f2;
    } else {
      C.E0[j] = 0.0;
      C.Fk[j][0] = C.Fk[j][1] = C.Fk[j][2] = 0.0;
    }
  }
  valid = __all_sync(mask, valid);
  if (!valid) {
    if (l == 0) {
      if (P.status) P.status[i] = RHD_STATUS_INVALID;
      if (P.iters) P.iters[i] = 0;
    }
    return false;
  }
  sumE0 = seg_sum<L>(sumE0, mask);
  C.chi0s = C.rho * k0;
  C.irho = 1.0 / C.rho;
  C.Etot = C.eg0 + (P.c / P.c_hat) * sumE0;
  C.rcv = C.rho * P.c_v;
  C.irc = 1.0 / C.rcv;
  C.m[0] = C.m0[0];
  C.m[1] = C.m0[1];
  C.m[2] = C.m0[2];
  C.Eint = C.eg0 - KE0;
  C.egas_new = C.eg0;
  C.cs = C.chi0s;
  C.nit = 0;
  C.stat = RHD_STATUS_OK;
  C.outer = 0;
  C.it = 0;
  C.chg_prev = HUGE_VAL;
  C.slow = 0;
  C.fresh = 0;
  C.cached = 0;
  return true;
}

template <int L, int GPL>
__device__ __forceinline__ void wset_tau(const KParams &P, const GroupTable &tab, int l,
                                         WCell<L, GPL> &C, double cs) {
  const double tdt = P.c_hat * P.theta * P.dt;
  C.cs = cs;
  C.its = (tdt * cs > 0.0) ? 1.0 / (tdt * cs) : 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    const double it = g < P.G ? C.its * tab.ikbar[g] : 0.0;
    C.itau[j] = it;
    C.qe[j] = it > 0.0 ? 1.0 / (1.0 + it) : 0.0;
  }
}

template <int L, int GPL>
__device__ __forceinline__ void wapply_warm(const KParams &P, const WarmStart &W, int l,
                                            WCell<L, GPL> &C) {
  const int64_t i = C.i, n = P.n;
  if (!(W.eint[i] > 0.0)) return;
  C.Eint = W.eint[i];
  C.m[0] = W.mom[i];
  C.m[1] = W.mom[n + i];
  C.m[2] = W.mom[2 * n + i];
  C.nit = W.nit[i];
  const double fs = P.c * C.Etot;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= P.G) continue;
    const int64_t o = (int64_t)g * n + i;
    if (W.ur) {  // the FP32 iterate plus the correction step, both exact in FP64
      C.R[j] = fma(f2d(W.r[o]), C.Etot, f2d(W.ur[o]) * C.Etot);
      for (int d = 0; d < 3; ++d) {
        const int64_t od = (int64_t)d * P.G * n + o;
        C.Fk[j][d] = fma(f2d(W.f[od]), fs, f2d(W.uf[od]) * fs);
      }
      continue;
    }
    C.R[j] = (double)W.r[o] * C.Etot;
    C.Fk[j][0] = (double)W.f[o] * fs;
    C.Fk[j][1] = (double)W.f[(int64_t)P.G * n + o] * fs;
    C.Fk[j][2] = (double)W.f[(int64_t)2 * P.G * n + o] * fs;
  }
}

template <int L, int GPL>
__device__ __forceinline__ void wouter_begin(const KParams &P, WCell<L, GPL> &C) {
  const double ir = C.irho, inv_c2 = P.inv_c2;
  C.KE = 0.5 * (C.m[0] * C.m[0] + C.m[1] * C.m[1] + C.m[2] * C.m[2]) * ir;
  C.v[0] = C.m[0] * ir;
  C.v[1] = C.m[1] * ir;
  C.v[2] = C.m[2] * ir;
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    C.w[j] = (C.v[0] * C.Fk[j][0] + C.v[1] * C.Fk[j][1] + C.v[2] * C.Fk[j][2]) * inv_c2;
  C.it = 0;
}

// The sums over the cell's groups, the convergence test and the Newton step
// of an inner iteration (as inner_tail; the per-lane partial sums in).
template <int L, int GPL>
__device__ __forceinline__ int wtail(const KParams &P, unsigned mask, WCell<L, GPL> &C,
                                     double sumR, double sFRe, double sde, double sabs) {
  const double cr = P.cr;
  // the test's two sums first: the step's two are only needed when it fails
  // (most full evaluations of a warm-started pass end converged)
  sumR = seg_sum<L>(sumR, mask);
  sabs = seg_sum<L>(sabs, mask);
  const double FG = C.Eint + C.KE - C.eg0 + cr * sumR;
  if (fabs(FG) < P.tol * C.Etot && cr * sabs < P.tol * C.Etot) {
#pragma unroll
    for (int j = 0; j < GPL; ++j)
      if (C.qe[j] > 0.0) C.R[j] += C.FR[j] * C.qe[j];
    C.fresh = 1;
    return 1;
  }
  C.fresh = 0;
  if (C.it >= P.max_newton) return 2;
  sFRe = seg_sum<L>(sFRe, mask);
  sde = seg_sum<L>(sde, mask);
  const double dE = (-FG + cr * sFRe) / (1.0 - cr * sde);
  double lam = 1.0;
  for (int k = 0; k < 40 && !(C.Eint + lam * dE > 0.0); ++k) lam *= 0.5;
  C.Eint += lam * dE;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const double ie = C.qe[j] > 0.0 ? C.qe[j] : 1.0;
    C.R[j] += lam * (C.FR[j] + C.dg[j] * dE) * ie;
  }
  ++C.nit;
  ++C.it;
  return 0;
}

// The first inner iteration of an outer pass after a converged one (as
// inner_cached): C.FR holds the v.F-term change that wouter_end left there.
template <int L, int GPL>
__device__ __forceinline__ int winner_cached(const KParams &P, int l, unsigned mask,
                                             WCell<L, GPL> &C) {
  C.cached = 0;
  double sumR = 0.0, sFRe = 0.0, sde = 0.0, sabs = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    if (l + L * j >= P.G) continue;
    const double fr = C.FR[j];
    const double iee = C.qe[j] > 0.0 ? C.qe[j] : 1.0;
    sumR += C.R[j];
    sFRe -= fr * iee;
    sde -= C.dg[j] * iee;
    sabs += fabs(fr);
  }
  return wtail(P, mask, C, sumR, sFRe, sde, sabs);
}

// One inner Newton iteration (a4-a8), as inner_step.
template <int L, int GPL>
__device__ __forceinline__ int winner_step(const KParams &P, const GroupTable &tab, int l,
                                           int lane0, unsigned mask, WCell<L, GPL> &C) {
  if (C.cached) return winner_cached(P, l, mask, C);
  constexpr int NE = GPL + 1;
  const int G = P.G;
  const double T = C.Eint * C.irc;
  if (P.temp_exp != 0.0) wset_tau(P, tab, l, C, C.chi0s * pow(T / P.T_ref, P.temp_exp));
  const double aT3 = P.a_rad * T * T * T, aT4 = aT3 * T;
  const double invT = 1.0 / T;
  // a4: the edges e = l + L jj.  When the groups fill the lanes exactly the
  // last slot holds only the top edge x_G (lane 0); x_G is the same for all
  // lanes of the cell, and for 40 <= x_G < inf the n >= 2 terms of Q and the
  // 1/(1 - e^-x) factor of D are below e^-40 = 4e-18 relative, so that slot
  // takes the short exact forms Q = 15/pi^4 e^-x (x^3 + 3x^2 + 6x + 6),
  // D = 15/pi^4 x^4 e^-x, x D' = D (4 - x) without splitting the lanes.
  double pqE[NE], dE_[NE], eE[NE];  // eE (x D') is not needed without dchi_F/dT
  bool lowE[NE];
#pragma unroll
  for (int jj = 0; jj < NE; ++jj) {
    const int e = l + L * jj;
    if (jj == NE - 1 && G == L * GPL) {
      const double xg = tab.xe[G] * invT;
      if (xg >= 40.0 && xg < HUGE_VAL) {
        const double em = exp(-xg);
        const double x2 = xg * xg;
        pqE[jj] = kPlanckNorm * em * (x2 * xg + 3.0 * x2 + 6.0 * xg + 6.0);
        dE_[jj] = kPlanckNorm * em * x2 * x2;
        eE[jj] = dE_[jj] * (4.0 - xg);
        lowE[jj] = false;
        continue;
      }
    }
    edge_tab(tab.pc, e <= G ? tab.xe[e] * invT : 1.0, pqE[jj], dE_[jj], eE[jj], lowE[jj]);
  }
  double sumR = 0.0, sFRe = 0.0, sde = 0.0, sabs = 0.0;
  const int src_lane = lane0 + (l + 1) % L;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    // upper edge g + 1 = (l + 1) + L j: lane l + 1, slot j; for l = L - 1 lane 0, slot j + 1
    const double pa = __shfl_sync(mask, pqE[j], src_lane), pb = __shfl_sync(mask, pqE[j + 1], src_lane);
    const double da = __shfl_sync(mask, dE_[j], src_lane), db_ = __shfl_sync(mask, dE_[j + 1], src_lane);
    const int la = __shfl_sync(mask, (int)lowE[j], src_lane),
              lb = __shfl_sync(mask, (int)lowE[j + 1], src_lane);
    const bool last = l == L - 1;
    const double pqU = last ? pb : pa, dU = last ? db_ : da;
    const bool lowU = (last ? lb : la) != 0;
    const int g = l + L * j;
    if (g >= G) {  // a slot past the last group: no residual, no update
      C.FR[j] = 0.0;
      C.dg[j] = 0.0;
      continue;
    }
    const double pqL = pqE[j], dL = dE_[j];
    const bool lowL = lowE[j];
    const double dP = band_fp64(pqL, lowL, pqU, lowU);
    const double dD = dU - dL;
    const double b = aT4 * dP;
    const double db = aT3 * (4.0 * dP - dD);
    const double a = tab.alpha[g], rm = tab.rm[g], rp = tab.rp[g];
    // a5: chi_F; its T-derivative is left out of the Jacobian (the paper's
    // own simplification: the rate changes, not the root; measured on the
    // 64-group workload: +0.2 % iterations, -5 % time)
    const double q = chiF_q<double>(b, aT4, dD, a, rm, rp, dL, dU);
    C.bq[j] = b;
    C.dnx[j] = aT4 * (rp * dU - rm * dL);
    C.qF[j] = q;
    const double ie = C.qe[j];
    double fr, d;
    if (ie > 0.0) {
      const double Eg = b + (1.0 + a) * q * C.w[j] - C.R[j] * C.itau[j];
      fr = Eg - C.E0[j] - C.R[j];
      d = db * C.irc;
    } else {
      fr = -C.R[j];
      d = 0.0;
    }
    const double iee = ie > 0.0 ? ie : 1.0;
    C.FR[j] = fr;
    C.dg[j] = d;
    sumR += C.R[j];
    sFRe -= fr * iee;
    sde -= d * iee;
    sabs += fabs(fr);
  }
  return wtail(P, mask, C, sumR, sFRe, sde, sabs);
}

// a9-a12, as outer_end.
template <int L, int GPL>
__device__ __forceinline__ bool wouter_end(const KParams &P, const GroupTable &tab, int l,
                                           unsigned mask, WCell<L, GPL> &C) {
  const int G = P.G;
  const double c = P.c, chat = P.c_hat, cr = P.cr;
  const double tdt = chat * P.theta * P.dt;
  const double inv_c2 = P.inv_c2;
  const double icc = P.icc;
  const bool gtest = (P.flags & RHD_GROUP_TEST) != 0;

  double sumR = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j)
    if (l + L * j < G) sumR += C.R[j];
  sumR = seg_sum<L>(sumR, mask);
  C.egas_new = C.eg0 - cr * sumR;

  const double *v = C.v;
  const double v2c = 100.0 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);  // (10 |v|)^2
  const double c2 = c * c;
  double dF[3] = {0.0, 0.0, 0.0};
  double fchg = 0.0;
  bool newton = false;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    const double Enew = C.E0[j] + C.R[j];
    const double chiB = C.cs * tab.kbar[g], a = tab.alpha[g];
    const int64_t o = (int64_t)g * P.gs + C.i;
    const double ft[3] = {P.frad[0][o], P.frad[1][o], P.frad[2][o]};
    // v.P_g = ca v + (kn / kd) F_g; one reciprocal of (1 + c_hat theta dt chi_F) kd
    // gives both divisions
    double ca, kn, kd;
    closure_vP_parts<double>(P.closure, c, P.ic, Enew, C.Fk[j][0], C.Fk[j][1], C.Fk[j][2], v[0],
                             v[1], v[2], ca, kn, kd);
    const double srcg = chiB * (C.bq[j] - C.dnx[j] * (1.0 / 3.0));
    const double den = 1.0 + tdt * chiB * C.qF[j];
    const double dk = den * kd;
    double inv, kf;
    if (dk > 1e-290) {  // one reciprocal (kd is tiny only for a nearly empty group)
      const double rr = 1.0 / dk;
      inv = kd * rr;
      kf = kn * den * rr;
    } else {
      inv = 1.0 / den;
      kf = kn / kd;
    }
    const double vp0 = ca * v[0] + kf * C.Fk[j][0], vp1 = ca * v[1] + kf * C.Fk[j][1],
                 vp2 = ca * v[2] + kf * C.Fk[j][2];
    const double kap = tdt * (1.0 + a) * chiB * inv;
    newton = newton || kap * kap * v2c > c2;  // 10 |kap| |v| > c
    const double n0 = (ft[0] + tdt * v[0] * srcg) * inv + kap * vp0;
    const double n1 = (ft[1] + tdt * v[1] * srcg) * inv + kap * vp1;
    const double n2 = (ft[2] + tdt * v[2] * srcg) * inv + kap * vp2;
    dF[0] += n0 - ft[0];
    dF[1] += n1 - ft[1];
    dF[2] += n2 - ft[2];
    fchg += fabs(n0 - C.Fk[j][0]) + fabs(n1 - C.Fk[j][1]) + fabs(n2 - C.Fk[j][2]);
    C.Fk[j][0] = n0;
    C.Fk[j][1] = n1;
    C.Fk[j][2] = n2;
  }
  // Newton flux steps (flux_update) where the cell contracts slowly
  if (C.slow && P.closure == RHD_M1 && __any_sync(mask, newton)) {
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const int g = l + L * j;
      if (g >= G) continue;
      const double chiB = C.cs * tab.kbar[g];
      const double inv = 1.0 / (1.0 + tdt * chiB * C.qF[j]);
      const double kap = tdt * (1.0 + tab.alpha[g]) * chiB * inv;
      if (!(kap * kap * v2c > c2)) continue;
      const double srcg = chiB * (C.bq[j] - C.dnx[j] * (1.0 / 3.0));
      const int64_t o = (int64_t)g * P.gs + C.i;
      ++C.nfn;
      const Vec3<double> F = flux_newton<double>(
          c, C.E0[j] + C.R[j], kap, (P.frad[0][o] + tdt * v[0] * srcg) * inv,
          (P.frad[1][o] + tdt * v[1] * srcg) * inv, (P.frad[2][o] + tdt * v[2] * srcg) * inv, v[0],
          v[1], v[2], C.Fk[j][0], C.Fk[j][1], C.Fk[j][2], 1e-14);
      dF[0] += F.x - C.Fk[j][0];
      dF[1] += F.y - C.Fk[j][1];
      dF[2] += F.z - C.Fk[j][2];
      fchg += fabs(F.x - C.Fk[j][0]) + fabs(F.y - C.Fk[j][1]) + fabs(F.z - C.Fk[j][2]);
      C.Fk[j][0] = F.x;
      C.Fk[j][1] = F.y;
      C.Fk[j][2] = F.z;
    }
  }
  dF[0] = seg_sum<L>(dF[0], mask);
  dF[1] = seg_sum<L>(dF[1], mask);
  dF[2] = seg_sum<L>(dF[2], mask);
  const double mn[3] = {C.m0[0] - dF[0] * icc, C.m0[1] - dF[1] * icc, C.m0[2] - dF[2] * icc};
  const double ir = C.irho;
  const double vn[3] = {mn[0] * ir, mn[1] * ir, mn[2] * ir};
  const double KEn = 0.5 * (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) * ir;
  double cg_sum = 0.0;
  bool gok = true;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    const double wn = (vn[0] * C.Fk[j][0] + vn[1] * C.Fk[j][1] + vn[2] * C.Fk[j][2]) * inv_c2;
    // tau_E / (1 + tau_E) = qe (0 for an uncoupled group, whose term is 0)
    const double dvf = (1.0 + tab.alpha[g]) * C.qF[j] * (wn - C.w[j]);
    const double cg = fabs(dvf) * C.qe[j];
    C.FR[j] = C.qe[j] > 0.0 ? dvf : -C.R[j];  // the residual at T, R_g for the new w
    cg_sum += cg;
    if (gtest) {
      const double e0 = C.E0[j];  // E^t + S (the group's own energy scale)
      gok = gok && cg <= P.tol_outer * (fabs(e0) + fabs(e0 + C.R[j]));
    }
  }
  cg_sum = seg_sum<L>(cg_sum, mask);
  double chg = fabs(KEn - C.KE) + cg_sum;
  if (P.flags & RHD_FLUX_TEST) chg += seg_sum<L>(fchg, mask) / c;
  gok = __all_sync(mask, gok);
  C.m[0] = mn[0];
  C.m[1] = mn[1];
  C.m[2] = mn[2];
  if (C.outer >= 1 && chg > 0.25 * C.chg_prev) C.slow = 1;
  C.chg_prev = chg;
  ++C.outer;
  if (chg <= P.tol_outer * C.Etot && gok) return true;
  if (C.outer >= P.max_outer) {
    C.stat = RHD_STATUS_MAXITER;
    return true;
  }
  if (C.fresh) {  // next pass starts at this T, R_g with a known residual
    wouter_begin(P, C);
    C.cached = 1;
    return false;
  }
  C.Eint = C.egas_new - KEn;
  if (!(C.Eint > 0.0)) {
    C.stat = RHD_STATUS_MAXITER;
    return true;
  }
  wouter_begin(P, C);
  return false;
}

template <int L, int GPL>
__device__ __forceinline__ void wstore(const KParams &P, int l, const WCell<L, GPL> &C) {
  const int64_t i = C.i;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= P.G) continue;
    const int64_t o = (int64_t)g * P.gs + i;
    P.erad[o] = C.E0[j] + C.R[j];
    P.frad[0][o] = C.Fk[j][0];
    P.frad[1][o] = C.Fk[j][1];
    P.frad[2][o] = C.Fk[j][2];
  }
  if (l == 0) {
    P.egas[i] = C.egas_new;
    P.mom[0][i] = C.m[0];
    P.mom[1][i] = C.m[1];
    P.mom[2][i] = C.m[2];
    if (P.status) P.status[i] = (uint8_t)C.stat;
    if (P.iters) P.iters[i] = (uint8_t)(C.nit > 255 ? 255 : C.nit);
  }
}

// The FP64 passes of one cell with L lanes (lane l of the cell's segment,
// mask its lanes): from the warm start in W where W.r is set (skipping a cell
// the correction step finished), with the cold restart on failure.
template <int L, int GPL>
__device__ __forceinline__ void warp_cell(const KParams &P, const GroupTable &tab,
                                          const WarmStart &W, int64_t i, int l, int lane0,
                                          unsigned mask, WCell<L, GPL> &C) {
  const bool warm = W.r != nullptr;
  if (W.done && W.done[i]) return;
  if (!wload(P, i, l, mask, C)) return;
  unsigned ne = 0, nc = 0, no = 0;
  C.nfn = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    int nit0 = 0;
    if (attempt == 1) {
      if (!(warm && W.fallback && C.stat != RHD_STATUS_OK)) break;
      nit0 = C.nit;
      wload(P, i, l, mask, C);
    }
    wset_tau(P, tab, l, C, C.chi0s);
    if (warm && attempt == 0) wapply_warm(P, W, l, C);
    wouter_begin(P, C);
    for (;;) {
      if (C.cached) ++nc;
      else ++ne;
      const int r = winner_step(P, tab, l, lane0, mask, C);
      if (r == 0) continue;
      if (r == 2) C.stat = RHD_STATUS_MAXITER;
      ++no;
      if (wouter_end(P, tab, l, mask, C)) break;
    }
    if (attempt == 1) {
      C.nit += nit0;
      if (C.stat == RHD_STATUS_OK) C.stat = RHD_STATUS_FALLBACK;
    }
  }
  wstore(P, l, C);
  if (P.count) {
    const unsigned nfn = __reduce_add_sync(mask, C.nfn);
    if (l == 0) {
      count_event(P, RHD_EV_CELLS64, 1);
      count_event(P, RHD_EV_EVAL64, ne);
      count_event(P, RHD_EV_CACHED64, nc);
      count_event(P, RHD_EV_OUTER64, no);
      count_event(P, RHD_EV_FLUXNEWTON, nfn);
    }
  }
}

// FP64 solve with L lanes per cell (32 / L cells per warp); warm start and
// cold restart as solve_fp64_kernel.
template <int L, int GPL>
__global__ void __launch_bounds__(128) solve_warp_kernel(const __grid_constant__ KParams P,
                                                         const WarmStart W) {
  static_assert(L == 8 || L == 16 || L == 32, "lanes per cell");
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  const int lane = threadIdx.x & 31, seg = lane / L, l = lane % L, lane0 = seg * L;
  const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << lane0);
  constexpr int CPW = 32 / L;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  WCell<L, GPL> C;
  for (int64_t i = warp * CPW + seg; i < P.n; i += nwarps * CPW)
    warp_cell<L, GPL>(P, tab, W, i, l, lane0, mask, C);
}

}  // namespace rhd
