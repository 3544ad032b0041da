// rhd_fp64.cuh -- the FP64 passes of the per-cell implicit source-term update.
//
// One thread owns one cell at a time.  The per-group arrays of a cell live in
// thread-local storage; loads of the state are coalesced because the cell
// index is the fastest index of every group array.  The algorithm is the
// paper's (Sec. 3):
//   outer pass k (v, F_g frozen at the k-th iterate):
//     inner Newton-Raphson over x = (E_gas, R_1..R_Ng):
//       residual F_G, F_R,g of eq. FGFR with R_g of eq. Rnew (c_hat/c factor
//       included), Jacobian entries after eq. linear (chi_B/chi_E = 1 here,
//       and the T-derivative of chi_F in the work term is kept),
//       arrowhead elimination of eq. matrix, convergence test after eq. matrix,
//       then each R_g from its own row at the converged T;
//     conservative write-back E_g = E_g^t + R_g + S_g,
//       E_gas = E_gas^t - (c/c_hat) sum_g R_g;
//     flux update eq. numF1 with the outdated velocity v_k, P_g from the
//       closure of (E_g^new, F_g^k);
//     momentum update (rho v) = (rho v)^t - (c c_hat)^-1 sum_g (F_g^new - F_g^t);
//     stop when the v,F-terms of R_g (and the kinetic energy, which sets T)
//     changed by less than tol_outer E_tot.
// The gas energy is carried as E_int = E_gas - E_kin (E_kin frozen within an
// inner solve, so the Newton steps in E_gas and E_int are the same).
//
// The steps are written as a per-lane state machine (outer_begin, inner_step,
// outer_end) so that a lane whose cell has converged takes its next cell while
// the other lanes of its warp keep iterating: every Newton evaluation then runs
// with (nearly) full warps, whatever the spread of iteration counts.
#pragma once
#include "rhd_common.cuh"

namespace rhd {

// eq. chiDiff as q = chi_F / chi_E, from b_g, (4pi/c)Delta_g(nu B_nu) = aT4 dD
// and the edge values; held to [min, max] of chi_0 / chi_E over the group.
// Also dq/dT (0 where held): with db = db_g/dT and the edge terms
// d(aT4 D)/dT = aT3 (4 D - x dD/dx) (eU, eL = x dD/dx at the edges).
template <typename R>
__device__ __forceinline__ R chiF_ratio(R b, R aT4, R dD, R a, R rm, R rp, R dL, R dU, R db,
                                        R aT3, R eL, R eU, R &dq) {
  const R X = rp * dU - rm * dL;
  const R den = R(4.0 / 3.0) * b - R(1.0 / 3.0) * aT4 * dD;
  R q = R(1);
  dq = R(0);
  if (den > R(0)) {
    const R iden = R(1) / den;
    q = (R(4.0 / 3.0) * b + R(1.0 / 3.0) * (a * b - aT4 * X)) * iden;
    const R dX = aT3 * (R(4) * X - (rp * eU - rm * eL));
    const R dnum = R(4.0 / 3.0) * db + R(1.0 / 3.0) * (a * db - dX);
    const R dden = R(4.0 / 3.0) * db - R(1.0 / 3.0) * aT3 * (R(4) * dD - (eU - eL));
    dq = (dnum - q * dden) * iden;
  }
  const R lo = fmin(rm, rp), hi = fmax(rm, rp);
  if (q < lo || q > hi) dq = R(0);
  return fmin(fmax(q, lo), hi);
}

// eq. chiDiff alone (no T-derivative), held as in chiF_ratio.
template <typename R>
__device__ __forceinline__ R chiF_q(R b, R aT4, R dD, R a, R rm, R rp, R dL, R dU) {
  const R X = rp * dU - rm * dL;
  const R den = R(4.0 / 3.0) * b - R(1.0 / 3.0) * aT4 * dD;
  R q = R(1);
  if (den > R(0)) q = (R(4.0 / 3.0) * b + R(1.0 / 3.0) * (a * b - aT4 * X)) / den;
  return fmin(fmax(q, fmin(rm, rp)), fmax(rm, rp));
}

// Per-cell constants and the FP64 iterate of one cell.
struct Cell {
  int64_t i;
  double rho, irho, m0[3], eg0, chi0s, Etot, rcv, irc;  // irho = 1/rho
  double m[3];     // momentum of the current outer iterate
  double v[3];     // its velocity (frozen during the inner solve)
  double KE;       // its kinetic energy (frozen during the inner solve)
  double Eint;     // internal energy of the current inner iterate
  double egas_new; // written-back total gas energy
  double cs;       // rho kappa0 (T/T_ref)^p of the last evaluation
  double its;      // 1 / (c_hat theta dt cs)
  double chg_prev; // outer-test change of the previous pass
  int nit, stat, it, outer;
  int slow;        // the outer iteration contracted slowly: Newton flux steps on
  int fresh;       // the last inner step converged: FR_g ~ 0 at the current T, R_g
  int cached;      // A.FR holds the residual at the current T, R_g (see inner_cached)
  int use_cache;   // take the cached first iteration of a pass (see outer_end)
  unsigned nfn;    // group flux updates solved by Newton steps
};

// Thread-local per-group arrays of the FP64 passes.
template <int MAXG>
struct Arr64 {
  double R[MAXG], w[MAXG], FR[MAXG], dg[MAXG], qe[MAXG];
  double bq[MAXG], dnx[MAXG], qF[MAXG];
  double Fk[3 * MAXG];
};

// Load and validate one cell (step a1); false = invalid (status written).
template <int MAXG>
__device__ __forceinline__ bool load_cell(const KParams &P, int64_t i, Cell &C, Arr64<MAXG> &A) {
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
  double sumE0 = 0.0, sumS = 0.0;
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    const double e = P.erad[o], s = P.src ? P.src[o] : 0.0;
    const double f0 = P.frad[0][o], f1 = P.frad[1][o], f2 = P.frad[2][o];
    valid = valid && isfinite(e) && isfinite(s) && isfinite(f0) && isfinite(f1) && isfinite(f2);
    sumE0 += e;
    sumS += s;
    A.Fk[3 * g] = f0;
    A.Fk[3 * g + 1] = f1;
    A.Fk[3 * g + 2] = f2;
    A.R[g] = 0.0;
  }
  if (!valid) {
    if (P.status) P.status[i] = RHD_STATUS_INVALID;
    if (P.iters) P.iters[i] = 0;
    return false;
  }
  C.chi0s = C.rho * k0;
  C.irho = 1.0 / C.rho;
  C.Etot = C.eg0 + (P.c / P.c_hat) * (sumE0 + sumS);  // energy at the start (reading: c/c_hat)
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
  C.use_cache = 0;  // set by the kernels that take the cached iteration
  return true;
}

// 1/tau_E and -1/e_g = tau_E/(1 + tau_E) per group for opacity scale cs.
// ikE: per-group 1/(chi_E / cs) of the cell (free slopes), else the table's.
template <int MAXG>
__device__ __forceinline__ void set_tau(const KParams &P, const GroupTable &tab, Cell &C,
                                        Arr64<MAXG> &A, double cs, const double *ikE = nullptr) {
  const double tdt = P.c_hat * P.theta * P.dt;
  C.cs = cs;
  C.its = (tdt * cs > 0.0) ? 1.0 / (tdt * cs) : 0.0;
  for (int g = 0; g < P.G; ++g) {
    const double it = C.its * (ikE ? ikE[g] : tab.ikbar[g]);  // 1/tau_E (0: uncoupled)
    A.qe[g] = it > 0.0 ? 1.0 / (1.0 + it) : 0.0;
  }
}

// a3: the terms frozen for one outer pass.
template <int MAXG>
__device__ __forceinline__ void outer_begin(const KParams &P, Cell &C, Arr64<MAXG> &A) {
  const double ir = C.irho, inv_c2 = P.inv_c2;
  C.KE = 0.5 * (C.m[0] * C.m[0] + C.m[1] * C.m[1] + C.m[2] * C.m[2]) * ir;
  C.v[0] = C.m[0] * ir;
  C.v[1] = C.m[1] * ir;
  C.v[2] = C.m[2] * ir;
  for (int g = 0; g < P.G; ++g)
    A.w[g] = (C.v[0] * A.Fk[3 * g] + C.v[1] * A.Fk[3 * g + 1] + C.v[2] * A.Fk[3 * g + 2]) * inv_c2;
  C.it = 0;
}

// a8 and the Newton step of a7, after the residual of every group is in
// A.FR/A.dg and its sums are taken: the convergence test (then each R_g from
// its own row, return 1), the iteration cap (return 2), or the arrowhead
// elimination of eq. matrix and the step (return 0).
template <int MAXG>
__device__ __forceinline__ int inner_tail(const KParams &P, Cell &C, Arr64<MAXG> &A, double sumR,
                                          double sFRe, double sde, double sabs) {
  const int G = P.G;
  const double cr = P.cr;
  const double FG = C.Eint + C.KE - C.eg0 + cr * sumR;
  // a8: convergence test
  if (fabs(FG) < P.tol * C.Etot && cr * sabs < P.tol * C.Etot) {
    // each R_g from its own row of eq. FGFR at the converged T (the arrowhead
    // rows with dE = 0): groups far below E_tot, which the aggregate test
    // cannot see, end consistent with T to round-off
    for (int g = 0; g < G; ++g)
      if (A.qe[g] > 0.0) A.R[g] += A.FR[g] * A.qe[g];
    C.fresh = 1;
    return 1;
  }
  C.fresh = 0;
  if (C.it >= P.max_newton) return 2;
  // a7: arrowhead elimination of eq. matrix: dE from the reduced first row,
  // then each dR_g from its own row
  const double dE = (-FG + cr * sFRe) / (1.0 - cr * sde);
  double lam = 1.0;
  for (int k = 0; k < 40 && !(C.Eint + lam * dE > 0.0); ++k) lam *= 0.5;
  C.Eint += lam * dE;
  for (int g = 0; g < G; ++g) {
    const double ie = A.qe[g] > 0.0 ? A.qe[g] : 1.0;
    A.R[g] += lam * (A.FR[g] + A.dg[g] * dE) * ie;
  }
  ++C.nit;
  ++C.it;
  return 0;
}

// The first inner iteration of an outer pass after a converged one.  T and
// R_g are still those of the last full evaluation, where each row of eq. FGFR
// was solved to round-off (R_g += FR_g qe_g), and the outer step changed only
// v (so E_kin) and F_g: the residual of row g is then exactly its v.F_g term,
// (1 + alpha) (chi_F/chi_E) (w_new - w_old), which outer_end left in A.FR,
// and b_g, chi_F, dF_R,g/dE_gas are unchanged.  The test and the Newton step
// are those of a full evaluation; the next evaluation is a full one at the
// stepped T.
template <int MAXG>
__device__ __forceinline__ int inner_cached(const KParams &P, Cell &C, Arr64<MAXG> &A) {
  C.cached = 0;
  double sumR = 0.0, sFRe = 0.0, sde = 0.0, sabs = 0.0;
  for (int g = 0; g < P.G; ++g) {
    const double fr = A.FR[g];
    const double iee = A.qe[g] > 0.0 ? A.qe[g] : 1.0;
    sumR += A.R[g];
    sFRe -= fr * iee;
    sde -= A.dg[g] * iee;
    sabs += fabs(fr);
  }
  return inner_tail(P, C, A, sumR, sFRe, sde, sabs);
}

// One inner Newton iteration (a4-a8): evaluate the residual at the current
// iterate; if the convergence test passes, set each R_g from its own row and
// return 1; at the iteration cap return 2; else take the Newton step, return 0.
template <int MAXG, bool CACHE = false>
__device__ __forceinline__ int inner_step(const KParams &P, const GroupTable &tab, Cell &C,
                                          Arr64<MAXG> &A) {
  if (CACHE && C.cached) return inner_cached(P, C, A);
  const int G = P.G;
  const int64_t i = C.i;
  const double T = C.Eint * C.irc;
  if (P.temp_exp != 0.0) set_tau(P, tab, C, A, C.chi0s * pow(T / P.T_ref, P.temp_exp));
  const double aT3 = P.a_rad * T * T * T, aT4 = aT3 * T;
  const double invT = 1.0 / T;
  double pqL, dL, eL;
  bool lowL;
  edge_tab(tab.pc, tab.xe[0] * invT, pqL, dL, eL, lowL);
  double sumR = 0.0, sFRe = 0.0, sde = 0.0, sabs = 0.0;
  for (int g = 0; g < G; ++g) {
    double pqU, dU, eU;
    bool lowU;
    edge_tab(tab.pc, tab.xe[g + 1] * invT, pqU, dU, eU, lowU);
    const int64_t o = (int64_t)g * P.gs + i;
    const double dP = band_fp64(pqL, lowL, pqU, lowU);
    const double dD = dU - dL;
    const double b = aT4 * dP;
    const double db = aT3 * (4.0 * dP - dD);  // d b_g / dT
    const double a = tab.alpha[g], rm = tab.rm[g], rp = tab.rp[g];
    // a5: chi_F; its T-derivative is left out of the Jacobian (the paper's
    // own simplification; the rate changes, not the root)
    const double q = chiF_q<double>(b, aT4, dD, a, rm, rp, dL, dU);
    A.bq[g] = b;
    A.dnx[g] = aT4 * (rp * dU - rm * dL);  // (4pi/c) Delta_g(nu chi_0 B_nu) / chi_E
    A.qF[g] = q;
    // a6: F_R,g of eq. FGFR, E_g(T, R_g) from eq. Rnew solved for E_g
    const double ie = A.qe[g];  // = -1/e_g
    double fr, d;
    if (ie > 0.0) {
      const double Eg = b + (1.0 + a) * q * A.w[g] - A.R[g] * C.its * tab.ikbar[g];
      const double s = P.src ? P.src[o] : 0.0;
      fr = Eg - P.erad[o] - A.R[g] - s;
      // a7: dF_R,g/dE_gas = (1/C_v) db_g/dT at fixed R_g (chi_B/chi_E = 1 in
      // PPL and PC)
      d = db * C.irc;
    } else {
      fr = -A.R[g];  // uncoupled group: R_g = 0
      d = 0.0;
    }
    const double iee = ie > 0.0 ? ie : 1.0;  // -1/e_g (e_g = -1 when uncoupled)
    A.FR[g] = fr;
    A.dg[g] = d;
    sumR += A.R[g];
    sFRe -= fr * iee;
    sde -= d * iee;
    sabs += fabs(fr);
    pqL = pqU;
    dL = dU;
    eL = eU;
    lowL = lowU;
  }
  return inner_tail(P, C, A, sumR, sFRe, sde, sabs);
}

// a9-a12 after an inner solve: write-back, flux and momentum update, outer
// test.  Returns true when the cell is done (converged or at a cap); else the
// next outer pass has been set up.
// The Newton part of flux_update for the groups whose eq. numF1 step
// contracts by less than 1/2 per outer pass (kE[g] = chi_E / cs; bq = chi_B
// b_g / chi_E).  Fk holds the eq. numF1 values
// and is updated; returns the change of their sum and its l1 size.  Out of
// line (few cells take it) with scalar and array arguments only, so that the
// caller's cell state stays in registers.
__device__ __noinline__ FluxDelta flux_newton_pass(
    int G, int64_t i, int64_t gs, const double *erad, const double *src, const double *ft0p,
    const double *ft1p, const double *ft2p, const double *kE, const double *alpha,
    const double *R, const double *bq, const double *dnx, const double *qF, double *Fk, double c,
    double tdt, double cs, double v0, double v1, double v2) {
  const double vmag = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  FluxDelta d = {0.0, 0.0, 0.0, 0.0, 0};
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * gs + i;
    const double chiE = cs * kE[g];
    const double inv = 1.0 / (1.0 + tdt * chiE * qF[g]);
    const double kap = tdt * (1.0 + alpha[g]) * chiE * inv;
    if (!(10.0 * fabs(kap) * vmag > c)) continue;
    ++d.n;
    const double s = src ? src[o] : 0.0;
    const double Enew = erad[o] + R[g] + s;
    const double srcg = chiE * (bq[g] - dnx[g] * (1.0 / 3.0));
    const Vec3<double> F = flux_newton<double>(
        c, Enew, kap, (ft0p[o] + tdt * v0 * srcg) * inv, (ft1p[o] + tdt * v1 * srcg) * inv,
        (ft2p[o] + tdt * v2 * srcg) * inv, v0, v1, v2, Fk[3 * g], Fk[3 * g + 1], Fk[3 * g + 2],
        1e-14);
    d.x += F.x - Fk[3 * g];
    d.y += F.y - Fk[3 * g + 1];
    d.z += F.z - Fk[3 * g + 2];
    d.l1 += fabs(F.x - Fk[3 * g]) + fabs(F.y - Fk[3 * g + 1]) + fabs(F.z - Fk[3 * g + 2]);
    Fk[3 * g] = F.x;
    Fk[3 * g + 1] = F.y;
    Fk[3 * g + 2] = F.z;
  }
  return d;
}

// kE: per-group chi_E / cs of the cell (free slopes), else the table's kbar.
template <int MAXG>
__device__ __forceinline__ bool outer_end(const KParams &P, const GroupTable &tab, Cell &C,
                                          Arr64<MAXG> &A, const double *kE = nullptr) {
  const double *kq = kE ? kE : tab.kbar;
  const int G = P.G;
  const int64_t i = C.i;
  const double c = P.c, chat = P.c_hat, cr = P.cr;
  const double tdt = chat * P.theta * P.dt;
  const double inv_c2 = P.inv_c2;
  const double icc = P.icc;
  const bool gtest = (P.flags & RHD_GROUP_TEST) != 0;

  // ---- a9: conservative energy write-back
  double sumR = 0.0;
  for (int g = 0; g < G; ++g) sumR += A.R[g];
  C.egas_new = C.eg0 - cr * sumR;

  // ---- a10: flux update, eq. fupdate (outdated velocity v_k): eq. numF1 for
  // every group, then flux_newton_pass where the closure's dependence on F
  // needs it (see flux_update)
  const double *v = C.v;
  const double v2c = 100.0 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);  // (10 |v|)^2
  const double c2 = c * c;
  double dF[3] = {0.0, 0.0, 0.0};
  double fchg = 0.0;  // sum_g |F_g,new - F_g,old|_1 (RHD_FLUX_TEST)
  bool newton = false;
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    const double s = P.src ? P.src[o] : 0.0;
    const double Enew = P.erad[o] + A.R[g] + s;
    const double chiE = C.cs * kq[g], a = tab.alpha[g];  // A.bq holds chi_B b_g / chi_E
    // v.P_g = ca v + (kn / kd) F_g; one reciprocal of (1 + c_hat theta dt chi_F) kd
    // gives both divisions
    double ca, kn, kd;
    closure_vP_parts<double>(P.closure, c, P.ic, Enew, A.Fk[3 * g], A.Fk[3 * g + 1],
                             A.Fk[3 * g + 2], v[0], v[1], v[2], ca, kn, kd);
    const double srcg = chiE * (A.bq[g] - A.dnx[g] * (1.0 / 3.0));
    const double den = 1.0 + tdt * chiE * A.qF[g];
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
    const double vp0 = ca * v[0] + kf * A.Fk[3 * g], vp1 = ca * v[1] + kf * A.Fk[3 * g + 1],
                 vp2 = ca * v[2] + kf * A.Fk[3 * g + 2];
    const double kap = tdt * (1.0 + a) * chiE * inv;
    newton = newton || kap * kap * v2c > c2;  // 10 |kap| |v| > c
    const double ft0 = P.frad[0][o], ft1 = P.frad[1][o], ft2 = P.frad[2][o];
    const double n0 = (ft0 + tdt * v[0] * srcg) * inv + kap * vp0;
    const double n1 = (ft1 + tdt * v[1] * srcg) * inv + kap * vp1;
    const double n2 = (ft2 + tdt * v[2] * srcg) * inv + kap * vp2;
    dF[0] += n0 - ft0;
    dF[1] += n1 - ft1;
    dF[2] += n2 - ft2;
    fchg += fabs(n0 - A.Fk[3 * g]) + fabs(n1 - A.Fk[3 * g + 1]) + fabs(n2 - A.Fk[3 * g + 2]);
    A.Fk[3 * g] = n0;
    A.Fk[3 * g + 1] = n1;
    A.Fk[3 * g + 2] = n2;
  }
  if (newton && C.slow && P.closure == RHD_M1) {
    const FluxDelta d =
        flux_newton_pass(G, i, P.gs, P.erad, P.src, P.frad[0], P.frad[1], P.frad[2], kq,
                         tab.alpha, A.R, A.bq, A.dnx, A.qF, A.Fk, c, tdt, C.cs, v[0], v[1], v[2]);
    dF[0] += d.x;
    dF[1] += d.y;
    dF[2] += d.z;
    fchg += d.l1;
    C.nfn += d.n;
  }
  // ---- a11: momentum update
  const double mn[3] = {C.m0[0] - dF[0] * icc, C.m0[1] - dF[1] * icc, C.m0[2] - dF[2] * icc};
  // ---- a12: outer test on the change of the v,F-terms of R_g, taken as their
  // effect on R_g after the implicit energy solve (divided by
  // 1 + c_hat theta dt chi_E), plus the change of the kinetic energy, which
  // moves T = (E_gas - E_kin)/(rho c_v) and with it every term of R_g
  const double ir = C.irho;
  const double vn[3] = {mn[0] * ir, mn[1] * ir, mn[2] * ir};
  const double KEn = 0.5 * (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) * ir;
  double chg = fabs(KEn - C.KE) + ((P.flags & RHD_FLUX_TEST) ? fchg / c : 0.0);
  bool gok = true;
  for (int g = 0; g < G; ++g) {
    const double wn =
        (vn[0] * A.Fk[3 * g] + vn[1] * A.Fk[3 * g + 1] + vn[2] * A.Fk[3 * g + 2]) * inv_c2;
    const double tauE = tdt * C.cs * kq[g];
    const double dvf = (1.0 + tab.alpha[g]) * A.qF[g] * (wn - A.w[g]);
    const double cg = fabs(tauE * dvf) / (1.0 + tauE);
    chg += cg;
    if (C.use_cache) A.FR[g] = A.qe[g] > 0.0 ? dvf : -A.R[g];  // residual at T, R_g, new w
    if (gtest) {
      const int64_t o = (int64_t)g * P.gs + i;
      const double s = P.src ? P.src[o] : 0.0;
      gok = gok && cg <= P.tol_outer * (fabs(P.erad[o]) + fabs(s) + fabs(P.erad[o] + A.R[g] + s));
    }
  }
  C.m[0] = mn[0];
  C.m[1] = mn[1];
  C.m[2] = mn[2];
  // a pass that removed less than 3/4 of the previous change turns the
  // Newton flux steps on for the rest of this cell's passes
  if (C.outer >= 1 && chg > 0.25 * C.chg_prev) C.slow = 1;
  C.chg_prev = chg;
  ++C.outer;
  if (chg <= P.tol_outer * C.Etot && gok) return true;
  if (C.outer >= P.max_outer) {
    C.stat = RHD_STATUS_MAXITER;
    return true;
  }
  if (C.fresh && C.use_cache) {
    // the next inner solve starts at this T and R_g, where its first
    // residual is known without evaluating the groups (inner_cached)
    outer_begin(P, C, A);
    C.cached = 1;
    return false;
  }
  // otherwise from the written-back gas energy
  C.Eint = C.egas_new - KEn;
  if (!(C.Eint > 0.0)) {
    C.stat = RHD_STATUS_MAXITER;
    return true;
  }
  outer_begin(P, C, A);
  return false;
}

// Store the cell (a13).
template <int MAXG>
__device__ __forceinline__ void store_cell(const KParams &P, const Cell &C, const Arr64<MAXG> &A) {
  const int64_t i = C.i;
  for (int g = 0; g < P.G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    const double s = P.src ? P.src[o] : 0.0;
    P.erad[o] = P.erad[o] + A.R[g] + s;
    P.frad[0][o] = A.Fk[3 * g];
    P.frad[1][o] = A.Fk[3 * g + 1];
    P.frad[2][o] = A.Fk[3 * g + 2];
  }
  P.egas[i] = C.egas_new;
  P.mom[0][i] = C.m[0];
  P.mom[1][i] = C.m[1];
  P.mom[2][i] = C.m[2];
  if (P.status) P.status[i] = (uint8_t)C.stat;
  if (P.iters) P.iters[i] = (uint8_t)(C.nit > 255 ? 255 : C.nit);
}

// The warm start a previous FP32 pass leaves in the workspace (see
// rhd_mixed.cuh); r == nullptr means a cold start (R_g = 0, E_gas = E_gas^t).
struct WarmStart {
  const double *eint;  // [n] internal energy
  const double *mom;   // [3][n] momentum
  const float *r;      // [G][n] R_g / E_tot
  const float *f;      // [3][G][n] F_g / (c E_tot)
  const uint8_t *nit;  // [n] FP32 Newton iterations
  int fallback;        // a cell whose warm-started solve fails is solved again from the cold start
  const float *ur;     // [G][n] correction step of R_g / E_tot (rhd_correct.cuh), or null
  const float *uf;     // [3][G][n] correction step of F_g / (c E_tot), or null
  const uint8_t *done; // [n] 1: the correction step finished the cell (skip it), or null
};

template <int MAXG>
__device__ __forceinline__ void apply_warm(const KParams &P, const WarmStart &W, Cell &C,
                                           Arr64<MAXG> &A) {
  const int64_t i = C.i, n = P.n;
  if (!(W.eint[i] > 0.0)) return;  // no usable guess: the cold start stays
  C.Eint = W.eint[i];
  C.m[0] = W.mom[i];
  C.m[1] = W.mom[n + i];
  C.m[2] = W.mom[2 * n + i];
  C.nit = W.nit[i];
  const double fs = P.c * C.Etot;
  for (int g = 0; g < P.G; ++g) {
    const int64_t o = (int64_t)g * n + i;
    if (W.ur) {  // the FP32 iterate plus the correction step, both exact in FP64
      A.R[g] = fma(f2d(W.r[o]), C.Etot, f2d(W.ur[o]) * C.Etot);
      for (int d = 0; d < 3; ++d) {
        const int64_t od = (int64_t)d * P.G * n + o;
        A.Fk[3 * g + d] = fma(f2d(W.f[od]), fs, f2d(W.uf[od]) * fs);
      }
      continue;
    }
    A.R[g] = (double)W.r[o] * C.Etot;
    A.Fk[3 * g] = (double)W.f[o] * fs;
    A.Fk[3 * g + 1] = (double)W.f[(int64_t)P.G * n + o] * fs;
    A.Fk[3 * g + 2] = (double)W.f[(int64_t)2 * P.G * n + o] * fs;
  }
}

// The FP64 passes of cell i, one cell per thread.  With a warm start (W.r)
// the first attempt starts from it; if that attempt does not converge and
// W.fallback is set, the cell is solved again from the cold start (status
// FALLBACK if that converges).  A cell the correction step finished (W.done)
// is skipped.  CACHE: take the cached first iteration of each outer pass.
template <int MAXG, bool CACHE = false>
__device__ __forceinline__ void fp64_cell(const KParams &P, const GroupTable &tab,
                                          const WarmStart &W, int64_t i, Cell &C,
                                          Arr64<MAXG> &A) {
  const bool warm = W.r != nullptr;
  if (W.done && W.done[i]) return;
  if (!load_cell(P, i, C, A)) return;
  C.use_cache = CACHE;
  C.nfn = 0;
  unsigned ne = 0, nc = 0, no = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    int nit0 = 0;
    if (attempt == 1) {
      if (!(warm && W.fallback && C.stat != RHD_STATUS_OK)) break;
      nit0 = C.nit;
      load_cell(P, i, C, A);
      C.use_cache = CACHE;
    }
    set_tau(P, tab, C, A, C.chi0s);
    if (warm && attempt == 0) apply_warm(P, W, C, A);
    outer_begin(P, C, A);
    for (;;) {
      if (CACHE && C.cached) ++nc;
      else ++ne;
      const int r = inner_step<MAXG, CACHE>(P, tab, C, A);
      if (r == 0) continue;
      if (r == 2) C.stat = RHD_STATUS_MAXITER;
      ++no;
      if (outer_end(P, tab, C, A)) break;
    }
    if (attempt == 1) {
      C.nit += nit0;
      if (C.stat == RHD_STATUS_OK) C.stat = RHD_STATUS_FALLBACK;
    }
  }
  store_cell(P, C, A);
  count_event(P, RHD_EV_CELLS64, 1);
  count_event(P, RHD_EV_EVAL64, ne);
  count_event(P, RHD_EV_CACHED64, nc);
  count_event(P, RHD_EV_OUTER64, no);
  count_event(P, RHD_EV_FLUXNEWTON, C.nfn);
}

// FP64 solve, one cell per thread: each thread walks the cells i, i + stride,
// ..., finishing each before the next.  The lanes of a warp hold different
// cells here, so a cached iteration on some lanes runs beside full
// evaluations on others and saves nothing (measured: +50 % time at 16 and 32
// groups, and the extra path costs registers); CACHE is instantiated for
// RHD_CELL_PER_THREAD, which runs the warp mapping's algorithm to count its
// operations.
template <int MAXG, bool CACHE = false>
__global__ void __launch_bounds__(128) solve_fp64_kernel(const __grid_constant__ KParams P,
                                                         const WarmStart W) {
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  Arr64<MAXG> A;
  Cell C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride)
    fp64_cell<MAXG, CACHE>(P, tab, W, i, C, A);
}

}  // namespace rhd
