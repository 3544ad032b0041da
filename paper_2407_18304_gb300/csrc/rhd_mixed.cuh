// rhd_mixed.cuh -- the mixed-precision form of the per-cell update.
//
// Phase A runs the paper's inner/outer iteration (same steps as rhd_fp64.cuh)
// in FP32, on variables scaled by the cell's total energy E_tot so that FP32's
// range suffices: R~_g = R_g / E_tot, E~ = E / E_tot, f_g = F_g / (c E_tot),
// beta = v / c.  Only the quantities that cancel -- the internal energy
// E_int = E_gas - E_kin and the momentum -- stay in FP64.
// Phase B takes the phase-A iterate as the warm start of the FP64 outer loop
// (rhd_fp64.cuh): the residual of eq. FGFR and the Planck-integral differences
// are evaluated in FP64, the Newton correction is applied, the paper's
// convergence test is checked in FP64 at the caller's tolerance, and the
// conservative write-back, flux and momentum updates are FP64.
// The phases are two lane-persistent launches; phase A leaves its iterate in a
// workspace (WarmStart, rhd_fp64.cuh), so each launch keeps full warps on its
// own kind of arithmetic.
#pragma once
#include "rhd_fp64.cuh"

namespace rhd {

constexpr int kNB32 = 9;   // Bernoulli terms for FP32 (x < 2)
constexpr int kNQ32 = 10;  // exponential terms for FP32 (x >= 2)

__constant__ float c_bern_f[kNB32];
__constant__ float c_bern3_f[kNB32];
__constant__ float c_invn_f[kNQ32 + 1];

// FP32 edge values, same split and series as edge_fp64, cut at FP32 precision.
__device__ __forceinline__ void edge_fp32(float x, float &pq, float &d, float &ed, bool &low) {
  const float K = (float)kPlanckNorm;
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
  if (x < 2.0f) {
    const float z = x * x;
    float s1 = c_bern_f[kNB32 - 1], s3 = c_bern3_f[kNB32 - 1];
#pragma unroll
    for (int j = kNB32 - 2; j >= 0; --j) {
      s1 = fmaf(s1, z, c_bern_f[j]);
      s3 = fmaf(s3, z, c_bern3_f[j]);
    }
    const float x3 = z * x;
    const float xr = fmaf(z, s1, fmaf(-0.5f, x, 1.0f));
    pq = K * x3 * fmaf(z, s3, fmaf(-0.125f, x, 1.0f / 3.0f));
    d = K * x3 * xr;
    ed = d * (4.0f - xr - x);
    low = true;
  } else {
    const float e1 = __expf(-x);
    int nmax = (int)(18.5f / x) + 1;
    if (nmax > kNQ32) nmax = kNQ32;
    const float x2 = x * x, x3 = x2 * x, sx = 6.0f * x, tx2 = 3.0f * x2;
    float en = 1.0f, sum = 0.0f;
    for (int n = 1; n <= nmax; ++n) {
      en *= e1;
      const float inv = c_invn_f[n];
      float h = fmaf(6.0f, inv, sx);
      h = fmaf(h, inv, tx2);
      h = fmaf(h, inv, x3);
      sum = fmaf(en * inv, h, sum);
    }
    pq = K * sum;
    const float inv1 = __fdividef(1.0f, 1.0f - e1);
    d = K * x3 * x * e1 * inv1;
    ed = d * (4.0f - x * inv1);
    low = false;
  }
}

__device__ __forceinline__ float band_fp32(float pqL, bool lowL, float pqU, bool lowU) {
  if (!lowL) return pqL - pqU;
  if (lowU) return pqU - pqL;
  return (1.0f - pqU) - pqL;
}

template <int MAXG>
struct Arr32 {
  float R[MAXG], FR[MAXG], dg[MAXG], qe[MAXG], itau[MAXG], tau[MAXG], e0[MAXG], w[MAXG];
  float b[MAXG], dnx[MAXG], q[MAXG];
  float f[3 * MAXG], ft[3 * MAXG];
};

// FP32-phase scalars of one cell beyond Cell: the frozen scaled velocity.
struct Cell32 {
  float be[3];
  double sE;  // 1 / E_tot
};

// tau_g = c_hat theta dt chi_E,g, 1/tau_g and tau/(1+tau) for opacity scale cs.
template <int MAXG>
__device__ __forceinline__ void set_tau32(const KParams &P, const GroupTable &tab, Arr32<MAXG> &B,
                                          double cs) {
  const double tdt = P.c_hat * P.theta * P.dt;
  for (int g = 0; g < P.G; ++g) {
    const float t = (float)(tdt * cs * tab.kbar[g]);
    B.tau[g] = t;
    B.itau[g] = t > 0.0f ? 1.0f / t : 0.0f;
    B.qe[g] = t > 0.0f ? t / (1.0f + t) : 0.0f;
  }
}

// Load one cell into the FP32 phase (validation as in load_cell).
template <int MAXG>
__device__ __forceinline__ bool load_cell32(const KParams &P, const GroupTable &tab, int64_t i,
                                            Cell &C, Cell32 &D, Arr32<MAXG> &B) {
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
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    const double e = P.erad[o] + (P.src ? P.src[o] : 0.0);
    valid = valid && isfinite(e) && isfinite(P.frad[0][o]) && isfinite(P.frad[1][o]) &&
            isfinite(P.frad[2][o]);
    sumE0 += e;
  }
  if (!valid) return false;  // the FP64 launch writes the status
  C.chi0s = C.rho * k0;
  C.irho = 1.0 / C.rho;
  C.Etot = C.eg0 + P.cr * sumE0;
  C.rcv = C.rho * P.c_v;
  C.irc = 1.0 / C.rcv;
  C.m[0] = C.m0[0];
  C.m[1] = C.m0[1];
  C.m[2] = C.m0[2];
  C.Eint = C.eg0 - KE0;
  C.nit = 0;
  C.outer = 0;
  C.chg_prev = HUGE_VAL;
  C.slow = 0;
  D.sE = 1.0 / C.Etot;
  const double fs = D.sE / P.c;
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    B.e0[g] = (float)((P.erad[o] + (P.src ? P.src[o] : 0.0)) * D.sE);
    for (int d = 0; d < 3; ++d) {
      const float f = (float)(P.frad[d][o] * fs);
      B.f[3 * g + d] = f;
      B.ft[3 * g + d] = f;
    }
    B.R[g] = 0.0f;
  }
  set_tau32(P, tab, B, C.chi0s);
  return true;
}

template <int MAXG>
__device__ __forceinline__ void outer_begin32(const KParams &P, Cell &C, Cell32 &D,
                                              Arr32<MAXG> &B) {
  const double irc_ = C.irho * P.ic;  // 1/(rho c)
  C.KE = 0.5 * (C.m[0] * C.m[0] + C.m[1] * C.m[1] + C.m[2] * C.m[2]) * C.irho;
  for (int d = 0; d < 3; ++d) D.be[d] = (float)(C.m[d] * irc_);
  for (int g = 0; g < P.G; ++g)
    B.w[g] = D.be[0] * B.f[3 * g] + D.be[1] * B.f[3 * g + 1] + D.be[2] * B.f[3 * g + 2];
  C.it = 0;
}

// One FP32 inner iteration (same steps as inner_step, scaled variables);
// returns 0 (continue), 1 (converged at FP32 resolution) or 2 (cap).
template <int MAXG>
__device__ __forceinline__ int inner_step32(const KParams &P, const GroupTable &tab, Cell &C,
                                            Cell32 &D, Arr32<MAXG> &B) {
  const int G = P.G;
  const float cr = (float)P.cr;
  const double Etot = C.Etot, sE = D.sE;
  const float tol32 = 1e-7f;  // near FP32 resolution: the correction step then needs one Newton step
  const int max_it = P.max_newton < 32 ? P.max_newton : 32;
  const double T = C.Eint * C.irc;
  if (P.temp_exp != 0.0) set_tau32(P, tab, B, C.chi0s * pow(T / P.T_ref, P.temp_exp));
  const double aT3 = P.a_rad * T * T * T;
  const float aT4s = (float)(aT3 * T * sE);
  const float aT3s = (float)(aT3 * sE);
  const float kT = (float)(Etot * C.irc);  // dT / dE~_int
  const float invT = (float)(1.0 / T);
  float pqL, dL, eL;
  bool lowL;
  edge_fp32(tab.xef[0] * invT, pqL, dL, eL, lowL);
  float sumR = 0.0f, sFRe = 0.0f, sde = 0.0f, sabs = 0.0f;
  for (int g = 0; g < G; ++g) {
    float pqU, dU, eU;
    bool lowU;
    edge_fp32(tab.xef[g + 1] * invT, pqU, dU, eU, lowU);
    const float dP = band_fp32(pqL, lowL, pqU, lowU);
    const float dD = dU - dL;
    const float b = aT4s * dP;
    const float dbs = aT3s * (4.0f * dP - dD);  // d b~_g / dT
    const float a = tab.alphaf[g], rm = tab.rmf[g], rp = tab.rpf[g];
    float dq;
    const float q = chiF_ratio<float>(b, aT4s, dD, a, rm, rp, dL, dU, dbs, aT3s, eL, eU, dq);
    B.b[g] = b;
    B.dnx[g] = aT4s * (rp * dU - rm * dL);
    B.q[g] = q;
    const float ie = B.qe[g];
    float fr, d;
    if (ie > 0.0f) {
      const float Eg = b + (1.0f + a) * q * B.w[g] - B.R[g] * B.itau[g];
      fr = Eg - B.e0[g] - B.R[g];
      d = (dbs + (1.0f + a) * dq * B.w[g]) * kT;  // dF~_R,g / dE~_int
    } else {
      fr = -B.R[g];
      d = 0.0f;
    }
    const float iee = ie > 0.0f ? ie : 1.0f;
    B.FR[g] = fr;
    B.dg[g] = d;
    sumR += B.R[g];
    sFRe -= fr * iee;
    sde -= d * iee;
    sabs += fabsf(fr);
    pqL = pqU;
    dL = dU;
    eL = eU;
    lowL = lowU;
  }
  const float FG = (float)((C.Eint + C.KE - C.eg0) * sE) + cr * sumR;
  if (fabsf(FG) < tol32 && cr * sabs < tol32) return 1;
  if (C.it >= max_it) return 2;
  const float dE = (-FG + cr * sFRe) / (1.0f - cr * sde);
  double lam = 1.0;
  for (int k = 0; k < 40 && !(C.Eint + lam * (double)dE * Etot > 0.0); ++k) lam *= 0.5;
  C.Eint += lam * (double)dE * Etot;
  const float lf = (float)lam;
  for (int g = 0; g < G; ++g) {
    const float ie = B.qe[g] > 0.0f ? B.qe[g] : 1.0f;
    B.R[g] += lf * (B.FR[g] + B.dg[g] * dE) * ie;
  }
  ++C.nit;
  ++C.it;
  return fabsf(dE) < 1e-8f ? 1 : 0;  // a step below FP32 resolution of E_tot ends it
}

// FP32 write-back, flux update eq. numF1, momentum update and outer test;
// true when the phase is done for this cell.
template <int MAXG>
__device__ __forceinline__ bool outer_end32(const KParams &P, const GroupTable &tab, Cell &C,
                                            Cell32 &D, Arr32<MAXG> &B) {
  const int G = P.G;
  const double Etot = C.Etot, irc_ = C.irho * P.ic;
  const float cr = (float)P.cr;
  float sR = 0.0f;
  for (int g = 0; g < G; ++g) sR += B.R[g];
  const double egas_new = C.eg0 - (double)cr * (double)sR * Etot;
  float df[3] = {0.0f, 0.0f, 0.0f};
  const float bmag = sqrtf(D.be[0] * D.be[0] + D.be[1] * D.be[1] + D.be[2] * D.be[2]);
  for (int g = 0; g < G; ++g) {
    const float En = B.e0[g] + B.R[g];
    const float t = B.tau[g], a = tab.alphaf[g];
    const float srcg = t * (B.b[g] - B.dnx[g] * (1.0f / 3.0f));
    const float inv = 1.0f / (1.0f + t * B.q[g]);
    const float base[3] = {(B.ft[3 * g] + D.be[0] * srcg) * inv,
                           (B.ft[3 * g + 1] + D.be[1] * srcg) * inv,
                           (B.ft[3 * g + 2] + D.be[2] * srcg) * inv};
    const float kap = (1.0f + a) * t * inv;
    float F[3] = {B.f[3 * g], B.f[3 * g + 1], B.f[3 * g + 2]};
    flux_update<float>(P.closure, 1.0f, En, kap, base, D.be, bmag, F, 1e-6f, C.slow != 0);
    df[0] += F[0] - B.ft[3 * g];
    df[1] += F[1] - B.ft[3 * g + 1];
    df[2] += F[2] - B.ft[3 * g + 2];
    B.f[3 * g] = F[0];
    B.f[3 * g + 1] = F[1];
    B.f[3 * g + 2] = F[2];
  }
  const double mf = Etot * P.icc * P.c;  // E_tot / c_hat = (c E_tot)/(c c_hat)
  const double mn[3] = {C.m0[0] - mf * df[0], C.m0[1] - mf * df[1], C.m0[2] - mf * df[2]};
  const double KEn = 0.5 * (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) * C.irho;
  const float bn[3] = {(float)(mn[0] * irc_), (float)(mn[1] * irc_), (float)(mn[2] * irc_)};
  float chg = (float)(fabs(KEn - C.KE) * D.sE);
  for (int g = 0; g < G; ++g) {
    const float wn = bn[0] * B.f[3 * g] + bn[1] * B.f[3 * g + 1] + bn[2] * B.f[3 * g + 2];
    const float t = B.tau[g];
    chg += fabsf(t * (1.0f + tab.alphaf[g]) * B.q[g] * (wn - B.w[g])) / (1.0f + t);
  }
  C.m[0] = mn[0];
  C.m[1] = mn[1];
  C.m[2] = mn[2];
  if (C.outer >= 1 && chg > 0.25f * (float)C.chg_prev) C.slow = 1;  // as in outer_end
  C.chg_prev = chg;
  C.Eint = egas_new - KEn;  // start of the next pass (or of the FP64 phase)
  if (!(C.Eint > 0.0)) C.Eint = C.eg0 - C.KE;
  ++C.outer;
  if (chg <= 3e-8f || C.outer >= P.max_outer) return true;
  outer_begin32(P, C, D, B);
  return false;
}

// Workspace view of the warm start (writable side of WarmStart).
struct WarmOut {
  double *eint, *mom;
  float *r, *f;
  uint8_t *nit;
  float *ur, *uf;  // the correction step (rhd_correct.cuh)
  uint8_t *done;   // [n] cells the correction step finished
};

template <int MAXG>
__device__ __forceinline__ void store_warm(const KParams &P, const WarmOut &W, const Cell &C,
                                           const Arr32<MAXG> &B) {
  const int64_t i = C.i, n = P.n;
  W.eint[i] = C.Eint;
  W.mom[i] = C.m[0];
  W.mom[n + i] = C.m[1];
  W.mom[2 * n + i] = C.m[2];
  W.nit[i] = (uint8_t)(C.nit > 255 ? 255 : C.nit);
  for (int g = 0; g < P.G; ++g) {
    const int64_t o = (int64_t)g * n + i;
    W.r[o] = B.R[g];
    W.f[o] = B.f[3 * g];
    W.f[(int64_t)P.G * n + o] = B.f[3 * g + 1];
    W.f[(int64_t)2 * P.G * n + o] = B.f[3 * g + 2];
  }
}

// The FP32 passes of cells i, i + stride, ... < end, one cell per thread,
// lane-persistent: a thread takes its next cell as soon as its current one is
// stored, so the lanes of a warp stay busy while their cells take different
// iteration counts (every lane of the warp must call this).  S.r non-null:
// each cell starts from S (E_int and R_g / E_tot; a surrogate's guess)
// instead of the cold start.  S may alias W (each thread reads its cell's
// start before it writes that cell's result).
template <int MAXG>
__device__ __forceinline__ void fp32_cells(const KParams &P, const GroupTable &tab,
                                           const WarmOut &W, const WarmStart &S, int64_t i,
                                           int64_t end, int64_t stride) {
  Arr32<MAXG> B;
  Cell C;
  Cell32 D;
  unsigned ne = 0, no = 0;
  auto next = [&]() -> bool {
    ne = no = 0;
    while (i < end) {
      if (load_cell32(P, tab, i, C, D, B)) {
        if (S.r && S.eint[i] > 0.0) {
          C.Eint = S.eint[i];
          for (int g = 0; g < P.G; ++g) B.R[g] = S.r[(int64_t)g * P.n + i];
        }
        outer_begin32(P, C, D, B);
        return true;
      }
      i += stride;
    }
    return false;
  };
  bool active = next();
  while (__any_sync(0xffffffffu, active)) {
    if (active) {
      const int r = inner_step32(P, tab, C, D, B);
      ++ne;
      if (r != 0) ++no;
      if (r != 0 && outer_end32(P, tab, C, D, B)) {
        store_warm(P, W, C, B);
        count_event(P, RHD_EV_CELLS32, 1);
        count_event(P, RHD_EV_EVAL32, ne);
        count_event(P, RHD_EV_OUTER32, no);
        i += stride;
        active = next();
      }
    }
  }
}

// Phase A launch: the FP32 passes over the whole grid; writes the warm start.
template <int MAXG>
__global__ void __launch_bounds__(128) warm_fp32_kernel(const __grid_constant__ KParams P,
                                                        const WarmOut W, const WarmStart S) {
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  fp32_cells<MAXG>(P, tab, W, S, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, P.n,
                   (int64_t)gridDim.x * blockDim.x);
}

}  // namespace rhd
