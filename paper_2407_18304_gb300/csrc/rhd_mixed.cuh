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
// conservative write-back, flux and momentum updates are FP64.  Phase B usually
// needs one correction and one confirming evaluation.
#pragma once
#include "rhd_fp64.cuh"

namespace rhd {

constexpr int kNB32 = 9;   // Bernoulli terms for FP32 (x < 2)
constexpr int kNQ32 = 10;  // exponential terms for FP32 (x >= 2)

__constant__ float c_bern_f[kNB32];
__constant__ float c_bern3_f[kNB32];
__constant__ float c_invn_f[kNQ32 + 1];

// FP32 edge values, same split and series as edge_fp64, cut at FP32 precision.
__device__ __forceinline__ void edge_fp32(float x, float &pq, float &d, bool &low) {
  const float K = (float)kPlanckNorm;
  if (!(x > 0.0f)) {
    pq = 0.0f;
    d = 0.0f;
    low = true;
    return;
  }
  if (isinf(x)) {
    pq = 0.0f;
    d = 0.0f;
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
    pq = K * x3 * fmaf(z, s3, fmaf(-0.125f, x, 1.0f / 3.0f));
    d = K * x3 * fmaf(z, s1, fmaf(-0.5f, x, 1.0f));
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
    d = __fdividef(K * x3 * x * e1, 1.0f - e1);
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
  float f[3 * MAXG];
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

// Phase A: the FP32 inner/outer iteration.  On return the cell's FP64 iterate
// (Eint, m, R, Fk) holds the FP32 solution as the warm start of phase B.
template <int MAXG>
__device__ __forceinline__ void fp32_phase(const KParams &P, const GroupTable &tab, Cell &C,
                                           Arr64<MAXG> &A, Arr32<MAXG> &B) {
  const int G = P.G;
  const int64_t i = C.i;
  const double c = P.c, chat = P.c_hat;
  const float cr = (float)(c / chat);
  const double Etot = C.Etot, sE = 1.0 / Etot;
  const float tol32 = 2e-6f, tolo32 = 1e-6f;
  const bool tdep = P.temp_exp != 0.0;
  const double rho = C.rho;
  const int max_it = P.max_newton < 32 ? P.max_newton : 32;

  // scaled start values
  for (int g = 0; g < G; ++g) {
    const int64_t o = (int64_t)g * P.gs + i;
    const double s = P.src ? P.src[o] : 0.0;
    B.e0[g] = (float)((P.erad[o] + s) * sE);
    const double fs = sE / c;
    B.f[3 * g] = (float)(A.Fk[3 * g] * fs);
    B.f[3 * g + 1] = (float)(A.Fk[3 * g + 1] * fs);
    B.f[3 * g + 2] = (float)(A.Fk[3 * g + 2] * fs);
    B.R[g] = 0.0f;
  }
  set_tau32(P, tab, B, C.chi0s);

  for (int outer = 0; outer < P.max_outer; ++outer) {
    const double KE = 0.5 * (C.m[0] * C.m[0] + C.m[1] * C.m[1] + C.m[2] * C.m[2]) / rho;
    const float be[3] = {(float)(C.m[0] / (rho * c)), (float)(C.m[1] / (rho * c)),
                         (float)(C.m[2] / (rho * c))};
    for (int g = 0; g < G; ++g)
      B.w[g] = be[0] * B.f[3 * g] + be[1] * B.f[3 * g + 1] + be[2] * B.f[3 * g + 2];

    for (int it = 0; it <= max_it; ++it) {
      const double T = C.Eint * C.irc;
      if (tdep) set_tau32(P, tab, B, C.chi0s * pow(T / P.T_ref, P.temp_exp));
      const double aT3 = P.a_rad * T * T * T;
      const float aT4s = (float)(aT3 * T * sE);
      const float kd = (float)(aT3 * C.irc);  // a_R T^3 / (rho c_v): d~_g = kd (4 dP - dD)
      const float invT = (float)(1.0 / T);
      float pqL, dL;
      bool lowL;
      edge_fp32(tab.xef[0] * invT, pqL, dL, lowL);
      float sumR = 0.0f, sFRe = 0.0f, sde = 0.0f, sabs = 0.0f;
      for (int g = 0; g < G; ++g) {
        float pqU, dU;
        bool lowU;
        edge_fp32(tab.xef[g + 1] * invT, pqU, dU, lowU);
        const float dP = band_fp32(pqL, lowL, pqU, lowU);
        const float dD = dU - dL;
        const float b = aT4s * dP;
        const float a = tab.alphaf[g], rm = tab.rmf[g], rp = tab.rpf[g];
        const float q = chiF_ratio<float>(b, aT4s, dD, a, rm, rp, dL, dU);
        B.b[g] = b;
        B.dnx[g] = aT4s * (rp * dU - rm * dL);
        B.q[g] = q;
        const float ie = B.qe[g];
        float fr, d;
        if (ie > 0.0f) {
          const float Eg = b + (1.0f + a) * q * B.w[g] - B.R[g] * B.itau[g];
          fr = Eg - B.e0[g] - B.R[g];
          d = kd * (4.0f * dP - dD);
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
        lowL = lowU;
      }
      const float FG = (float)((C.Eint + KE - C.eg0) * sE) + cr * sumR;
      if (fabsf(FG) < tol32 && cr * sabs < tol32) break;
      if (it == max_it) break;
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
      if (fabsf(dE) < 1e-8f) break;  // step below FP32 resolution of E_tot
    }

    // write-back (energies stay scaled), flux update eq. numF1, momentum
    float sR = 0.0f;
    for (int g = 0; g < G; ++g) sR += B.R[g];
    const double egas_new = C.eg0 - (double)cr * (double)sR * Etot;
    float df[3] = {0.0f, 0.0f, 0.0f};
    for (int g = 0; g < G; ++g) {
      const int64_t o = (int64_t)g * P.gs + i;
      const float En = B.e0[g] + B.R[g];
      float vp0, vp1, vp2;
      closure_vP<float>(P.closure, 1.0f, En, B.f[3 * g], B.f[3 * g + 1], B.f[3 * g + 2], be[0],
                        be[1], be[2], vp0, vp1, vp2);
      const float t = B.tau[g], a = tab.alphaf[g];
      const float srcg = t * (B.b[g] - B.dnx[g] * (1.0f / 3.0f));
      const float kP = (1.0f + a) * t;
      const float inv = 1.0f / (1.0f + t * B.q[g]);
      const double fs = sE / c;
      const float ft0 = (float)(P.frad[0][o] * fs), ft1 = (float)(P.frad[1][o] * fs),
                  ft2 = (float)(P.frad[2][o] * fs);
      const float n0 = (ft0 + be[0] * srcg + kP * vp0) * inv;
      const float n1 = (ft1 + be[1] * srcg + kP * vp1) * inv;
      const float n2 = (ft2 + be[2] * srcg + kP * vp2) * inv;
      df[0] += n0 - ft0;
      df[1] += n1 - ft1;
      df[2] += n2 - ft2;
      B.f[3 * g] = n0;
      B.f[3 * g + 1] = n1;
      B.f[3 * g + 2] = n2;
    }
    const double mf = Etot / chat;  // (c E_tot)/(c c_hat)
    const double mn[3] = {C.m0[0] - mf * df[0], C.m0[1] - mf * df[1], C.m0[2] - mf * df[2]};
    const double KEn = 0.5 * (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) / rho;
    const float bn[3] = {(float)(mn[0] / (rho * c)), (float)(mn[1] / (rho * c)),
                         (float)(mn[2] / (rho * c))};
    float chg = (float)(fabs(KEn - KE) * sE);
    for (int g = 0; g < G; ++g) {
      const float wn = bn[0] * B.f[3 * g] + bn[1] * B.f[3 * g + 1] + bn[2] * B.f[3 * g + 2];
      const float t = B.tau[g];
      chg += fabsf(t * (1.0f + tab.alphaf[g]) * B.q[g] * (wn - B.w[g])) / (1.0f + t);
    }
    C.m[0] = mn[0];
    C.m[1] = mn[1];
    C.m[2] = mn[2];
    C.Eint = egas_new - KEn;  // start of the next pass (or of phase B)
    if (!(C.Eint > 0.0)) C.Eint = C.eg0 - KE;
    if (chg <= tolo32) break;
  }
  // hand over to phase B
  for (int g = 0; g < G; ++g) {
    A.R[g] = (double)B.R[g] * Etot;
    const double fs = c * Etot;
    A.Fk[3 * g] = (double)B.f[3 * g] * fs;
    A.Fk[3 * g + 1] = (double)B.f[3 * g + 1] * fs;
    A.Fk[3 * g + 2] = (double)B.f[3 * g + 2] * fs;
  }
}

template <int MAXG>
__global__ void __launch_bounds__(128) solve_mixed_kernel(const __grid_constant__ KParams P) {
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  Arr64<MAXG> A;
  Arr32<MAXG> B;
  Cell C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    if (!load_cell(P, i, C, A)) continue;
    fp32_phase(P, tab, C, A, B);
    set_tau(P, tab, C, A, C.chi0s);
    fp64_outer(P, tab, C, A, P.max_outer);
    store_cell(P, C, A);
  }
}

}  // namespace rhd
