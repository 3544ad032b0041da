// rhd_pplfree.cuh -- FP64 passes with free-slope PPL mean opacities.
//
// Appendix A replaces the fixed spectral index alpha_Q = -1 of B_nu and E_nu
// inside each group (Sec. 2.2.2) by indices fitted to the group values: edge
// slopes s_(g+1/2) = ln(Qbar_(g+1)/Qbar_g) / ln(nubar_(g+1)/nubar_g) (eq. sg,
// Qbar_g = Q_g/(nu_g+ - nu_g-), nubar_g = sqrt(nu_g+ nu_g-)), then alpha_Q,g =
// minmod(s_(g-1/2), s_(g+1/2)) between the end groups and -1 at both ends
// (eq. minmod).  The mean opacities follow from eq. chiQg with those indices.
//
// When the indices are refreshed is not fixed by the paper; here
//   alpha_B from b_g(T) at every Newton evaluation (B_nu is a function of the
//     iterate's T alone), with its T-derivative in the Jacobian so the inner
//     iteration stays a Newton iteration in T;
//   alpha_E once per cell from the radiation energy the update starts from,
//     E_g^t + S_g (a fixed chi_E keeps the O(N_g) arrowhead elimination: an
//     index from the iterate's E_g would couple neighbouring rows).
// A slope whose group values are not both positive is undefined, and a group
// with an undefined edge slope takes -1, like the end groups.
//
// Everything else is the fixed-slope FP64 pass of rhd_fp64.cuh with chi_B /
// chi_E != 1: the residual of eq. FGFR uses E_g = (chi_B/chi_E) b_g +
// (1 + alpha) (chi_F/chi_E) v.F_g/c^2 - R_g / (c_hat theta dt chi_E), and eq.
// chiDiff takes chi_B and chi_E separately.  One cell per thread.
#pragma once
#include "rhd_fp64.cuh"

namespace rhd {

// Per-group constants of the slope fit, in shared memory after the group table:
//   lr[g]  = ln r_g = ln(nu_g+ / nu_g-)
//   lw[g]  = ln(w_g / w_(g+1)), w = nu+ - nu-  (so ln(Qbar_(g+1)/Qbar_g) =
//            ln(Q_(g+1)/Q_g) + lw[g])
//   ils[g] = 1 / ln(nubar_(g+1)/nubar_g) = 2 / ln(nu_(g+2)/nu_g)
//   km[g]  = khat at the lower edge;  ra[g] = r_g^alpha_chi
struct FreeGeom {
  const double *lr, *lw, *ils, *km, *ra;
};
constexpr int kFreeArrays = 5;

// word offset of FreeGeom after the tables (the group table ends with floats)
__host__ __device__ __forceinline__ size_t free_geom_offset(int G) {
  return (table_bytes(G) + sizeof(double) - 1) / sizeof(double);
}
__host__ __device__ __forceinline__ size_t free_table_bytes(int G) {
  return sizeof(double) * (free_geom_offset(G) + (size_t)kFreeArrays * G);
}

// After build_table: all threads; ends with __syncthreads().
__device__ inline FreeGeom build_free_geom(const KParams &P, const GroupTable &tab, double *sm) {
  const int G = P.G;
  double *lr = sm, *lw = lr + G, *ils = lw + G, *km = ils + G, *ra = km + G;
  for (int t = threadIdx.x; t < G; t += blockDim.x) {
    const double n0 = P.edges[t], n1 = P.edges[t + 1];
    lr[t] = log(n1 / n0);
    if (t + 1 < G) {
      const double n2 = P.edges[t + 2];
      lw[t] = log((n1 - n0) / (n2 - n1));
      ils[t] = 2.0 / log(n2 / n0);
    } else {
      lw[t] = 0.0;
      ils[t] = 0.0;
    }
    km[t] = tab.kbar[t] * tab.rm[t];
    ra[t] = tab.rp[t] / tab.rm[t];
  }
  __syncthreads();
  return FreeGeom{lr, lw, ils, km, ra};
}

// phi(z) = (e^z - 1)/z, 1 at z = 0
__device__ __forceinline__ double phi_expm1(double z) {
  if (fabs(z) < 1e-6) return 1.0 + z * (0.5 + z * (1.0 / 6.0 + z * (1.0 / 24.0)));
  return expm1(z) / z;
}

// phi(z2) / phi(z1) without overflow when both are large and positive
__device__ __forceinline__ double phi_ratio(double z2, double z1) {
  if (z1 > 1.0 && z2 > 1.0) return exp(z2 - z1) * (z1 / z2) * (expm1(-z2) / expm1(-z1));
  return phi_expm1(z2) / phi_expm1(z1);
}

// psi(z) = d ln phi / dz = e^z/(e^z - 1) - 1/z (series 1/2 + z/12 - z^3/720
// + z^5/30240 near 0, from (1/2) coth(z/2) = 1/z + z/12 - ...)
__device__ __forceinline__ double psi_expm1(double z) {
  if (fabs(z) < 0.1) {
    const double z2 = z * z;
    return 0.5 + z * (1.0 / 12.0 + z2 * (-1.0 / 720.0 + z2 * (1.0 / 30240.0)));
  }
  if (z > 0.0) return -1.0 / expm1(-z) - 1.0 / z;
  return 1.0 + 1.0 / expm1(z) - 1.0 / z;
}

// eq. sg for the edge between g and g+1 from the group values qa = Q_g,
// qb = Q_(g+1); false when undefined
__device__ __forceinline__ bool edge_slope(double qa, double qb, double lw, double ils,
                                           double &s) {
  if (!(qa > 0.0) || !(qb > 0.0)) return false;
  s = (log(qb / qa) + lw) * ils;
  return isfinite(s);
}

// eq. minmod with the derivative of the selected slope
__device__ __forceinline__ double minmod_d(double a, double da, double b, double db,
                                           double &d) {
  if (a > 0.0 && b > 0.0) {
    d = a < b ? da : db;
    return a < b ? a : b;
  }
  if (a < 0.0 && b < 0.0) {
    d = a > b ? da : db;
    return a > b ? a : b;
  }
  d = 0.0;
  return 0.0;
}

// Per-cell free-slope arrays: chi_E / cs and the edge values of chi_0 / chi_E
// (set once from E_g^t + S_g), and the band fractions and edge D values of
// the current evaluation.
template <int MAXG>
struct FreeArr {
  double kE[MAXG], ikE[MAXG], rmE[MAXG], rpE[MAXG];
  double fP[MAXG], fD[MAXG + 1];
};

// chi_E of every group from alpha_E of Q_g = E_g^t + S_g (eqs. sg, minmod,
// chiQg).
template <int MAXG>
__device__ __forceinline__ void set_free_E(const KParams &P, const GroupTable &tab,
                                           const FreeGeom &fg, const Cell &C, FreeArr<MAXG> &F) {
  const int G = P.G;
  const int64_t i = C.i;
  auto Qg = [&](int g) {
    const int64_t o = (int64_t)g * P.gs + i;
    return P.erad[o] + (P.src ? P.src[o] : 0.0);
  };
  double q1 = Qg(0), sl = 0.0;
  bool okl = false;
  for (int g = 0; g < G; ++g) {
    const double q2 = g + 1 < G ? Qg(g + 1) : 0.0;
    double sr = 0.0;
    const bool okr = g + 1 < G && edge_slope(q1, q2, fg.lw[g], fg.ils[g], sr);
    double aE = -1.0, dummy;
    if (g > 0 && g + 1 < G && okl && okr) aE = minmod_d(sl, 0.0, sr, 0.0, dummy);
    const double a = tab.alpha[g], lr = fg.lr[g];
    const double z1 = (aE + 1.0) * lr;
    const double ratio = phi_ratio(z1 + a * lr, z1);  // chi_E / chi_0(nu_g-)
    const double k = fg.km[g] * ratio;
    F.kE[g] = k;
    F.ikE[g] = 1.0 / k;
    F.rmE[g] = 1.0 / ratio;
    F.rpE[g] = fg.ra[g] / ratio;
    q1 = q2;
    sl = sr;
    okl = okr;
  }
}

// One inner Newton iteration with free slopes (a4-a8; see inner_step).
template <int MAXG>
__device__ __forceinline__ int inner_step_free(const KParams &P, const GroupTable &tab,
                                               const FreeGeom &fg, Cell &C, Arr64<MAXG> &A,
                                               FreeArr<MAXG> &F) {
  const int G = P.G;
  const int64_t i = C.i;
  const double T = C.Eint * C.irc;
  if (P.temp_exp != 0.0) set_tau(P, tab, C, A, C.chi0s * pow(T / P.T_ref, P.temp_exp), F.ikE);
  const double aT3 = P.a_rad * T * T * T, aT4 = aT3 * T;
  const double invT = 1.0 / T;
  // band fractions and edge values of every group first: alpha_B of a group
  // needs its neighbours' b_g
  {
    double pqL, dL, eL;
    bool lowL;
    edge_tab(tab.pc, tab.xe[0] * invT, pqL, dL, eL, lowL);
    F.fD[0] = dL;
    for (int g = 0; g < G; ++g) {
      double pqU, dU, eU;
      bool lowU;
      edge_tab(tab.pc, tab.xe[g + 1] * invT, pqU, dU, eU, lowU);
      F.fP[g] = band_fp64(pqL, lowL, pqU, lowU);
      F.fD[g + 1] = dU;
      pqL = pqU;
      lowL = lowU;
    }
  }
  // edge slope of ln b against ln nu and its T-derivative: b_g = aT4 fP_g and
  // d fP_g/dT = -(D(x_g+) - D(x_g-))/T, so d ln(b_(g+1)/b_g)/dT =
  // (dD_g/fP_g - dD_(g+1)/fP_(g+1))/T
  auto slopeB = [&](int g, double &s, double &ds) {
    if (!edge_slope(F.fP[g], F.fP[g + 1], fg.lw[g], fg.ils[g], s)) return false;
    const double r0 = (F.fD[g + 1] - F.fD[g]) / F.fP[g];
    const double r1 = (F.fD[g + 2] - F.fD[g + 1]) / F.fP[g + 1];
    ds = (r0 - r1) * fg.ils[g] * invT;
    return true;
  };
  double sl = 0.0, dsl = 0.0;
  bool okl = false;
  double sumR = 0.0, sFRe = 0.0, sde = 0.0, sabs = 0.0;
  for (int g = 0; g < G; ++g) {
    double sr = 0.0, dsr = 0.0;
    const bool okr = g + 1 < G && slopeB(g, sr, dsr);
    double aB = -1.0, daB = 0.0;
    if (g > 0 && g + 1 < G && okl && okr) aB = minmod_d(sl, dsl, sr, dsr, daB);
    sl = sr;
    dsl = dsr;
    okl = okr;
    const int64_t o = (int64_t)g * P.gs + i;
    const double dL = F.fD[g], dU = F.fD[g + 1];
    const double dD = dU - dL;
    const double b = aT4 * F.fP[g];
    const double db = aT3 * (4.0 * F.fP[g] - dD);
    const double a = tab.alpha[g], lr = fg.lr[g];
    // chi_B / chi_E (eq. chiQg) and d ln chi_B / dT through alpha_B
    const double z1 = (aB + 1.0) * lr, z2 = z1 + a * lr;
    const double beta = fg.km[g] * phi_ratio(z2, z1) * F.ikE[g];
    const double dlk = lr * (psi_expm1(z2) - psi_expm1(z1)) * daB;
    const double rm = F.rmE[g], rp = F.rpE[g];
    // eq. chiDiff over chi_E, held to [min, max] of chi_0 / chi_E over the group
    const double X = rp * dU - rm * dL;
    const double den = (4.0 / 3.0) * b - (1.0 / 3.0) * aT4 * dD;
    double q = 1.0;
    if (den > 0.0) q = ((beta + 1.0 / 3.0) * b + (1.0 / 3.0) * (a * b - aT4 * X)) / den;
    q = fmin(fmax(q, fmin(rm, rp)), fmax(rm, rp));
    const double bq = beta * b;
    A.bq[g] = bq;
    A.dnx[g] = aT4 * X;
    A.qF[g] = q;
    const double ie = A.qe[g];
    double fr, d;
    if (ie > 0.0) {
      const double Eg = bq + (1.0 + a) * q * A.w[g] - A.R[g] * C.its * F.ikE[g];
      const double s = P.src ? P.src[o] : 0.0;
      fr = Eg - P.erad[o] - A.R[g] - s;
      d = (beta * db + bq * dlk) * C.irc;  // d(chi_B b_g / chi_E)/dT / C_v
    } else {
      fr = -A.R[g];
      d = 0.0;
    }
    const double iee = ie > 0.0 ? ie : 1.0;
    A.FR[g] = fr;
    A.dg[g] = d;
    sumR += A.R[g];
    sFRe -= fr * iee;
    sde -= d * iee;
    sabs += fabs(fr);
  }
  return inner_tail(P, C, A, sumR, sFRe, sde, sabs);
}

// FP64 solve with free slopes, one cell per thread (see solve_fp64_kernel).
template <int MAXG>
__global__ void __launch_bounds__(128) solve_free_kernel(const __grid_constant__ KParams P,
                                                         const WarmStart W) {
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  const FreeGeom fg = build_free_geom(P, tab, sm + free_geom_offset(P.G));
  Arr64<MAXG> A;
  FreeArr<MAXG> F;
  Cell C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool warm = W.r != nullptr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    if (!load_cell(P, i, C, A)) continue;
    set_free_E(P, tab, fg, C, F);
    for (int attempt = 0; attempt < 2; ++attempt) {
      int nit0 = 0;
      if (attempt == 1) {
        if (!(warm && W.fallback && C.stat != RHD_STATUS_OK)) break;
        nit0 = C.nit;
        load_cell(P, i, C, A);
      }
      set_tau(P, tab, C, A, C.chi0s, F.ikE);
      if (warm && attempt == 0) apply_warm(P, W, C, A);
      outer_begin(P, C, A);
      for (;;) {
        const int r = inner_step_free(P, tab, fg, C, A, F);
        if (r == 0) continue;
        if (r == 2) C.stat = RHD_STATUS_MAXITER;
        if (outer_end(P, tab, C, A, F.kE)) break;
      }
      if (attempt == 1) {
        C.nit += nit0;
        if (C.stat == RHD_STATUS_OK) C.stat = RHD_STATUS_FALLBACK;
      }
    }
    store_cell(P, C, A);
  }
}

}  // namespace rhd
