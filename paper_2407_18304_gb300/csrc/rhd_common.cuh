// rhd_common.cuh -- launch parameters, the per-grid group table and the FP64
// Planck / closure building blocks shared by the solver kernels.
//
// Notation follows He, Wibking & Krumholz (2024): x = h nu / (k_B T); the
// group Planck integral b_g = 4 pi B_g / c = a_R T^4 [P(x_g+) - P(x_g-)] with
// P(x) = (15/pi^4) int_0^x t^3/(e^t-1) dt (eq. Qg applied to B_nu); the edge
// term D(x) = (15/pi^4) x^4/(e^x-1) = nu (4 pi B_nu / c) / (a_R T^4), so that
// (4 pi/c) Delta_g(nu B_nu) = a_R T^4 [D(x_g+) - D(x_g-)] (Sec. 2.2.1) and
// (4 pi/c) Delta_g(nu chi_0 B_nu) = a_R T^4 [chi_0(nu_g+) D(x_g+) -
// chi_0(nu_g-) D(x_g-)] with chi_0 at each edge from group g's own powerlaw.
#pragma once
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/rhd.h"
#include "planck_table.h"

namespace rhd {

constexpr int kMaxG = RHD_MAX_GROUPS;
constexpr int kMaxSeg = RHD_MAX_SEGMENTS;
constexpr int kNB = 18;  // Bernoulli terms of the small-x series (x < 2)
constexpr int kNQ = 21;  // exponential terms of the large-x series (x >= 2)
constexpr double kPlanckNorm = 0.15398973382026502;  // 15 / pi^4
constexpr double kXSplit = 2.0;

// Everything one launch needs, passed by value (about 8 KB; the group table
// is built from it inside each CTA).
struct KParams {
  const double *rho;
  double *mom[3];
  double *egas;
  const double *kappa0;
  double *erad;
  double *frad[3];
  const double *src;
  uint8_t *status;
  uint8_t *iters;
  int64_t n;   // cells
  int64_t gs;  // group stride
  double c_v, theta, dt, c, c_hat, a_rad, h_over_k;
  double cr, ic, inv_c2, icc;  // c / c_hat, 1 / c, 1 / c^2, 1 / (c c_hat) (set with c, c_hat)
  double tol, tol_outer;
  int max_newton, max_outer, closure, flags;
  int G, mode, n_seg, has_table;
  int count;  // 1: add this launch's events to g_events (rhd_events_start/stop)
  double nu_ref, temp_exp, T_ref;
  double edges[kMaxG + 1];
  double nu_break[kMaxSeg];
  double seg_logk[kMaxSeg];
  double seg_beta[kMaxSeg];
  double khat_g[kMaxG];
  double alpha_g[kMaxG];
};

// Shared-memory group table, structure of arrays:
//   xe[G+1]  h nu_e / k_B of every edge (x_e = xe[e] / T)
//   kbar[G]  PPL fixed-slope mean opacity shape khat_g- (r^a - 1)/(a ln r)
//            (eq. chiQg with alpha_Q = -1), so chi_B = chi_E = rho kappa0 kbar
//   ikbar[G] 1 / kbar
//   rm[G]    khat_g- / kbar   (chi_0 at the lower edge over chi_E)
//   rp[G]    khat_g- r^a / kbar (chi_0 at the upper edge over chi_E)
//   alpha[G] in-group powerlaw index a
// and FP32 copies xef[G+1], rmf, rpf, alphaf (read by the FP32 iterations, so
// they never convert).
struct GroupTable {
  const double *xe, *kbar, *ikbar, *rm, *rp, *alpha;
  const float *xef, *rmf, *rpf, *alphaf;
  const double *pc;  // the Planck-integral polynomials (planck_table.h layout, see edge_tab)
};

// Shared-memory layout of a CTA's tables: the Planck polynomials first
// (kPlanckWords doubles: coefficients [kDeg + 1][kSeg], centres [kSeg],
// inverse half-widths [kSeg]), then the group table of the grid.
constexpr int kPlanckWords = (planck_table::kDeg + 3) * planck_table::kSeg;
constexpr int kTableArrays = 6;
__host__ __device__ __forceinline__ size_t group_table_bytes(int G) {
  return sizeof(double) * (kTableArrays * G + 1) + sizeof(float) * (4 * G + 1);
}
__host__ __device__ __forceinline__ size_t table_bytes(int G) {
  return sizeof(double) * kPlanckWords + group_table_bytes(G);
}

__constant__ double c_planck[kPlanckWords];

// Event counters of the update (include/rhd.h, RHD_EV_*): what each launch
// did, per cell, added once per cell by one lane when KParams::count is set.
__device__ unsigned long long g_events[RHD_EVENTS];

__device__ __forceinline__ void count_event(const KParams &P, int k, unsigned long long v) {
  if (P.count && v) atomicAdd(&g_events[k], v);
}

// Copy the Planck polynomials to sm (all threads; the caller synchronises).
__device__ __forceinline__ void load_planck(double *sm) {
  for (int t = threadIdx.x; t < kPlanckWords; t += blockDim.x) sm[t] = c_planck[t];
}

// khat from the piecewise law; right = 1 takes the segment above a breakpoint
// that coincides with nu, right = 0 the one below.
__device__ inline double law_logk(const KParams &P, double nu, int right) {
  int s = 0;
  for (int b = 0; b < P.n_seg - 1; ++b) {
    const double nb = P.nu_break[b];
    if (right ? (nb <= nu) : (nb < nu)) s = b + 1;
  }
  return P.seg_logk[s] + P.seg_beta[s] * log(nu / P.nu_ref);
}

// (r^a - 1)/(a ln r), 1 at a = 0 (Taylor near 0)
__device__ inline double ppl_mean_factor(double a, double lr) {
  const double z = a * lr;
  if (fabs(z) < 1e-6) return 1.0 + z * (0.5 + z * (1.0 / 6.0 + z * (1.0 / 24.0)));
  return expm1(z) / z;
}

// Build the group table in shared memory (step a2): all threads of the CTA
// take part; ends with __syncthreads().
__device__ inline GroupTable build_table(const KParams &P, double *smem) {
  const int G = P.G;
  load_planck(smem);
  double *sm = smem + kPlanckWords;
  double *xe = sm, *kbar = sm + G + 1, *ikbar = kbar + G, *rm = ikbar + G, *rp = rm + G,
         *alp = rp + G;
  for (int t = threadIdx.x; t <= G; t += blockDim.x) {
    xe[t] = P.h_over_k * P.edges[t];  // inf stays inf, 0 stays 0
    if (t == G) continue;
    const double n0 = P.edges[t], n1 = P.edges[t + 1];
    if (P.mode != RHD_PC) {  // PPL, fixed or free slopes: same per-group law
      const double lr = log(n1 / n0);
      double lk0, a;
      if (P.has_table) {
        lk0 = log(P.khat_g[t]);
        a = P.alpha_g[t];
      } else {
        lk0 = law_logk(P, n0, 1);
        a = (law_logk(P, n1, 0) - lk0) / lr;
      }
      const double mf = ppl_mean_factor(a, lr);
      kbar[t] = exp(lk0) * mf;
      ikbar[t] = 1.0 / kbar[t];
      rm[t] = 1.0 / mf;
      rp[t] = exp(a * lr) / mf;
      alp[t] = a;
    } else {
      double k0;
      if (P.has_table) {
        k0 = P.khat_g[t];
      } else {
        double centre;
        if (n0 == 0.0 && isinf(n1)) centre = P.nu_ref;
        else if (n0 == 0.0) centre = 0.5 * n1;
        else if (isinf(n1)) centre = 2.0 * n0;
        else centre = sqrt(n0 * n1);
        k0 = exp(law_logk(P, centre, 1));
      }
      kbar[t] = k0;
      ikbar[t] = 1.0 / k0;
      rm[t] = 1.0;
      rp[t] = 1.0;
      alp[t] = 0.0;
    }
  }
  float *xef = reinterpret_cast<float *>(alp + G), *rmf = xef + G + 1, *rpf = rmf + G,
        *alf = rpf + G;
  __syncthreads();
  for (int t = threadIdx.x; t <= G; t += blockDim.x) {
    xef[t] = (float)xe[t];
    if (t == G) continue;
    rmf[t] = (float)rm[t];
    rpf[t] = (float)rp[t];
    alf[t] = (float)alp[t];
  }
  __syncthreads();
  return GroupTable{xe, kbar, ikbar, rm, rp, alp, xef, rmf, rpf, alf, smem};
}

// Decomposition of a positive normal double without FP64 instructions (on
// GB300 an FP64 instruction, conversions included, costs 64 FP32 ones): from
// the bit pattern, x = m 2^ex with m in [0.5, 1) (as frexp), m cut to FP32.
__device__ __forceinline__ float frexp_f(double x, int &ex) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  ex = ((hi >> 20) & 0x7FF) - 1022;
  const unsigned frac = ((unsigned)(hi & 0xFFFFF) << 3) | ((unsigned)lo >> 29);
  return __int_as_float((int)((126u << 23) | frac));
}

// x 2^-sh as FP32 from the bit pattern (mantissa cut, not rounded; 0 below
// FP32's normal range, +-inf above it).
__device__ __forceinline__ float scaled_f(double x, int sh) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int E = (hi >> 20) & 0x7FF;
  const unsigned sign = (unsigned)hi & 0x80000000u;
  if (E == 0) return __int_as_float((int)sign);
  const int fe = E - 1023 - sh + 127;
  if (fe <= 0) return __int_as_float((int)sign);
  if (fe >= 255) return __int_as_float((int)(sign | 0x7F800000u));
  const unsigned frac = ((unsigned)(hi & 0xFFFFF) << 3) | ((unsigned)lo >> 29);
  return __int_as_float((int)(sign | ((unsigned)fe << 23) | frac));
}

// A float widened to double from its bit pattern (exact for normal numbers;
// zero and FP32 subnormals give 0, which at E_tot scale is below FP64's
// resolution of the sums they enter).  No FP64 instruction.
__device__ __forceinline__ double f2d(float f) {
  const int b = __float_as_int(f);
  const int e = (b >> 23) & 0xFF;
  if (e == 0) return 0.0;
  const unsigned sign = (unsigned)b & 0x80000000u;
  const unsigned man = (unsigned)b & 0x7FFFFFu;
  const unsigned he = e == 0xFF ? 0x7FFu : (unsigned)(e + 896);
  return __hiloint2double((int)(sign | (he << 20) | (man >> 3)), (int)((man & 7u) << 29));
}

// A group energy that carries a feature: positive, finite, not below about
// 1.3e-290 (exponent field >= 60), tested on the bits.
__device__ __forceinline__ bool usable_energy(double x) {
  const int hi = __double2hiint(x);
  return hi >= 0 && ((hi >> 20) & 0x7FF) >= 60 && ((hi >> 20) & 0x7FF) < 0x7FF;
}

// Allow `kernel` smem bytes of dynamic shared memory on the current device.
// The attribute belongs to the (kernel, device) pair, so the largest size set
// so far is remembered per device (one table per kernel instance, under a
// lock: launches may come from several host threads).
constexpr int kAttrDevices = 64;
template <auto kernel>
cudaError_t allow_smem(size_t smem) {
  static std::mutex mu;
  static size_t done[kAttrDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kAttrDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev] >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done[dev] = smem;
  return e;
}

// (This header is compiled into exactly one translation unit, rhd.cu.)

// FP64 edge values: pq = P(x) when low (x < 2), else Q(x) = 1 - P(x);
// d = D(x) = (15/pi^4) x^4/(e^x-1) and ed = x dD/dx = D (4 - x e^x/(e^x-1)).
// One expm1 and one division give x/(e^x - 1) and e^-x = 1/(expm1(x) + 1); P and Q come from the
// piecewise polynomials of planck_table.h (P = 15/pi^4 x^3 g(x) below x = 2,
// Q = 15/pi^4 x^3 e^-x h(x) above), the segment read off the exponent and two
// leading mantissa bits of x: every x takes the same instructions, so the
// lanes of a warp never split on the value of x.  Beyond the table (x >= 1024)
// e^-x is 0 in FP64 and the polynomial is evaluated at its centre.
__device__ __forceinline__ void edge_tab(const double *pc, double x, double &pq, double &d,
                                         double &ed, bool &low) {
  using namespace planck_table;
  if (!(x > 0.0)) {
    pq = 0.0;
    d = 0.0;
    ed = 0.0;
    low = true;
    return;
  }
  if (isinf(x)) {
    pq = 0.0;
    d = 0.0;
    ed = 0.0;
    low = false;
    return;
  }
  const double em = expm1(x);
  double xr, emx;  // x/(e^x - 1), e^-x
  if (x < 300.0) {  // one reciprocal of (e^x - 1) e^x serves both (no overflow below 354)
    const double ep = em + 1.0;
    const double r = 1.0 / (em * ep);
    xr = x * ep * r;
    emx = em * r;
  } else {
    xr = x / em;
    emx = 1.0 / (em + 1.0);
  }
  const double x3 = x * x * x;
  d = kPlanckNorm * x3 * xr;
  ed = d * (4.0 - xr - x);  // x e^x/(e^x-1) = x/(e^x-1) + x
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7FF) - 1023;
  int sg = 1 + (e - kEMin) * kSub + ((hi >> 18) & 3);
  sg = e < kEMin ? 0 : (e > kEMax ? kSeg - 1 : sg);
  const double *cen = pc + (kDeg + 1) * kSeg, *ih = cen + kSeg;
  const double u = e > kEMax ? 0.0 : (x - cen[sg]) * ih[sg];
  double p = pc[kDeg * kSeg + sg];
#pragma unroll
  for (int k = kDeg - 1; k >= 0; --k) p = fma(p, u, pc[k * kSeg + sg]);
  low = x < kXSplit;
  pq = kPlanckNorm * x3 * p * (low ? 1.0 : emx);
}

// Planck fraction of the band between a lower and an upper edge value.
__device__ __forceinline__ double band_fp64(double pqL, bool lowL, double pqU, bool lowU) {
  if (!lowL) return pqL - pqU;            // Q(x-) - Q(x+): no 1 - 1 cancellation
  if (lowU) return pqU - pqL;             // P(x+) - P(x-)
  return (1.0 - pqU) - pqL;               // edges straddle the split
}

// v . P_g for the closure P(E, F) applied to one group (Sec. 2.1).  M1:
// P = E [iso I + dir n n^T], n = F/|F|, iso = (1 - chi)/2, dir = (3 chi - 1)/2
// with Levermore's chi(f) = (3 + 4 f^2)/(5 + 2 sqrt(4 - 3 f^2)), f = |F|/(cE).
// Multiplying numerator and denominator by 5 - 2 sqrt(4 - 3 f^2) turns the
// denominator into 3 (3 + 4 f^2), so chi = (5 - 2 s)/3 with s = sqrt(4 - 3 f^2):
// iso = (s - 1)/3 and dir = 2 - s = 3 f^2 / (2 + s).  With S = cE s =
// sqrt(4 (cE)^2 - 3 |F|^2) that is
//   v . P = [(S - cE)/3 v + 3 (v . F) F / (2 cE + S)] / c,
// one square root and one division.  f >= 1 is held at 1 (chi = 1):
// v . P = E (v . F) F / |F|^2.
template <typename R>
__device__ __forceinline__ void closure_vP(int closure, R c, R E, R F0, R F1, R F2, R v0, R v1,
                                           R v2, R &o0, R &o1, R &o2) {
  const R fn2 = F0 * F0 + F1 * F1 + F2 * F2;
  if (closure == RHD_M1 && E > R(0) && fn2 > R(0)) {
    const R cE = c * E, cE2 = cE * cE;
    const R vF = v0 * F0 + v1 * F1 + v2 * F2;
    if (fn2 < cE2) {
      const R S = sqrt(R(4) * cE2 - R(3) * fn2);
      const R ic = R(1) / c;
      const R a = (S - cE) * (R(1) / R(3)) * ic;
      const R k = R(3) * vF * ic / (R(2) * cE + S);
      o0 = a * v0 + k * F0;
      o1 = a * v1 + k * F1;
      o2 = a * v2 + k * F2;
    } else {
      const R k = E * vF / fn2;
      o0 = k * F0;
      o1 = k * F1;
      o2 = k * F2;
    }
    return;
  }
  const R e3 = E * (R(1) / R(3));
  o0 = e3 * v0;
  o1 = e3 * v1;
  o2 = e3 * v2;
}

// closure_vP in parts for a caller that divides by another positive quantity
// as well (the flux update): v . P = a v + (kn / kd) F with kd > 0, so that
// one reciprocal serves both divisions.  ic = 1 / c.
template <typename R>
__device__ __forceinline__ void closure_vP_parts(int closure, R c, R ic, R E, R F0, R F1, R F2,
                                                 R v0, R v1, R v2, R &a, R &kn, R &kd) {
  const R fn2 = F0 * F0 + F1 * F1 + F2 * F2;
  if (closure == RHD_M1 && E > R(0) && fn2 > R(0)) {
    const R cE = c * E, cE2 = cE * cE;
    const R vF = v0 * F0 + v1 * F1 + v2 * F2;
    if (fn2 < cE2) {
      const R S = sqrt(R(4) * cE2 - R(3) * fn2);
      a = (S - cE) * (R(1) / R(3)) * ic;
      kn = R(3) * vF * ic;
      kd = R(2) * cE + S;
    } else {
      a = R(0);
      kn = E * vF;
      kd = fn2;
    }
    return;
  }
  a = E * (R(1) / R(3));
  kn = R(0);
  kd = R(1);
}

// v . P_g and M = d(v . P_g)/dF_g at fixed E_g for the M1 closure of
// closure_vP (Levermore's Eddington factor chi(f), f = |F|/(cE) held at 1):
// with n = F/|F|, vn = v . n,
//   v . P = E [iso v + dir vn n],  iso = (1 - chi)/2,  dir = (3 chi - 1)/2,
//   M = (iso'/c) v n^T + (dir'/c) vn n n^T
//       + (E dir/|F|) [n (v - vn n)^T + vn (I - n n^T)],
// iso' = -chi'/2, dir' = 3 chi'/2 (chi' = 0 where f is held at 1).  F = 0
// gives P = E/3 I and M = 0 (dir vanishes like f^2).
template <typename R>
__device__ __forceinline__ void closure_vP_jac(R c, R E, const R F[3], const R v[3], R vP[3],
                                               R M[9]) {
  const R fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
  if (!(E > R(0)) || !(fn2 > R(0))) {
    for (int k = 0; k < 3; ++k) vP[k] = E * v[k] * (R(1) / R(3));
    for (int k = 0; k < 9; ++k) M[k] = R(0);
    return;
  }
  const R fn = sqrt(fn2), inv = R(1) / fn;
  R f = fn / (c * E);
  const bool held = f > R(1);
  if (held) f = R(1);
  const R f2 = f * f;
  const R sq = sqrt(R(4) - R(3) * f2), num = R(3) + R(4) * f2, den = R(5) + R(2) * sq;
  const R chi = num / den;
  const R dchi = held ? R(0) : (R(8) * f * den + R(6) * f * num / sq) / (den * den);
  const R iso = R(0.5) * (R(1) - chi), dir = R(0.5) * (R(3) * chi - R(1));
  const R n[3] = {F[0] * inv, F[1] * inv, F[2] * inv};
  const R vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  const R a = -R(0.5) * dchi / c, b = R(1.5) * dchi * vn / c, e = E * dir * inv;
  for (int r = 0; r < 3; ++r) {
    vP[r] = E * (iso * v[r] + dir * vn * n[r]);
    for (int q = 0; q < 3; ++q) {
      const R id = r == q ? R(1) : R(0);
      M[3 * r + q] = a * v[r] * n[q] + b * n[r] * n[q] + e * (n[r] * (v[q] - vn * n[q]) +
                                                               vn * (id - n[r] * n[q]));
    }
  }
}

template <typename R>
struct Vec3 {
  R x, y, z;
};

// Sum of the flux changes of a Newton flux pass (x, y, z) and of their
// absolute values (l1).
struct FluxDelta {
  double x, y, z, l1;
  unsigned n;  // groups solved by Newton steps
};

// Newton steps of flux_update from F (kept out of line: taken by few groups,
// and inlined it would raise the register count of the whole solve loop;
// scalars in and out, so that nothing of the caller has to leave registers).
template <typename R>
__device__ __noinline__ Vec3<R> flux_newton(R c, R E, R kap, R b0, R b1, R b2, R v0, R v1, R v2,
                                            R F0, R F1, R F2, R eps) {
  const R base[3] = {b0, b1, b2}, v[3] = {v0, v1, v2};
  R F[3] = {F0, F1, F2}, vP[3], M[9];
  const Vec3<R> keep = {F0, F1, F2};
  for (int it = 0; it < 8; ++it) {
    closure_vP_jac<R>(c, E, F, v, vP, M);
    const R r0 = F[0] - base[0] - kap * vP[0], r1 = F[1] - base[1] - kap * vP[1],
            r2 = F[2] - base[2] - kap * vP[2];
    // the scale includes the terms that cancel in r (base against kap v.P)
    const R sc = c * E + fmax(fabs(F[0]), fmax(fabs(F[1]), fabs(F[2]))) +
                 fmax(fabs(base[0]), fmax(fabs(base[1]), fabs(base[2]))) +
                 fabs(kap) * fmax(fabs(vP[0]), fmax(fabs(vP[1]), fabs(vP[2])));
    if (fmax(fabs(r0), fmax(fabs(r1), fabs(r2))) <= eps * sc) break;
    // J = I - kap M; d = J^-1 r by the adjugate
    const R j00 = R(1) - kap * M[0], j01 = -kap * M[1], j02 = -kap * M[2];
    const R j10 = -kap * M[3], j11 = R(1) - kap * M[4], j12 = -kap * M[5];
    const R j20 = -kap * M[6], j21 = -kap * M[7], j22 = R(1) - kap * M[8];
    const R c00 = j11 * j22 - j12 * j21, c01 = j12 * j20 - j10 * j22, c02 = j10 * j21 - j11 * j20;
    const R idet = R(1) / (j00 * c00 + j01 * c01 + j02 * c02);
    const R d0 = (c00 * r0 + (j02 * j21 - j01 * j22) * r1 + (j01 * j12 - j02 * j11) * r2) * idet;
    const R d1 = (c01 * r0 + (j00 * j22 - j02 * j20) * r1 + (j02 * j10 - j00 * j12) * r2) * idet;
    const R d2 = (c02 * r0 + (j01 * j20 - j00 * j21) * r1 + (j00 * j11 - j01 * j10) * r2) * idet;
    if (!(isfinite(d0) && isfinite(d1) && isfinite(d2))) return keep;  // the eq. numF1 value
    F[0] -= d0;
    F[1] -= d1;
    F[2] -= d2;
    if (fmax(fabs(d0), fmax(fabs(d1), fabs(d2))) <= eps * sc) break;  // quadratic: done
  }
  if (!(isfinite(F[0]) && isfinite(F[1]) && isfinite(F[2]))) return keep;
  return Vec3<R>{F[0], F[1], F[2]};
}

// Flux update of one group, eq. fupdate with P_g at the new flux:
//   F = base + kap (v . P_g(E, F)),
//   base = (F^t + c_hat theta dt v src_g) / (1 + c_hat chi_F theta dt),
//   kap = c_hat theta dt (1 + alpha) chi_E / (1 + c_hat chi_F theta dt).
// F holds the lagged flux on entry.  The first step takes P_g at the lagged
// flux (eq. numF1).  Repeating that step contracts by at most 5 |kap| |v| / c
// per outer pass (|M| <= 5 |v| / c), and where v chi_E / chi_F is of order c
// it oscillates around the solution for hundreds of passes; so in a cell whose
// outer iteration has been seen to contract slowly (slow), for the groups
// where the bound exceeds 1/2 (M1 closure only: the Eddington P_g does not
// depend on F), Newton steps on the closure's dependence on F follow (flux_newton: at most
// 8, stopped once the residual F - base - kap v.P or the last step is below
// eps times the size of the terms; a non-finite step keeps the eq. numF1
// value).  Both forms have the same fixed point.
template <typename R>
__device__ __forceinline__ void flux_update(int closure, R c, R E, R kap, const R base[3],
                                            const R v[3], R vmag, R F[3], R eps, bool slow) {
  R vP[3];
  closure_vP<R>(closure, c, E, F[0], F[1], F[2], v[0], v[1], v[2], vP[0], vP[1], vP[2]);
  for (int k = 0; k < 3; ++k) F[k] = base[k] + kap * vP[k];
  if (slow && closure == RHD_M1 && R(10) * fabs(kap) * vmag > c) {
    const Vec3<R> r = flux_newton<R>(c, E, kap, base[0], base[1], base[2], v[0], v[1], v[2],
                                     F[0], F[1], F[2], eps);
    F[0] = r.x;
    F[1] = r.y;
    F[2] = r.z;
  }
}

}  // namespace rhd
