// rhd_correct.cuh -- the correction step of the mixed form: one FP64
// evaluation of the residual of the fully coupled per-cell system at the FP32
// passes' result, and one Newton step on that system whose Jacobian is built
// and solved in FP32 (iterative refinement: the residual carries the FP64
// accuracy, the Jacobian only the rate).
//
// The paper's inner/outer iteration (Sec. 3) converges to the root of
//   F_G   = E_int + E_kin(m) - E_gas^t + (c/c_hat) sum_g R_g               (eq. FGFR)
//   F_R,g = E_g(T, R_g, w_g) - (E_g^t + S_g) - R_g,   E_g from eq. Rnew,
//           w_g = v.F_g / c^2                                             (eq. FGFR)
//   F_F,g = F_g - base_g - kap_g v.P_g(E_g^t + S_g + R_g, F_g)            (eq. fupdate,
//           base_g = (F_g^t + c_hat theta dt v (chi_B b_g - delta chi_g/3)) / (1 + c_hat theta dt chi_F),
//           kap_g = c_hat theta dt (1 + alpha) chi_E / (1 + c_hat theta dt chi_F))   eq. numF1)
// with the momentum of eq. vupdate, m = m^t - (c c_hat)^-1 sum_g (F_g - F_g^t),
// v = m / rho, and T = E_int / (rho c_v).  Unknowns: E_int, R_g, F_g.
//
// Its Jacobian is bordered block-diagonal: a group's four unknowns (R_g, F_g)
// couple to one another, and to the other groups only through E_int (by T)
// and through v (by the sum of the fluxes).  So each group's 4x4 block is
// eliminated with its five right-hand sides (the residual, the E_int column,
// the three v columns): u_g = p_g + q_g x + S_g beta.  The sums over the groups
// turn the E_int row and the momentum relation into a 4x4 system for
// (x, beta); then every group's step follows -- O(N_g) work, like the
// paper's arrowhead elimination of eq. matrix.
//
// Scaled FP32 variables: x = dE_int / E_tot, r_g = dR_g / E_tot,
// f_g = dF_g / (c E_tot), beta = dv / c; residual rows F_G and F_R,g divided
// by E_tot, F_F,g by c E_tot.  The step is left in a second workspace (U,
// FP32) beside the FP32 iterate (W); the FP64 passes start from W + U, which
// together carry the corrected iterate to FP64 precision.
#pragma once
#include "rhd_warp32.cuh"

namespace rhd {

// The correction kernel's output for the cells it does not finish: the
// accumulated step (r_g, f_g) from the FP32 iterate, and per cell whether the
// cell is finished (1: its final state is written; the FP64 passes skip it).
struct CorrOut {
  float *ur;      // [G][n]
  float *uf;      // [3][G][n]
  uint8_t *done;  // [n]
  int from_step;  // 1: ur, uf already hold a step from the FP32 iterate (rhd_refine.cuh),
                  // and the correction starts from the FP32 iterate plus that step
};

// The closure in units with c = 1 (E, F / c, v / c): v.P, M = d(v.P)/dF at
// fixed E, dE = d(v.P)/dE at fixed F, and P itself (d(v.P)/dv).  M1 as in
// closure_vP_jac (Levermore's chi(f), f held at 1); Eddington P = E/3 I.
__device__ __forceinline__ void closure_full32(int closure, float E, const float F[3],
                                               const float v[3], float vP[3], float M[9],
                                               float Pm[9], float dE[3]) {
  const float fn2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
  if (closure != RHD_M1 || !(E > 0.0f) || !(fn2 > 0.0f)) {
    const float e3 = E * (1.0f / 3.0f);
    for (int k = 0; k < 3; ++k) {
      vP[k] = e3 * v[k];
      dE[k] = v[k] * (1.0f / 3.0f);
    }
    for (int k = 0; k < 9; ++k) {
      M[k] = 0.0f;
      Pm[k] = (k % 4 == 0) ? e3 : 0.0f;
    }
    return;
  }
  const float fn = sqrtf(fn2), inv = 1.0f / fn;
  float f = fn / E;
  const bool held = f > 1.0f;
  if (held) f = 1.0f;
  const float f2 = f * f;
  const float sq = sqrtf(4.0f - 3.0f * f2), num = 3.0f + 4.0f * f2, den = 5.0f + 2.0f * sq;
  const float chi = num / den;
  const float dchi = held ? 0.0f : (8.0f * f * den + 6.0f * f * num / sq) / (den * den);
  const float iso = 0.5f * (1.0f - chi), dir = 0.5f * (3.0f * chi - 1.0f);
  const float n[3] = {F[0] * inv, F[1] * inv, F[2] * inv};
  const float vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  const float a = -0.5f * dchi, b = 1.5f * dchi * vn, e = E * dir * inv;
  // dE: d/dE of E (iso v + dir vn n) at fixed F, with df/dE = -f/E
  const float ie = iso + 0.5f * f * dchi, de = dir - 1.5f * f * dchi;
  for (int r = 0; r < 3; ++r) {
    vP[r] = E * (iso * v[r] + dir * vn * n[r]);
    dE[r] = ie * v[r] + de * vn * n[r];
    for (int q = 0; q < 3; ++q) {
      const float id = r == q ? 1.0f : 0.0f;
      M[3 * r + q] = a * v[r] * n[q] + b * n[r] * n[q] +
                     e * (n[r] * (v[q] - vn * n[q]) + vn * (id - n[r] * n[q]));
      Pm[3 * r + q] = E * (iso * id + dir * n[r] * n[q]);
    }
  }
}

// One group's block of the bordered system, u = (r_g, f_g):
//   [A00 A0^T] u = rhs - c x - B beta
//   [Af0 Aff ]
// eliminated through its (r_g) row (A00 <= -1 never vanishes): the 3x3 Schur
// complement K = Aff - Af0 A0^T / A00 is inverted by its adjugate.  Output:
// u = p + q x + S beta (S row-major 4x3).  false when K is singular.
struct GBlock {
  float p[4], q[4], S[12];
};

__device__ __forceinline__ bool group_block(float A00, const float A0[3], const float Af0[3],
                                            const float Aff[9], float c0, const float cF[3],
                                            const float B0[3], const float BF[9], float rhs0,
                                            const float rhsF[3], GBlock &o) {
  const float ia = 1.0f / A00;
  float K[9];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) K[3 * r + q] = Aff[3 * r + q] - Af0[r] * A0[q] * ia;
  const float k00 = K[4] * K[8] - K[5] * K[7], k01 = K[2] * K[7] - K[1] * K[8],
              k02 = K[1] * K[5] - K[2] * K[4];
  const float k10 = K[5] * K[6] - K[3] * K[8], k11 = K[0] * K[8] - K[2] * K[6],
              k12 = K[2] * K[3] - K[0] * K[5];
  const float k20 = K[3] * K[7] - K[4] * K[6], k21 = K[1] * K[6] - K[0] * K[7],
              k22 = K[0] * K[4] - K[1] * K[3];
  const float det = K[0] * k00 + K[1] * k10 + K[2] * k20;
  if (!(fabsf(det) > 1e-30f) || !isfinite(det)) return false;
  const float id = 1.0f / det;
  const float Ki[9] = {k00 * id, k01 * id, k02 * id, k10 * id, k11 * id,
                       k12 * id, k20 * id, k21 * id, k22 * id};
  auto col = [&](float t0, const float tF[3], float &o0, float o1[3]) {
    // solve [A00 A0; Af0 Aff] y = (t0, tF)
    const float s[3] = {tF[0] - Af0[0] * t0 * ia, tF[1] - Af0[1] * t0 * ia,
                        tF[2] - Af0[2] * t0 * ia};
    for (int r = 0; r < 3; ++r) o1[r] = Ki[3 * r] * s[0] + Ki[3 * r + 1] * s[1] + Ki[3 * r + 2] * s[2];
    o0 = (t0 - A0[0] * o1[0] - A0[1] * o1[1] - A0[2] * o1[2]) * ia;
  };
  float y1[3];
  col(rhs0, rhsF, o.p[0], y1);
  o.p[1] = y1[0];
  o.p[2] = y1[1];
  o.p[3] = y1[2];
  const float ncF[3] = {-cF[0], -cF[1], -cF[2]};
  col(-c0, ncF, o.q[0], y1);
  o.q[1] = y1[0];
  o.q[2] = y1[1];
  o.q[3] = y1[2];
  for (int l = 0; l < 3; ++l) {
    const float nB[3] = {-BF[l], -BF[3 + l], -BF[6 + l]};
    col(-B0[l], nB, o.S[l], y1);
    o.S[3 + l] = y1[0];
    o.S[6 + l] = y1[1];
    o.S[9 + l] = y1[2];
  }
  return true;
}

// The FP32 Jacobian block of one group at the iterate, with the FP64
// residual (scaled) as right-hand side.  Edge values (P or Q, D, x dD/dx) at
// the lower (L) and upper (U) edge at the iterate's T; aT4s = a_R T^4 / E_tot,
// dTs = a_R T^3 / (rho c_v) (d/dx of the scaled Planck terms per unit x);
// tau = c_hat theta dt chi_E (0: the group is uncoupled); Eg = E_g / E_tot;
// f = F_g / (c E_tot); be = v / c.
__device__ __forceinline__ bool group_jac32(int closure, float tau, float a, float rm, float rp,
                                            float pqL, bool lowL, float dL, float eL, float pqU,
                                            bool lowU, float dU, float eU, float aT4s, float dTs,
                                            float Eg, const float f[3], const float be[3],
                                            float rR, const float rF[3], GBlock &o) {
  const float rhsF[3] = {-rF[0], -rF[1], -rF[2]};
  if (!(tau > 0.0f)) {  // uncoupled: R_g = 0, F_g = F_g^t, no coupling
    const float z3[3] = {0.0f, 0.0f, 0.0f};
    const float I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const float z9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    return group_block(-1.0f, z3, z3, I9, 0.0f, z3, z3, z9, -rR, rhsF, o);
  }
  const float dP = band_fp32(pqL, lowL, pqU, lowU);
  const float dD = dU - dL;
  const float b = aT4s * dP;
  const float dbs = dTs * (4.0f * dP - dD);
  float dq;
  const float q = chiF_ratio<float>(b, aT4s, dD, a, rm, rp, dL, dU, dbs, dTs, eL, eU, dq);
  const float X = rp * dU - rm * dL;
  const float s = b - aT4s * X * (1.0f / 3.0f);                       // (chi_B b - dchi/3) / chi_E
  const float ds = dbs - dTs * (4.0f * X - (rp * eU - rm * eL)) * (1.0f / 3.0f);
  const float inv = 1.0f / (1.0f + tau * q);
  const float kap = (1.0f + a) * tau * inv;
  const float a1 = (1.0f + a) * q;
  float vP[3], M[9], Pm[9], dE[3];
  closure_full32(closure, Eg, f, be, vP, M, Pm, dE);
  const float w = be[0] * f[0] + be[1] * f[1] + be[2] * f[2];
  const float A0[3] = {a1 * be[0], a1 * be[1], a1 * be[2]};
  const float Af0[3] = {-kap * dE[0], -kap * dE[1], -kap * dE[2]};
  float Aff[9], BF[9];
  const float ts = inv * tau * s;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      Aff[3 * r + c] = (r == c ? 1.0f : 0.0f) - kap * M[3 * r + c];
      BF[3 * r + c] = -((r == c ? ts : 0.0f) + kap * Pm[3 * r + c]);
    }
  const float c0 = dbs + (1.0f + a) * dq * w;
  // d F_F / dx: through chi_F (q) in both the denominator and kap, and
  // through the source term; base + kap v.P is F_g at the root
  const float cF[3] = {inv * tau * (dq * f[0] - be[0] * ds), inv * tau * (dq * f[1] - be[1] * ds),
                       inv * tau * (dq * f[2] - be[2] * ds)};
  const float B0[3] = {a1 * f[0], a1 * f[1], a1 * f[2]};
  return group_block(-(1.0f + 1.0f / tau), A0, Af0, Aff, c0, cF, B0, BF, -rR, rhsF, o);
}

// The 4x4 system in (x, beta) after the groups are eliminated:
//   (1 + cr sum q_R) x + (m c / E_tot + cr sum S_R) . beta = -F_G / E_tot - cr sum p_R
//   mu sum q_F x + (I + mu sum S_F) beta = -mu sum p_F,   mu = E_tot / (rho c c_hat)
// sums: [0] p_R, [1] q_R, [2..4] S_R, [5..7] p_F, [8..10] q_F, [11..19] S_F.
// Gaussian elimination with partial pivoting; false if singular.
__device__ __forceinline__ bool global_solve(const float s[20], float rG, float cr,
                                             const float mc[3], float mu, float &x,
                                             float beta[3]) {
  float A[4][5];
  A[0][0] = 1.0f + cr * s[1];
  for (int k = 0; k < 3; ++k) A[0][1 + k] = mc[k] + cr * s[2 + k];
  A[0][4] = -rG - cr * s[0];
  for (int r = 0; r < 3; ++r) {
    A[1 + r][0] = mu * s[8 + r];
    for (int k = 0; k < 3; ++k) A[1 + r][1 + k] = (r == k ? 1.0f : 0.0f) + mu * s[11 + 3 * r + k];
    A[1 + r][4] = -mu * s[5 + r];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabsf(A[r][c]) > fabsf(A[piv][c])) piv = r;
    if (!(fabsf(A[piv][c]) > 0.0f)) return false;
    if (piv != c)
      for (int k = 0; k < 5; ++k) {
        const float t = A[c][k];
        A[c][k] = A[piv][k];
        A[piv][k] = t;
      }
    const float ip = 1.0f / A[c][c];
    for (int r = c + 1; r < 4; ++r) {
      const float fct = A[r][c] * ip;
      for (int k = c; k < 5; ++k) A[r][k] -= fct * A[c][k];
    }
  }
  float y[4];
  for (int r = 3; r >= 0; --r) {
    float t = A[r][4];
    for (int k = r + 1; k < 4; ++k) t -= A[r][k] * y[k];
    y[r] = t / A[r][r];
  }
  x = y[0];
  beta[0] = y[1];
  beta[1] = y[2];
  beta[2] = y[3];
  return isfinite(x) && isfinite(beta[0]) && isfinite(beta[1]) && isfinite(beta[2]);
}

// Dynamic shared memory of the correction kernel: the group table, then
// GPL * 20 floats per thread for the group blocks.
__host__ __device__ __forceinline__ size_t correct_smem_bytes(int G, int GPL, int threads) {
  return ((table_bytes(G) + 15) & ~(size_t)15) + sizeof(float) * 20 * GPL * threads;
}
__device__ __forceinline__ float *correct_blocks(double *sm, int G) {
  return reinterpret_cast<float *>(reinterpret_cast<char *>(sm) + ((table_bytes(G) + 15) & ~(size_t)15));
}

// A step is taken only when it is small against the cell's energy scale:
// the FP32 passes leave the iterate at FP32 accuracy, so a larger step means
// they stopped at a cap, and the FP64 passes take the cell from there.
constexpr float kMaxStep = 1e-2f;
// Newton steps on the coupled system before a cell is left to the FP64 passes.
constexpr int kMaxCorrections = 3;

// The cell's state and iterate of the correction kernel, per lane: groups
// g = l + L j (the layout of rhd_warp.cuh).
template <int GPL>
struct CCell {
  double E0[GPL], R[GPL], F[GPL][3], ft[GPL][3];  // E^t + S, iterate, F^t
  float rw[GPL], fw[GPL][3];                       // the FP32 iterate (scaled)
  float rR[GPL], rF[GPL][3], q[GPL], qe[GPL];      // scaled residual, chi_F/chi_E, tau/(1+tau)
};

// The correction step with L lanes per cell: from the FP32 passes' iterate
// (W), Newton steps on the coupled system -- each an FP64 evaluation of the
// residual followed, unless the paper's tests already hold, by an FP32
// Jacobian step -- until the paper's inner test (after eq. matrix) and outer
// test (the change one more outer pass would make, readings of Sec. 3) hold
// on the FP64 residual.  A cell that meets them is finished here exactly as
// an FP64 pass finishes it: each R_g from its own row, the flux update of
// eq. numF1, the conservative write-back of E_g, E_gas and the momentum in
// FP64.  Any other cell is left to the FP64 passes with its iterate in
// W + U.
// The correction step of cell i with L lanes (lane = the thread's lane in
// its warp; the cell's segment is lanes lane0 .. lane0 + L - 1), gb this
// warp's slice of the group blocks in shared memory.
template <int L, int GPL>
__device__ __forceinline__ void correct_cell(const KParams &P, const GroupTable &tab,
                                             const WarmOut &W, const CorrOut &U, float *gb,
                                             int64_t i, int lane, CCell<GPL> &C) {
  constexpr int NE = GPL + 1;
  const int seg = lane / L, l = lane % L, lane0 = seg * L;
  const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << lane0);
  const int G = P.G;
  const int64_t n = P.n;
  const double c = P.c, tdt = P.c_hat * P.theta * P.dt;
  const int src_lane = lane0 + (l + 1) % L;
  const float tol = (float)P.tol, tol_o = (float)P.tol_outer, crf = (float)P.cr;
  // ---- the cell, validated as the FP64 passes validate it; an invalid
  // cell or one without an FP32 iterate is left to them
  const double Eint0 = W.eint[i];
  const double rho = P.rho[i];
  const double k0 = P.kappa0 ? P.kappa0[i] : 1.0;
  const double m0[3] = {P.mom[0][i], P.mom[1][i], P.mom[2][i]};
  const double eg0 = P.egas[i];
  bool valid = Eint0 > 0.0 && rho > 0.0 && isfinite(rho) && isfinite(eg0) && isfinite(k0) &&
               k0 >= 0.0 && isfinite(m0[0]) && isfinite(m0[1]) && isfinite(m0[2]);
  valid = valid && eg0 - 0.5 * (m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2]) / rho > 0.0;
  double sumE0 = 0.0;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    C.E0[j] = 0.0;
    C.rw[j] = 0.0f;
    for (int d = 0; d < 3; ++d) {
      C.fw[j][d] = 0.0f;
      C.ft[j][d] = 0.0;
    }
    if (g < G && valid) {
      const int64_t o = (int64_t)g * P.gs + i;
      const double e = P.erad[o], sg = P.src ? P.src[o] : 0.0;
      C.E0[j] = e + sg;
      valid = valid && isfinite(e) && isfinite(sg);
      sumE0 += C.E0[j];
      const int64_t ow = (int64_t)g * n + i;
      C.rw[j] = W.r[ow];
      for (int d = 0; d < 3; ++d) {
        C.ft[j][d] = P.frad[d][o];
        valid = valid && isfinite(C.ft[j][d]);
        C.fw[j][d] = W.f[(int64_t)d * G * n + ow];
      }
    }
  }
  if (!__all_sync(mask, valid)) {
    if (l == 0) U.done[i] = 0;
    return;
  }
  sumE0 = seg_sum<L>(sumE0, mask);
  const double Et = eg0 + P.cr * sumE0;
  int shE;
  const float imE = 1.0f / frexp_f(Et, shE);
  const float imEc = imE * (float)P.ic;
  const double fs = c * Et;
  // the iterate in FP64 (the FP32 iterate, plus the refinement step when it ran)
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    if (U.from_step && l + L * j < G) {
      const int64_t ow = (int64_t)(l + L * j) * n + i;
      C.R[j] = fma(f2d(C.rw[j]), Et, f2d(U.ur[ow]) * Et);
      for (int d = 0; d < 3; ++d)
        C.F[j][d] = fma(f2d(C.fw[j][d]), fs, f2d(U.uf[(int64_t)d * G * n + ow]) * fs);
    } else {
      C.R[j] = f2d(C.rw[j]) * Et;
      for (int d = 0; d < 3; ++d) C.F[j][d] = f2d(C.fw[j][d]) * fs;
    }
  }
  double Eint = Eint0;
  const double irho = 1.0 / rho;
  const double rcv = rho * P.c_v, irc = 1.0 / rcv;
  int shV;
  const float imV = 1.0f / frexp_f(rho * c, shV);
  const float mu = scaled_f(Et * irho * P.icc, 0);  // E_tot / (rho c c_hat)
  double cs = rho * k0;  // rho kappa0 (T/T_ref)^p
  double its = (tdt * cs > 0.0) ? 1.0 / (tdt * cs) : 0.0;
  int et = 0;
  float mt = tdt * cs > 0.0 ? frexp_f(tdt * cs, et) : 0.0f;  // c_hat theta dt cs = mt 2^et
  int nit = W.nit[i], steps = 0, nres = 0;
  bool finished = false, ok = true;
  for (int k = 0; k <= kMaxCorrections; ++k) {
    ++nres;
    // ---- FP64 residual at the iterate: its momentum (eq. vupdate) and the
    // sum of R_g, summed exactly
    double dF[3] = {0.0, 0.0, 0.0}, sumR = 0.0;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      if (l + L * j >= G) continue;
      sumR += C.R[j];
      for (int d = 0; d < 3; ++d) dF[d] += C.F[j][d] - C.ft[j][d];
    }
    for (int d = 0; d < 3; ++d) dF[d] = seg_sum<L>(dF[d], mask);
    sumR = seg_sum<L>(sumR, mask);
    const double m[3] = {m0[0] - dF[0] * P.icc, m0[1] - dF[1] * P.icc, m0[2] - dF[2] * P.icc};
    const double v[3] = {m[0] * irho, m[1] * irho, m[2] * irho};
    const double KE = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) * irho;
    const double T = Eint * irc;
    if (P.temp_exp != 0.0) {  // the opacity scale follows T (otherwise set once per cell)
      cs = rho * k0 * pow(T / P.T_ref, P.temp_exp);
      its = (tdt * cs > 0.0) ? 1.0 / (tdt * cs) : 0.0;
      mt = tdt * cs > 0.0 ? frexp_f(tdt * cs, et) : 0.0f;
    }
    const double aT3 = P.a_rad * T * T * T, aT4 = aT3 * T;
    const double invT = 1.0 / T;
    double pqE[NE], dE_[NE], eE[NE];
    bool lowE[NE];
#pragma unroll
    for (int jj = 0; jj < NE; ++jj) {
      const int e = l + L * jj;
      if (jj == NE - 1 && G == L * GPL) {  // the top edge alone (see winner_step)
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
    // the same edge values in FP32 for the Jacobian (bit-pattern cut, no FP64 instruction)
    float pqF[NE], dF_[NE], eF[NE];
    bool lowF[NE];
#pragma unroll
    for (int jj = 0; jj < NE; ++jj) {
      pqF[jj] = scaled_f(pqE[jj], 0);
      dF_[jj] = scaled_f(dE_[jj], 0);
      eF[jj] = scaled_f(eE[jj], 0);
      lowF[jj] = lowE[jj];
    }
    const float be[3] = {scaled_f(m[0], shV) * imV, scaled_f(m[1], shV) * imV,
                         scaled_f(m[2], shV) * imV};
    float sabs = 0.0f, sdf[3] = {0.0f, 0.0f, 0.0f}, sfl = 0.0f;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const double pa = __shfl_sync(mask, pqE[j], src_lane), pb = __shfl_sync(mask, pqE[j + 1], src_lane);
      const double da = __shfl_sync(mask, dE_[j], src_lane), db_ = __shfl_sync(mask, dE_[j + 1], src_lane);
      const int la = __shfl_sync(mask, (int)lowE[j], src_lane),
                lb = __shfl_sync(mask, (int)lowE[j + 1], src_lane);
      const bool last = l == L - 1;
      const double pqU = last ? pb : pa, dU = last ? db_ : da;
      const bool lowU = (last ? lb : la) != 0;
      const int g = l + L * j;
      C.rR[j] = 0.0f;
      C.rF[j][0] = C.rF[j][1] = C.rF[j][2] = 0.0f;
      C.q[j] = 0.0f;
      C.qe[j] = 0.0f;
      if (g >= G) continue;
      const double dP = band_fp64(pqE[j], lowE[j], pqU, lowU);
      const double dD = dU - dE_[j];
      const double b = aT4 * dP;
      const double a = tab.alpha[g], rm = tab.rm[g], rp = tab.rp[g];
      const double q = chiF_q<double>(b, aT4, dD, a, rm, rp, dE_[j], dU);
      const double dnx = aT4 * (rp * dU - rm * dE_[j]);
      const double chiB = cs * tab.kbar[g];
      const double Enew = C.E0[j] + C.R[j];
      const double w = (v[0] * C.F[j][0] + v[1] * C.F[j][1] + v[2] * C.F[j][2]) * P.inv_c2;
      const double FR = chiB > 0.0 ? b + (1.0 + a) * q * w - C.R[j] * its * tab.ikbar[g] - Enew
                                   : -C.R[j];
      // the flux residual F - (eq. numF1 at this iterate), as wouter_end forms it
      double ca, kn, kd;
      closure_vP_parts<double>(P.closure, c, P.ic, Enew, C.F[j][0], C.F[j][1], C.F[j][2], v[0],
                               v[1], v[2], ca, kn, kd);
      const double srcg = chiB * (b - dnx * (1.0 / 3.0));
      const double den = 1.0 + tdt * chiB * q;
      const double dk = den * kd;
      double inv, kf;
      if (dk > 1e-290) {
        const double rr = 1.0 / dk;
        inv = kd * rr;
        kf = kn * den * rr;
      } else {
        inv = 1.0 / den;
        kf = kn / kd;
      }
      const double kap = tdt * (1.0 + a) * chiB * inv;
      C.rR[j] = scaled_f(FR, shE) * imE;
      for (int d = 0; d < 3; ++d) {
        const double vp = ca * v[d] + kf * C.F[j][d];
        // eq. numF1 at the iterate: the cell's flux if this evaluation finishes
        // it (the state's array holds it meanwhile; F^t stays in C.ft)
        const double Fn = (C.ft[j][d] + tdt * v[d] * srcg) * inv + kap * vp;
        P.frad[d][(int64_t)g * P.gs + i] = Fn;
        const double FF = C.F[j][d] - Fn;
        C.rF[j][d] = scaled_f(FF, shE) * imEc;
        sdf[d] += C.rF[j][d];
        sfl += fabsf(C.rF[j][d]);
      }
      const float tau = mt * scaled_f(tab.kbar[g], -et);
      C.q[j] = scaled_f(q, 0);
      C.qe[j] = tau > 0.0f ? tau / (1.0f + tau) : 0.0f;
      sabs += fabsf(C.rR[j]);
    }
    // ---- the paper's tests on this residual: the inner test, and the
    // outer test on the change one more outer pass would make (fluxes
    // F - F_F, momentum and kinetic energy from them, the v.F terms of R_g
    // after the implicit solve), taken to first order in the change
    const double FG = Eint + KE - eg0 + P.cr * sumR;
    sabs = seg_sumf<L>(sabs, mask);
    for (int d = 0; d < 3; ++d) sdf[d] = seg_sumf<L>(sdf[d], mask);
    const float db[3] = {mu * sdf[0], mu * sdf[1], mu * sdf[2]};  // d(v/c)
    const float cf = (float)c;
    const float mc[3] = {scaled_f(m[0], shE) * imE * cf, scaled_f(m[1], shE) * imE * cf,
                         scaled_f(m[2], shE) * imE * cf};  // m c / E_tot
    float cg = 0.0f;
    bool gok = true;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const int g = l + L * j;
      if (g >= G) continue;
      float dw = 0.0f;
      for (int d = 0; d < 3; ++d)
        dw += db[d] * (C.fw[j][d] - C.rF[j][d]) - be[d] * C.rF[j][d];
      const float cgg = fabsf((1.0f + tab.alphaf[g]) * C.q[j] * dw) * C.qe[j];
      cg += cgg;
      if (P.flags & RHD_GROUP_TEST) {
        const float e0 = scaled_f(C.E0[j], shE) * imE;
        gok = gok && cgg <= tol_o * (fabsf(e0) + fabsf(e0 + C.rw[j]));
      }
    }
    float chg = fabsf(mc[0] * db[0] + mc[1] * db[1] + mc[2] * db[2]) + seg_sumf<L>(cg, mask);
    if (P.flags & RHD_FLUX_TEST) chg += seg_sumf<L>(sfl, mask);
    gok = __all_sync(mask, gok);
    if (fabs(FG) < P.tol * Et && crf * sabs < tol && chg <= tol_o && gok) {
      finished = true;
      break;
    }
    if (k == kMaxCorrections || !ok) break;
    // ---- FP32 Jacobian at the iterate, group blocks, sums, the step
    const float rG = scaled_f(FG, shE) * imE;
    const float eint = scaled_f(Eint, shE) * imE;
    const float aT4s = scaled_f(aT4, shE) * imE;
    const float dTs = aT4s / eint;
    float sums[20];
    for (int t = 0; t < 20; ++t) sums[t] = 0.0f;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const float pa = __shfl_sync(mask, pqF[j], src_lane), pb = __shfl_sync(mask, pqF[j + 1], src_lane);
      const float da = __shfl_sync(mask, dF_[j], src_lane), db_ = __shfl_sync(mask, dF_[j + 1], src_lane);
      const float ea = __shfl_sync(mask, eF[j], src_lane), eb = __shfl_sync(mask, eF[j + 1], src_lane);
      const int la = __shfl_sync(mask, (int)lowF[j], src_lane),
                lb = __shfl_sync(mask, (int)lowF[j + 1], src_lane);
      const bool last = l == L - 1;
      const int g = l + L * j;
      if (g >= G) {
        for (int t = 0; t < 20; ++t) gb[(j * 20 + t) * 32 + lane] = 0.0f;
        continue;
      }
      const float tau = mt * scaled_f(tab.kbar[g], -et);
      const float Eg = scaled_f(C.E0[j] + C.R[j], shE) * imE;
      const float fcur[3] = {scaled_f(C.F[j][0], shE) * imEc, scaled_f(C.F[j][1], shE) * imEc,
                             scaled_f(C.F[j][2], shE) * imEc};
      GBlock blk;
      ok = group_jac32(P.closure, tau, tab.alphaf[g], tab.rmf[g], tab.rpf[g], pqF[j], lowF[j],
                       dF_[j], eF[j], last ? pb : pa, (last ? lb : la) != 0, last ? db_ : da,
                       last ? eb : ea, aT4s, dTs, Eg, fcur, be, C.rR[j], C.rF[j], blk) && ok;
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
    float x = 0.0f, beta[3] = {0.0f, 0.0f, 0.0f};
    ok = global_solve(sums, rG, crf, mc, mu, x, beta) && ok;
    ok = ok && fabsf(x) < kMaxStep;
    float u[GPL][4];
#pragma unroll
    for (int j = 0; j < GPL; ++j)
      for (int t = 0; t < 4; ++t) {
        u[j][t] = gb[(j * 20 + t) * 32 + lane] + gb[(j * 20 + 4 + t) * 32 + lane] * x +
                  gb[(j * 20 + 8 + 3 * t) * 32 + lane] * beta[0] +
                  gb[(j * 20 + 9 + 3 * t) * 32 + lane] * beta[1] +
                  gb[(j * 20 + 10 + 3 * t) * 32 + lane] * beta[2];
        ok = ok && fabsf(u[j][t]) < kMaxStep;
      }
    ok = __all_sync(mask, ok);
    if (!ok) break;  // the iterate stays the last good one
    // ---- take the step (FP64)
    Eint += f2d(x) * Et;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      if (l + L * j >= G) continue;
      C.R[j] += f2d(u[j][0]) * Et;
      for (int d = 0; d < 3; ++d) C.F[j][d] += f2d(u[j][1 + d]) * fs;
    }
    ++nit;
    ++steps;
  }
  if (l == 0) {
    count_event(P, RHD_EV_CELLSC, 1);
    count_event(P, RHD_EV_RESID64, nres);
    count_event(P, RHD_EV_STEP32, steps);
    count_event(P, RHD_EV_FINISH64, finished ? 1 : 0);
  }
  if (finished) {
    // ---- the end of a converged pass, as the FP64 passes end it: each
    // R_g from its own row, the flux update (F - F_F), the conservative
    // write-back of E_g, E_gas and the momentum in FP64
    double sR = 0.0, sF[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const int g = l + L * j;
      if (g >= G) continue;
      const double R = C.R[j] + f2d(C.rR[j] * C.qe[j]) * Et;
      const int64_t o = (int64_t)g * P.gs + i;
      P.erad[o] = C.E0[j] + R;
      sR += R;
      for (int d = 0; d < 3; ++d) sF[d] += P.frad[d][o] - C.ft[j][d];
    }
    sR = seg_sum<L>(sR, mask);
    for (int d = 0; d < 3; ++d) sF[d] = seg_sum<L>(sF[d], mask);
    if (l == 0) {
      P.egas[i] = eg0 - P.cr * sR;
      for (int d = 0; d < 3; ++d) P.mom[d][i] = m0[d] - sF[d] * P.icc;
      if (P.status) P.status[i] = RHD_STATUS_OK;
      if (P.iters) P.iters[i] = (uint8_t)(nit > 255 ? 255 : nit);
      U.done[i] = 1;
    }
    return;
  }
  // ---- not finished: the FP64 passes start from W + U (the FP32 iterate
  // and the steps taken here and by the refinement; none when no step was
  // taken), from F^t
  const bool moved = steps || U.from_step;
#pragma unroll
  for (int j = 0; j < GPL; ++j) {
    const int g = l + L * j;
    if (g >= G) continue;
    for (int d = 0; d < 3; ++d) P.frad[d][(int64_t)g * P.gs + i] = C.ft[j][d];
    if (!steps && U.from_step) continue;  // U holds the refinement's step already
    const int64_t o = (int64_t)g * n + i;
    U.ur[o] = steps ? scaled_f(C.R[j] - f2d(C.rw[j]) * Et, shE) * imE : 0.0f;
    for (int d = 0; d < 3; ++d)
      U.uf[(int64_t)d * G * n + o] =
          steps ? scaled_f(C.F[j][d] - f2d(C.fw[j][d]) * fs, shE) * imEc : 0.0f;
  }
  double dF[3] = {0.0, 0.0, 0.0};
  if (moved) {
#pragma unroll
    for (int j = 0; j < GPL; ++j)
      if (l + L * j < G)
        for (int d = 0; d < 3; ++d) dF[d] += C.F[j][d] - C.ft[j][d];
    for (int d = 0; d < 3; ++d) dF[d] = seg_sum<L>(dF[d], mask);
  }
  if (l == 0) {
    if (moved) {
      W.eint[i] = Eint;
      for (int d = 0; d < 3; ++d) W.mom[(int64_t)d * n + i] = m0[d] - dF[d] * P.icc;
      W.nit[i] = (uint8_t)(nit > 255 ? 255 : nit);
    }
    U.done[i] = 0;
  }
}

// Warp w's slice of the group blocks (p, q, S: 20 floats per group slot,
// lane-fastest: no bank conflicts) that a cell keeps in shared memory between
// the elimination and the step; blocks is the CTA's first slice.
template <int GPL>
__device__ __forceinline__ float *warp_blocks(float *blocks, int w) {
  return blocks + w * (GPL * 20 * 32);
}

template <int L, int GPL>
__global__ void __launch_bounds__(128) correct_warp_kernel(const __grid_constant__ KParams P,
                                                           const WarmOut W, const CorrOut U) {
  extern __shared__ double sm[];
  const GroupTable tab = build_table(P, sm);
  const int lane = threadIdx.x & 31, seg = lane / L;
  float *gb = warp_blocks<GPL>(correct_blocks(sm, P.G), threadIdx.x / 32);
  constexpr int CPW = 32 / L;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  CCell<GPL> C;
  for (int64_t i = warp * CPW + seg; i < P.n; i += nwarps * CPW)
    correct_cell<L, GPL>(P, tab, W, U, gb, i, lane, C);
}

}  // namespace rhd
