/* rhd_oracle.c -- FP64 CPU oracle (test infrastructure only; see rhd_oracle.h).
 *
 * Plain and slow on purpose: every formula is written out as the paper states
 * it, the implicit system is solved as a whole by a generic Newton method with
 * a finite-difference Jacobian and a dense partial-pivot LU, and nothing is
 * blocked, fused or reordered.  Compile with -ffp-contract=off (round to
 * nearest, no FMA contraction).
 */
#include "rhd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Planck integrals                                                          */
/* ------------------------------------------------------------------------ */
/* Normalisation: 4 pi B_nu / c integrates to a_R T^4 over all frequencies, so
 * with x = h nu / (k_B T)
 *   4 pi B_nu / c dnu = a_R T^4 (15/pi^4) x^3/(e^x - 1) dx.
 * P(x) is the fraction of a_R T^4 below x.  Two series (Widger & Woodall
 * 1976, Bull. Am. Meteorol. Soc. 57, 1217):
 *   small x: int_0^x t^3/(e^t-1) dt = sum_k B_k x^(k+3) / (k! (k+3))
 *            (generating function t/(e^t-1) = sum_k B_k t^k / k!, Bernoulli B_k)
 *   large x: int_x^inf t^3/(e^t-1) dt
 *            = sum_n e^(-n x) (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4).
 * The even Bernoulli numbers are taken from B_2j = (-1)^(j+1) 2 (2j)! zeta(2j)
 * / (2 pi)^(2j), so the small-x coefficient of x^(2j+3) is
 *   c_j = (-1)^(j+1) 2 zeta(2j) / ((2 pi)^(2j) (2j+3)).                     */
#define ORC_NBERN 48
static double orc_bern_c[ORC_NBERN + 1];
static int orc_bern_ready = 0;

static void orc_init_series(void) {
  if (orc_bern_ready) return;
  for (int j = 1; j <= ORC_NBERN; ++j) {
    double zeta;
    if (j == 1) {
      zeta = ORC_PI * ORC_PI / 6.0;
    } else if (j == 2) {
      zeta = ORC_PI * ORC_PI * ORC_PI * ORC_PI / 90.0;
    } else {
      /* direct sum; the tail beyond n = 2000 is below 2000^(1-2j)/(2j-1) */
      zeta = 0.0;
      for (int n = 2000; n >= 1; --n) zeta += pow((double)n, -2.0 * j);
    }
    double sign = (j % 2 == 1) ? 1.0 : -1.0;
    orc_bern_c[j] = sign * 2.0 * zeta / (pow(2.0 * ORC_PI, 2.0 * j) * (2.0 * j + 3.0));
  }
  orc_bern_ready = 1;
}

static double orc_norm15(void) { return 15.0 / (ORC_PI * ORC_PI * ORC_PI * ORC_PI); }

/* int_0^x t^3/(e^t-1) dt for 0 <= x < 2 */
static double orc_lower_integral(double x) {
  double x2 = x * x, x3 = x2 * x;
  double sum = x3 / 3.0 - x3 * x / 8.0;
  double pw = x3 * x2; /* x^(2j+3), j = 1 */
  for (int j = 1; j <= ORC_NBERN; ++j) {
    double term = orc_bern_c[j] * pw;
    sum += term;
    if (fabs(term) < 1e-20 * fabs(sum)) break;
    pw *= x2;
  }
  return sum;
}

/* int_x^inf t^3/(e^t-1) dt for x >= 2 */
static double orc_upper_integral(double x) {
  double sum = 0.0;
  double e1 = exp(-x), en = 1.0;
  for (int n = 1; n <= 200; ++n) {
    en *= e1;
    double dn = (double)n;
    double term = en * (x * x * x / dn + 3.0 * x * x / (dn * dn) + 6.0 * x / (dn * dn * dn) +
                        6.0 / (dn * dn * dn * dn));
    sum += term;
    if (term < 1e-20 * sum) break;
  }
  return sum;
}

double orc_planck_P(double x) {
  orc_init_series();
  if (!(x > 0.0)) return 0.0;
  if (isinf(x)) return 1.0;
  if (x < 2.0) return orc_norm15() * orc_lower_integral(x);
  return 1.0 - orc_norm15() * orc_upper_integral(x);
}

double orc_planck_Q(double x) {
  orc_init_series();
  if (!(x > 0.0)) return 1.0;
  if (isinf(x)) return 0.0;
  if (x < 2.0) return 1.0 - orc_norm15() * orc_lower_integral(x);
  return orc_norm15() * orc_upper_integral(x);
}

double orc_planck_band(double x0, double x1) {
  /* the complement difference avoids 1 - 1 cancellation in the Wien tail */
  if (x0 >= 2.0) return orc_planck_Q(x0) - orc_planck_Q(x1);
  return orc_planck_P(x1) - orc_planck_P(x0);
}

/* (15/pi^4) x^4 / (e^x - 1): the value of nu * 4 pi B_nu / c per a_R T^4 */
static double orc_nu_B(double x) {
  if (!(x > 0.0) || isinf(x)) return 0.0;
  if (x > 700.0) return orc_norm15() * x * x * x * x * exp(-x);
  return orc_norm15() * x * x * x * x / expm1(x);
}

/* ------------------------------------------------------------------------ */
/* PPL mean opacities (Sec. 2.2.2, eq. chiQg)                                */
/* ------------------------------------------------------------------------ */
/* (r^a - 1)/a, and ln r at a = 0 (the special case named after eq. chiQg) */
static double orc_pow_bracket(double a, double r) {
  double lr = log(r);
  double z = a * lr;
  if (z == 0.0) return lr;
  if (fabs(z) < 1e-5) return lr * (1.0 + z / 2.0 + z * z / 6.0 + z * z * z / 24.0);
  return expm1(z) / a;
}

double orc_ppl_mean_opacity(double chi_minus, double alpha_chi, double alpha_Q, double r) {
  return chi_minus * orc_pow_bracket(alpha_chi + alpha_Q + 1.0, r) /
         orc_pow_bracket(alpha_Q + 1.0, r);
}

/* ------------------------------------------------------------------------ */
/* Group table from a piecewise-powerlaw opacity law                         */
/* ------------------------------------------------------------------------ */
static double orc_law_logk(double nu, int right, int32_t n_seg, const double *nu_break,
                           const double *seg_logk, const double *seg_beta, double nu_ref) {
  int s = 0;
  for (int b = 0; b < n_seg - 1; ++b) {
    if (right ? (nu_break[b] <= nu) : (nu_break[b] < nu)) s = b + 1;
  }
  return seg_logk[s] + seg_beta[s] * log(nu / nu_ref);
}

int orc_group_table(int32_t n_groups, const double *edges, int32_t mode, int32_t n_seg,
                    const double *nu_break, const double *seg_logk, const double *seg_beta,
                    double nu_ref, double *khat_minus_out, double *alpha_out) {
  if (n_groups < 1 || n_seg < 1 || !(nu_ref > 0.0)) return -1;
  for (int g = 0; g < n_groups; ++g) {
    double n0 = edges[g], n1 = edges[g + 1];
    if (!(n1 > n0) || n0 < 0.0) return -1;
    if (mode == ORC_PPL_FIXED) {
      if (!(n0 > 0.0) || isinf(n1)) return -1;
      double lk0 = orc_law_logk(n0, 1, n_seg, nu_break, seg_logk, seg_beta, nu_ref);
      double lk1 = orc_law_logk(n1, 0, n_seg, nu_break, seg_logk, seg_beta, nu_ref);
      khat_minus_out[g] = exp(lk0);
      alpha_out[g] = (lk1 - lk0) / log(n1 / n0);
    } else {
      double centre;
      if (n0 == 0.0 && isinf(n1)) centre = nu_ref; /* one group spanning all frequencies */
      else if (n0 == 0.0) centre = 0.5 * n1;
      else if (isinf(n1)) centre = 2.0 * n0;
      else centre = sqrt(n0 * n1);
      khat_minus_out[g] =
          exp(orc_law_logk(centre, 1, n_seg, nu_break, seg_logk, seg_beta, nu_ref));
      alpha_out[g] = 0.0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* PPL slopes fitted to the group values (Appendix A)                        */
/* ------------------------------------------------------------------------ */
/* eq. sg: slope between groups g and g+1 of Qbar against nubar in log-log;
 * NAN when either Qbar is not positive or the slope is not finite */
static double orc_edge_slope(const double *edges, const double *Q, int g) {
  double qa = Q[g] / (edges[g + 1] - edges[g]);
  double qb = Q[g + 1] / (edges[g + 2] - edges[g + 1]);
  if (!(qa > 0.0) || !(qb > 0.0)) return NAN;
  double nua = sqrt(edges[g] * edges[g + 1]);
  double nub = sqrt(edges[g + 1] * edges[g + 2]);
  double s = log(qb / qa) / log(nub / nua);
  return isfinite(s) ? s : NAN;
}

static double orc_minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

void orc_ppl_free_slopes(int32_t n_groups, const double *edges, const double *Q,
                         double *alpha_out) {
  for (int g = 0; g < n_groups; ++g) alpha_out[g] = -1.0; /* eq. minmod, first and last */
  for (int g = 1; g + 1 < n_groups; ++g) {
    double sl = orc_edge_slope(edges, Q, g - 1);
    double sr = orc_edge_slope(edges, Q, g);
    if (isnan(sl) || isnan(sr)) continue; /* reading: undefined slope -> -1 */
    alpha_out[g] = orc_minmod(sl, sr);
  }
}

/* ------------------------------------------------------------------------ */
/* Group terms at temperature T                                              */
/* ------------------------------------------------------------------------ */
void orc_group_terms(const orc_params *p, const orc_groups *gt, double chi0_scale, double T,
                     const double *erad0, double *b, double *dnb, double *dnxb, double *chiB,
                     double *chiE, double *chiF) {
  orc_init_series();
  const int G = gt->n_groups;
  double fac = p->a_rad * T * T * T * T;
  double tfac = (p->temp_exponent != 0.0) ? pow(T / p->T_ref, p->temp_exponent) : 1.0;
  double *bg = (double *)malloc(sizeof(double) * 3 * (size_t)G);
  double *aB = bg + G, *aE = aB + G;
  /* b_g = 4 pi B_g / c of every group first: the Appendix A slopes of B_nu
   * need the neighbours */
  for (int g = 0; g < G; ++g) {
    double n0 = gt->edges[g], n1 = gt->edges[g + 1];
    double x0 = p->h * n0 / (p->k_B * T);
    double x1 = isinf(n1) ? INFINITY : p->h * n1 / (p->k_B * T);
    bg[g] = fac * orc_planck_band(x0, x1);
  }
  /* spectral indices of B_nu and E_nu inside each group: -1 (fixed slope), or
   * Appendix A from b_g(T) and from the starting radiation energy */
  for (int g = 0; g < G; ++g) aB[g] = aE[g] = -1.0;
  if (gt->free_slopes) {
    orc_ppl_free_slopes(G, gt->edges, bg, aB);
    if (erad0) orc_ppl_free_slopes(G, gt->edges, erad0, aE);
  }
  for (int g = 0; g < G; ++g) {
    double n0 = gt->edges[g], n1 = gt->edges[g + 1];
    double x0 = p->h * n0 / (p->k_B * T);
    double x1 = isinf(n1) ? INFINITY : p->h * n1 / (p->k_B * T);
    double alpha = gt->alpha[g];
    /* (4 pi/c) Delta_g(nu B_nu) */
    double d0 = orc_nu_B(x0), d1 = orc_nu_B(x1);
    double dnbg = fac * (d1 - d0);
    /* chi_0 at the two edges of the group, from the group's own powerlaw */
    double chim = chi0_scale * tfac * gt->khat_minus[g];
    double chip = (alpha == 0.0) ? chim : chim * pow(n1 / n0, alpha);
    double dnxbg = fac * (chip * d1 - chim * d0);
    /* eq. chiQg for B_nu and E_nu (PC: chi_0 is flat, any spectrum gives chim) */
    double chiBg = (alpha == 0.0) ? chim : orc_ppl_mean_opacity(chim, alpha, aB[g], n1 / n0);
    double chiEg = (alpha == 0.0) ? chim : orc_ppl_mean_opacity(chim, alpha, aE[g], n1 / n0);
    /* eq. chiDiff.  The exact diffusion-limit flux mean is a positively
     * weighted mean of chi_0 over the group (weight B_nu - dB_nu/dln(nu)/3 > 0),
     * so it lies between the smallest and largest chi_0 inside the group; the
     * PPL estimate is held to that range (it can leave it, even turn negative,
     * for steep in-group slopes).  When b_g underflows the estimate is chi_E. */
    double den = (4.0 / 3.0) * bg[g] - dnbg / 3.0;
    double chiFg;
    if (den > 0.0)
      chiFg = ((chiBg + chiEg / 3.0) * bg[g] + (alpha * chiEg * bg[g] - dnxbg) / 3.0) / den;
    else
      chiFg = chiEg;
    double chlo = chim < chip ? chim : chip, chhi = chim < chip ? chip : chim;
    if (chiFg < chlo) chiFg = chlo;
    if (chiFg > chhi) chiFg = chhi;
    if (b) b[g] = bg[g];
    if (dnb) dnb[g] = dnbg;
    if (dnxb) dnxb[g] = dnxbg;
    if (chiB) chiB[g] = chiBg;
    if (chiE) chiE[g] = chiEg;
    if (chiF) chiF[g] = chiFg;
  }
  free(bg);
}

/* ------------------------------------------------------------------------ */
/* Closure (Sec. 2.1: applied group by group)                                */
/* ------------------------------------------------------------------------ */
void orc_closure(int32_t closure, double c, double E, const double F[3], double P[9]) {
  double fn = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  double chi = 1.0 / 3.0;
  double n[3] = {0.0, 0.0, 0.0};
  if (closure == ORC_CLOSURE_M1 && E > 0.0 && fn > 0.0) {
    /* Levermore (1984): Eddington factor of the reduced flux f = |F|/(cE) */
    double f = fn / (c * E);
    if (f > 1.0) f = 1.0;
    chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
    for (int i = 0; i < 3; ++i) n[i] = F[i] / fn;
  }
  double iso = 0.5 * (1.0 - chi), dir = 0.5 * (3.0 * chi - 1.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[3 * i + j] = E * ((i == j ? iso : 0.0) + dir * n[i] * n[j]);
}

/* ------------------------------------------------------------------------ */
/* Linear algebra                                                            */
/* ------------------------------------------------------------------------ */
void orc_arrowhead_solve(int32_t n, double a00, const double *top, const double *left,
                         const double *diag, const double *rhs, double *x) {
  /* cancel the first-row entries 2..n+1 with rows 2..n+1, solve for x_0 ... */
  double a = a00, r = rhs[0];
  for (int g = 0; g < n; ++g) {
    a -= top[g] * left[g] / diag[g];
    r -= top[g] * rhs[g + 1] / diag[g];
  }
  x[0] = r / a;
  /* ... then substitute x_0 into each remaining row */
  for (int g = 0; g < n; ++g) x[g + 1] = (rhs[g + 1] - left[g] * x[0]) / diag[g];
}

int orc_dense_solve(int32_t n, double *A, double *b, double *x) {
  int *piv = (int *)malloc(sizeof(int) * (size_t)n);
  if (!piv) return -1;
  for (int k = 0; k < n; ++k) {
    int pr = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(A[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        pr = i;
      }
    }
    piv[k] = pr;
    if (best == 0.0) {
      free(piv);
      return -1;
    }
    if (pr != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)pr * n + j];
        A[(size_t)pr * n + j] = t;
      }
      double t = b[k];
      b[k] = b[pr];
      b[pr] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * x[j];
    x[i] = s / A[(size_t)i * n + i];
  }
  free(piv);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The coupled implicit system of one cell                                   */
/* ------------------------------------------------------------------------ */
/* Unknowns y = (E_int, rho v (3), E_g (G), F_g (3G, group-major)), with the
 * total gas energy E_gas = E_int + |rho v|^2/(2 rho) (Sec. 3, dual energy).
 * The equations are eqs. egupdate, eupdate, vupdate, fupdate, each written in
 * a form with the same root:
 *   [gas]  E_gas - E_gas^t + (c/c_hat) sum_g (E_g - E_g^t - S_g) = 0
 *          (eq. egupdate with R_g replaced by E_g - E_g^t - S_g from eq. FGFR)
 *   [E_g]  E_g - (E_g^t + S_g + A_g) / (1 + c_hat theta dt chi_E) = 0,
 *          A_g = c_hat theta dt [chi_B b_g + (1 + alpha) chi_F v.F_g / c^2]
 *          (eq. eupdate with -c_hat G^0_g theta dt from eq. G0_3, i.e. R_g of
 *          eq. Rnew including the c_hat/c factor of -c_hat G^0 theta dt)
 *   [F_g]  F_g - {F_g^t + c_hat theta dt [v (chi_B b_g - dnxb_g/3)
 *                 + (1 + alpha) chi_E v.P_g]} / (1 + c_hat chi_F theta dt) = 0
 *          (eq. fupdate with -G^i_g from eq. G1_3, chi_P^(ji) ~ chi_E)
 *   [mom]  rho v - (rho v)^t + (c c_hat)^-1 sum_g (F_g - F_g^t) = 0
 *          (eq. vupdate with sum_g G_g theta dt from eq. fupdate)
 * T = E_int / (rho c_v) and v = rho v / rho are those of the unknowns, so the
 * system is fully implicit (Sec. 3, last paragraph). */
typedef struct {
  const orc_params *p;
  const orc_groups *gt;
  int G;
  double rho, chi0s, m0[3], egas0, Etot, Eint0;
  const double *E0, *F0, *S; /* E0[g], F0[3g+d], S[g] (S may be NULL) */
  const double *Es;           /* E0[g] + S[g]: the spectrum that sets alpha_E (free slopes) */
  double *b, *dnb, *dnxb, *chiB, *chiE, *chiF;
} orc_cell;

static int orc_residual(const orc_cell *c, const double *y, double *r) {
  const orc_params *p = c->p;
  int G = c->G;
  double Eint = y[0];
  double T = Eint / (c->rho * p->c_v);
  if (!(T > 0.0) || !isfinite(T)) return -1;
  double m[3] = {y[1], y[2], y[3]};
  double v[3] = {m[0] / c->rho, m[1] / c->rho, m[2] / c->rho};
  double KE = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / c->rho;
  orc_group_terms(p, c->gt, c->chi0s, T, c->Es, c->b, c->dnb, c->dnxb, c->chiB, c->chiE,
                  c->chiF);
  double tdt = p->c_hat * p->theta * p->dt;
  double sumR = 0.0, dF[3] = {0.0, 0.0, 0.0};
  for (int g = 0; g < G; ++g) {
    double alpha = c->gt->alpha[g];
    double E = y[4 + g];
    const double *F = y + 4 + G + 3 * g;
    const double *F0 = c->F0 + 3 * g;
    double S = c->S ? c->S[g] : 0.0;
    double chiE = c->chiE[g];
    double w = (v[0] * F[0] + v[1] * F[1] + v[2] * F[2]) / (p->c * p->c);
    double A = tdt * (c->chiB[g] * c->b[g] + (1.0 + alpha) * c->chiF[g] * w);
    r[4 + g] = E - (c->E0[g] + S + A) / (1.0 + tdt * chiE);
    sumR += E - c->E0[g] - S;
    double P[9];
    orc_closure(p->closure, p->c, E, F, P);
    double src = c->chiB[g] * c->b[g] - c->dnxb[g] / 3.0;
    for (int i = 0; i < 3; ++i) {
      double vP = v[0] * P[0 * 3 + i] + v[1] * P[1 * 3 + i] + v[2] * P[2 * 3 + i];
      double num = F0[i] + tdt * (v[i] * src + (1.0 + alpha) * chiE * vP);
      r[4 + G + 3 * g + i] = F[i] - num / (1.0 + tdt * c->chiF[g]);
      dF[i] += F[i] - F0[i];
    }
  }
  r[0] = Eint + KE - c->egas0 + (p->c / p->c_hat) * sumR;
  for (int i = 0; i < 3; ++i) r[1 + i] = m[i] - c->m0[i] + dF[i] / (p->c * p->c_hat);
  for (int k = 0; k < 4 + 4 * G; ++k)
    if (!isfinite(r[k])) return -1;
  return 0;
}

/* Scales: each equation (and its own unknown) against the magnitude of its
 * terms -- the start value, the current value and the value the equation
 * solves for (unknown minus residual).  r is the residual at y. */
static void orc_row_scales(const orc_cell *c, const double *y, const double *r, double *sig) {
  const orc_params *p = c->p;
  int G = c->G;
  double mscale = fabs(c->m0[0]) + fabs(c->m0[1]) + fabs(c->m0[2]) + c->Etot / p->c_hat;
  sig[0] = c->Etot;
  for (int i = 0; i < 3; ++i) sig[1 + i] = mscale;
  for (int g = 0; g < G; ++g) {
    double S = c->S ? fabs(c->S[g]) : 0.0;
    double E = y[4 + g];
    double e = fabs(c->E0[g]) + S + fabs(E) + fabs(E - r[4 + g]);
    if (!(e > 1e-300)) e = 1e-300;
    sig[4 + g] = e;
    const double *F0 = c->F0 + 3 * g;
    const double *F = y + 4 + G + 3 * g;
    const double *rF = r + 4 + G + 3 * g;
    double fs = p->c * e + fabs(F0[0]) + fabs(F0[1]) + fabs(F0[2]);
    for (int i = 0; i < 3; ++i) fs += fabs(F[i] - rF[i]);
    for (int i = 0; i < 3; ++i) sig[4 + G + 3 * g + i] = fs;
  }
}

static double orc_norm_inf(int n, const double *r, const double *sig) {
  double m = 0.0;
  for (int k = 0; k < n; ++k) {
    double a = fabs(r[k]) / sig[k];
    if (a > m) m = a;
  }
  return m;
}

static double orc_norm_2(int n, const double *r, const double *sig) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += (r[k] / sig[k]) * (r[k] / sig[k]);
  return sqrt(s);
}

/* Newton on the coupled system; returns iterations, writes best y. */
static int orc_newton(orc_cell *c, double *y, double *work, double *final_res, int *ok) {
  const orc_params *p = c->p;
  int n = 4 + 4 * c->G;
  double *r = work;
  double *sig = r + n;
  double *rp = sig + n;
  double *rm = rp + n;
  double *dy = rm + n;
  double *ytry = dy + n;
  double *rhs = ytry + n;
  double *J = rhs + n; /* n*n */
  double tol = p->tol > 0.0 ? p->tol : 1e-14;
  *ok = 0;
  if (orc_residual(c, y, r) != 0) {
    *final_res = INFINITY;
    return 0;
  }
  orc_row_scales(c, y, r, sig);
  double nrm = orc_norm_inf(n, r, sig);
  int it = 0, stall = 0;
  while (it < p->max_iter) {
    if (nrm <= tol) {
      *ok = 1;
      break;
    }
    /* central-difference Jacobian; steps relative to the unknown, or to its
     * scale when the unknown itself is far below it (E_int: its own value) */
    for (int j = 0; j < n; ++j) {
      double yj = y[j];
      double h = (j == 0) ? 6e-6 * fabs(yj) : 6e-6 * fmax(fabs(yj), 1e-4 * sig[j]);
      y[j] = yj + h;
      int e1 = orc_residual(c, y, rp);
      y[j] = yj - h;
      int e2 = orc_residual(c, y, rm);
      y[j] = yj;
      if (e1 != 0 || e2 != 0) {
        /* one-sided step away from the invalid side */
        y[j] = yj + h;
        e1 = orc_residual(c, y, rp);
        y[j] = yj;
        if (e1 != 0) {
          *final_res = nrm;
          return it;
        }
        for (int i = 0; i < n; ++i) J[(size_t)i * n + j] = (rp[i] - r[i]) / h * sig[j] / sig[i];
      } else {
        for (int i = 0; i < n; ++i)
          J[(size_t)i * n + j] = (rp[i] - rm[i]) / (2.0 * h) * sig[j] / sig[i];
      }
    }
    /* rows and columns both scaled by the magnitude of their own variable */
    for (int i = 0; i < n; ++i) rhs[i] = -r[i] / sig[i];
    if (orc_dense_solve(n, J, rhs, dy) != 0) break;
    for (int i = 0; i < n; ++i) dy[i] *= sig[i];
    /* backtracking: keep T > 0 and finite, and reduce the scaled 2-norm */
    double n2 = orc_norm_2(n, r, sig);
    double lam = 1.0;
    int accepted = 0;
    for (int k = 0; k < 40; ++k) {
      for (int i = 0; i < n; ++i) ytry[i] = y[i] + lam * dy[i];
      if (orc_residual(c, ytry, rp) == 0) {
        double n2t = orc_norm_2(n, rp, sig);
        if (n2t < (1.0 - 1e-4 * lam) * n2 || k == 39) {
          accepted = 1;
          break;
        }
      }
      lam *= 0.5;
    }
    ++it;
    if (!accepted) break;
    memcpy(y, ytry, sizeof(double) * (size_t)n);
    memcpy(r, rp, sizeof(double) * (size_t)n);
    orc_row_scales(c, y, r, sig);
    double nn = orc_norm_inf(n, r, sig);
    /* stop at the round-off floor: no decrease over four iterations */
    stall = (nn > 0.5 * nrm && nn < 1e-10) ? stall + 1 : 0;
    nrm = nn;
    if (stall >= 4) break;
  }
  /* converged: below the target, or stalled at the round-off floor near it */
  if (nrm <= tol || (stall >= 4 && nrm <= 100.0 * tol)) *ok = 1;
  *final_res = nrm;
  return it;
}

int32_t orc_max_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_source_update(int64_t n_cells, const orc_params *p, const orc_groups *gt,
                      const double *rho, double *mom, double *egas, const double *kappa0,
                      double *erad, double *frad, const double *src, int32_t *iters,
                      double *resid, int32_t *status, int32_t n_threads) {
  if (!p || !gt || n_cells < 0 || gt->n_groups < 1 || !rho || !mom || !egas || !erad || !frad)
    return -1;
  orc_init_series();
  const int G = gt->n_groups;
  const int n = 4 + 4 * G;
  const size_t wsz = (size_t)7 * n + (size_t)n * n + (size_t)2 * n + (size_t)8 * G;
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
  {
    double *work = (double *)malloc(sizeof(double) * wsz);
    double *y = work + 7 * n + (size_t)n * n;
    double *E0 = y + n;
    double *F0 = E0 + G;    /* 3G */
    double *S = F0 + 3 * G; /* G */
    double *scratch = S + G; /* 5G needed, 2G + n left over is plenty */
    double *tb = scratch, *tdnb = tb + G, *tdnxb = tdnb + G;
    double *tchiB = (double *)malloc(sizeof(double) * 4 * (size_t)G);
    double *tchiE = tchiB + G, *tchiF = tchiE + G, *Es = tchiF + G;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int64_t i = 0; i < n_cells; ++i) {
      double r_i = rho[i];
      double m0[3] = {mom[i], mom[n_cells + i], mom[2 * n_cells + i]};
      double eg0 = egas[i];
      double k0 = kappa0 ? kappa0[i] : 1.0;
      int valid = (r_i > 0.0) && isfinite(r_i) && isfinite(eg0) && isfinite(k0) && k0 >= 0.0;
      double KE0 = 0.0;
      for (int d = 0; d < 3; ++d) {
        valid = valid && isfinite(m0[d]);
        KE0 += 0.5 * m0[d] * m0[d] / r_i;
      }
      double Eint0 = eg0 - KE0;
      valid = valid && (Eint0 > 0.0);
      double sumE0 = 0.0, sumS = 0.0;
      for (int g = 0; g < G; ++g) {
        E0[g] = erad[(size_t)g * n_cells + i];
        S[g] = src ? src[(size_t)g * n_cells + i] : 0.0;
        valid = valid && isfinite(E0[g]) && isfinite(S[g]);
        sumE0 += E0[g];
        sumS += S[g];
        for (int d = 0; d < 3; ++d) {
          F0[3 * g + d] = frad[((size_t)d * G + g) * n_cells + i];
          valid = valid && isfinite(F0[3 * g + d]);
        }
      }
      if (!valid) {
        if (status) status[i] = 3;
        if (iters) iters[i] = 0;
        if (resid) resid[i] = 0.0;
        continue;
      }
      orc_cell c;
      c.p = p;
      c.gt = gt;
      c.G = G;
      c.rho = r_i;
      c.chi0s = r_i * k0;
      for (int d = 0; d < 3; ++d) c.m0[d] = m0[d];
      c.egas0 = eg0;
      /* E_tot at the start of the step; c/c_hat converts radiation energy to the
       * gas-energy equation's units (Sec. 3, convergence test) */
      c.Etot = eg0 + (p->c / p->c_hat) * (sumE0 + sumS);
      c.Eint0 = Eint0;
      c.E0 = E0;
      c.F0 = F0;
      c.S = S;
      c.b = tb;
      c.dnb = tdnb;
      c.dnxb = tdnxb;
      c.chiB = tchiB;
      c.chiE = tchiE;
      c.chiF = tchiF;
      for (int g = 0; g < G; ++g) Es[g] = E0[g] + S[g];
      c.Es = Es;
      y[0] = Eint0;
      for (int d = 0; d < 3; ++d) y[1 + d] = m0[d];
      for (int g = 0; g < G; ++g) {
        y[4 + g] = E0[g];
        for (int d = 0; d < 3; ++d) y[4 + G + 3 * g + d] = F0[3 * g + d];
      }
      double res = 0.0;
      int ok = 0;
      int it = orc_newton(&c, y, work, &res, &ok);
      /* conservative write-back (Sec. 3): E_g = E_g^t + R_g + S_g,
       * E_gas = E_gas^t - (c/c_hat) sum R_g, (rho v) = (rho v)^t - (c c_hat)^-1
       * sum (F_g - F_g^t), with R_g = E_g - E_g^t - S_g of the root */
      double sumR = 0.0, dF[3] = {0.0, 0.0, 0.0};
      for (int g = 0; g < G; ++g) {
        double Eg = y[4 + g];
        sumR += Eg - E0[g] - S[g];
        erad[(size_t)g * n_cells + i] = Eg;
        for (int d = 0; d < 3; ++d) {
          double Fg = y[4 + G + 3 * g + d];
          dF[d] += Fg - F0[3 * g + d];
          frad[((size_t)d * G + g) * n_cells + i] = Fg;
        }
      }
      egas[i] = eg0 - (p->c / p->c_hat) * sumR;
      for (int d = 0; d < 3; ++d) mom[(size_t)d * n_cells + i] = m0[d] - dF[d] / (p->c * p->c_hat);
      if (iters) iters[i] = it;
      if (resid) resid[i] = res;
      if (status) status[i] = ok ? 0 : 2;
    }
    free(tchiB);
    free(work);
  }
  return 0;
}
