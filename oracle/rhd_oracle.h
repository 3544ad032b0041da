/* rhd_oracle.h -- FP64 CPU oracle for the implicit multigroup matter-radiation
 * source-term update of He, Wibking & Krumholz (2024), "A novel numerical
 * method for mixed-frame multigroup radiation-hydrodynamics ...".
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no source, header,
 * table or helper with the CUDA library; the two are written separately from
 * the paper.
 *
 * What it computes: for every cell, the root of the fully coupled implicit
 * system of Sec. 3 -- eqs. egupdate, eupdate (energies), vupdate, fupdate
 * (momenta) -- with the four-force of eqs. G0_3 and G1_3 (Sec. 2.2.2), the
 * PPL fixed-slope mean opacities of eq. chiQg with alpha_Q = -1 (Sec. 2.2.2),
 * (or the Appendix A slopes, free_slopes), the diffusion-limit flux-mean
 * opacity of eq. chiDiff, and a group-by-group
 * closure for P_g (Sec. 2.1).  The root is found by a plain Newton iteration
 * on all 4+4*N_g unknowns with a finite-difference Jacobian and a dense
 * partial-pivot LU; the paper's conservative write-back (Sec. 3, after the
 * convergence test, and the momentum update after eq. numF1) is applied to the
 * root so that total energy and momentum are conserved to round-off.
 *
 * Layout of the batch arrays (all host memory, FP64):
 *   per cell   [n_cells]              rho, egas, kappa0 (may be NULL => 1)
 *   momentum   [3][n_cells]           rho*v components
 *   per group  [n_groups][n_cells]    erad, src (src may be NULL => 0)
 *   flux       [3][n_groups][n_cells] F_g components
 */
#ifndef RHD_ORACLE_H
#define RHD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CLOSURE_M1 = 0, ORC_CLOSURE_EDDINGTON = 1 };
enum { ORC_PPL_FIXED = 0, ORC_PC = 1, ORC_PPL_FREE = 2 };

typedef struct {
  double c, c_hat, a_rad, h, k_B; /* constants (cgs or any consistent units) */
  double c_v;                     /* specific heat per unit mass: E_int = rho*c_v*T */
  double theta;                   /* IMEX stage weight (1 or 1/2), Sec. 3 */
  double dt;                      /* time step */
  double temp_exponent, T_ref;    /* optional (T/T_ref)^p opacity factor */
  double tol;                     /* scaled-residual target of the coupled Newton */
  int32_t max_iter;               /* Newton iteration cap */
  int32_t closure;                /* ORC_CLOSURE_M1 | ORC_CLOSURE_EDDINGTON */
} orc_params;

/* Per-group opacity table (Sec. 2.2.2): chi_0(nu) = rho*kappa0*khat_minus[g]*
 * (nu/nu_minus)^alpha[g] inside group g.  PC mode is alpha = 0 (Sec. 2.2.1).
 * free_slopes = 0: the spectral indices alpha_Q of B_nu and E_nu inside every
 * group are -1 (PPL fixed slope, Sec. 2.2.2).  free_slopes = 1: they come from
 * the group values by the edge slopes and minmod of Appendix A -- alpha_B from
 * b_g(T) at the temperature of every evaluation, alpha_E from the radiation
 * energy the update starts from, E_g^t + S_g. */
typedef struct {
  int32_t n_groups;
  const double *edges;      /* [n_groups+1] lab-frame group edges, increasing */
  const double *khat_minus; /* [n_groups] opacity shape at the lower edge */
  const double *alpha;      /* [n_groups] powerlaw index inside the group */
  int32_t free_slopes;      /* 0: alpha_Q = -1; 1: Appendix A slopes */
} orc_groups;

/* Cumulative Planck fraction P(x) = (15/pi^4) int_0^x t^3/(e^t-1) dt and its
 * complement Q(x) = 1 - P(x). */
double orc_planck_P(double x);
double orc_planck_Q(double x);
/* Fraction of a_R T^4 in the band [x0, x1] (x0 <= x1; x1 may be +inf). */
double orc_planck_band(double x0, double x1);

/* PPL mean opacity of eq. chiQg for a powerlaw spectrum of index alpha_Q:
 * chi_Q = chi_minus * [(r^(aQ+1)-1)/(aQ+1)]^-1 * [(r^(aX+aQ+1)-1)/(aX+aQ+1)],
 * each bracket replaced by ln r when its exponent is zero. */
double orc_ppl_mean_opacity(double chi_minus, double alpha_chi, double alpha_Q, double r);

/* Spectral indices alpha_Q,g of a radiation quantity from its group values
 * Q[g] (Appendix A, eqs. sg and minmod): the edge slopes s_(g+1/2) =
 * ln(Qbar_(g+1)/Qbar_g) / ln(nubar_(g+1)/nubar_g) with Qbar_g = Q_g/(nu_g+ -
 * nu_g-) and nubar_g = sqrt(nu_g+ nu_g-); alpha = -1 for the first and the
 * last group and minmod(s_(g-1/2), s_(g+1/2)) between.  Reading: a slope
 * whose Qbar is not positive on either side (or whose value is not finite) is
 * undefined, and a group with an undefined edge slope takes -1 like the edge
 * groups.  minmod(a, b) = the one of smaller magnitude when a and b have the
 * same sign, else 0.  Edges must be finite and > 0. */
void orc_ppl_free_slopes(int32_t n_groups, const double *edges, const double *Q,
                         double *alpha_out);

/* Group table from a piecewise-powerlaw opacity law (Sec. 2.2.2):
 * khat(nu) = exp(seg_logk[s] + seg_beta[s]*ln(nu/nu_ref)) in segment s, the
 * segments separated by n_seg-1 increasing breakpoints nu_break.  PPL_FIXED:
 * khat_minus = right-continuous value at nu_minus, alpha = ln(khat(nu_plus-)/
 * khat(nu_minus+))/ln r.  PC: khat at the log-centre of the group (nu_plus/2
 * for a group starting at 0, 2 nu_minus for one ending at infinity, nu_ref for
 * a single group covering both), alpha = 0.
 * Returns 0, or -1 on bad input. */
int orc_group_table(int32_t n_groups, const double *edges, int32_t mode, int32_t n_seg,
                    const double *nu_break, const double *seg_logk, const double *seg_beta,
                    double nu_ref, double *khat_minus_out, double *alpha_out);

/* Group-integrated Planck terms and mean opacities at temperature T for one
 * cell (chi0_scale = rho*kappa0).  erad0: [n_groups] radiation energy whose
 * spectral indices set chi_E when gt->free_slopes (may be NULL otherwise).
 * Outputs, each [n_groups]:
 *   b     = 4 pi B_g / c
 *   dnb   = (4 pi / c) Delta_g(nu B_nu)
 *   dnxb  = (4 pi / c) Delta_g(nu chi_0 B_nu)
 *   chiB, chiE (eq. chiQg), chiF (eq. chiDiff).  Any output pointer may be NULL. */
void orc_group_terms(const orc_params *p, const orc_groups *gt, double chi0_scale, double T,
                     const double *erad0, double *b, double *dnb, double *dnxb, double *chiB,
                     double *chiE, double *chiF);

/* Closure P_g(E_g, F_g): M1 (Levermore 1984) or Eddington; P is 3x3 row-major. */
void orc_closure(int32_t closure, double c, double E, const double F[3], double P[9]);

/* Arrowhead system of eq. matrix: row 0 = (a00, top[0..n-1]), row 1+g =
 * (left[g], 0.., diag[g], ..0).  Solves J x = rhs by the paper's elimination
 * (Sec. 3, after eq. matrix).  x has n+1 entries. */
void orc_arrowhead_solve(int32_t n, double a00, const double *top, const double *left,
                         const double *diag, const double *rhs, double *x);
/* Dense partial-pivot LU solve of A x = b (A is n x n row-major, overwritten). */
int orc_dense_solve(int32_t n, double *A, double *b, double *x);

/* The batch source update (see the top of this file).  Returns 0 or -1 on bad
 * arguments.  Per cell: iters[i] = Newton iterations, resid[i] = final scaled
 * residual (max-norm), status[i] = 0 converged, 2 not converged within
 * max_iter (the best iterate is written back), 3 invalid input (untouched).
 * n_threads <= 0 uses the OpenMP default. */
int orc_source_update(int64_t n_cells, const orc_params *p, const orc_groups *gt,
                      const double *rho, double *mom, double *egas, const double *kappa0,
                      double *erad, double *frad, const double *src, int32_t *iters,
                      double *resid, int32_t *status, int32_t n_threads);

/* Number of OpenMP threads a parallel region of this library would use. */
int32_t orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
