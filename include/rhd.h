/* rhd.h -- C ABI of the GB300 library for the implicit multigroup
 * matter-radiation source-term update of He, Wibking & Krumholz (2024),
 * "A novel numerical method for mixed-frame multigroup radiation-hydrodynamics
 * with GPU acceleration implemented in the QUOKKA code".
 *
 * One call advances, in every cell independently, the implicit stage of Sec. 3:
 * eqs. egupdate and eupdate (gas and group energies), vupdate and fupdate (gas
 * momentum and group fluxes), with the four-force of eqs. G0_3 / G1_3 and the
 * piecewise-powerlaw (PPL) mean opacities of Sec. 2.2.2.  Per cell it runs the
 * paper's inner Newton-Raphson over x = (E_gas, R_1..R_Ng) with the arrowhead
 * Jacobian of eq. matrix, eliminated in O(N_g), the convergence test after
 * eq. matrix, the conservative energy write-back, the closed-form flux update
 * eq. numF1, the momentum update that follows it, and the outer iteration of
 * the last paragraph of Sec. 3.
 *
 * Units are the caller's (cgs in the paper, Table 1); the constants are fields
 * so that dimensionless test units work as well.  The radiation constant and
 * the Planck shape are used as 4 pi B_nu / c = a_R T^4 (15/pi^4) x^3/(e^x-1)
 * dx/dnu with x = h nu / (k_B T), i.e. the group Planck integrals sum to
 * a_R T^4 over all frequencies.
 *
 * Memory: every array pointer in rhd_state_t is a DEVICE pointer owned by the
 * caller; the library never frees or keeps it.  Arrays in rhd_groups_t and
 * rhd_opacity_law_t are HOST pointers, read during the call (they are packed
 * into the launch).  Calls are asynchronous on `stream` (a cudaStream_t passed
 * as void*, NULL = the legacy default stream).  Per-cell problems never fail a
 * call; they are reported in status[].  Negative return values are errors;
 * rhd_strerror() names them.  Not thread-safe for concurrent calls that share
 * a context.
 */
#ifndef RHD_H
#define RHD_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define RHD_OK 0
#define RHD_EINVAL (-1)   /* a pointer, size or parameter is invalid */
#define RHD_EEDGES (-2)   /* group edges not strictly increasing, or not finite and > 0 for PPL */
#define RHD_ELAW (-3)     /* opacity law rejected (segment count, breakpoints, nu_ref) */
#define RHD_ECUDA (-4)    /* a CUDA call failed (launch, copy, device query) */
#define RHD_ENOMEM (-5)   /* workspace allocation failed */
#define RHD_ESIZE (-6)    /* a size exceeds a compiled limit (groups, segments, grids) */
#define RHD_EIO (-7)      /* a file could not be opened, read or written, or is not a saved surrogate */

/* compiled limits */
#define RHD_MAX_GROUPS 256
#define RHD_MAX_SEGMENTS 64

/* rhd_state_t.precision */
#define RHD_FP64 0  /* every step in FP64 */
#define RHD_MIXED 1 /* FP32 Newton; FP64 Planck differences, final residual, write-back */

/* rhd_state_t.closure (Sec. 2.1: applied group by group) */
#define RHD_M1 0        /* Levermore (1984) M1 closure, the paper's default */
#define RHD_EDDINGTON 1 /* P = E/3 I (used by the paper's radiative-shock test) */

/* rhd_opacity_law_t.mode */
#define RHD_PPL_FIXED 0 /* piecewise powerlaw, alpha_Q = -1 (Sec. 2.2.2, favoured) */
#define RHD_PC 1        /* piecewise constant (Sec. 2.2.1) */
#define RHD_PPL_FREE 2  /* piecewise powerlaw opacity with the spectral indices alpha_Q of
                           B_nu and E_nu fitted to the group values (Appendix A, eqs. sg and
                           minmod; -1 in the first and last group and next to a group value
                           that is not positive): alpha_B from b_g(T) at every Newton
                           evaluation (with its T-derivative in the Jacobian), alpha_E from
                           E_g^t + S_g of the cell.  Runs the FP64 passes with one cell per
                           thread in either precision (the FP32 passes of RHD_MIXED are not
                           built for it, so a warm start from them is skipped); not accepted
                           by the batched interface (RHD_ELAW). */

/* rhd_state_t.flags */
#define RHD_GROUP_TEST 1 /* the outer iteration also stops only when, in every group,
                            the change of the v,F-terms of R_g is below tol_outer times
                            that group's own energy (the paper's test is relative to
                            E_tot, which leaves groups far below E_tot loosely converged) */
#define RHD_CELL_PER_THREAD 4 /* run every pass with one cell per thread (the other mapping
                                 spreads a cell's 33..128 groups over a warp's lanes, and in
                                 the mixed form's FP32 passes 1..32 groups over 8 or 16; same
                                 equations and results to rounding, slower at those sizes;
                                 for comparison and for counting the algorithm's operations
                                 without the lane-replicated per-cell work: under this flag
                                 the thread mapping also takes the warp mapping's cached first
                                 iteration of each outer pass, which it otherwise skips) */
#define RHD_LANES_16 8 /* 33..64 groups: the warp kernels (FP64 passes; the mixed form's FP32
                          passes, first correction step and correction) spread a cell over
                          16 lanes with 4 groups each (two cells per warp) instead of 32
                          lanes with 2 groups each; same equations and results to rounding,
                          a different balance of registers, shuffles, per-cell work repeated
                          on every lane of a cell, and cells in flight; no effect on other
                          group counts or with RHD_CELL_PER_THREAD */
#define RHD_FLUX_TEST 2  /* the outer iteration also stops only when the change of the
                            group fluxes, sum_g |F_g,new - F_g,old|_1 / c, is below
                            tol_outer E_tot (the paper's test sees F_g only through the
                            v.F terms of R_g, so flux components normal to v can still be
                            moving when it passes) */

/* per-cell status codes written to rhd_state_t.status */
#define RHD_STATUS_OK 0
#define RHD_STATUS_FALLBACK 1 /* converged after a fallback start */
#define RHD_STATUS_MAXITER 2  /* an iteration cap was reached; the last iterate is written back */
#define RHD_STATUS_INVALID 3  /* rho <= 0, E_int <= 0, non-finite or negative input: cell untouched */

/* One grid's cell state, FP64 structure of arrays.  Per-cell arrays have
 * n_cells entries; per-group arrays are [n_groups][group_stride] with the
 * cell index fastest (group g of cell i at g*group_stride + i). */
typedef struct {
  const double *rho;    /* in    gas density, > 0 */
  double *mom[3];       /* inout gas momentum density rho*v, one array per component */
  double *egas;         /* inout total gas energy density (internal + kinetic) */
  const double *kappa0; /* in    opacity normaliser: chi_0(nu) = rho*kappa0*khat(nu); NULL = 1 */
  double *erad;         /* inout E_g, lab frame */
  double *frad[3];      /* inout F_g components, lab frame */
  const double *src;    /* in    optional radiation source S_g of eq. FGFR; NULL = 0 */
  uint8_t *status;      /* out   per-cell status (RHD_STATUS_*); NULL = not written */
  uint8_t *iters;       /* out   Newton iterations summed over outer passes, saturating
                                 at 255; NULL = not written */
  int64_t group_stride; /* elements between groups in erad/frad/src; 0 = n_cells */
  double c_v;           /* specific heat per unit mass: E_int = rho*c_v*T */
  double theta;         /* IMEX stage weight: 1 (first stage) or 1/2 (second), Sec. 3 */
  double c, c_hat, a_rad, h, k_B; /* speed of light, reduced speed of light, radiation
                                     constant, Planck and Boltzmann constants */
  double tol;           /* Newton tolerance epsilon of the convergence test (paper: 1e-11);
                           <= 0 selects 1e-11 */
  double tol_outer;     /* outer-iteration tolerance (paper: 1e-13); <= 0 selects 1e-13 */
  int32_t max_newton;   /* Newton cap per inner solve; <= 0 selects 64 */
  int32_t max_outer;    /* outer-iteration cap; <= 0 selects 16 */
  int32_t precision;    /* RHD_FP64 | RHD_MIXED */
  int32_t closure;      /* RHD_M1 | RHD_EDDINGTON */
  int32_t flags;        /* 0, or RHD_GROUP_TEST | RHD_FLUX_TEST | RHD_CELL_PER_THREAD |
                           RHD_LANES_16 */
} rhd_state_t;

/* Lab-frame group edges (Sec. 2.1, eq. Qg: contiguous groups).  HOST array of
 * n_groups+1 strictly increasing frequencies; PPL needs them finite and > 0,
 * PC also accepts a first edge of 0 and a last edge of +inf. */
typedef struct {
  int32_t n_groups; /* 1 .. RHD_MAX_GROUPS */
  const double *edges;
} rhd_groups_t;

/* Opacity shape khat(nu), chi_0 = rho*kappa0*khat(nu)*(T/T_ref)^temp_exponent.
 * Either a piecewise powerlaw law -- segment s (s = 0..n_seg-1, separated by
 * the n_seg-1 increasing breakpoints nu_break) has khat = exp(seg_logk[s] +
 * seg_beta[s]*ln(nu/nu_ref)) -- or, when khat_gminus is non-NULL, a per-group
 * table given directly (the paper lets the user give the slopes, Sec. 2.2.2).
 * PPL_FIXED takes khat_gminus = khat just above nu_g- and alpha_g =
 * ln(khat(nu_g+)/khat(nu_g-))/ln(nu_g+/nu_g-) (Sec. 2.2.2, the tabulated-opacity
 * slope; a breakpoint on an edge belongs to the group above it); PPL_FREE takes the
 * same table.  PC takes khat
 * at the logarithmic group centre and alpha = 0.  All arrays are HOST memory. */
typedef struct {
  int32_t mode;            /* RHD_PPL_FIXED | RHD_PC | RHD_PPL_FREE */
  int32_t n_seg;           /* 1 .. RHD_MAX_SEGMENTS (ignored when khat_gminus != NULL) */
  const double *nu_break;  /* [n_seg-1] */
  const double *seg_logk;  /* [n_seg] natural log of khat at nu_ref for the segment's powerlaw */
  const double *seg_beta;  /* [n_seg] powerlaw index of the segment */
  double nu_ref;           /* > 0 */
  const double *khat_gminus; /* [n_groups] optional per-group table: khat at the lower edge */
  const double *alpha_g;     /* [n_groups] its in-group slopes (PC: ignored, alpha = 0) */
  double temp_exponent, T_ref; /* optional (T/T_ref)^p factor; p = 0 disables it */
} rhd_opacity_law_t;

/* Advance every cell of one grid by one implicit source-term stage of length
 * dt (in place).  n_cells may be 0.  Returns RHD_OK or a negative RHD_E* code
 * (then nothing was launched).  The first call on a device initialises the
 * library's constant tables on that device (synchronously), so make it before
 * any stream capture.  RHD_FP64 runs the paper's inner/outer iteration (Sec. 3)
 * in FP64.  RHD_MIXED runs it in FP32 to FP32 resolution, takes a first Newton
 * step on the coupled per-cell system from a float-float residual, then
 * evaluates that system's residual in FP64, applies the paper's convergence
 * tests to it and writes back in FP64 (another FP32-Jacobian step where the
 * tests fail; the FP64 iteration for any cell left over), so its result
 * meets the same tolerances and conserves energy and momentum to FP64
 * round-off.  The mixed form uses a per-device workspace of 32 bytes per
 * cell-group + 34 bytes per cell (grown on demand; RHD_ENOMEM if that fails). */
int rhd_source_update(rhd_state_t *state, const rhd_groups_t *groups,
                      const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                      void *stream);

/* ---- One radiation step of the two-stage IMEX integrator -----------------------
 * Sec. 3, eqs. imex1 and imex2, with the transport terms left out (a single
 * zone, or a caller that applies transport elsewhere).  Stage 1 is the implicit
 * source update of rhd_source_update over dt with theta = 1, from U^(n) to
 * U^(n+1/2).  Stage 2's explicit part is then U^(n) + (dt/2) S(U^(n+1/2)), and
 * with no transport dt S(U^(n+1/2)) = U^(n+1/2) - U^(n) (stage 1), so stage 2
 * starts from (U^(n) + U^(n+1/2))/2 (E_gas, rho v, E_g, F_g) and makes the
 * implicit update with theta = 1/2.  state->theta is ignored; state->src must
 * be NULL (RHD_EINVAL otherwise: a per-stage source is the caller's to split).
 * status is the worse of the two stages, iters their sum (held at 255).  The
 * library keeps U^(n) in a per-device workspace (8 (4 + 4 N_g) + 2 bytes per
 * cell, grown on demand); otherwise as rhd_source_update. */
int rhd_imex_step(rhd_state_t *state, const rhd_groups_t *groups,
                  const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells, void *stream);

/* ---- Batched uneven grids --------------------------------------------------
 * Many independent grids (own cell count, N_g <= RHD_MAX_GROUPS_BATCHED, own
 * opacity law, dt and parameters) in a few persistent launches: a device work
 * queue hands (grid, cell-tile) items to the CTAs, each CTA keeps the group
 * table of its current grid in shared memory, and every cell is solved by the
 * same per-cell algorithm as rhd_source_update -- the FP64 form's passes, or
 * the mixed form's three phases (FP32 passes, correction step, FP64 passes for
 * the cells the correction leaves), each grid's phases handing over through
 * its own part of the context's workspace.  The grids fall into
 * RHD_BATCH_BUCKETS buckets by group count (bucket 0: 1..16, 1: 17..32, 2:
 * 33..64 groups); the grids of a bucket share a mapping of cells to lanes and
 * their own queues, and the buckets run side by side on separate streams.  A
 * mapping is a number of lanes per cell: 1 (one cell per thread) or a segment
 * of 8, 16 or 32 lanes of a warp, each lane holding (the bucket's largest
 * group count / lanes) groups in registers; the passes and the correction step
 * have a mapping each (rhd_context_set_mapping lists the choices).  The
 * defaults are the one-grid call's mappings, so that a batched call gives
 * every cell exactly as rhd_source_update gives it; rhd_context_autotune
 * picks them by timing.  RHD_CELL_PER_THREAD has no effect here.  The call is
 * recorded once as a CUDA graph (descriptor upload, queue reset, table setup,
 * the phases) and replayed while the number of grids, the work items and the
 * mappings are unchanged.  A context owns the workspace (descriptors, tables,
 * queue heads; mixed form 32 bytes per cell-group + 34 per cell of every
 * grid, grown on demand), the graph and the tuned mappings; it is not
 * thread-safe, and a call waits (host side) for the previous call of the same
 * context to finish reading its host staging buffers.  The operation on each
 * cell is the implicit source update of Sec. 3 (the same as
 * rhd_source_update); batching several grids into one launch has no
 * counterpart in the paper, which updates one patch at a time.
 * Errors: RHD_EINVAL (null context or grids, n_grids < 1, grids of mixed
 * precision, or a per-grid check of rhd_source_update failing), RHD_ELAW (free
 * slopes), RHD_ESIZE (n_grids > RHD_MAX_GRIDS or a grid with more than
 * RHD_MAX_GROUPS_BATCHED groups), RHD_ENOMEM, RHD_ECUDA; on any error nothing
 * was launched. */
#define RHD_MAX_GROUPS_BATCHED 64
#define RHD_MAX_GRIDS 4096
#define RHD_BATCH_BUCKETS 3

typedef struct rhd_context rhd_context_t;

typedef struct {
  rhd_state_t state;               /* as for rhd_source_update (group_stride allowed) */
  rhd_groups_t groups;
  rhd_opacity_law_t opacity_law;
  double dt;
  int64_t n_cells;
} rhd_grid_t;

/* Create / destroy a context on the current device.  The first batched call
 * allocates the workspace (make it before any stream capture). */
int rhd_context_create(rhd_context_t **ctx);
int rhd_context_destroy(rhd_context_t *ctx);

/* Advance every grid (in place).  All grids must use the same precision. */
int rhd_source_update_batched(rhd_context_t *ctx, const rhd_grid_t *grids, int32_t n_grids,
                              void *stream);

/* Pick each bucket's mappings and the CTA shape by timing them on these
 * grids: per bucket (on its own grids) every mapping of the passes, then
 * (mixed form) every mapping of the correction step; then the CTA size x cells
 * per work item of the one-cell-per-thread mapping (threads 64, 128, 256;
 * items of 1, 4 or 16 CTAs' worth of cells).  Each candidate is timed as the
 * best of two uncaptured calls.  The grids' state is saved to a temporary
 * device copy first and restored after each candidate, so it is unchanged on
 * return; the call synchronizes the stream.  On an error the mappings are
 * left as they were. */
int rhd_context_autotune(rhd_context_t *ctx, const rhd_grid_t *grids, int32_t n_grids,
                         void *stream);

/* The CTA shape of the one-cell-per-thread mapping (threads per CTA, cells
 * per work item). */
int rhd_context_shape(const rhd_context_t *ctx, int32_t *threads, int32_t *cells_per_item);

/* Read or set bucket `bucket`'s mappings, as lanes per cell: `passes` for the
 * FP32 and FP64 passes (bucket 0: 0, 1 or 8; bucket 1: 0, 1, 8, 16 or 32;
 * bucket 2: 0, 1, 16 or 32), `correction` for the mixed form's correction
 * step (bucket 0: 8; bucket 1: 8 or 16; bucket 2: 16 or 32).  Passes 0 means
 * the one-grid call's mapping for the call's precision: in the mixed form 8,
 * 16 and 32 lanes (its FP32 passes' mapping, which the FP64 passes of the
 * cells the correction leaves follow), in the FP64 form 1, 1 and 32.
 * Defaults: passes 0, 0, 0; correction 8, 16, 32.  RHD_EINVAL for another
 * bucket or mapping (nothing changed). */
int rhd_context_mapping(const rhd_context_t *ctx, int32_t bucket, int32_t *passes,
                        int32_t *correction);
int rhd_context_set_mapping(rhd_context_t *ctx, int32_t bucket, int32_t passes,
                            int32_t correction);

/* ---- Learned warm start ----------------------------------------------------
 * A small MLP (features 2 N_g + 4 -> 128 -> 128 -> 128 -> N_g + 1, GELU, BF16
 * weights and activations, FP32 accumulation on the tensor cores; FP32 master
 * parameters, Adam) that maps a cell's state to a guess of the result of the
 * implicit update: ln(T_new / T) and ln(E_g,new / E_g).  The guess becomes the
 * starting point of the Newton iteration of Sec. 3, which still runs to the
 * caller's tolerance; a cell whose warm-started solve does not converge is
 * solved again from the cold start (status RHD_STATUS_FALLBACK).  The paper
 * has no counterpart: it always starts from the state at the beginning of the
 * step.  Features of a cell: ln rho, ln T, ln(E_g / a_R T^4) (N_g),
 * |F_g| / (c E_g) (N_g), |v| / c, ln(c rho kappa0 dt); both features and
 * targets are standardised with moments fitted on the training set.
 * All float pointers are DEVICE pointers, row-major [rows][columns].  A
 * surrogate belongs to the device current at creation and is not thread-safe. */
#define RHD_SURROGATE_MAX_GROUPS 64

typedef struct rhd_surrogate rhd_surrogate_t;

/* Create with random initial weights (seeded); 1 <= n_groups <= 64. */
int rhd_surrogate_create(int32_t n_groups, uint64_t seed, rhd_surrogate_t **s);
int rhd_surrogate_destroy(rhd_surrogate_t *s);
/* n_features = 2 n_groups + 4, n_outputs = n_groups + 1, n_params = length of the flat
 * parameter vector [W1 (128 x n_features), b1, W2, b2, W3, b3, W4 (n_outputs x 128), b4]. */
int rhd_surrogate_dims(const rhd_surrogate_t *s, int32_t *n_features, int32_t *n_outputs,
                       int64_t *n_params);
/* Raw features x [n_cells][n_features] of a grid (state as for rhd_source_update). */
int rhd_surrogate_features(const rhd_surrogate_t *s, const rhd_state_t *state,
                           const rhd_groups_t *groups, const rhd_opacity_law_t *opacity_law,
                           double dt, int64_t n_cells, float *x, void *stream);
/* Raw targets y [n_cells][n_outputs] from the same grid before and after an update. */
int rhd_surrogate_targets(const rhd_surrogate_t *s, const rhd_state_t *before,
                          const rhd_state_t *after, const rhd_groups_t *groups,
                          const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                          float *y, void *stream);
/* Fit the standardisation (per-column mean and deviation) on n >= 2 samples. */
int rhd_surrogate_fit_normalization(rhd_surrogate_t *s, const float *x, const float *y, int64_t n,
                                    void *stream);
/* Copy the flat FP32 parameters and/or the standardisation [x_mean, x_sd, y_mean, y_sd]
 * out (set = 0) or in (set = 1; setting parameters resets the Adam state).  Either
 * pointer may be NULL. */
int rhd_surrogate_params(rhd_surrogate_t *s, float *params, float *normalization, int32_t set,
                         void *stream);
/* Mean squared error (standardised targets) and its gradient with respect to the
 * flat parameters on rows [0, n) of raw x, y (n a multiple of 8); loss and grad
 * may be NULL. */
int rhd_surrogate_loss_grad(rhd_surrogate_t *s, const float *x, const float *y, int64_t n,
                            float *loss, float *grad, void *stream);
/* One Adam step (lr; beta 0.9, 0.999; eps 1e-8) on the batch of rows
 * (perm_mult (first + j) + perm_add) mod n_rows, j < batch (batch a multiple of 8;
 * perm_mult coprime with n_rows makes each epoch a permutation).  loss (device
 * float, may be NULL) is incremented by the batch's mean squared error. */
int rhd_surrogate_train_step(rhd_surrogate_t *s, const float *x, const float *y, int64_t n_rows,
                             int64_t first, int64_t batch, int64_t perm_mult, int64_t perm_add,
                             float lr, float *loss, void *stream);
/* Raw outputs y [n][n_outputs] for raw features x [n][n_features]. */
int rhd_surrogate_predict(rhd_surrogate_t *s, const float *x, int64_t n, float *y, void *stream);
/* 1 if a tensor-core wait of this surrogate ever timed out (results then invalid). */
int rhd_surrogate_error(rhd_surrogate_t *s, int32_t *flag);
/* Test support for the bounded waits (no counterpart in the paper): with on != 0
 * the surrogate's tensor-core GEMMs (training and rhd_surrogate_predict) issue no
 * MMA, so each one's first barrier wait gives up after a few polls with nothing
 * asynchronous in flight; the kernel sets the error flag that rhd_surrogate_error
 * reads, releases its tensor memory and returns, and the device stays usable.
 * Outputs of calls made meanwhile are meaningless; on = 0 restores the normal
 * path (the flag stays set for this surrogate). */
int rhd_surrogate_test_wait_timeout(rhd_surrogate_t *s, int32_t on);
/* Save the network (parameters and standardisation, not the Adam moments) to a
 * file: a 32-byte header -- the 8 bytes "RHDMLP1\0", int32 n_groups,
 * n_features, n_outputs, int32 0 (padding), int64 n_params -- then n_params FP32
 * parameters and 2 (n_features + n_outputs) FP32 standardisation values, all
 * little-endian.  Synchronises the device.  RHD_EIO when the file cannot be
 * written. */
int rhd_surrogate_save(rhd_surrogate_t *s, const char *path);
/* Save the training state as well: the same header with the magic "RHDMLP2\0",
 * the same parameters and standardisation, then the Adam first and second
 * moments (n_params FP32 each) and the int64 count of Adam steps taken.  A
 * surrogate loaded from it continues training exactly where this one stands
 * (the training step is deterministic: the same batches give the same
 * parameters bit for bit).  Synchronises the device.  RHD_EIO when the file
 * cannot be written. */
int rhd_surrogate_checkpoint(rhd_surrogate_t *s, const char *path);
/* Create a surrogate on the current device from a file rhd_surrogate_save wrote
 * (Adam moments zero and step count 0, so training resumes with a fresh
 * optimiser state) or rhd_surrogate_checkpoint wrote (moments and step count
 * restored).  RHD_EIO when the file cannot be read or its header or length does
 * not match. */
int rhd_surrogate_load(const char *path, rhd_surrogate_t **out);
/* rhd_source_update (FP64 or mixed form, from state->precision) started from the
 * surrogate's guess; groups->n_groups must equal the surrogate's.  Same results to
 * the caller's tolerance; status RHD_STATUS_FALLBACK marks cells that needed the
 * cold start.  Uses the library's per-device workspace like the mixed form.  The
 * guess comes from one persistent tensor-core kernel (features, the four layers
 * with the activations kept on chip, the Newton start) over all n_cells. */
int rhd_source_update_warm(rhd_surrogate_t *s, rhd_state_t *state, const rhd_groups_t *groups,
                           const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                           void *stream);
/* The Newton start rhd_source_update_warm takes, without solving: eint [n_cells]
 * (DEVICE, FP64) gets the guess of the internal energy (-1 where the cell is
 * invalid or the guess is not finite: cold start), r [n_groups][n_cells]
 * (DEVICE, FP32, cell fastest) the guess of R_g / E_tot.  The state is read only. */
int rhd_surrogate_warm_start(rhd_surrogate_t *s, const rhd_state_t *state,
                             const rhd_groups_t *groups, const rhd_opacity_law_t *opacity_law,
                             double dt, int64_t n_cells, double *eint, float *r, void *stream);

/* ---- Host-resident state --------------------------------------------------------
 * rhd_source_update (surrogate == NULL) or rhd_source_update_warm (surrogate !=
 * NULL) for a grid whose state lives in HOST memory: every pointer of *state is a
 * host pointer (page-locked memory lets the copies overlap the solve; pageable
 * memory works, serialised), with the layout of rhd_state_t (group_stride of the
 * host arrays; 0 = n_cells).  The cells go through the GPU in chunks of
 * chunk_cells (0 = 2^20): chunk k+1 is copied in and chunk k-1 copied out on two
 * copy streams while chunk k is solved, through three device staging sets of the
 * library (grown on demand, per device, never freed: 3 x chunk x (8 (6 + 5 N_g) + 2)
 * bytes).  Each chunk is one rhd_source_update / rhd_source_update_warm call, so
 * the results are those of the device entry, cell for cell.  Synchronous: returns
 * when the host arrays (E_gas, rho v, E_g, F_g, status, iters) hold the result,
 * or with the first error (every transfer started has then ended).  Calls on the
 * same device must not overlap. */
int rhd_source_update_host(rhd_state_t *state, const rhd_groups_t *groups,
                           const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                           rhd_surrogate_t *surrogate, int64_t chunk_cells);

/* ---- Benchmark support -------------------------------------------------------
 * Time the solver launches of every rhd_source_update / rhd_source_update_warm
 * call this thread makes between rhd_profile_start and rhd_profile_stop, with
 * CUDA events recorded on the call's stream right before and after each launch.
 * rhd_profile_stop synchronizes those events and returns the number of timed
 * launches and their summed duration in milliseconds, over all kinds of launch.
 * Not part of the method; no counterpart in the paper. */
int rhd_profile_start(void);
int rhd_profile_stop(int32_t *launches, double *total_ms);

/* The same events around each kind of launch: after rhd_profile_stop,
 * rhd_profile_kernel returns the launches of one kind and their summed
 * duration (RHD_EINVAL for an unknown kind). */
#define RHD_KERNEL_FP32 0       /* the mixed form's FP32 passes */
#define RHD_KERNEL_CORRECTION 1 /* its correction step (FP64 residual, FP32 Newton step) */
#define RHD_KERNEL_FP64 2       /* the FP64 passes (the FP64 form; the mixed form's fallback) */
#define RHD_KERNEL_INFERENCE 3  /* the learned warm start's fused inference */
#define RHD_KERNEL_REFINE 4     /* the correction's first step (float-float residual) */
#define RHD_KERNELS 5
int rhd_profile_kernel(int32_t kind, int32_t *launches, double *total_ms);

/* ---- Event counts ------------------------------------------------------------
 * Counters of what the update calls of this thread did between rhd_events_start
 * and rhd_events_stop, summed over cells (a cell of N_g groups contributes each
 * event once, not per group): the benchmark multiplies them by the operations
 * per event of the counting model to get the algorithmic operations of a call.
 * rhd_events_start zeroes the counters of the current device; rhd_events_stop
 * synchronizes the device and copies RHD_EVENTS counters to counts.  Counting
 * costs one atomic add per event and cell; calls on other threads and the
 * batched entry are not counted.  Not part of the method; no counterpart in the
 * paper. */
#define RHD_EV_CELLS32 0     /* cells through the FP32 passes */
#define RHD_EV_EVAL32 1      /* FP32 inner evaluations (a4-a8) */
#define RHD_EV_OUTER32 2     /* FP32 outer passes (a9-a12) */
#define RHD_EV_CELLSC 3      /* cells through the correction step */
#define RHD_EV_RESID64 4     /* FP64 evaluations of the coupled residual */
#define RHD_EV_STEP32 5      /* FP32 Newton steps on the coupled system */
#define RHD_EV_FINISH64 6    /* cells the correction step finished */
#define RHD_EV_CELLS64 7     /* cells through the FP64 passes */
#define RHD_EV_EVAL64 8      /* FP64 inner evaluations */
#define RHD_EV_CACHED64 9    /* FP64 inner iterations taken from cached group terms */
#define RHD_EV_OUTER64 10    /* FP64 outer passes */
#define RHD_EV_FLUXNEWTON 11 /* group flux updates solved by Newton steps (slow cells) */
#define RHD_EV_INFER 12      /* cells through the warm start's inference */
#define RHD_EV_RESIDDF 13    /* float-float evaluations of the coupled residual */
#define RHD_EV_STEPDF 14     /* Newton steps taken from them */
#define RHD_EVENTS 15
int rhd_events_start(void);
int rhd_events_stop(uint64_t *counts);

/* The mixed-precision form without any device allocation.  Some callers
 * cannot let a library call cudaMalloc: a host that hands every byte of HBM
 * to its own memory pool up front, a latency-bound loop where a first-call
 * allocation (which synchronizes the device) is not acceptable, or code that
 * must never fail for lack of memory in the middle of a run.  This entry point
 * computes the same result as rhd_source_update with precision = RHD_MIXED
 * (state->precision is ignored) but keeps the FP32 pass's warm start in a
 * file-scope device array of RHD_NOALLOC_BYTES that every GPU loading the
 * library holds until process exit.  The caller still passes all inputs and
 * outputs.  Size limit: n_cells * (32 * n_groups + 34) + 1024 <=
 * RHD_NOALLOC_BYTES (64 MiB; at most 32,232 cells at 64 groups, 122,908 at 16);
 * larger calls return RHD_ESIZE and launch nothing.  The paper has no counterpart: this is a
 * deployment variant of the same kernels.  The first call on a device looks up
 * the array's device address (and initialises the constant tables), so make
 * it before any stream capture.  All calls share the one array and nothing in
 * it needs to start at zero (each call writes every slot it reads), but calls
 * that overlap on the GPU (other streams, other threads) race on it: serialise
 * them. */
#define RHD_NOALLOC_BYTES ((int64_t)64 << 20)
int rhd_source_update_noalloc(rhd_state_t *state, const rhd_groups_t *groups,
                              const rhd_opacity_law_t *opacity_law, double dt, int64_t n_cells,
                              void *stream);

/* Text for a return code. */
const char *rhd_strerror(int code);

/* Library version (major*10000 + minor*100 + patch). */
int rhd_version(void);

#ifdef __cplusplus
}
#endif
#endif
