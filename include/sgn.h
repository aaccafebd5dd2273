/*
 * sgn.h — C ABI of the GB300 (sm_103a) library for the preconditioned constraint solve of
 * the Serre-Green-Naghdi (SGN) equations and the time integrators built on it.
 *
 * Paper: L. Feng, D. Shirokoff, W. Choi, "Preconditioning and Linearly Implicit Time
 * Integration for the Serre-Green-Naghdi Equations" (arXiv 2506.16045).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns sgn_status; no C++ exception crosses this boundary and the
 *    library never aborts the process.  sgn_last_error() gives a message for the last
 *    failure on a context.
 *  - Array arguments are DEVICE pointers owned by the caller (for example the data_ptr of
 *    a CUDA tensor), contiguous, float64.  The library owns only the workspace inside
 *    sgn_ctx, sgn_layout and sgn_state objects.
 *  - Calls are asynchronous on the given stream (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream).  A call that returns host-side information (info/out
 *    arrays) synchronises that stream first and says so.
 *  - Batches: a layout packs `count` independent periodic instances.  The real fields of
 *    instance i occupy [off_i, off_i + N_i) of every packed scalar array, with
 *    off_i = N_0 + ... + N_{i-1} and N_i = nx*ny.  A 1d vector field is one packed array;
 *    a 2d vector field is two packed planes: x components of all instances first, then y
 *    components (the plane stride is the layout's total point count P).  A 2d scalar field
 *    is row-major [ny][nx] (x fastest).
 *  - Grid (§6.1): x_j = j Lx/nx; spectral derivatives D = F^{-1}(iK)F with
 *    k_j = 2 pi j/L, j = -n/2+1..n/2-1, and the n/2 wavenumber set to 0.
 *    Sizes: a power of two (1d 8 <= nx <= 16384, where nx = 16384 runs each solve and
 *    right-hand side on a thread-block cluster of two CTAs; 2d 8 <= nx, ny <= 1024), or
 *    n = 2^a 3^b 5^c with a >= 1 (1d 6 <= nx <= 16384; 2d 6 <= nx, ny <= 1024) on generic
 *    kernels (see sgn_layout_create for what they serve).
 */
#ifndef SGN_H
#define SGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SGN_OK = 0,
  SGN_ERR_INVALID_ARG = 1,        /* null pointer, bad count, inconsistent grids */
  SGN_ERR_UNSUPPORTED_SIZE = 2,   /* a size outside the supported set (sgn_layout_create) */
  SGN_ERR_NOMEM = 3,              /* device allocation failed */
  SGN_ERR_CUDA = 4,               /* a CUDA runtime call failed (message in sgn_last_error) */
  SGN_ERR_NOT_CONVERGED = 5,      /* PCG hit maxit (or the refinement cap) before rtol */
  SGN_ERR_BREAKDOWN = 6,          /* NaN/Inf or p.Gp <= 0 inside PCG */
  SGN_ERR_NONPOSITIVE_DEPTH = 7,  /* eta_min <= 0 (or NaN): the theorem needs eta > 0 */
  SGN_ERR_PENDING = 8,            /* serving: request not finished */
  SGN_ERR_TIMEOUT = 9,            /* a bounded device wait gave up */
  SGN_ERR_REJECTED = 10           /* serving: request footprint above the memory budget */
} sgn_status;

typedef struct sgn_ctx sgn_ctx;
typedef struct sgn_layout sgn_layout;
typedef struct sgn_state sgn_state;
typedef void* sgn_stream;         /* cudaStream_t */

/* One periodic grid.  dim = 1: ny must be 1 and Ly is ignored.  g is the gravity constant
 * (the paper sets g = 1 after non-dimensionalising, §2.1; it is kept explicit here). */
typedef struct {
  int dim;
  int nx, ny;
  double Lx, Ly;
  double g;
} sgn_grid;

/* Preconditioner A = sigma I - alpha grad(div) (Def:A, §4) and the bound kappa_ub on the
 * condition number of A^{-1}G (Theorem 4.1).  flat = 1 when max|grad h| <= 1e-12. */
typedef struct {
  double sigma, alpha, kappa_ub;
  int flat;
} sgn_precond;

typedef enum {
  SGN_COEF_OPT = 0,               /* Eq:FlatbathCoeff / Eq:Optcoeff / Eq:Optcoeffb (§4) */
  SGN_COEF_REPLACEMENT = 1        /* sigma**, alpha** of the replacement remark (§4) */
} sgn_coef_kind;

typedef enum {
  SGN_PREC_FP64 = 0,              /* every operation in float64 */
  SGN_PREC_MIXED = 1              /* float32 inner PCG (matvecs, FFTs, vectors) with float64
                                     dot accumulation, inside float64 iterative refinement */
} sgn_precision;

typedef struct {
  int iters;                      /* PCG iterations (summed over refinements when mixed) */
  int refinements;                /* float32 inner solves (mixed), 0 for FP64 */
  double rel_resid_Ainv;          /* sqrt(r.A^{-1}r)/sqrt(b.A^{-1}b) at exit (float64 residual) */
  int status;                     /* sgn_status of this instance */
} sgn_pcg_info;

/* ---------------------------------------------------------------------------------- */
/* Context and layouts                                                                 */
/* ---------------------------------------------------------------------------------- */

/* Creates a context on `device` (made current for the call).  Allocates the twiddle
 * tables (~640 KB).  workspace_bytes is a hint (0 = grow on demand). */
sgn_status sgn_create(sgn_ctx** ctx, int device, size_t workspace_bytes);
void sgn_destroy(sgn_ctx* ctx);
const char* sgn_last_error(const sgn_ctx* ctx);
const char* sgn_status_string(sgn_status s);

/* Packs `count` instances (host array `grids`).  1d batches may mix sizes.  1d sizes: a
 * power of two with 8 <= n <= 16384, or n = 2^a 3^b 5^c (a >= 1) with 6 <= n <= 16384
 * (the grids of §6.1 at sizes such as 96, 384, 1536 or 12288).  The latter run on generic
 * kernels (one CTA per instance, a mixed-radix transform in shared memory up to n = 6144,
 * in a global buffer of the layout above) for the spectral gradient,
 * the coefficients, G, A^{-1}, PCG (both precisions), GMRES, the right-hand side and the
 * RK4 / Adams-Bashforth steppers; dealiasing, SBDF2 (sgn_step_linimp), the non-constraint
 * stepper and sgn_pcg1d_noalloc take powers of two only (SGN_ERR_UNSUPPORTED_SIZE).  2d
 * sides: powers of two with 8 <= n <= 1024, or n = 2^a 3^b 5^c (a >= 1) with
 * 6 <= n <= 1024 (such as 384 x 240).  A 2d grid with a side that is not a power of two
 * runs on generic kernels (full complex spectra, mixed-radix row and column passes) for
 * the same calls as the 1d generic sizes, with device-driven solves (one cached graph per
 * precision) and float64 right-hand sides; it takes no batches, no
 * inner-solve forms (sgn_layout_set_form2d, sgn_profile_inner2d) and the same power-of-two
 * options as 1d.  Other sizes: SGN_ERR_UNSUPPORTED_SIZE.  A 2d layout of
 * count > 1 (at most 32) is a batch of instances on one grid (every sgn_grid equal); it
 * serves sgn_spectral_grad, sgn_precond_coeffs, sgn_apply_operator, sgn_precond_solve,
 * sgn_pcg and sgn_pcg_async, whose mixed-precision solves advance the float32 inner PCG of
 * every instance in one persistent launch per refinement pass; sgn_gmres, sgn_rhs and
 * states take single 2d instances (SGN_ERR_INVALID_ARG).  Allocates the layout's device
 * descriptors and
 * spectral workspace.  Every call on a layout (and on the states bound to it) uses that
 * workspace, so calls on one layout must be ordered: issue them on one stream, or order
 * the streams; independent work runs concurrently on separate layouts. */
sgn_status sgn_layout_create(sgn_ctx* ctx, int count, const sgn_grid* grids, sgn_layout** out);
void sgn_layout_destroy(sgn_layout* lay);
/* Total packed points P (per component). */
long long sgn_layout_points(const sgn_layout* lay);
/* Kernel forms of a 1d layout's size classes.  The solve and the right-hand side of the
 * instances of n = 2^log2n run on one CTA per instance (ctas = 1, n <= 8192) or on a
 * thread-block cluster of two CTAs per instance that splits the instance's points and
 * modes between them (ctas = 2, n = 4096, 8192 and 16384; the only form of n = 16384).
 * The two forms agree up to rounding (their dot products add in another order).  A batch
 * that fills the GPU runs fastest on one CTA per instance; a few large instances run with
 * less latency on clusters.  Default: 1 below n = 16384.  set_form: SGN_ERR_INVALID_ARG on
 * a 2d layout or bad arguments, SGN_ERR_UNSUPPORTED_SIZE for a form the size lacks.
 * States step with the new forms from their next step. */
sgn_status sgn_layout_set_form(sgn_layout* lay, int log2n, int ctas);
sgn_status sgn_layout_get_form(const sgn_layout* lay, int log2n, int* ctas);
/* The same with separate forms for the solve and the right-hand side of the class (the
 * solve hands u_x to the right-hand side in natural point order under either form, so any
 * pair is valid).  sgn_layout_set_form(l, c) is set_forms(l, c, c); get_form reports the
 * solve's form. */
sgn_status sgn_layout_set_forms(sgn_layout* lay, int log2n, int solve_ctas, int rhs_ctas);
sgn_status sgn_layout_get_forms(const sgn_layout* lay, int log2n, int* solve_ctas,
                                int* rhs_ctas);

/* Kernel form of a 2d layout's float32 inner solves (the mixed-precision PCG).
 * inner = 0: one persistent cooperative launch per inner solve, whose CTAs (four
 * independent thread groups each) run the column passes, the row passes with the pointwise
 * step and the vector updates behind grid-wide barriers (the default); inner = 1: four
 * kernels per inner iteration inside a device-side loop.  tile_width: half-spectrum columns
 * per column unit of the persistent form (0 or 1: one column).  Both forms run the same PCG
 * (§3.2) and agree up to rounding.  SGN_ERR_INVALID_ARG on a 1d layout or bad arguments,
 * SGN_ERR_UNSUPPORTED_SIZE for another tile width. */
sgn_status sgn_layout_set_form2d(sgn_layout* lay, int inner, int tile_width);
sgn_status sgn_layout_get_form2d(const sgn_layout* lay, int* inner, int* tile_width);
/* Radix plan of the persistent 2d inner solve's transforms (§6.1 D by FFT): the stages of a
 * length-2^k transform have radices up to max_radix (8, the default, or 16), split as evenly
 * as possible (1024 = 8 x 8 x 4 x 4 with 8; 16 x 8 x 8 with 16).  Both plans compute the
 * same transform and agree up to rounding.  0 restores the default.  SGN_ERR_INVALID_ARG on
 * a 1d layout or another value, SGN_ERR_UNSUPPORTED_SIZE on a grid with a side that is not a
 * power of two.  sgn_state_autotune times the plans with the inner-solve forms. */
sgn_status sgn_layout_set_radix2d(sgn_layout* lay, int max_radix);
sgn_status sgn_layout_get_radix2d(const sgn_layout* lay, int* max_radix);
/* Threads per unit of the persistent 2d inner solve (a unit is one half-spectrum column or
 * one pair of rows, whose three transforms one thread group computes): 128 (four groups per
 * CTA), 256 (two groups per CTA: each unit in about half the time, half as many units in
 * flight), or 0, the default: 256 when the solve's largest phase has at most one unit per
 * 256-thread group of the grid (a single 512^2 instance), else 128.  Every choice runs the
 * same PCG (§3.2) and the results agree up to rounding.  The getter returns the setting (0
 * for the default).  SGN_ERR_INVALID_ARG on a 1d layout or another value,
 * SGN_ERR_UNSUPPORTED_SIZE on a grid with a side that is not a power of two. */
sgn_status sgn_layout_set_unit_threads2d(sgn_layout* lay, int threads);
sgn_status sgn_layout_get_unit_threads2d(const sgn_layout* lay, int* threads);

/* offsets[0..count]: start of each instance in a packed scalar array (host array). */
sgn_status sgn_layout_offsets(const sgn_layout* lay, long long* offsets);

/* ---------------------------------------------------------------------------------- */
/* Hot-path operations                                                                 */
/* ---------------------------------------------------------------------------------- */

/* Spectral gradient (§6.1): gradf = D f.  f: packed scalar [P]; gradf: packed vector
 * ([P] in 1d, [2P] in 2d).  Used for grad h (the discrete bathymetry slope). */
sgn_status sgn_spectral_grad(sgn_ctx* ctx, const sgn_layout* lay, const double* f, double* gradf,
                             sgn_stream stream);

/* Preconditioner coefficients (Eq:MaxMinWaveFields, Eq:FlatbathCoeff, Eq:Optcoeff,
 * Eq:Optcoeffb; replacement coefficients of §4).  eta: [P]; gradh: vector.  out: HOST
 * array [count]; the call synchronises the stream.  Returns SGN_ERR_NONPOSITIVE_DEPTH if
 * some instance has eta_min <= 0. */
sgn_status sgn_precond_coeffs(sgn_ctx* ctx, const sgn_layout* lay, const double* eta,
                              const double* gradh, sgn_coef_kind kind, sgn_precond* out,
                              sgn_stream stream);

/* Constraint operator (Def:G, §2.2):
 *   Gu = eta u - grad(eta^3/3 div u) - grad(eta^2/2 grad h.u) + eta^2/2 grad h (div u)
 *        + eta grad h (grad h.u).
 * eta: [P]; gradh, u, Gu: vectors.  float64. */
sgn_status sgn_apply_operator(sgn_ctx* ctx, const sgn_layout* lay, const double* eta,
                              const double* gradh, const double* u, double* Gu, sgn_stream stream);

/* Preconditioner solve z = A^{-1} r with A = sigma I - alpha grad(div) (Def:A): per
 * Fourier mode 1/(sigma + alpha k^2) in 1d, (sigma I + alpha k k^T)^{-1} in 2d.  P: HOST
 * array [count] of coefficients (from sgn_precond_coeffs or the caller). */
sgn_status sgn_precond_solve(sgn_ctx* ctx, const sgn_layout* lay, const sgn_precond* P,
                             const double* r, double* z, sgn_stream stream);

/* Preconditioned conjugate gradients for G_{eta,h} x = b with preconditioner A (§3.2,
 * Eq:PCGLinSyst; §4).  x holds the initial guess on entry and the solution on exit.
 * Stops when sqrt(r.A^{-1}r) <= rtol sqrt(b.A^{-1}b).  P: HOST array [count] or NULL to
 * compute the optimal coefficients per instance on the device.  prec = SGN_PREC_MIXED runs
 * float32 PCG inner solves inside float64 iterative refinement (the refinement residual
 * b - Gx, the dot accumulations and x are float64).  info: HOST array [count] or NULL;
 * when non-NULL the call synchronises the stream and returns the worst instance status. */
sgn_status sgn_pcg(sgn_ctx* ctx, const sgn_layout* lay, const double* eta, const double* gradh,
                   const sgn_precond* P, const double* b, double* x, double rtol, int maxit,
                   sgn_precision prec, sgn_pcg_info* info, sgn_stream stream);

/* The solve of sgn_pcg without any host synchronisation: the report goes to DEVICE
 * memory.  The preconditioner coefficients are the optimal ones (Eq:Optcoeff, §4), computed
 * per instance on the device, as the time steppers use them.  info: DEVICE array [count]
 * of sgn_pcg_info, written on `stream` after the solve; read it once the stream (or an
 * event recorded on it after this call) has completed.  Returns SGN_OK when the work was
 * issued; each instance's outcome (SGN_ERR_NOT_CONVERGED, SGN_ERR_BREAKDOWN,
 * SGN_ERR_NONPOSITIVE_DEPTH) is in its info.status.  A 2d solve on a stream that is being
 * captured takes the host-driven path, which synchronises. */
sgn_status sgn_pcg_async(sgn_ctx* ctx, const sgn_layout* lay, const double* eta,
                         const double* gradh, const double* b, double* x, double rtol, int maxit,
                         sgn_precision prec, sgn_pcg_info* info, sgn_stream stream);

/* Restarted GMRES(restart) for G_{eta,h} x = b, right-preconditioned by the A of §4: the
 * Krylov option besides sgn_pcg.  G is symmetric positive definite, where PCG (§3.2) is the
 * paper's method and the cheaper one; GMRES is the solver for a non-symmetric variant of
 * the operator and a cross-check of PCG.  Textbook method in the A^{-1} inner product
 * <u, v> = u . A^{-1} v: Arnoldi on G A^{-1} (classical Gram-Schmidt with one
 * reorthogonalisation), Givens rotations, x += A^{-1} V y per cycle.  Each iterate minimises
 * sqrt(r.A^{-1}r), the residual measure of sgn_pcg's stopping rule; the Euclidean residual
 * of a fine grid has a rounding floor near eps ||G|| that this measure damps.  float64
 * throughout.  Each instance stops when sqrt(r.A^{-1}r) <= rtol sqrt(b.A^{-1}b): inside a
 * cycle through the rotated right-hand side, and on the true residual at every restart.
 * maxit bounds the Arnoldi steps over all cycles; b = 0 gives x = 0 in 0 steps.
 *   P: per-instance coefficients, or NULL to compute them (Eq:Optcoeff) as sgn_pcg does.
 *   x: in: initial guess, out: solution.  restart: 1..SGN_GMRES_MAX_RESTART.
 *   info: HOST array [count] or NULL; iters = Arnoldi steps, refinements = cycles,
 *   rel_resid_Ainv = the final true sqrt(r.A^{-1}r) / sqrt(b.A^{-1}b), status.
 * The call allocates 2 (restart + 2) vectors of the layout's packed size on the stream,
 * synchronises the stream every four Arnoldi steps and at the end of each cycle (the host
 * drives the cycles) and before returning, and returns the worst instance status (SGN_ERR_NOT_CONVERGED at maxit,
 * SGN_ERR_BREAKDOWN on NaN/Inf, SGN_ERR_NONPOSITIVE_DEPTH from the coefficients). */
#define SGN_GMRES_MAX_RESTART 64
sgn_status sgn_gmres(sgn_ctx* ctx, const sgn_layout* lay, const double* eta, const double* gradh,
                     const sgn_precond* P, const double* b, double* x, double rtol, int restart,
                     int maxit, sgn_pcg_info* info, sgn_stream stream);

/* Right-hand side of the DAE form (Eq:DAE_DSWE, §5): f_eta = -div(eta u),
 * f_U = -g eta grad(zeta) - div(eta u (x) u) + F(eta, u, h) with F from Def:bigF and
 * (u.grad)^2 h read as u.grad(u.grad h).  zeta = eta - h.  float64. */
sgn_status sgn_rhs(sgn_ctx* ctx, const sgn_layout* lay, const double* eta, const double* u,
                   const double* h, const double* gradh, double* f_eta, double* f_U,
                   sgn_stream stream);

/* ---------------------------------------------------------------------------------- */
/* Time integration (§5)                                                               */
/* ---------------------------------------------------------------------------------- */

typedef struct {
  double rtol;                    /* constraint-solve tolerance (stopping rule of sgn_pcg) */
  int maxit;                      /* PCG iteration cap per solve */
  sgn_precision prec;             /* FP64 or MIXED constraint solves */
  sgn_coef_kind coef;             /* preconditioner coefficients for the PCG solves */
  double rtol_inner;              /* mixed: float32 inner tolerance; 0 = adaptive: each inner
                                     solve targets 0.3 rtol / (current residual ratio),
                                     clamped to [1e-6, 0.1] */
  int max_refine;                 /* mixed: refinement cap (0 = 12) */
} sgn_opts;

typedef struct {
  long long solves;               /* constraint solves since init */
  long long iterations;           /* PCG iterations since init */
  int max_iters;                  /* largest iteration count of one solve */
  int status;                     /* worst status seen (sticky) */
  double t;                       /* simulated time of instance 0 */
  long long step;                 /* steps taken */
  double flops32;                 /* algorithmic float32 flops of the PCG solves */
  double flops64;                 /* algorithmic flops of the solves' high-precision part:
                                     float64 for SGN_PREC_FP64, double-float (pairs of
                                     float32) for SGN_PREC_MIXED */
  long long refinements;          /* SGN_PREC_MIXED: float32 inner solves (refinement passes
                                     less one per solve) since init; 0 for FP64 */
  long long sbdf2_stability_warnings; /* SBDF2 instance-steps whose eta_max had grown past
                                     (4/3)^(1/3) of its value at sgn_state_init: A is fixed
                                     from the initial data (§6.5), and the generalised
                                     eigenvalues of A^{-1} G then may leave SBDF2's
                                     zero-stability interval (0, 4/3) (§5.4).  A warning, not
                                     an error: re-initialise the state to refresh A */
} sgn_state_stats;

/* Binds caller-owned packed arrays: eta [P], U (vector), u (vector), h [P], gradh (vector,
 * written by sgn_state_init).  Allocates the library-owned stage/history workspace. */
sgn_status sgn_state_create(sgn_ctx* ctx, const sgn_layout* lay, double* eta, double* U,
                            double* u, const double* h, double* gradh, sgn_state** out);
/* gradh = D h, U = G_{eta,h} u (Eq:DSWEcf4), clears history and counters. */
sgn_status sgn_state_init(sgn_state* st, sgn_stream stream);
/* Classical RK4 with one constraint solve per stage 2..4 and one for u_{n+1} (Eq:ERK,
 * §5.1); U stages start from U_n.  dt: HOST array [count] (per-instance step).  The stage-4
 * solve starts from 2 u^(3) - u_n (u extrapolated to its stage time), which changes only
 * the initial guess. */
sgn_status sgn_step_rk4(sgn_state* st, const double* dt, int nsteps, const sgn_opts* opts,
                        sgn_stream stream);
/* Adams-Bashforth of order 2..4 (Eq:AB, Table 1, §5.2), one solve per step; the first
 * order-1 steps after init are RK4 steps of the same dt. */
sgn_status sgn_step_abk(sgn_state* st, int order, const double* dt, int nsteps,
                        const sgn_opts* opts, sgn_stream stream);
/* RK4 on the non-constraint form of the SGN equations (Eq:dswe; the remark of §5 that the
 * same time discretisations apply to it), 1d and 2d.  The state advances (eta, u) with the
 * RK4 tableau of sgn_step_rk4; each stage takes eta_t = -div(eta u) and u_t from
 * G_{eta,h} u_t = M, where M collects the u_t-free terms of Eq:MomEq
 * (M = -eta (u.grad)u - g eta grad zeta + grad(eta^3 Q/3 + eta^2 S/2)
 *  - grad h (eta^2 Q/2 + eta S), Q = u.grad(div u) - (div u)^2, S = u.grad(grad h.u)),
 * solved by the PCG of sgn_pcg with the options (warm start from the previous u_t; the
 * stage at c = 1 from 2 u_t(c = 1/2) - u_t(c = 0)).
 * U = G u is refreshed after every step, so other steppers can continue from the state.
 * Right-hand side transforms: 1d in float64, or double-float on the mixed path; 2d in
 * float64.  SGN_ERR_INVALID_ARG for a state with a forcing or dealiasing set. */
sgn_status sgn_step_rk4_nc(sgn_state* st, const double* dt, int nsteps, const sgn_opts* opts,
                           sgn_stream stream);
/* Linearly implicit SBDF2 (Eq:MM with Table 1's SBDF2 row, §5.3): one A-solve per step,
 * no Krylov iteration; A fixed from the state at init (§6.5).  The first step after init
 * is an RK4 step. */
sgn_status sgn_step_linimp(sgn_state* st, const double* dt, int nsteps, const sgn_opts* opts,
                           sgn_stream stream);
/* External forcing of the time steppers, as Test 1 of §6.4 (manufactured solutions) adds
 * to the SGN equations: a finite Fourier series in time,
 *   f_eta += sum_k cos(omega_k t + theta_k) phi_eta_k,  f_U += sum_k cos(omega_k t + theta_k) phi_U_k,
 * added to every right-hand side evaluation of sgn_step_rk4 / _abk / _linimp at its stage
 * time t (per instance; t = 0 at sgn_state_init, advanced by each instance's dt).
 * phi_eta: DEVICE array [nterms][P] packed like eta; phi_U: DEVICE array [nterms][d P]
 * packed like U.  Both stay owned by the caller and are read at every step, so they must
 * outlive the state's use of them.  omega, theta: HOST arrays [nterms], copied.
 * 0 <= nterms <= SGN_MAX_FORCING; nterms = 0 removes the forcing.  SGN_ERR_INVALID_ARG on a
 * bad count, a null array with nterms > 0, or a non-finite omega / theta. */
#define SGN_MAX_FORCING 16
sgn_status sgn_state_set_forcing(sgn_state* st, int nterms, const double* phi_eta,
                                 const double* phi_U, const double* omega, const double* theta);
/* Dealiasing of a state (on = 1; 0 turns it off; default off, as in the paper's runs).
 * The paper reports that large solitary waves destabilise over long times without
 * dealiasing and that dealiasing (there by zero padding) helps (§6.4, Test 2).  Here it is
 * Orszag's 2/3 rule: every new time level has the Fourier modes |j| > n/3 (2d: |jx| > nx/3
 * or |jy| > ny/3) of zeta = eta - h and of U set to zero before u is solved from it (RK4,
 * AB2-4), and of u as well in the SBDF2 step, whose u is not solved from U; intermediate
 * RK4 stages are not projected.  Transforms: 1d in float64, or double-float on the mixed
 * path; 2d in float64.  Applies from the next step call. */
sgn_status sgn_state_set_dealias(sgn_state* st, int on);
/* Autotuner of the layout's kernel forms (sgn_layout_set_forms) on this state's own
 * problem: for every combination of forms of the n = 4096 and 8192 classes (solve and
 * right-hand side chosen separately: up to 16 combinations), one untimed and three timed
 * RK4 steps with these dt (HOST [count]) and options, each from the same state, in two
 * passes keeping each combination's faster one.  The default (one CTA per instance) stays
 * unless another combination is at least 3% faster; the choice stays set on the layout.
 * The state (eta, U, u, time, counters) is restored afterwards, so tuning leaves no trace
 * on the solution.  Allocates and frees 3 P doubles; synchronises `stream`; best_ms
 * (nullable, host) receives the chosen time per step.  A 1d state without such classes is
 * left as it is.  For a 2d state it chooses the layout's inner-solve form, radix plan and
 * threads per unit (sgn_layout_set_form2d, sgn_layout_set_radix2d and
 * sgn_layout_set_unit_threads2d: the persistent launch with radix-8 stages and units sized
 * by their count, with 128 or with 256 threads per unit, with radix-16 stages, or four
 * kernels per inner iteration) the same way: each candidate timed on RK4 steps from the same
 * state in two passes, the default (persistent, radix 8, units sized by their count) kept
 * unless another is at least 3% faster, the state restored.  A 2d grid with a side that is
 * not a power of two has one form: nothing to choose. */
sgn_status sgn_state_autotune(sgn_state* st, const double* dt, const sgn_opts* opts,
                              sgn_stream stream, double* best_ms);
/* Synchronises the stream used by the last step call and reports counters. */
sgn_status sgn_state_get_stats(sgn_state* st, sgn_state_stats* out);
void sgn_state_free(sgn_state* st);

/* ---------------------------------------------------------------------------------- */
/* Serving: continuous batching of constraint solves and SGN runs on one GPU            */
/* ---------------------------------------------------------------------------------- */

/* A server admits requests against a device-memory budget, keeps their state on the
 * device, and advances every admitted request concurrently: 1d RK4 runs move together
 * through one batched launch per kernel (per-instance dt), pending 1d solves run as one
 * batched PCG, and 2d or multistep runs advance in per-request chunks.  Requests that
 * arrive while others run join at the next chunk boundary as memory frees up.  The paper
 * has no counterpart; each result equals the request run alone (RK4 is a one-step method
 * and every instance is computed by its own CTAs, so batching does not change a result). */
typedef struct sgn_server sgn_server;

typedef enum { SGN_REQ_SOLVE = 0, SGN_REQ_RUN = 1 } sgn_req_kind;
typedef enum {
  SGN_SCHEME_RK4 = 0,      /* Eq:ERK */
  SGN_SCHEME_AB2 = 2,      /* Eq:AB, Table 1 */
  SGN_SCHEME_AB3 = 3,
  SGN_SCHEME_AB4 = 4,
  SGN_SCHEME_LINIMP = 5    /* Eq:MM (SBDF2) */
} sgn_scheme;

typedef struct {
  sgn_req_kind kind;
  sgn_grid grid;           /* one instance */
  sgn_scheme scheme;       /* RUN only */
  double dt;               /* RUN only */
  int nsteps;              /* RUN only */
  sgn_opts opts;           /* solve options (rtol, maxit, precision, coefficients) */
  const double* eta;       /* [N] depth eta = h + zeta (the PCG coefficient for SOLVE) */
  const double* u_or_b;    /* RUN: initial velocity u; SOLVE: right-hand side b (vector) */
  const double* h;         /* [N] bathymetry (grad h = D h is formed on the device) */
  int host_memory;         /* 1: eta, u_or_b, h are host pointers; 0: device pointers */
} sgn_request;

typedef struct {
  sgn_status status;
  const double* eta;       /* RUN: final eta (device, library-owned until release); SOLVE: NULL */
  const double* u;         /* RUN: final u; SOLVE: the solution x (vector) */
  const double* U;         /* RUN: final U = G u; SOLVE: NULL */
  sgn_pcg_info info;       /* SOLVE: the solve report; RUN: iters = PCG iterations of the run */
  double t_submit, t_admit, t_done;   /* seconds on sgn_clock() */
} sgn_result;

/* Starts a server (a worker thread with its own stream) on the context's device.
 * budget_fraction of the device's total memory bounds the admitted requests' footprint
 * (0 = 0.8). */
sgn_status sgn_server_create(sgn_ctx* ctx, double budget_fraction, sgn_server** out);
/* Copies the request's arrays (host or device) to the device and queues it; returns a
 * ticket.  SGN_ERR_REJECTED when its footprint exceeds the whole budget; validation errors
 * as for the corresponding direct calls. */
sgn_status sgn_batch_submit(sgn_server* srv, const sgn_request* req, uint64_t* ticket);
/* SGN_ERR_PENDING until the request is done; then fills *out (arrays stay valid until
 * sgn_result_release) and returns the request's status. */
sgn_status sgn_batch_poll(sgn_server* srv, uint64_t ticket, sgn_result* out);
sgn_status sgn_result_release(sgn_server* srv, uint64_t ticket);
/* Finishes all queued work, then stops the worker and frees everything. */
void sgn_server_destroy(sgn_server* srv);
/* The monotonic clock of the t_* fields, in seconds. */
double sgn_clock(void);

/* ---------------------------------------------------------------------------------- */
/* Allocation-free solve (no counterpart in the paper)                                 */
/* ---------------------------------------------------------------------------------- */

#define SGN_NOALLOC_MAX_N 8192

/* The solve of sgn_pcg for ONE 1d instance (nx = n, period L), for callers that cannot
 * allocate device memory once their run has started: a fixed, pre-reserved memory pool,
 * an embedded or certified host whose heap is frozen after start-up, or a callback inside
 * someone else's time loop where calling the CUDA allocator is not allowed.  It needs no
 * sgn_ctx or sgn_layout and calls no cudaMalloc, cudaFree or other allocating routine: its
 * scratch (six half spectra of n/2 + 1 complex doubles), twiddle tables and solve record
 * live in file-scope static device arrays that every GPU loading the library holds until
 * the process exits (about 1 MB per device).
 *
 * Arguments are as for sgn_pcg (device pointers eta, gradh, b and x of n doubles; x holds
 * the initial guess and receives the solution) with the optimal coefficients computed on
 * the device.  n must be a power of two with 8 <= n <= SGN_NOALLOC_MAX_N; a larger or
 * other n returns SGN_ERR_UNSUPPORTED_SIZE without doing anything.  info (host, nullable):
 * when non-NULL the call synchronises the stream and returns the instance status.
 *
 * Works on the current device.  The first call on a device does a one-time set-up (symbol
 * address lookups and the twiddle-table kernel) and synchronises the stream.  Under
 * CUDA's default lazy module loading that
 * first call is also where the driver loads this library's kernels and places the static
 * arrays in device memory, so a caller whose memory is frozen after start-up must make
 * the first call during start-up, before the freeze: "no allocation" holds from the
 * second call on.  Every call shares the same static scratch, which
 * keeps the last call's contents (the solve writes each scratch slot before reading it,
 * and clears the solve record itself): calls that overlap on the GPU (different streams,
 * or different host threads on one device) race with each other and must be serialised
 * by the caller. */
sgn_status sgn_pcg1d_noalloc(int n, double L, const double* eta, const double* gradh,
                             const double* b, double* x, double rtol, int maxit,
                             sgn_precision prec, sgn_pcg_info* info, sgn_stream stream);

/* ---------------------------------------------------------------------------------- */
/* Profiling aid (no counterpart in the paper)                                         */
/* ---------------------------------------------------------------------------------- */

/* When on, CUDA events bracket every PCG and right-hand-side launch group on the stream
 * it runs on.  sgn_profile_read synchronises those events, returns the summed device
 * milliseconds and the number of launch groups of each kind, and clears the record. */
sgn_status sgn_profile_enable(sgn_ctx* ctx, int on);
sgn_status sgn_profile_read(sgn_ctx* ctx, double* pcg_ms, long long* pcg_calls, double* rhs_ms,
                            long long* rhs_calls);
/* Profiling of a 2d layout's persistent inner solves.  Reports what was recorded since the
 * previous call (the summed device milliseconds of the persistent launches, their number,
 * and the inner PCG iterations they ran), synchronising those events, then starts (on = 1)
 * or stops (on = 0) recording.  While recording, mixed solves on the layout take the
 * host-driven refinement loop (a stream synchronisation per pass) so that every persistent
 * launch is bracketed by CUDA events on the solve's stream; results are unchanged.
 * SGN_ERR_INVALID_ARG on a 1d layout. */
sgn_status sgn_profile_inner2d(sgn_layout* lay, int on, double* ms, long long* launches,
                               long long* iterations);

#ifdef __cplusplus
}
#endif
#endif /* SGN_H */
