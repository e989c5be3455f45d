/*
 * mk.h -- C ABI of libmk: the all-at-once space-time solve of the theta-scheme
 * system by FGMRES preconditioned with the multilevel Krylov (MK) cycle
 * (Erlangga, "Parallel-in-time Multilevel Krylov Methods: A Prototype").
 *
 * Problem (Sec. 1, Eq. (dae), Eq. (thetascheme); Sec. 3.3 model problem):
 *   u' = A_n u + g on (0,T], A_n = tau * (2nd-order FD Laplacian) on the unit
 *   interval (dim 1) or unit square (dim 2), n interior points per direction,
 *   h = 1/(n+1), zero Dirichlet boundaries.  theta-scheme with step dt:
 *     psi u_k = phi u_{k-1} + dt gbar_k,  psi = I - theta dt A_n,
 *     phi = I + (1-theta) dt A_n,  gbar_k = (1-theta) g_{k-1} + theta g_k.
 * All-at-once system (Sec. 2, Eq. (finesys)): A_h u_h = f_h, block lower
 *   bidiagonal (I, psi, ..., psi on the diagonal, -phi below), f_0 = u_0,
 *   f_k = dt gbar_k.
 *
 * Array layout at this boundary: dense, row-major, time-major FP64:
 *   1D: x[k][i], shape (n_t+1, nx);  2D: x[k][j][i], shape (n_t+1, ny, nx).
 * A spatial vector (u_0, gradients w.r.t. u_0) has shape (nx) / (ny, nx).
 *
 * Pointers: every array argument may point to device memory (current device)
 * or to host memory (pageable or pinned); the library detects which with
 * cudaPointerGetAttributes and stages host arrays through its own device
 * buffers.  The caller owns every array it passes; the library never keeps a
 * caller pointer after a call returns.  The library owns its workspace, created
 * by mk_create_problem / on the first solve with given options, and freed by
 * mk_destroy.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 * are stream-ordered.  When any output is in host memory, or `info` is
 * non-NULL, the call synchronises the stream before returning.
 *
 * Errors: every entry point returns an mk_status; nothing is thrown across the
 * ABI.  On error, outputs are unspecified unless stated otherwise.
 *
 * Thread safety: one problem must not be used by two host threads at once.
 */
#ifndef MK_H
#define MK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mk_status {
    MK_OK = 0,
    MK_ERR_INVALID = 1,        /* bad argument: sizes, theta not in [0,1], dt <= 0, NULL pointer,
                                  n_t not divisible by the coarsening, unsupported option */
    MK_ERR_NOMEM = 2,          /* device allocation failed */
    MK_ERR_CUDA = 3,           /* a CUDA runtime call failed (see mk_last_cuda_error) */
    MK_ERR_NONFINITE = 4,      /* NaN/Inf in an input or in the iteration */
    MK_ERR_NOT_CONVERGED = 5,  /* max_iters reached: u_out holds the last iterate, info the residual */
    MK_ERR_TIMEOUT = 6,        /* reserved: no entry point returns it.  The library's kernels
                                  never wait on one another (no spin on a flag or barrier);
                                  cross-block reductions finish in the last arriving block */
    MK_ERR_TOO_LARGE = 7       /* the input needs more than a fixed-size static buffer holds
                                  (mk_op_residual_noalloc) */
} mk_status;

/* Spatial operator A_n (Sec. 3.3): tau * second-order FD Laplacian, zero Dirichlet,
   nx (and ny) interior points, h = 1/(n+1) per direction. */
typedef struct mk_stencil {
    int32_t dim;   /* 1 or 2 */
    int32_t nx;    /* >= 1 */
    int32_t ny;    /* >= 1 in 2D, ignored (taken as 1) in 1D */
    double tau;    /* > 0 */
} mk_stencil;

#define MK_MAX_LEVELS 12

/* Options of one MK solve.  Fill with mk_default_opts, then override. */
typedef struct mk_solve_opts {
    double tol;          /* stop when ||f - A u||_2 / ||f||_2 < tol (Sec. 3.3.1 criterion); default 1e-12 */
    int32_t restart;     /* FGMRES(m) restart length on level 1; default 40 */
    int32_t max_iters;   /* total outer iterations; default 2000 */
    int32_t levels;      /* L >= 2: level 1 (fine) .. level L (coarsest, decoupled); default 3 */
    int32_t nu[MK_MAX_LEVELS];      /* time coarsening factor from level l to l+1 (entries 0..L-2); default 2 */
    int32_t space[MK_MAX_LEVELS];   /* 1: agglomerate space (pairs / 2x2) on that coarsening (Case 2, TS) */
    int32_t m_inner[MK_MAX_LEVELS]; /* fixed FGMRES iterations on level l+2 (entries 0..L-3); default 2,
                                       and 1 on the level just above the coarsest (Sec. 4.2) */
    int32_t n_cgs;       /* decoupled slabs on the coarsest level (Sec. 3.3.2); 0 = exact coupled
                            coarse solve (Sec. 3.3.1).  The eigenbasis solvers (1D uniform
                            operator in the mixed path, 2D) handle any slab length, the coupled
                            march included, in parallel over time; the other 1D solvers step
                            through each slab sequentially.  Default 16 */
    int32_t mu_mode;     /* 0: mu_l = lambda_max(A_l) (Sec. 3.1); 1: mu = 1; 2: mu = mu_value */
    double mu_value;
    int32_t precision;   /* 0: FP64 throughout.  1: mixed -- MK cycle, transfers, inner levels and
                            coarsest slabs in FP32; level-1 residual, Arnoldi, least squares and the
                            true-residual check in FP64 (the level-1 basis as double-float pairs).
                            2: mixed with an FP32 level-1 basis -- as 1, but the level-1 Arnoldi
                            vectors are FP32 (dot products summed in FP32 within a tile, in FP64
                            across tiles): half the level-1 basis traffic and memory.  The true
                            residual of every restart stays FP64, so each restart cycle refines
                            the FP64 iterate and the tolerance is met in FP64 as in mode 1. */
    int32_t use_graph;   /* 1: capture each restart cycle in a CUDA graph (default 1) */
    int32_t orth;        /* level-1 Arnoldi: 0 = one classical Gram-Schmidt pass; 1 = a second
                            pass when the norm drops below 1/sqrt(2) of its value (default);
                            2 = always two passes */
    int32_t autotune;    /* 1: when the hierarchy for these options is built, time the tile depth
                            of each level's 1D transfer kernels and the coarsest slab solver
                            variants on its own buffers and keep the fastest (a few ms, once per
                            hierarchy); 0: built-in heuristics (default; bitwise reproducible
                            across processes) */
    int32_t transfer;    /* intergrid operators of the two-level method (Sec. 3.2):
                            MK_TRANSFER_MK (default): Y, Z of Eq. (blockYZ) -- sums of nu steps,
                            optional space agglomeration -- and Galerkin coarse levels
                            (Eqs. (timecoarse1)-(timecoarse3)).
                            MK_TRANSFER_MGRIT: the paper's comparison method -- Y of Eq. (mgritY)
                            (injection of the coarse time points 0, nu, 2 nu, ...), Z of
                            Eq. (mgritZ) (ideal interpolation: the fine steps between two coarse
                            points follow psi x_k = phi x_{k-1} from the coarse value) and the
                            non-Galerkin coarse matrix of Eq. (coarsemat) (the theta-scheme with
                            step nu dt).  Requires dim = 1, levels = 2, space[0] = 0,
                            nu[0] >= 2 and n_t / nu[0] <= 65535; MK_ERR_INVALID otherwise.
                            mk_op_restrict, mk_op_interp_correct and mk_create_batch take
                            MK_TRANSFER_MK only. */
    int32_t inner_kernel; /* how the inner levels 2..L run in each outer iteration:
                            MK_INNER_AUTO (default) and MK_INNER_SEPARATE: one launch per step
                            (measured faster than the cooperative kernel in whole solves);
                            MK_INNER_COOP: the whole inner recursion (restrictions, inner FGMRES
                            iterations, coarsest solve, interpolations, Gram-Schmidt and least
                            squares) in one cooperative launch with grid-wide barriers --
                            requires dim = 1, precision 1, levels >= 3, nu = 2 and no space
                            agglomeration below level 2, and the sine-transform coarsest solver
                            (2(n+1) a power of two); MK_ERR_INVALID otherwise.  The
                            cooperative kernel holds every SM for its duration: do not run
                            other GPU work concurrently with such a solve (separate streams
                            included); batches never use it. */
    int32_t augment;     /* k >= 0 (default 0): FGMRES with recycled corrections, the flexible
                            form of augmented restarting.  The correction u_c - u_{c-1} of every
                            restart cycle c is kept (ring slot (c-1) mod k, in the cycle
                            precision); once k cycles have completed, the last k of each
                            cycle's `restart` directions are those corrections instead of
                            preconditioned basis vectors (the Arnoldi relation and the least
                            squares are unchanged: FGMRES accepts any direction).  Requires
                            k < restart and k <= 8; not in batches.  Memory: k more level-1
                            vectors. */
} mk_solve_opts;

#define MK_MAX_AUGMENT 8
#define MK_INNER_AUTO 0
#define MK_INNER_SEPARATE 1
#define MK_INNER_COOP 2

#define MK_TRANSFER_MK 0
#define MK_TRANSFER_MGRIT 1

typedef struct mk_solve_info {
    int32_t iterations;      /* outer FGMRES iterations */
    int32_t restarts;        /* completed restart cycles */
    double rel_residual;     /* final true ||f - A u|| / ||f|| (FP64) */
    double f_norm;           /* ||f||_2 */
    double solve_ms;         /* device time of the solve (CUDA events on `stream`) */
    int32_t kernel_launches; /* kernels launched by the solve */
    int32_t levels;          /* levels actually built */
} mk_solve_info;

typedef struct mk_problem mk_problem;

/* Defaults listed above. */
void mk_default_opts(mk_solve_opts *opts);

/* Alternate time-space coarsening schedule (Sec. 4.2, Table 3).  Fills opts->levels, nu[],
   space[], m_inner[] and n_cgs for a hierarchy of `levels` levels on a problem with nx (x ny)
   interior points, nt steps of size dt and diffusion tau; other fields are left as they are.
   Level l has the Courant number C_l = c_d tau dT_l / dX_l^2 (c_d = 2 in 1D, 3 in 2D, as the
   paper defines them in Sec. 3.3.1 and 3.3.2), with dT_l its step (a_l + b_l) and dX_l^2 =
   2^s h^2 after s pair / 2x2 agglomerations (the Galerkin operator of an agglomerated uniform
   stencil has twice the squared spacing).  Coarsening is in time (nu = 2, space kept) while
   C_l <= c_max; from the first level whose C_l exceeds c_max, space-only coarsenings (nu = 1,
   pairs / 2x2) and time coarsenings alternate, space first.  Inner FGMRES iterations: 2 on the
   intermediate levels, 1 on the level just above the coarsest (Sec. 4.2).
   Errors (opts untouched): MK_ERR_INVALID for a null opts, levels outside 2..MK_MAX_LEVELS,
   dim not 1 or 2, nx, ny, nt, n_cgs < 1, tau, dt, c_max <= 0, a time coarsening of a level
   whose n_t is odd, a space coarsening of a direction with fewer than 2 points, or a coarsest
   n_t not divisible by n_cgs.  Host only: no device is touched. */
mk_status mk_schedule_alternate(int32_t dim, int32_t nx, int32_t ny, int32_t nt, double tau,
                                double dt, int32_t levels, int32_t n_cgs, double c_max,
                                mk_solve_opts *opts);

/* Human-readable status name. */
const char *mk_status_string(mk_status s);

/* Last CUDA error string seen by the library on this thread ("" if none). */
const char *mk_last_cuda_error(void);

/* Number of library kernels launched since the library was loaded (all threads).  Kernels
   replayed from a captured CUDA graph count once per replay. */
int64_t mk_kernel_launch_count(void);

/* Kernel-class timing (no counterpart in the paper; measurement support).  When on, every
   library kernel launch is bracketed by a pair of CUDA events on its stream (inside captured
   graphs as event nodes), and the device time, algorithmic bytes and launch count are
   accumulated per (class, level) for launches that did work.  Classes: 0 restrict,
   1 interp_correct, 2 multidot, 3 update, 4 slab, 5 residual, 6 combine, 7 march, 8 other.
   Level is 1-based (the level the kernel runs on; 0 when not level-specific).
   Toggling invalidates captured graphs (they are re-captured on the next solve). */
void mk_set_profiling(int32_t on);
void mk_profile_reset(void);
mk_status mk_profile_read(int32_t cls, int32_t level, double *ms, double *bytes, int64_t *launches);
const char *mk_profile_class_name(int32_t cls);

/*
 * mk_create_problem -- set up A_h (Eq. (finesys)) for the theta-scheme with step dt over
 * nt steps, and the source part of f_h: f_k = dt((1-theta) g_{k-1} + theta g_k), k >= 1.
 *   A_n   : spatial operator (host struct).
 *   theta : in [0,1].   dt : > 0.   nt : >= 1.
 *   g     : (nt+1) x n source samples g_k = g(k dt), host or device, or NULL for g = 0.
 *           Copied; not retained.
 *   out   : receives the new problem (host pointer).
 * Errors: MK_ERR_INVALID, MK_ERR_NOMEM, MK_ERR_CUDA.
 */
mk_status mk_create_problem(const mk_stencil *A_n, double theta, double dt, int32_t nt,
                            const double *g, mk_problem **out);

/* Replace the source g of an existing problem ((nt+1) x n samples, host or device, or
   NULL for g = 0): recomputes f_k, k >= 1 (Eq. (finesys)).  Copied; not retained.
   Errors: MK_ERR_INVALID (NULL p), MK_ERR_NOMEM, MK_ERR_CUDA. */
mk_status mk_set_source(mk_problem *p, const double *g, void *stream);

/* Frees the problem and all its workspace.  NULL is ignored. */
void mk_destroy(mk_problem *p);

/* Frees the solver workspace the problem keeps for the options of its last solve (Krylov
   bases, level vectors, coarsest tables, captured graph); the next mk_solve rebuilds it.
   Synchronises the device first.  Errors: MK_ERR_INVALID (NULL p), MK_ERR_CUDA. */
mk_status mk_trim(mk_problem *p);

/*
 * mk_solve -- solve A_h u = f_h (f_0 = u0) by FGMRES (Algorithm 2) right-preconditioned by
 * the MK cycle Q (Eq. (Qh), substeps 4.1-4.5, recursion of Sec. 4.1, decoupled coarsest
 * level Eq. (Qhtilde)).  Initial guess u^0 = 0.
 *   u0    : n initial values.   opts: NULL = defaults.
 *   u_out : (nt+1) x n solution, caller-allocated.
 *   info  : host struct or NULL.
 * Errors: MK_ERR_INVALID (options incompatible with nt/n), MK_ERR_NONFINITE,
 *         MK_ERR_NOT_CONVERGED (u_out holds the last iterate), MK_ERR_NOMEM, MK_ERR_CUDA.
 */
mk_status mk_solve(mk_problem *p, const double *u0, const mk_solve_opts *opts,
                   double *u_out, mk_solve_info *info, void *stream);

/*
 * mk_solve_rhs -- same solver for an arbitrary right-hand side f ((nt+1) x n), u^0 = 0.
 * mk_solve(p, u0, ...) equals mk_solve_rhs with f_0 = u0 and the problem's source blocks.
 * Errors: as mk_solve (MK_ERR_INVALID also for a NULL f or u_out).
 */
mk_status mk_solve_rhs(mk_problem *p, const double *f, const mk_solve_opts *opts,
                       double *u_out, mk_solve_info *info, void *stream);

/*
 * mk_march -- sequential theta-march on the GPU, Eq. (timemarch): block forward
 * substitution of A_h u = f_h, FP64, one step after another (the baseline the MK
 * solve is compared with).  u_out: (nt+1) x n.  Each step is a direct solve of
 * (I - theta dt A_n) u_k = rhs: a tridiagonal solve in 1D (nx <= 4096), a sine-transform
 * solve in 2D (FFT in a direction whose n + 1 is a power of two up to 2048, the dense sine
 * matrix in one with n <= 1024).  Larger grids: MK_ERR_INVALID.  Allocates its staging
 * and step buffers per call; returns after the stream has finished the march.
 * Errors: MK_ERR_INVALID (NULL p, u0 or u_out; grid too large), MK_ERR_NOMEM, MK_ERR_CUDA.
 */
mk_status mk_march(mk_problem *p, const double *u0, double *u_out, void *stream);

/*
 * mk_adjoint -- discrete adjoint of Eq. (finesys) for a loss J(u).
 * Solves A_h^T lam = dJ/du with the same MK solver run on the time-reversed system
 * (A_h^T is block upper bidiagonal; reversing time gives the forward structure, psi and
 * phi being symmetric), then forms
 *   dJ/du0   = lam_0 = b_0 + phi lam_1,
 *   dJ/dg_k  = dt (theta lam_k + (1-theta) lam_{k+1})   (lam_{nt+1} = 0; no lam_0 term),
 *   dJ/dtau  = sum_{k>=1} dt lam_k^T Lhat (theta u_k + (1-theta) u_{k-1}),  Lhat = A_n / tau.
 *   u      : (nt+1) x n forward solution, or NULL when grad_tau is NULL.
 *   dJdu   : (nt+1) x n.
 *   grad_u0: n, or NULL.  grad_g: (nt+1) x n, or NULL.  grad_tau: one double, or NULL.
 *   lam_out: (nt+1) x n adjoint state, or NULL.
 * Errors: MK_ERR_INVALID (NULL p or dJdu, grad_tau without u, options as in mk_solve),
 *         MK_ERR_NOT_CONVERGED (the outputs are formed from the last adjoint iterate),
 *         MK_ERR_NONFINITE, MK_ERR_NOMEM, MK_ERR_CUDA.
 */
mk_status mk_adjoint(mk_problem *p, const double *u, const double *dJdu,
                     const mk_solve_opts *opts, double *grad_u0, double *grad_g,
                     double *grad_tau, double *lam_out, mk_solve_info *info, void *stream);

/* Problem geometry (host ints / doubles); NULL outputs are skipped.  Host only.
   Errors: MK_ERR_INVALID (NULL p). */
mk_status mk_problem_shape(const mk_problem *p, int32_t *dim, int32_t *nx, int32_t *ny, int32_t *nt,
                           double *theta, double *dt, double *tau);

/* mk_tune -- schedule autotuner for one problem: picks the knobs the method leaves free by
   timing complete solves of this problem (its source as set, initial state u0, host or
   device) to base->tol.  Starting from *base (NULL: defaults): with MK_TUNE_LEVELS in flags
   the level count 2 .. base->levels (base's nu and space, inner counts 2 and 1 above the
   coarsest, the exact coarse solve where it is parallel), then up to two passes (the second
   only if the first improved) of coordinate descent over
     - each inner iteration count m_inner (Sec. 4.1) +1 and -1, deepest level first;
     - n_cgs (Sec. 3.3.2) in {base, 16, 8, 4, 2, 1, 0} (0 is left out for the FP64 path in 1D,
       whose coupled coarse march is sequential);
     - restart (Algorithm 2) in {8, 12, 16, 24, 32, 40, 64} (with MK_TUNE_RESTART_CAP only
       those up to base->restart: the level-1 basis grows with it);
   keeping at each step the fastest candidate that converges within base->max_iters (others,
   and candidates the library rejects, are skipped).  Each candidate first runs one restart
   cycle (max_iters 1), which builds its hierarchy, tunes its tiles and captures its graph, so
   that the timed solves that follow measure the iterations alone.  At most max_trials timed
   solves (0: no limit; the one-cycle runs are not counted).
   *best receives the chosen options (tile autotuning on); info (may be NULL) the number of
   solves, the best solve's time and iterations and the wall time of the tuning.  Allocates
   one solution buffer for the trials and frees it, and frees the workspace of the last trial
   (as mk_trim).  Synchronises the device.
   Errors: MK_ERR_INVALID (NULL p, u0 or best), MK_ERR_NOMEM, MK_ERR_CUDA from a trial,
   MK_ERR_NOT_CONVERGED when no candidate converged (best unchanged). */
#define MK_TUNE_LEVELS 1
#define MK_TUNE_RESTART_CAP 2   /* restart candidates only up to base->restart (bounds memory) */
typedef struct mk_tune_info {
    int32_t trials;           /* timed solves run */
    int32_t best_iterations;  /* outer iterations of the chosen options */
    double best_ms;           /* device time of the chosen options' solve */
    double tune_ms;           /* wall time of the whole tuning */
} mk_tune_info;
mk_status mk_tune(mk_problem *p, const double *u0, const mk_solve_opts *base, int32_t flags,
                  int32_t max_trials, mk_solve_opts *best, mk_tune_info *info, void *stream);

/* ------------------------------------------------------------------------------------
 * Operator-level entry points.  Each runs one step of the hot path on dense FP64 arrays
 * of the given level so that it can be checked on its own.  `level` is 1-based
 * (1 = fine).  `precision` 0 computes in FP64, 1 in FP32 (inputs rounded to FP32 first,
 * as in the mixed cycle; outputs widened back to FP64).  The hierarchy is the one `opts`
 * describes (NULL = defaults).  Arrays are host or device as elsewhere; the entry points
 * allocate their staging buffers per call and return after the stream has finished.
 * Errors (all of them): MK_ERR_INVALID for a NULL problem or array, a level or precision
 * out of range, or options the problem rejects; MK_ERR_NOMEM; MK_ERR_CUDA.
 * ------------------------------------------------------------------------------------ */

typedef struct mk_level_desc {
    int32_t dim, nx, ny, nt;   /* spatial sizes and time steps on this level */
    double a, b;               /* (A x)_k = (I - aL) x_k - (I + bL) x_{k-1} */
    double mu;                 /* shift used when restricting from this level */
} mk_level_desc;

/* Level geometry and weights (Galerkin coarse operator of Eqs. (timecoarse1)-(timecoarse3)):
   a_{l+1} = nu a_l + (nu-1) b_l, b_{l+1} = b_l, nt_{l+1} = nt_l / nu; with
   transfer = MK_TRANSFER_MGRIT the coarse level is the theta-scheme of Eq. (coarsemat),
   a_2 = theta nu dt, b_2 = (1-theta) nu dt.
   If xcoef/ycoef are non-NULL they receive the spatial operator L_l = Y^T L_{l-1} Z as
   3 x nx (resp. 3 x ny) host doubles: rows lo, di, up.
   Errors: MK_ERR_INVALID (NULL p, level outside 1..levels, bad options), MK_ERR_NOMEM,
   MK_ERR_CUDA (the hierarchy for opts is built if it does not exist yet). */
mk_status mk_level_info(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                        mk_level_desc *desc, double *xcoef, double *ycoef);

/* f = f_h for initial state u0 (RHS assembly of Eq. (finesys)).  f: (nt+1) x n. */
mk_status mk_op_rhs(mk_problem *p, const double *u0, double *f, void *stream);

/* w = A_l x  (space-time stencil matvec). */
mk_status mk_op_apply(mk_problem *p, const mk_solve_opts *opts, int32_t level, int32_t precision,
                      const double *x, double *w, void *stream);

/* r = f - A_1 u and ||r||_2 (host double, may be NULL). */
mk_status mk_op_residual(mk_problem *p, const double *f, const double *u, double *r,
                         double *rnorm, void *stream);

/* vhat = Y^T (A_l v - mu_l v)  (substeps 4.1-4.2), level l -> l+1. */
mk_status mk_op_restrict(mk_problem *p, const mk_solve_opts *opts, int32_t level, int32_t precision,
                         const double *v, double *vhat, void *stream);

/* x = v - Z vt and w = A_l x  (substeps 4.4-4.5 fused with step 5), vt on level l+1. */
mk_status mk_op_interp_correct(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                               int32_t precision, const double *v, const double *vt,
                               double *x, double *w, void *stream);

/* The same step with the full argument set of the solve: x = sigma v - Z vt with
   vt = sum_{m < nvt} y_m vt_m (the scaled basis vector and the inner FGMRES combination of
   the coarser level, substeps 4.4-4.5 of Algorithm 2), and w = A_l x.  vt: nvt consecutive
   level-(l+1) arrays; y: nvt host doubles, or NULL with nvt = 1 (vt used as it is).
   precision 0: FP64; 1: FP32; 2: the level-1 path of the mixed solve -- v rounded to a
   double-float pair (hi, lo) and vt to FP32, x formed in FP32 from the leading part of v,
   w = A_1 x evaluated in double-float arithmetic and returned as hi + lo (level 1 only,
   opts->precision 1).  Errors as above; MK_ERR_INVALID also for nvt outside 1..8, y NULL
   with nvt > 1, or precision 2 with level != 1 or opts->precision != 1. */
mk_status mk_op_interp_combine(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                               int32_t precision, const double *v, double sigma,
                               const double *vt, int32_t nvt, const double *y, double *x,
                               double *w, void *stream);

/* x = Atilde_L^{-1} r on the coarsest level (decoupled slabs, Eq. (Qhtilde); n_cgs = 0: the
   exact coarse matrix; with MK_TRANSFER_MGRIT the theta-scheme of Eq. (coarsemat)). */
mk_status mk_op_coarsest(mk_problem *p, const mk_solve_opts *opts, int32_t precision,
                         const double *r, double *x, void *stream);

/* x = Q_l v: one full MK cycle from level l (inner FGMRES on intermediate levels); with
   MK_TRANSFER_MGRIT the two-level cycle with the transfers of Eqs. (mgritY), (mgritZ). */
mk_status mk_op_precond(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                        const double *v, double *x, void *stream);

/* One Arnoldi orthogonalisation (classical Gram-Schmidt, twice) of w against the j
   columns of V (j x N, orthonormal), N = (nt+1) n on level 1:
   h[0..j-1] = coefficients, h[j] = ||w'||, w <- w' / h[j].  h: host, j+1 doubles. */
mk_status mk_op_orthogonalize(mk_problem *p, int32_t j, const double *V, double *w,
                              double *h, void *stream);

/* Least squares y = argmin || beta e_1 - H y ||, H (j+1) x j column-major (host),
   solved on the device by Givens rotations.  y: host, j doubles; res: |g_{j+1}|. */
mk_status mk_op_lsq(int32_t j, const double *H, double beta, double *y, double *res, void *stream);

/* ---- Batches of independent problems (Sec. 4's method applied to many problems at once) ----

   A batch solves `count` independent problems of any sizes, dimensions, theta and tau
   together.  Every problem gets its own level hierarchy (built from opts[i], or the defaults
   when opts is NULL), and one CUDA graph holds one restart cycle of every problem, each on
   its own branch, so a replay of the graph advances all unconverged problems at once and
   the GPU overlaps their kernels.  A problem that has converged, failed or used max_iters
   is stopped through its own done flag; its branch then exits at once in later replays.
   With autotune != 0 the tile depth of each level's 1D transfer kernels and the coarsest
   slab solver variant (sine transform, partitioned, cyclic reduction) are chosen by timing
   them on the problem's own buffers at creation (a few milliseconds per problem).

   mk_create_batch: problems = count distinct handles (not owned; they must outlive the
     batch and keep their source); opts = NULL or count option structs.  The batch holds
     its hierarchies, graph and streams on the current device until mk_destroy_batch.
     The members' inner levels run as separate launches (inner_kernel = MK_INNER_AUTO is
     taken as MK_INNER_SEPARATE): their branches run concurrently, and a cooperative kernel
     sized to the whole GPU is not run beside other work.
     Errors: MK_ERR_INVALID (count < 1, a NULL or repeated handle, bad options, options
     with transfer != MK_TRANSFER_MK, inner_kernel = MK_INNER_COOP or augment > 0),
     MK_ERR_NOMEM, MK_ERR_CUDA.
   mk_solve_batch: u0[i] = initial state of problem i (nx or ny x nx), u_out[i] = its
     (nt+1) x n solution; each pointer host or device as elsewhere in this ABI.  infos =
     NULL or count structs (solve_ms and kernel_launches are those of the whole batch).
     Returns MK_OK when every problem converged, else the first non-OK status of a member
     (MK_ERR_NOT_CONVERGED, MK_ERR_NONFINITE); every u_out[i] holds that member's last
     iterate.  Synchronises `stream` before returning.  One batch must not be solved from
     two host threads at once. */
typedef struct mk_batch mk_batch;
mk_status mk_create_batch(mk_problem *const *problems, int32_t count, const mk_solve_opts *opts,
                          int32_t autotune, mk_batch **out);
mk_status mk_solve_batch(mk_batch *batch, const double *const *u0, double *const *u_out,
                         mk_solve_info *infos, void *stream);
void mk_destroy_batch(mk_batch *batch);

/* ---- Allocation-free residual (a library extension: the paper has no counterpart) ----

   r = f - A_h u on the fine level (Eq. (finesys)), its norm ||r||_2 and optionally the
   per-step norms ||r_k||_2, k = 0..n_t -- the same quantities as mk_op_residual, computed
   without allocating anything: no cudaMalloc/cudaFree, no staging buffer, no temporary
   level.  It is for callers that must not allocate while they run: a loop that works in
   a device-memory budget fixed at start-up, a caller that cannot afford the device-wide
   synchronisation that cudaFree implies, or a caller whose own allocator owns the device.
   mk_op_residual, by contrast, builds a temporary fine level and stages host arrays.

   f, u:        device pointers, dense (n_t+1) x n FP64 (the layout of this ABI).
   r:           device pointer to (n_t+1) x n doubles, or NULL to compute the norms only.
   rnorm:       device pointer to one double: ||f - A_h u||_2.
   rnorm_steps: device pointer to n_t+1 doubles (||r_k||_2), or NULL.
   Host pointers, and NULL f/u/rnorm, return MK_ERR_INVALID.  The call does not
   synchronise: the outputs are ready in the order of `stream`.

   Scratch: the reduction's partial sums live in one array of MK_NOALLOC_MAX_PARTIALS
   doubles in the library's static device memory (one copy per device, 512 KiB).  A call
   needs (n_t+1) * ceil(nx*ny / MK_NOALLOC_CHUNK) of them; above that it returns
   MK_ERR_TOO_LARGE and launches nothing.  The partial sums need no initial value; an
   arrival counter beside them must be zero when a launch starts -- it is zero when the
   library's device code is loaded, and every completed launch leaves it at zero.
   Set-up: the first call on each device looks up the scratch's address
   (cudaGetSymbolAddress, with that device current), which may load the library's device
   code; make that first call where loading device code is allowed.  The address is kept for
   the life of the process: after a device reset (cudaDeviceReset, or a primary-context
   reset by other code) the library's device code is reloaded and calls of this entry point
   are undefined.
   Concurrency: every call on a device uses the same scratch, so calls whose executions
   overlap on one device (other streams, other host threads, without event ordering)
   race and return wrong results.  Order them on one stream.  Calls on different devices
   are independent.  The results are deterministic (fixed reduction order). */
#define MK_NOALLOC_MAX_PARTIALS 65536
#define MK_NOALLOC_CHUNK 2048
mk_status mk_op_residual_noalloc(const mk_problem *p, const double *f, const double *u,
                                 double *r, double *rnorm, double *rnorm_steps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MK_H */
