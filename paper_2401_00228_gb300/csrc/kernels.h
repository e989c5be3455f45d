// Kernel launchers of libmk (internal).  Each launcher checks nothing but launch
// errors; argument validation happens at the ABI.
#pragma once

#include "mk_internal.h"

namespace mk {

// Per-level device scalars of an FGMRES process (one block of doubles + ints).
//   sigma[i]  : 1/||V_i|| (basis stored unnormalised, v_i = sigma_i V_i)
//   H         : (m+1) x m Hessenberg, column-major, ld = m+1
//   cs, sn, g : Givens rotations and rotated right-hand side (level 1)
//   y         : least-squares solution (combination of the X_i)
//   beta      : ||r_0|| of the current (re)start
struct KState {
    double *d;     // doubles, layout below
    int *flags;    // [0] done, [1] j_final, [2] reorth, [3] error, [4] iterations (total)
    int m;         // capacity (iterations per cycle)
    __host__ __device__ double *sigma() const { return d; }                       // m+1
    __host__ __device__ double *H() const { return d + (m + 1); }                  // (m+1)*m
    __host__ __device__ double *cs() const { return d + (m + 1) * (m + 1); }       // m
    __host__ __device__ double *sn() const { return cs() + m; }                    // m
    __host__ __device__ double *g() const { return sn() + m; }                     // m+1
    __host__ __device__ double *y() const { return g() + (m + 1); }                // m
    __host__ __device__ double *tmp() const { return y() + m; }                    // m+1
    __host__ __device__ double *misc() const { return tmp() + (m + 1); }           // 8
    // misc[0] = beta, misc[1] = tol * ||f|| (absolute target), misc[2] = ||w||^2 before
    // orthogonalisation, misc[3] = ||f||, misc[4] = last true residual norm,
    // misc[5] = raw result of the last reduction, misc[6] = last Givens residual estimate
    static int ndoubles(int m) { return (m + 1) + (m + 1) * m + 2 * m + (m + 1) + m + (m + 1) + 8; }
};

enum EpilogueKind {
    EPI_NONE = 0,
    EPI_BETA = 1,        // result[0] = ||v||^2 -> misc[0] = beta, sigma[0] = 1/beta (inner start)
    EPI_OUTER_START = 2, // same, and g = beta e1, done/j reset, level-1 convergence test
    EPI_OUTER_INIT = 3,  // first residual (= f): also ||f|| -> misc[3], tol*||f|| -> misc[1]
                         // (tol read from misc[7])
};

// ---- stencil family (stencil.cu) ------------------------------------------------------
template <typename Tsrc, typename Tdst>
void launch_pack(const Geom &g, const Tsrc *dense, Tdst *padded, cudaStream_t s);
template <typename Tsrc, typename Tdst>
void launch_unpack(const Geom &g, const Tsrc *padded, Tdst *dense, cudaStream_t s);
template <typename Tsrc, typename Tdst>
void launch_convert(int64_t n, const Tsrc *src, Tdst *dst, cudaStream_t s);

// f_k = dt((1-theta) g_{k-1} + theta g_k), k >= 1 (g dense -> f padded).
void launch_rhs_source(const Geom &g, double theta, double dt, const double *gdense, double *f,
                       cudaStream_t s);

// w = A x  (Tc = arithmetic type).
template <typename Tin, typename Tout, typename Tc>
void launch_apply(const Geom &g, const Weights &w, SpaceOp<Tc> L, const Tin *x, Tout *out,
                  cudaStream_t s);

// r = f - A u ; ||r||^2 reduced into the KState (epilogue kind as above); r may alias V_0.
void launch_residual(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                     const double *u, double *r, const ReduceScratch &rs, int slot,
                     KState ks, int epi, cudaStream_t s);

// vhat = sigma * Y^T (A v - mu v) from level f to level c.  If ks_c.d != nullptr the
// squared norm of vhat is reduced and the inner start epilogue (EPI_BETA) runs on ks_c.
// skip_if_done: early exit when *done != 0.
template <typename Tin, typename Tout, typename Tc>
void launch_restrict(const Geom &gf, const Geom &gc, int nu, bool space, const Weights &w,
                     SpaceOp<Tc> L, const Tin *v, const double *sigma, Tout *vhat,
                     const ReduceScratch &rs, int slot, KState ks_c, const int *done,
                     cudaStream_t s);

// x = sigma v - Z (sum_m yc[m] Xc_m) ; w = A x.  yc == nullptr means a single Xc with
// coefficient 1.
template <typename Tv, typename Tz, typename Tx, typename Tw, typename Tc>
void launch_interp(const Geom &gf, const Geom &gc, int nu, bool space, const Weights &w,
                   SpaceOp<Tc> L, const Tv *v, const double *sigma, const Tz *Xc, int mc,
                   int64_t xc_stride, const double *yc, Tx *x, Tw *wout, const int *done,
                   cudaStream_t s);

// ---- Krylov family (krylov.cu) --------------------------------------------------------
// Arnoldi step j on a process with state ks, vectors of length len (padded):
//   h_i = sigma_i <W, V_i>, i = 0..j   (multidot, partials + last block)
// close_mode != 0 (inner levels, last iteration j = m - 1, first pass): the new basis vector
// is not needed, so its norm comes from Pythagoras, ||w - sum h_i v_i||^2 = ||w||^2 - sum h_i^2,
// and the update epilogue of mode close_mode (the least squares) runs in this kernel.
template <typename TW, typename TV>
void launch_multidot(int64_t len, const TW *W, const TV *V, int64_t vstride, int j,
                     const ReduceScratch &rs, KState ks, bool second_pass, const int *done,
                     cudaStream_t s, int close_mode = 0);
//   V_{j+1} = W - sum_i h_i sigma_i V_i, ||.||^2 -> h_{j+1,j}, sigma_{j+1};
//   last block also runs the least-squares bookkeeping (Givens for the outer level,
//   final solve on the last inner iteration).
enum UpdateMode {
    UPD_REORTH = 1,     // request a second Gram-Schmidt pass when ||w'|| < ||w|| / sqrt(2)
    UPD_GIVENS = 2,     // outer level: Givens update, convergence test, y on completion
    UPD_INNER_LSQ = 4,  // inner level: least squares on the last iteration
    UPD_REORTH_ALWAYS = 8,  // always request the second Gram-Schmidt pass
    UPD_OUTER = UPD_REORTH | UPD_GIVENS,
    UPD_INNER = UPD_INNER_LSQ
};
template <typename TW, typename TV>
void launch_update(int64_t len, const TW *W, TV *V, int64_t vstride, int j, bool write_next,
                   const ReduceScratch &rs, KState ks, int mode, bool second_pass,
                   const int *done, cudaStream_t s);

// u += sum_{i < jf} y_i X_i (FP64 u), jf = flags[1] (outer) -- skip when nothing to add.
// aug (may be null): the correction sum y_i X_i also goes to ring slot flags[5] mod augk
// (slots xstride apart).
template <typename TX>
void launch_combine(int64_t len, double *u, const TX *X, int64_t xstride, KState ks,
                    cudaStream_t s, TX *aug = nullptr, int augk = 0);

// Small solve on the device: least squares of an explicit (j+1) x j Hessenberg by Givens,
// rotating H in place; gg: j+1 doubles of scratch.
void launch_lsq(int j, double *H, double beta, double *gg, double *y, double *res,
                cudaStream_t s);

// ---- level-1 kernels of the mixed solve with double-float vectors (dfkernels.cu) --------
void launch_residual_df(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                        const double *u, float2 *r, const ReduceScratch &rs, int slot, KState ks,
                        int epi, cudaStream_t s);
// the same with r rounded to FP32 (the FP32 level-1 basis)
void launch_residual_f32(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                        const double *u, float *r, const ReduceScratch &rs, int slot, KState ks,
                        int epi, cudaStream_t s);
// 2D coarsest slabs in the eigenbasis of Lx (+) Ly, all time rows at once (slab.cu): forward
// transform of every row, per-mode recurrence over each slab, inverse transform.  rh: scratch of
// (nt+1) nx ny values.  Three launches.
template <typename T>
void launch_slab_2d_fdm(const Geom &g, double a, double b, const T *Sx, const T *Sxi,
                        const T *lamx, const T *Sy, const T *Syi, const T *lamy, int n_cgs,
                        T *rh, const T *r, T *x, const int *done, cudaStream_t s);

// Sequential 2D theta-march with a sine-transform solve per step (march2d.cu): FP64, for the
// uniform fine-level operator.  Per direction the transform is an FFT when n + 1 is a power of
// two (march2d_transform_size != 0, twiddles tw) and otherwise the dense sine matrix S (n x n,
// n <= MARCH2D_DENSE_MAX).  u's plane 0 must hold u_0; t1 is nx ny doubles of scratch.
// 3 n_t launches.
constexpr int MARCH2D_DENSE_MAX = 1024;
int march2d_transform_size(int n);
cudaError_t march2d_set_attributes();
void launch_march_2d_dst(const Geom &g, double a, double b, double cx, double cy,
                         const double *lamx, const double *lamy, const double2 *twx,
                         const double2 *twy, const double *Sx, const double *Sy, const double *f,
                         double *u, double *t1, cudaStream_t s);

// Coarsest decoupled slabs by sine-transform diagonalisation (slab_dst.cu), FP32, for a
// uniform 1D operator.  dst_transform_size(n) = 2(n+1) when that is a power of two <= 4096,
// else 0 (not supported).  tab = [alpha (n) | beta (n)], tw = FFT twiddle table,
// rh = scratch (nt+1) x ldd.  Any slab length; n_cgs = 0 is the coupled march over all nt
// steps (the exact coarse solve).  Three launches.
int dst_transform_size(int n);
size_t dst_smem_bytes(int N2);
cudaError_t dst_set_attributes();
void launch_slab_1d_dst(const Geom &g, const float *tab, const float2 *tw, int N2, int n_cgs,
                        float *rh, int ldd, const float *r, float *x, const int *done,
                        cudaStream_t s);

// ---- inner levels of the 1D mixed cycle in one cooperative kernel (inner_coop.cu) -------
// Levels 2 .. L-1 (FP32, time coarsening by 2 without space agglomeration) and the
// sine-transform coarsest level L.  Level l's fixed FGMRES iterations, the restriction to
// l+1, the recursion, the interpolation with correction and matvec, the Gram-Schmidt
// reductions and the small least-squares problems all run inside one launch, the phases
// separated by grid-wide barriers of a cooperative launch.
struct CoopLevel {
    Geom g;
    float a, b, mu;
    const float *L;      // [lo | di | up] of the spatial operator, nx each
    float *V, *X, *W;    // basis (m+1 vectors), preconditioned vectors (m), w
    int64_t stride;
    int m;               // fixed inner iterations
    KState ks;
};
struct CoopCoarse {
    Geom g;
    const float *tab;    // [alpha (n) | beta (n)] of the per-mode recurrence
    const float2 *tw;    // FFT twiddles
    int N2, logN2, ldd, n_cgs;
    float *rh, *R, *X;   // transformed rows (nt+1) x ldd, right-hand side, solution
};
struct CoopParams {
    int nl;                          // intermediate levels: lv[0] is level 2, lv[nl-1] level L-1
    CoopLevel lv[MK_MAX_LEVELS];
    CoopCoarse c;
    double *partials;                // [slot][block]
    int max_blocks;
};
// Blocks of the cooperative launch (all co-resident) for an FFT length N2; 0 if the device
// cannot run it.
int coop_grid_size(int N2);
cudaError_t coop_set_attributes();
// The whole inner solve of level 2 (its right-hand side and beta already in lv[0].V and
// lv[0].ks by the level-1 restriction): X_2 and y_2 on return.
// Pdev: the parameters in device memory; N2: the coarsest level's FFT length.
void launch_inner_coop(const CoopParams *Pdev, int N2, int grid, const int *done, cudaStream_t s);

// Blocks per SM of the small-basis Gram-Schmidt launches that follow on this host thread
// (0: the default 4).
void set_krylov_hint(int blocks_per_sm);

// Tile depth (time steps per thread) for the tiled 1D transfer launches that follow on this
// host thread: restriction in {1, 2, 4, 8}, interpolation in {2, 4}; 0 = built-in heuristic.
void set_tile_hint(int kc_restrict, int kc_interp);

// Time-tiled 1D variants for nu = 2 (transfer1d.cu).  Each returns false, launching
// nothing, when the case is not covered (2D, nu != 2); the caller then uses the general
// kernel.  The caller brackets the launch (profiling, launch count).
template <typename Tin, typename Tout, typename Tc>
bool launch_restrict_1d_tiled(const Geom &gf, const Geom &gc, int nu, bool space,
                              const Weights &w, SpaceOp<Tc> L, const Tin *v, const double *sigma,
                              Tout *vhat, const ReduceScratch &rs, int slot, KState ks_c,
                              const int *done, cudaStream_t s);
template <typename Tv, typename Tz, typename Tx, typename Tw, typename Tc>
bool launch_interp_1d_tiled(const Geom &gf, const Geom &gc, int nu, bool space, const Weights &w,
                            SpaceOp<Tc> L, const Tv *v, const double *sigma, const Tz *Xc,
                            int mc, int64_t xc_stride, const double *yc, Tx *x, Tw *wout,
                            const int *done, cudaStream_t s);
// uniform_ab: nullptr, or the device values (a cx, b cx, a cy, b cy) as double-floats when the
// level's operator is cx tridiag(1, -2, 1) (+) cy tridiag(1, -2, 1) (then ca/cb are not read)
bool launch_interp_df_1d_tiled(const Geom &gf, const Geom &gc, int nu, bool space,
                               const float2 *ca, const float2 *cb, bool has_b, const float2 *v,
                               const double *sigma, const float *Xc, int mc, int64_t xc_stride,
                               const double *yc, float *x, float2 *wout, const int *done,
                               cudaStream_t s, const float2 *uniform_ab = nullptr);
// ca, cb: double-float a*L and b*L coefficient rows, [x: lo|di|up (3 nx) | y: (3 ny)]
void launch_interp_df(const Geom &gf, const Geom &gc, int nu, bool space, const float2 *ca,
                      const float2 *cb, bool has_b, const float2 *v, const double *sigma,
                      const float *Xc, int mc, int64_t xc_stride, const double *yc, float *x,
                      float2 *wout, const int *done, cudaStream_t s,
                      const float2 *uniform_ab = nullptr, bool uniform_square = false);
// u += sum_{i < jf} y_i X_i for FP32 X in double-float arithmetic (mixed level 1)
void launch_combine_df(int64_t len, double *u, const float *X, int64_t xstride, KState ks,
                       cudaStream_t s, float *aug = nullptr, int augk = 0);
// In place: the FP64 values of w become double-float pairs (same 8 bytes per element).
void launch_f64_to_df(int64_t len, void *w, const int *done, cudaStream_t s);
void launch_multidot_df(int64_t len, const float2 *W, const float2 *V, int64_t vstride, int j,
                        const ReduceScratch &rs, KState ks, bool second_pass, const int *done,
                        cudaStream_t s);
void launch_update_df(int64_t len, const float2 *W, float2 *V, int64_t vstride, int j,
                      const ReduceScratch &rs, KState ks, int mode, bool second_pass,
                      const int *done, cudaStream_t s);

// ---- MGRIT intergrid operators, 1D (mgrit.cu; Sec. 3.2 Eqs. (mgritY), (mgritZ)) ----------
// vhat_K = sigma ((A v)_{nu K} - mu v_{nu K}), K = 0 .. gc.nt (injection of the coarse points).
template <typename Tin, typename Tc>
void launch_inject_restrict_1d(const Geom &gf, const Geom &gc, int nu, const Weights &w,
                               SpaceOp<Tc> L, const Tin *v, const double *sigma, Tc *vhat,
                               const int *done, cudaStream_t s);
// Ideal interpolation, first part: rp row 1 + K (nu - 1) = (I + bL) xt_K, K < gc.nt, on the
// propagation geometry gp (gc.nt (nu - 1) steps; its other rows are left untouched).
template <typename Tc>
void launch_ideal_interp_rhs_1d(const Geom &gc, const Geom &gp, int nu, double b, SpaceOp<Tc> L,
                                const Tc *xt, Tc *rp, const int *done, cudaStream_t s);
// Ideal interpolation, last part: t_{nu K} = xt_K, t_{nu K + i} = xp row 1 + K (nu - 1) + i - 1.
template <typename Tc>
void launch_ideal_interp_gather_1d(const Geom &gf, const Geom &gc, const Geom &gp, int nu,
                                   const Tc *xt, const Tc *xp, Tc *t, const int *done,
                                   cudaStream_t s);

// ---- slab solvers (slab.cu) -----------------------------------------------------------
// 1D coarsest: n_cgs slabs x s steps, tridiagonal I - aL by parallel cyclic reduction with
// precomputed tables (alpha, gamma, binv in T); x_0 = r_0.
template <typename T>
void launch_slab_1d(const Geom &g, double b, SpaceOp<T> L, const T *alpha, const T *gamma,
                    const T *binv, int npad, int nlev, int n_cgs, const T *r, T *x,
                    const int *done, cudaStream_t s);
// 1D, one warp per slab: partitioned solver with the tables of spike_tables() in T.
// cls: PROF_SLAB or PROF_MARCH for the kernel-class timing.
int spike_block_size(int n);
int spike_threads(int n);
template <typename T>
bool slab_warp_supported(int n);
template <typename T>
void launch_slab_1d_warp(const Geom &g, double b, const T *tab, int U, int n_cgs, const T *r, T *x,
                         const int *done, cudaStream_t s, int cls);
// 2D coarsest: fast diagonalisation of I - a(Lx (+) Ly) with S, S^{-1} per direction.
template <typename T>
void launch_slab_2d(const Geom &g, double a, double b, SpaceOp<T> L, const T *Sx, const T *Sxi,
                    const T *lamx, const T *Sy, const T *Syi, const T *lamy, int n_cgs,
                    const T *r, T *x, const int *done, cudaStream_t s);

// Sequential 1D theta-march on the GPU (FP64): the same direct solver, one slab of nt steps
// with the coupling kept, in one CTA.
void launch_march_1d(const Geom &g, double b, SpaceOp<double> L, const double *alpha,
                     const double *gamma, const double *binv, int npad, int nlev,
                     const double *f, double *u, cudaStream_t s);

}  // namespace mk
