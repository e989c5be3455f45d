// Transfers of the comparison two-level method with MGRIT intergrid operators (Sec. 3.2,
// Eqs. (mgritY), (mgritZ)), 1D, time coarsening by nu >= 2.
//
//   Y^T injects the coarse time points: vhat_K = sigma ((A v)_{nu K} - mu v_{nu K}).
//   Z is the ideal interpolation [-(A_ff)^{-1} A_fc; I_c]: the coarse point nu K takes
//   xt_K and the fine points nu K + i (i = 1 .. nu - 1) follow the homogeneous march
//   psi x_{nu K + i} = phi x_{nu K + i - 1}.
//
// The march between coarse points runs through the decoupled slab solvers on a
// "propagation" geometry gp with n_T (nu - 1) steps: slab K holds the fine points of
// interval K, rows 1 + K (nu - 1) .. (K + 1)(nu - 1), and its first step's right-hand side
// is phi xt_K (every other row of that right-hand side stays zero).  The coarse operator
// keeps the fine operator L, so the fine coefficient rows serve on the coarse geometry.
#include "stencil_common.cuh"

namespace mk {

namespace {

constexpr int MG_THREADS = 256;

inline void mg_launch(int rows, int nx, dim3 &grid, dim3 &block) {
    const int bx = nx >= MG_THREADS ? MG_THREADS : ((nx + 31) / 32) * 32;
    block = dim3(bx, 1, 1);
    grid = dim3(rows, (nx + bx - 1) / bx, 1);
}

}  // namespace

// vhat_K = sigma ((A v)_{nu K} - mu v_{nu K}), K = 0 .. n_T; (A v)_0 = v_0.
template <typename Tin, typename Tc>
__global__ void __launch_bounds__(MG_THREADS) k_inject_restrict_1d(
    Geom gf, Geom gc, int nu, Tc a, Tc b, Tc mu, const Tc *__restrict__ cx,
    const Tin *__restrict__ v, const double *__restrict__ sigma, Tc *__restrict__ vhat,
    const int *__restrict__ done) {
    if (done && *done) return;
    const int K = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= gf.nx) return;
    const int k = nu * K;
    const Tc sig = sigma ? (Tc)(*sigma) : (Tc)1;
    const Tc *cy = nullptr;
    const int64_t idx = gf.at(k, 0, i);
    const Tc vk = ldv<Tc>(v, idx);
    Tc av = vk;
    if (K > 0) {
        const int64_t ip = gf.at(k - 1, 0, i);
        const Tc Lk = lap_at<1, Tc>(v, idx, i, 0, gf, cx, cy);
        const Tc Lp = lap_at<1, Tc>(v, ip, i, 0, gf, cx, cy);
        av = (vk - a * Lk) - (ldv<Tc>(v, ip) + b * Lp);
    }
    vhat[gc.at(K, 0, i)] = sig * (av - mu * vk);
}

// First-step right-hand sides of the propagation slabs: r_{1 + K(nu-1)} = phi xt_K,
// K = 0 .. n_T - 1, phi = I + bL.
template <typename Tc>
__global__ void __launch_bounds__(MG_THREADS) k_ideal_rhs_1d(Geom gc, Geom gp, int nu, Tc b,
                                                             const Tc *__restrict__ cx,
                                                             const Tc *__restrict__ xt,
                                                             Tc *__restrict__ rp,
                                                             const int *__restrict__ done) {
    if (done && *done) return;
    const int K = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= gc.nx) return;
    const Tc *cy = nullptr;
    const int64_t idx = gc.at(K, 0, i);
    rp[gp.at(1 + K * (nu - 1), 0, i)] = xt[idx] + b * lap_at<1, Tc>(xt, idx, i, 0, gc, cx, cy);
}

// t = Z xt on the fine geometry: coarse points from xt, fine points from the marched slabs.
template <typename Tc>
__global__ void __launch_bounds__(MG_THREADS) k_ideal_gather_1d(Geom gf, Geom gc, Geom gp, int nu,
                                                                const Tc *__restrict__ xt,
                                                                const Tc *__restrict__ xp,
                                                                Tc *__restrict__ t,
                                                                const int *__restrict__ done) {
    if (done && *done) return;
    const int k = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= gf.nx) return;
    const int K = k / nu, r = k - K * nu;
    t[gf.at(k, 0, i)] = (r == 0) ? xt[gc.at(K, 0, i)] : xp[gp.at(1 + K * (nu - 1) + (r - 1), 0, i)];
}

template <typename Tin, typename Tc>
void launch_inject_restrict_1d(const Geom &gf, const Geom &gc, int nu, const Weights &w,
                               SpaceOp<Tc> L, const Tin *v, const double *sigma, Tc *vhat,
                               const int *done, cudaStream_t s) {
    dim3 grid, block;
    mg_launch(gc.nt + 1, gf.nx, grid, block);
    prof_begin(s);
    k_inject_restrict_1d<Tin, Tc><<<grid, block, 0, s>>>(gf, gc, nu, (Tc)w.a, (Tc)w.b, (Tc)w.mu,
                                                        L.x, v, sigma, vhat, done);
    prof_end(s, PROF_RESTRICT,
             (double)(gc.nt + 1) * gf.nx * (2.0 * sizeof(Tin) + sizeof(Tc)));
    count_launch();
}

template <typename Tc>
void launch_ideal_interp_rhs_1d(const Geom &gc, const Geom &gp, int nu, double b, SpaceOp<Tc> L,
                                const Tc *xt, Tc *rp, const int *done, cudaStream_t s) {
    dim3 grid, block;
    mg_launch(gc.nt, gc.nx, grid, block);
    prof_begin(s);
    k_ideal_rhs_1d<Tc><<<grid, block, 0, s>>>(gc, gp, nu, (Tc)b, L.x, xt, rp, done);
    prof_end(s, PROF_INTERP, (double)gc.nt * gc.nx * 2.0 * sizeof(Tc));
    count_launch();
}

template <typename Tc>
void launch_ideal_interp_gather_1d(const Geom &gf, const Geom &gc, const Geom &gp, int nu,
                                   const Tc *xt, const Tc *xp, Tc *t, const int *done,
                                   cudaStream_t s) {
    dim3 grid, block;
    mg_launch(gf.nt + 1, gf.nx, grid, block);
    prof_begin(s);
    k_ideal_gather_1d<Tc><<<grid, block, 0, s>>>(gf, gc, gp, nu, xt, xp, t, done);
    prof_end(s, PROF_INTERP, (double)(gf.nt + 1) * gf.nx * 2.0 * sizeof(Tc));
    count_launch();
}

template void launch_inject_restrict_1d<double, double>(const Geom &, const Geom &, int,
                                                        const Weights &, SpaceOp<double>,
                                                        const double *, const double *, double *,
                                                        const int *, cudaStream_t);
template void launch_inject_restrict_1d<float2, float>(const Geom &, const Geom &, int,
                                                       const Weights &, SpaceOp<float>,
                                                       const float2 *, const double *, float *,
                                                       const int *, cudaStream_t);
template void launch_inject_restrict_1d<float, float>(const Geom &, const Geom &, int,
                                                      const Weights &, SpaceOp<float>,
                                                      const float *, const double *, float *,
                                                      const int *, cudaStream_t);
template void launch_ideal_interp_rhs_1d<double>(const Geom &, const Geom &, int, double,
                                                 SpaceOp<double>, const double *, double *,
                                                 const int *, cudaStream_t);
template void launch_ideal_interp_rhs_1d<float>(const Geom &, const Geom &, int, double,
                                                SpaceOp<float>, const float *, float *,
                                                const int *, cudaStream_t);
template void launch_ideal_interp_gather_1d<double>(const Geom &, const Geom &, const Geom &, int,
                                                    const double *, const double *, double *,
                                                    const int *, cudaStream_t);
template void launch_ideal_interp_gather_1d<float>(const Geom &, const Geom &, const Geom &, int,
                                                   const float *, const float *, float *,
                                                   const int *, cudaStream_t);

}  // namespace mk
