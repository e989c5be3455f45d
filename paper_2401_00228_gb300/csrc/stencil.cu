// Space-time stencil kernels: RHS assembly, layout conversion, matvec A_l x (K1),
// residual f - A u (K2), fused matvec-shift-restriction (K3) and fused
// interpolation-correction-matvec (K4).
//
// Operator (Sec. 2, Eq. (finesys), at any level of Sec. 3.2 / Sec. 4):
//   (A x)_0 = x_0,   (A x)_k = (x_k - a L x_k) - (x_{k-1} + b L x_{k-1}),
// with L = Lx (+) Ly a sum of per-direction tridiagonal operators.
//
// Mapping: one thread per spatial point (or per coarse aggregate), looping over a chunk of
// consecutive time steps, so that x_{k-1} and L x_{k-1} are carried in registers and each
// element is read from DRAM once (spatial neighbours come from L1/L2).  Loads are
// coalesced along i (the contiguous direction of the padded layout).
#include "kernels.h"
#include "reduce.cuh"
#include <type_traits>

#include "stencil_common.cuh"
#include "async_copy.cuh"

namespace mk {

// ---------------------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------------------
template <typename Tsrc, typename Tdst>
__global__ void k_pack(Geom g, const Tsrc *__restrict__ dense, Tdst *__restrict__ padded) {
    int64_t n = g.interior();
    int64_t npts = g.npts();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = e / npts;
        int64_t r = e - k * npts;
        int j = (int)(r / g.nx), i = (int)(r - (int64_t)j * g.nx);
        padded[g.at((int)k, j, i)] = cvt_to<Tdst>(dense[e]);
    }
}

template <typename Tsrc, typename Tdst>
__global__ void k_unpack(Geom g, const Tsrc *__restrict__ padded, Tdst *__restrict__ dense) {
    int64_t n = g.interior();
    int64_t npts = g.npts();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = e / npts;
        int64_t r = e - k * npts;
        int j = (int)(r / g.nx), i = (int)(r - (int64_t)j * g.nx);
        dense[e] = cvt_to<Tdst>(padded[g.at((int)k, j, i)]);
    }
}

template <typename Tsrc, typename Tdst>
__global__ void k_convert(int64_t n, const Tsrc *__restrict__ src, Tdst *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (Tdst)src[e];
}


template <typename Tsrc, typename Tdst>
void launch_pack(const Geom &g, const Tsrc *dense, Tdst *padded, cudaStream_t s) {
    k_pack<Tsrc, Tdst><<<grid_for(g.interior(), 256), 256, 0, s>>>(g, dense, padded);
    count_launch();
}
template <typename Tsrc, typename Tdst>
void launch_unpack(const Geom &g, const Tsrc *padded, Tdst *dense, cudaStream_t s) {
    k_unpack<Tsrc, Tdst><<<grid_for(g.interior(), 256), 256, 0, s>>>(g, padded, dense);
    count_launch();
}
template <typename Tsrc, typename Tdst>
void launch_convert(int64_t n, const Tsrc *src, Tdst *dst, cudaStream_t s) {
    k_convert<Tsrc, Tdst><<<grid_for(n, 256), 256, 0, s>>>(n, src, dst);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// RHS assembly (Eq. (finesys)): f_k = dt ((1-theta) g_{k-1} + theta g_k), k >= 1
// ---------------------------------------------------------------------------------------
__global__ void k_rhs_source(Geom g, double theta, double dt, const double *__restrict__ gd,
                             double *__restrict__ f) {
    int64_t npts = g.npts();
    int64_t n = (int64_t)g.nt * npts;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t km1 = e / npts;
        int64_t r = e - km1 * npts;
        int j = (int)(r / g.nx), i = (int)(r - (int64_t)j * g.nx);
        double gbar = (1.0 - theta) * gd[e] + theta * gd[e + npts];
        f[g.at((int)km1 + 1, j, i)] = dt * gbar;
    }
}

void launch_rhs_source(const Geom &g, double theta, double dt, const double *gdense, double *f,
                       cudaStream_t s) {
    k_rhs_source<<<grid_for((int64_t)g.nt * g.npts(), 256), 256, 0, s>>>(g, theta, dt, gdense, f);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// K1: w = A x
// ---------------------------------------------------------------------------------------
template <int DIM, typename Tin, typename Tout, typename Tc>
__global__ void __launch_bounds__(256) k_apply(Geom g, Tc a, Tc b, SpaceOp<Tc> L,
                                               const Tin *__restrict__ x,
                                               Tout *__restrict__ w, int kc) {
    int i, j, chunk;
    point_index<DIM>(i, j, chunk);
    if (i >= g.nx || j >= g.ny) return;
    int k0 = chunk * kc;
    int k1 = min(k0 + kc, g.nt + 1);
    Tc prev = 0, Lprev = 0;
    if (k0 > 0) {
        int64_t idx = g.at(k0 - 1, j, i);
        prev = ldv<Tc>(x, idx);
        Lprev = lap_at<DIM, Tc>(x, idx, i, j, g, L.x, L.y);
    }
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        int64_t idx = g.at(k, j, i);
        Tc cur = ldv<Tc>(x, idx);
        Tc Lc = lap_at<DIM, Tc>(x, idx, i, j, g, L.x, L.y);
        Tc r = (k == 0) ? cur : (cur - a * Lc) - (prev + b * Lprev);
        w[idx] = (Tout)r;
        prev = cur;
        Lprev = Lc;
    }
}

// w = A x element-wise in 2D (32 x 8 x 1 blocks over (i, j, k)); rows k and k-1 of x are read
// directly (neighbours from cache).
template <typename Tin, typename Tout, typename Tc>
__global__ void __launch_bounds__(256) k_apply_2d(Geom g, Tc a, Tc b, SpaceOp<Tc> L,
                                                  const Tin *__restrict__ x,
                                                  Tout *__restrict__ w,
                                                  const int *__restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t idx = g.at(k, j, i);
    const Tc cur = ldv<Tc>(x, idx);
    Tc r;
    if (k == 0) {
        r = cur;
    } else {
        const int64_t ip = idx - g.plane;
        const Tc Lc = lap_at<2, Tc>(x, idx, i, j, g, L.x, L.y);
        const Tc Lp = lap_at<2, Tc>(x, ip, i, j, g, L.x, L.y);
        r = (cur - a * Lc) - (ldv<Tc>(x, ip) + b * Lp);
    }
    w[idx] = (Tout)r;
}

template <typename Tin, typename Tout, typename Tc>
void launch_apply(const Geom &g, const Weights &w, SpaceOp<Tc> L, const Tin *x, Tout *out,
                  cudaStream_t s) {
    int kc = cap_kc(choose_kc(g.npts(), g.nt + 1), g.nt + 1, g.dim, g.nx, g.ny);
    int nch = (g.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(g.dim, g.nx, g.ny, nch);
    if (g.dim == 1)
        k_apply<1, Tin, Tout, Tc><<<l.grid, l.block, 0, s>>>(g, (Tc)w.a, (Tc)w.b, L, x, out, kc);
    else
        k_apply<2, Tin, Tout, Tc><<<l.grid, l.block, 0, s>>>(g, (Tc)w.a, (Tc)w.b, L, x, out, kc);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// K2: r = f - A u, ||r||^2
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_residual(Geom g, double a, double b, SpaceOp<double> L,
                                                  const double *__restrict__ f,
                                                  const double *__restrict__ u,
                                                  double *__restrict__ r, int kc,
                                                  ReduceScratch rs, int slot, KState ks, int epi) {
    int i, j, chunk;
    point_index<DIM>(i, j, chunk);
    double acc = 0.0;
    if (i < g.nx && j < g.ny) {
        int k0 = chunk * kc;
        int k1 = min(k0 + kc, g.nt + 1);
        double prev = 0, Lprev = 0;
        if (k0 > 0) {
            int64_t idx = g.at(k0 - 1, j, i);
            prev = u[idx];
            Lprev = lap_at<DIM, double>(u, idx, i, j, g, L.x, L.y);
        }
        for (int k = k0; k < k1; ++k) {
            int64_t idx = g.at(k, j, i);
            double cur = u[idx];
            double Lc = lap_at<DIM, double>(u, idx, i, j, g, L.x, L.y);
            double Au = (k == 0) ? cur : (cur - a * Lc) - (prev + b * Lprev);
            double rv = f[idx] - Au;
            r[idx] = rv;
            acc += rv * rv;
            prev = cur;
            Lprev = Lc;
        }
    }
    block_partial_and_finish(acc, rs, slot, ks, epi);
}

void launch_residual(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                     const double *u, double *r, const ReduceScratch &rs, int slot, KState ks,
                     int epi, cudaStream_t s) {
    int kc = cap_kc(choose_kc(g.npts(), g.nt + 1), g.nt + 1, g.dim, g.nx, g.ny);
    int nch = (g.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(g.dim, g.nx, g.ny, nch);
    prof_begin(s);
    if (g.dim == 1)
        k_residual<1><<<l.grid, l.block, 0, s>>>(g, w.a, w.b, L, f, u, r, kc, rs, slot, ks, epi);
    else
        k_residual<2><<<l.grid, l.block, 0, s>>>(g, w.a, w.b, L, f, u, r, kc, rs, slot, ks, epi);
    prof_end(s, PROF_RESIDUAL, 3.0 * 8.0 * (double)g.interior());
    count_launch();
}

// ---------------------------------------------------------------------------------------
// K3: vhat = sigma Y^T (A v - mu v)   (substeps 4.1-4.2)
//   Y^T sums the nu fine steps of each coarse block (Eq. (tcoarseZ), Y_k = Z_k) and, with
//   space agglomeration, averages each aggregate (Eq. (constructY)).  Block 0 maps to
//   block 0: (A v)_0 = v_0, so vhat_0 = sigma (1 - mu) Y^T v_0.
//   Thread -> coarse spatial point (aggregate), loop over a chunk of coarse blocks; the
//   fine points of the aggregate (1, 2 or 4) each carry their own (v_{k-1}, L v_{k-1}).
// ---------------------------------------------------------------------------------------
template <int DIM, bool SPACE, typename Tin, typename Tout, typename Tc, int NU = 0>
__global__ void __launch_bounds__(256) k_restrict(Geom gf, Geom gc, int nu_rt, Tc a, Tc b, Tc mu,
                                                  SpaceOp<Tc> L, const Tin *__restrict__ v,
                                                  const double *__restrict__ sigma,
                                                  Tout *__restrict__ vhat, int kc,
                                                  ReduceScratch rs, int slot, KState ks,
                                                  const int *__restrict__ done) {
    if (done && *done) return;
    constexpr int PX = SPACE ? 2 : 1;
    constexpr int PY = (SPACE && DIM == 2) ? 2 : 1;
    // NU > 0: the coarsening factor fixed at compile time (the fine steps of a coarse block
    // unrolled, their loads issued together)
    const int nu = NU > 0 ? NU : nu_rt;
    int I, J, chunk;
    point_index<DIM>(I, J, chunk);
    Tc acc2 = (Tc)0;   // per-thread and per-warp sums in the arithmetic type, FP64 across warps
    const bool active = I < gc.nx && J < gc.ny;
    const Tc scale = block_scalar<Tc>(sigma);
    if (active) {
        // fine points of this aggregate
        int ii[PX], jj[PY];
        int npx = 0, npy = 0;
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            ii[p] = PX * I + p;
            if (ii[p] < gf.nx) npx = p + 1;
        }
#pragma unroll
        for (int q = 0; q < PY; ++q) {
            jj[q] = (DIM == 2) ? PY * J + q : 0;
            if (jj[q] < gf.ny) npy = q + 1;
        }
        const Tc inv_count = (Tc)1 / (Tc)(npx * npy);
        Tc prev[PY][PX], Lprev[PY][PX];
        const int K0 = chunk * kc;
        const int K1 = min(K0 + kc, gc.nt + 1);
        // state at the fine step just before the chunk
        if (K0 > 0) {
            int kf = nu * (K0 - 1);
#pragma unroll
            for (int q = 0; q < PY; ++q)
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    prev[q][p] = 0;
                    Lprev[q][p] = 0;
                    if (p < npx && q < npy) {
                        int64_t idx = gf.at(kf, jj[q], ii[p]);
                        prev[q][p] = ldv<Tc>(v, idx);
                        Lprev[q][p] = lap_at<DIM, Tc>(v, idx, ii[p], jj[q], gf, L.x, L.y);
                    }
                }
        }
        for (int K = K0; K < K1; ++K) {
            Tc sum = 0;
            if (K == 0) {
#pragma unroll
                for (int q = 0; q < PY; ++q)
#pragma unroll
                    for (int p = 0; p < PX; ++p) {
                        if (p < npx && q < npy) {
                            int64_t idx = gf.at(0, jj[q], ii[p]);
                            Tc cur = ldv<Tc>(v, idx);
                            sum += cur - mu * cur;
                            prev[q][p] = cur;
                            Lprev[q][p] = lap_at<DIM, Tc>(v, idx, ii[p], jj[q], gf, L.x, L.y);
                        }
                    }
            } else {
#pragma unroll
                for (int s = 1; s <= (NU > 0 ? NU : nu); ++s) {
                    int kf = nu * (K - 1) + s;
#pragma unroll
                    for (int q = 0; q < PY; ++q)
#pragma unroll
                        for (int p = 0; p < PX; ++p) {
                            if (p < npx && q < npy) {
                                int64_t idx = gf.at(kf, jj[q], ii[p]);
                                Tc cur = ldv<Tc>(v, idx);
                                Tc Lc = lap_at<DIM, Tc>(v, idx, ii[p], jj[q], gf, L.x, L.y);
                                Tc Av = (cur - a * Lc) - (prev[q][p] + b * Lprev[q][p]);
                                sum += Av - mu * cur;
                                prev[q][p] = cur;
                                Lprev[q][p] = Lc;
                            }
                        }
                }
            }
            Tc outv = scale * (sum * inv_count);
            vhat[gc.at(K, J, I)] = (Tout)outv;
            acc2 += outv * outv;
        }
    }
    if (ks.d) block_partial_and_finish_t(acc2, rs, slot, ks, EPI_BETA);
}

// 2D specialisation of K3 for 2 x 2 agglomeration and nu = 2 (every coarsening of the 2D
// workloads): a thread owns the aggregate (I, J), i.e. fine points (2I, 2I+1) x (2J, 2J+1),
// and walks its chunk of coarse steps.  Each fine step it loads its 2 x 2 values and the two
// points of the rows 2J-1 and 2J+2 as four vector loads (the pair 2I, 2I+1 is 8- or 16-byte
// aligned: 2I is even and rows start at multiples of 8 elements); the x neighbours 2I-1 and
// 2I+2 come from the adjacent lanes by warp shuffles, and the two edge lanes of a warp load
// theirs.  Every lane runs the loop (lanes past the grid carry zeros and store nothing).
// Points outside the fine grid (the singleton edge of an odd size) are masked.
template <typename Tc>
__device__ __forceinline__ void ld_pair(const float2 *p, Tc &a, Tc &b) {
    const float4 q = *reinterpret_cast<const float4 *>(p);   // double-float pairs: hi parts
    a = (Tc)q.x;
    b = (Tc)q.z;
}
template <typename Tc>
__device__ __forceinline__ void ld_pair(const float *p, Tc &a, Tc &b) {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    a = (Tc)q.x;
    b = (Tc)q.y;
}
template <typename Tc>
__device__ __forceinline__ void ld_pair(const double *p, Tc &a, Tc &b) {
    const double2 q = *reinterpret_cast<const double2 *>(p);
    a = (Tc)q.x;
    b = (Tc)q.y;
}

template <typename Tin, typename Tout, typename Tc>
__global__ void __launch_bounds__(256) k_restrict_2d_ts(Geom gf, Geom gc, Tc a, Tc b, Tc mu,
                                                        SpaceOp<Tc> L, const Tin *__restrict__ v,
                                                        const double *__restrict__ sigma,
                                                        Tout *__restrict__ vhat, int kc,
                                                        ReduceScratch rs, int slot, KState ks,
                                                        const int *__restrict__ done) {
    if (done && *done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;   // blocks are 32 x 8: a warp is one row of 32 I's
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int chunk = blockIdx.z;
    const bool active = I < gc.nx && J < gc.ny;
    const int i0 = 2 * I, i1 = 2 * I + 1, j0 = 2 * J, j1 = 2 * J + 1;
    const bool in00 = active, in01 = active && i1 < gf.nx;              // (j0, i0), (j0, i1)
    const bool in10 = active && j1 < gf.ny, in11 = in10 && i1 < gf.nx;  // (j1, i0), (j1, i1)
    const Tc *cx = L.x, *cy = L.y;
    const int nxf = gf.nx, nyf = gf.ny;
    // coefficients of the thread's columns and rows (0 where masked)
    const Tc xl0 = in00 ? cx[i0] : (Tc)0, xd0 = in00 ? cx[nxf + i0] : (Tc)0, xu0 = in00 ? cx[2 * nxf + i0] : (Tc)0;
    const Tc xl1 = in01 ? cx[i1] : (Tc)0, xd1 = in01 ? cx[nxf + i1] : (Tc)0, xu1 = in01 ? cx[2 * nxf + i1] : (Tc)0;
    const Tc yl0 = in00 ? cy[j0] : (Tc)0, yd0 = in00 ? cy[nyf + j0] : (Tc)0, yu0 = in00 ? cy[2 * nyf + j0] : (Tc)0;
    const Tc yl1 = in10 ? cy[j1] : (Tc)0, yd1 = in10 ? cy[nyf + j1] : (Tc)0, yu1 = in10 ? cy[2 * nyf + j1] : (Tc)0;
    const int npts = (int)in00 + (int)in01 + (int)in10 + (int)in11;
    const Tc inv_count = npts > 0 ? (Tc)1 / (Tc)npts : (Tc)0;
    const Tc scale = block_scalar<Tc>(sigma);
    // values and Laplacians of the four points at fine step kf
    auto step = [&](int kf, Tc (&c)[4], Tc (&l)[4]) {
        const int64_t r0 = gf.at(kf, j0, 0);
        Tc u0a = 0, u0b = 0, u1a = 0, u1b = 0, dna = 0, dnb = 0, upa = 0, upb = 0;
        if (active) {
            ld_pair<Tc>(v + r0 + i0, u0a, u0b);                 // row j0
            ld_pair<Tc>(v + r0 + gf.ldx + i0, u1a, u1b);        // row j1 (the zero row at ny)
            ld_pair<Tc>(v + r0 - gf.ldx + i0, dna, dnb);        // row j0 - 1 (zero below j = 0)
            ld_pair<Tc>(v + r0 + 2 * gf.ldx + i0, upa, upb);    // row j1 + 1
        }
        // x neighbours: 2I - 1 is the left lane's second column, 2I + 2 the right lane's first
        Tc l0 = __shfl_up_sync(FULL, u0b, 1), l1 = __shfl_up_sync(FULL, u1b, 1);
        Tc r0v = __shfl_down_sync(FULL, u0a, 1), r1v = __shfl_down_sync(FULL, u1a, 1);
        if (lane == 0) {
            l0 = active ? ldv<Tc>(v, r0 + i0 - 1) : (Tc)0;
            l1 = active ? ldv<Tc>(v, r0 + gf.ldx + i0 - 1) : (Tc)0;
        }
        if (lane == 31) {
            r0v = active ? ldv<Tc>(v, r0 + i1 + 1) : (Tc)0;
            r1v = active ? ldv<Tc>(v, r0 + gf.ldx + i1 + 1) : (Tc)0;
        }
        c[0] = u0a; c[1] = u0b; c[2] = u1a; c[3] = u1b;
        // the order of lap_at: x part, then the y part added
        l[0] = (xd0 * u0a + xl0 * l0 + xu0 * u0b) + (yd0 * u0a + yl0 * dna + yu0 * u1a);
        l[1] = (xd1 * u0b + xl1 * u0a + xu1 * r0v) + (yd0 * u0b + yl0 * dnb + yu0 * u1b);
        l[2] = (xd0 * u1a + xl0 * l1 + xu0 * u1b) + (yd1 * u1a + yl1 * u0a + yu1 * upa);
        l[3] = (xd1 * u1b + xl1 * u1a + xu1 * r1v) + (yd1 * u1b + yl1 * u0b + yu1 * upb);
    };
    const bool m[4] = {in00, in01, in10, in11};
    Tc prev[4] = {0, 0, 0, 0}, Lprev[4] = {0, 0, 0, 0};
    const int K0 = chunk * kc;
    const int K1 = min(K0 + kc, gc.nt + 1);
    if (K0 > 0) step(2 * (K0 - 1), prev, Lprev);
    Tc acc2 = (Tc)0;   // per-thread and per-warp sums in the arithmetic type, FP64 across warps
    for (int K = K0; K < K1; ++K) {
        Tc sum = 0;
        if (K == 0) {
            Tc c[4], l[4];
            step(0, c, l);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (m[q]) sum += c[q] - mu * c[q];
                prev[q] = c[q];
                Lprev[q] = l[q];
            }
        } else {
            Tc c1[4], l1[4], c2[4], l2[4];
            step(2 * K - 1, c1, l1);
            step(2 * K, c2, l2);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (m[q]) {
                    const Tc av1 = (c1[q] - a * l1[q]) - (prev[q] + b * Lprev[q]);
                    sum += av1 - mu * c1[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (m[q]) {
                    const Tc av2 = (c2[q] - a * l2[q]) - (c1[q] + b * l1[q]);
                    sum += av2 - mu * c2[q];
                }
                prev[q] = c2[q];
                Lprev[q] = l2[q];
            }
        }
        if (active) {
            const Tc outv = scale * (sum * inv_count);
            vhat[gc.at(K, J, I)] = (Tout)outv;
            acc2 += outv * outv;
        }
    }
    if (ks.d) block_partial_and_finish_t(acc2, rs, slot, ks, EPI_BETA);
}

// 1D specialisation of K3: one thread per coarse column; each fine value is loaded once and
// its spatial neighbours come from the adjacent lanes (warp shuffles; the two edge lanes of
// a warp load their outer neighbour).  With agglomeration a thread owns the fine pair
// (2I, 2I+1).  Every lane of a warp runs the loop (lanes past the grid carry zeros).
template <bool SPACE, typename Tin, typename Tout, typename Tc>
__global__ void __launch_bounds__(256) k_restrict_1d(Geom gf, Geom gc, int nu, Tc a, Tc b, Tc mu,
                                                     SpaceOp<Tc> L, const Tin *__restrict__ v,
                                                     const double *__restrict__ sigma,
                                                     Tout *__restrict__ vhat, int kc,
                                                     ReduceScratch rs, int slot, KState ks,
                                                     const int *__restrict__ done) {
    if (done && *done) return;
    const unsigned FULL = 0xffffffffu;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int nf = gf.nx;
    const bool active = I < gc.nx;
    const int p0 = SPACE ? 2 * I : I;           // fine points of this column
    const int p1 = SPACE ? 2 * I + 1 : I;
    const bool has0 = p0 < nf, has1 = SPACE && p1 < nf;
    const Tc *cx = L.x;
    const Tc lo0 = has0 ? cx[p0] : (Tc)0, di0 = has0 ? cx[nf + p0] : (Tc)0, up0 = has0 ? cx[2 * nf + p0] : (Tc)0;
    const Tc lo1 = has1 ? cx[p1] : (Tc)0, di1 = has1 ? cx[nf + p1] : (Tc)0, up1 = has1 ? cx[2 * nf + p1] : (Tc)0;
    const Tc inv_count = SPACE ? ((Tc)1 / (Tc)(has1 ? 2 : 1)) : (Tc)1;
    const Tc scale = block_scalar<Tc>(sigma);
    auto fine = [&](int k, int p) -> Tc { return (p >= 0 && p < nf) ? ldv<Tc>(v, gf.at(k, 0, p)) : (Tc)0; };
    // values and Laplacians of the thread's fine points at fine step k
    auto row = [&](int k, Tc &c0, Tc &c1, Tc &l0, Tc &l1) {
        c0 = has0 ? ldv<Tc>(v, gf.at(k, 0, p0)) : (Tc)0;
        c1 = has1 ? ldv<Tc>(v, gf.at(k, 0, p1)) : (Tc)0;
        Tc left, right;
        if (SPACE) {
            left = __shfl_up_sync(FULL, c1, 1);
            right = __shfl_down_sync(FULL, c0, 1);
            if (lane == 0) left = fine(k, p0 - 1);
            if (lane == 31) right = fine(k, p1 + 1);
            l0 = di0 * c0 + lo0 * left + up0 * c1;
            l1 = di1 * c1 + lo1 * c0 + up1 * right;
        } else {
            left = __shfl_up_sync(FULL, c0, 1);
            right = __shfl_down_sync(FULL, c0, 1);
            if (lane == 0) left = fine(k, p0 - 1);
            if (lane == 31) right = fine(k, p0 + 1);
            l0 = di0 * c0 + lo0 * left + up0 * right;
            l1 = (Tc)0;
        }
    };
    Tc acc2 = (Tc)0;   // per-thread and per-warp sums in the arithmetic type, FP64 across warps
    const int K0 = blockIdx.y * kc;
    const int K1 = min(K0 + kc, gc.nt + 1);
    Tc pr0 = 0, pr1 = 0, Lp0 = 0, Lp1 = 0;
    if (K0 > 0) row(nu * (K0 - 1), pr0, pr1, Lp0, Lp1);
    for (int K = K0; K < K1; ++K) {
        Tc sum = 0;
        if (K == 0) {
            Tc c0, c1, l0, l1;
            row(0, c0, c1, l0, l1);
            sum = (c0 - mu * c0) + (c1 - mu * c1);
            pr0 = c0;
            pr1 = c1;
            Lp0 = l0;
            Lp1 = l1;
        } else {
            for (int st = 1; st <= nu; ++st) {
                const int kf = nu * (K - 1) + st;
                Tc c0, c1, l0, l1;
                row(kf, c0, c1, l0, l1);
                Tc Av0 = (c0 - a * l0) - (pr0 + b * Lp0);
                sum += Av0 - mu * c0;
                if (SPACE) {
                    Tc Av1 = (c1 - a * l1) - (pr1 + b * Lp1);
                    sum += Av1 - mu * c1;
                }
                pr0 = c0;
                pr1 = c1;
                Lp0 = l0;
                Lp1 = l1;
            }
        }
        if (active) {
            Tc outv = scale * (sum * inv_count);
            vhat[gc.at(K, 0, I)] = (Tout)outv;
            acc2 += outv * outv;
        }
    }
    if (ks.d) block_partial_and_finish_t(acc2, rs, slot, ks, EPI_BETA);
}

template <typename Tin, typename Tout, typename Tc>
void launch_restrict(const Geom &gf, const Geom &gc, int nu, bool space, const Weights &w,
                     SpaceOp<Tc> L, const Tin *v, const double *sigma, Tout *vhat,
                     const ReduceScratch &rs, int slot, KState ks_c, const int *done,
                     cudaStream_t s) {
    int kc = choose_kc(gc.npts() * (space ? (gf.dim == 2 ? 4 : 2) : 1) * nu, gc.nt + 1);
    if (gf.dim == 2) {
        // a thread walks its chunk of coarse steps serially: enough chunks for one full wave
        // of 2048 threads per SM, but at least four fine steps per chunk (the fine step before
        // each chunk is read again)
        const int64_t want = (int64_t)g_num_sms * 2048;
        const int64_t k2 = (gc.npts() * (int64_t)(gc.nt + 1)) / want;
        const int kmin = (4 + nu - 1) / nu;
        if (k2 < kc) kc = k2 < kmin ? kmin : (int)k2;
    }
    kc = cap_kc(kc, gc.nt + 1, gf.dim, gc.nx, gc.ny);
    int nch = (gc.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(gf.dim, gc.nx, gc.ny, nch);
    Tc a = (Tc)w.a, b = (Tc)w.b, mu = (Tc)w.mu;
#define MK_RESTRICT(D, S)                                                                     \
    do {                                                                                      \
        if (nu == 2)                                                                          \
            k_restrict<D, S, Tin, Tout, Tc, 2><<<l.grid, l.block, 0, s>>>(                    \
                gf, gc, nu, a, b, mu, L, v, sigma, vhat, kc, rs, slot, ks_c, done);           \
        else                                                                                  \
            k_restrict<D, S, Tin, Tout, Tc><<<l.grid, l.block, 0, s>>>(                       \
                gf, gc, nu, a, b, mu, L, v, sigma, vhat, kc, rs, slot, ks_c, done);           \
    } while (0)
#define MK_RESTRICT1(S) \
    k_restrict_1d<S, Tin, Tout, Tc><<<l.grid, l.block, 0, s>>>(gf, gc, nu, a, b, mu, L, v, sigma, \
                                                                vhat, kc, rs, slot, ks_c, done)
    prof_begin(s);
    if (launch_restrict_1d_tiled<Tin, Tout, Tc>(gf, gc, nu, space, w, L, v, sigma, vhat, rs, slot,
                                                ks_c, done, s)) {
        // 1D, nu = 2: time-tiled kernel (transfer1d.cu)
    } else if (gf.dim == 1) {
        if (space) MK_RESTRICT1(true); else MK_RESTRICT1(false);
    } else if (space && nu == 2) {
        // 2 x 2 agglomeration with nu = 2: aggregate-per-thread kernel with vector loads
        k_restrict_2d_ts<Tin, Tout, Tc><<<l.grid, l.block, 0, s>>>(gf, gc, a, b, mu, L, v, sigma,
                                                                    vhat, kc, rs, slot, ks_c, done);
    } else {
        if (space) MK_RESTRICT(2, true); else MK_RESTRICT(2, false);
    }
#undef MK_RESTRICT
#undef MK_RESTRICT1
    prof_end(s, PROF_RESTRICT, (double)gf.interior() * sizeof(Tin) + (double)gc.interior() * sizeof(Tout));
    count_launch();
}

// ---------------------------------------------------------------------------------------
// K4: x = sigma v - Z vt,  w = A x      (substeps 4.4-4.5 and step 5 of Algorithm 2)
//   vt = sum_m yc[m] Xc_m (the inner FGMRES solution of the coarser level, combined on
//   the fly).  (Z vt)_0 = Z vt_0, (Z vt)_k = Z vt_{ceil(k/nu)}; in space Z copies the
//   aggregate value to its members (Eq. (constructZ)).
// ---------------------------------------------------------------------------------------
template <int DIM, bool SPACE, typename Tv, typename Tz, typename Tx>
struct XEval {
    const Tv *v;
    Tx sigma;
    const Tz *Xc;
    int mc;             // 0: a single coarse vector with coefficient 1
    int64_t xc_stride;
    Tx y[MK_MAX_INNER]; // combination coefficients, converted once per thread
    Geom gf, gc;
    int nu;

    // x at fine (k, j, i); zero outside the interior (Dirichlet)
    __device__ __forceinline__ Tx operator()(int k, int j, int i) const {
        if (i < 0 || i >= gf.nx || j < 0 || j >= gf.ny) return (Tx)0;
        int K = (k == 0) ? 0 : (k - 1) / nu + 1;
        int I = SPACE ? (i >> 1) : i;
        int J = (SPACE && DIM == 2) ? (j >> 1) : j;
        int64_t cidx = gc.at(K, J, I);
        Tx zt;
        if (mc == 0) {
            zt = (Tx)Xc[cidx];
        } else {
            zt = (Tx)0;
#pragma unroll
            for (int m = 0; m < MK_MAX_INNER; ++m)
                if (m < mc) zt = fma_rn(y[m], (Tx)Xc[cidx + m * xc_stride], zt);
        }
        return fma_rn(sigma, (Tx)v[gf.at(k, j, i)], -zt);
    }
};

template <int DIM, bool SPACE, typename Tv, typename Tz, typename Tx, typename Tw, typename Tc>
__global__ void __launch_bounds__(256) k_interp(Geom gf, Geom gc, int nu, Tc a, Tc b,
                                                SpaceOp<Tc> L, const Tv *__restrict__ v,
                                                const double *__restrict__ sigma,
                                                const Tz *__restrict__ Xc, int mc,
                                                int64_t xc_stride,
                                                const double *__restrict__ yc,
                                                Tx *__restrict__ xout, Tw *__restrict__ wout,
                                                int kc, const int *__restrict__ done) {
    if (done && *done) return;
    int i, j, chunk;
    point_index<DIM>(i, j, chunk);
    if (i >= gf.nx || j >= gf.ny) return;
    XEval<DIM, SPACE, Tv, Tz, Tx> X;
    X.v = v;
    X.sigma = sigma ? (Tx)(*sigma) : (Tx)1;
    X.Xc = Xc;
    X.mc = yc ? mc : 0;
    X.xc_stride = xc_stride;
    for (int m = 0; m < MK_MAX_INNER; ++m) X.y[m] = (yc && m < mc) ? (Tx)yc[m] : (Tx)0;
    X.gf = gf;
    X.gc = gc;
    X.nu = nu;
    const Tc *cx = L.x;
    const Tc *cy = L.y;
    auto lap = [&](int k, Tc c) -> Tc {
        Tc s = cx[gf.nx + i] * c + cx[i] * (Tc)X(k, j, i - 1) + cx[2 * gf.nx + i] * (Tc)X(k, j, i + 1);
        if (DIM == 2) {
            Tc sy = cy[gf.ny + j] * c + cy[j] * (Tc)X(k, j - 1, i) + cy[2 * gf.ny + j] * (Tc)X(k, j + 1, i);
            s = s + sy;
        }
        return s;
    };
    int k0 = chunk * kc;
    int k1 = min(k0 + kc, gf.nt + 1);
    Tc prev = 0, Lprev = 0;
    if (k0 > 0) {
        prev = (Tc)X(k0 - 1, j, i);
        Lprev = lap(k0 - 1, prev);
    }
    for (int k = k0; k < k1; ++k) {
        Tx xs = X(k, j, i);
        Tc cur = (Tc)xs;
        Tc Lc = lap(k, cur);
        Tc r = (k == 0) ? cur : (cur - a * Lc) - (prev + b * Lprev);
        int64_t idx = gf.at(k, j, i);
        xout[idx] = xs;
        wout[idx] = (Tw)r;
        prev = cur;
        Lprev = Lc;
    }
}

// 1D specialisation of K4: x is formed once per point and its spatial neighbours come from
// the adjacent lanes (warp shuffles).  Row base pointers and the coarse block index K(k)
// are advanced once per time step (no division per point), and the combination
// vt = sum_m y_m Xc_m is specialised on the number of coarse directions MC (0: a single
// vector with coefficient 1; 1; 2; -1: any count up to MK_MAX_INNER).
template <bool SPACE, int MC, typename Tv, typename Tz, typename Tx, typename Tw, typename Tc>
__global__ void __launch_bounds__(256) k_interp_1d(Geom gf, Geom gc, int nu, Tc a, Tc b,
                                                   SpaceOp<Tc> L, const Tv *__restrict__ v,
                                                   const double *__restrict__ sigma,
                                                   const Tz *__restrict__ Xc, int mc,
                                                   int64_t xc_stride,
                                                   const double *__restrict__ yc,
                                                   Tx *__restrict__ xout, Tw *__restrict__ wout,
                                                   int kc, const int *__restrict__ done) {
    if (done && *done) return;
    const unsigned FULL = 0xffffffffu;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int nx = gf.nx;
    const bool act = i < nx;
    const Tx sig = sigma ? (Tx)(*sigma) : (Tx)1;
    constexpr int NY = MC > 0 ? MC : MK_MAX_INNER;
    Tx y[NY];
#pragma unroll
    for (int m = 0; m < NY; ++m) y[m] = (yc && m < mc) ? (Tx)yc[m] : (Tx)0;
    const Tc *cx = L.x;
    const Tc clo = act ? cx[i] : (Tc)0, cdi = act ? cx[nx + i] : (Tc)0,
             cup = act ? cx[2 * nx + i] : (Tc)0;
    auto xval = [&](const Tv *vr, const Tz *zr, int ii) -> Tx {
        if (ii < 0 || ii >= nx) return (Tx)0;
        const Tz *zp = zr + (SPACE ? (ii >> 1) : ii);
        Tx zt;
        if (MC == 0) {
            zt = (Tx)zp[0];
        } else if (MC == 1) {
            zt = mul_rn(y[0], (Tx)zp[0]);
        } else if (MC == 2) {
            zt = fma_rn(y[NY > 1 ? 1 : 0], (Tx)zp[xc_stride], mul_rn(y[0], (Tx)zp[0]));
        } else {
            zt = (Tx)0;
#pragma unroll
            for (int m = 0; m < NY; ++m)
                if (m < mc) zt = fma_rn(y[m], (Tx)zp[m * xc_stride], zt);
        }
        return fma_rn(sig, ldv<Tx>(vr, ii), -zt);
    };
    const int k0 = blockIdx.y * kc;
    const int k1 = min(k0 + kc, gf.nt + 1);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    // coarse block of fine step k: 0 for k = 0, (k-1)/nu + 1 otherwise (tracked incrementally)
    int K = (kstart == 0) ? 0 : (kstart - 1) / nu + 1;
    int ph = (kstart == 0) ? nu - 1 : (kstart - 1) % nu;
    Tc prev = 0, Lprev = 0;
    for (int k = kstart; k < k1; ++k) {
        if (k > kstart) {
            if (ph == nu - 1) {
                ++K;
                ph = 0;
            } else {
                ++ph;
            }
        }
        const Tv *vr = v + gf.guard + (int64_t)k * gf.plane;
        const Tz *zr = Xc + gc.guard + (int64_t)K * gc.plane;
        Tx xc = xval(vr, zr, i);
        Tx xl = __shfl_up_sync(FULL, xc, 1), xr = __shfl_down_sync(FULL, xc, 1);
        if (lane == 0) xl = xval(vr, zr, i - 1);
        if (lane == 31) xr = xval(vr, zr, i + 1);
        Tc cur = (Tc)xc;
        Tc Lc = cdi * cur + clo * (Tc)xl + cup * (Tc)xr;
        if (k >= k0) {
            Tc r = (k == 0) ? cur : (cur - a * Lc) - (prev + b * Lprev);
            if (act) {
                int64_t idx = gf.guard + (int64_t)k * gf.plane + i;
                xout[idx] = xc;
                wout[idx] = (Tw)r;
            }
        }
        prev = cur;
        Lprev = Lc;
    }
}

template <typename T>
__device__ __forceinline__ void st_pair_t(T *p, T a, T b);
template <>
__device__ __forceinline__ void st_pair_t<float>(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void st_pair_t<double>(double *p, double a, double b) {
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}

// 2D K4 with 2 x 2 aggregates in FP32, walked in time.  A thread owns the aggregate (I, J): the
// fine points (2I, 2I+1) x (2J, 2J+1), which share one coarse value (Z vt)_{K(k)}.  Per fine
// step it forms x at those four points and at the two points of each adjacent row (2J-1, 2J+2:
// the aggregates J-1 and J+1); the columns 2I-1 and 2I+2 come from the neighbouring lanes by
// warp shuffles (the first and last lane form them itself).  x_{k-1} and L x_{k-1} stay in
// registers from the previous step, so x and w are written once per point and v read once per
// point from HBM (the adjacent rows are the neighbouring threads' rows, served by the caches).
// The arithmetic is that of k_apply_2d (lap_at's order: x part, then the y part added;
// w_k = (x_k - a L x_k) - (x_{k-1} + b L x_{k-1})).  MC: the number of coarse directions
// combined (0: Xc itself).
// The loads of later steps are staged in shared memory: every thread copies its own words of
// step k+2 (the four row pairs, the outer columns of the first and last lane, the coarse
// values) into a three-stage ring with cp.async while it computes step k, and reads back only
// what it copied (cp.async.wait_group orders that, no block barrier), so about two steps of
// loads stay in flight at the register count of one (a register-staged version with one step
// ahead took 266 us against 208 us per level-1 launch on the 255^2 x 1024 workload).  Fields are
// laid out field-major (word t of a field belongs to thread t): a warp's accesses are
// conflict-free.  Row starts are multiples of eight elements and i0 is even, so the paired
// accesses are 8-byte aligned; a row is read only where it is interior.
constexpr int I2C_STAGES = 3;
constexpr int I2C_THREADS = 256;
__host__ __device__ constexpr int i2c_fields(int nz) { return 10 + 4 * nz; }   // floats per thread and stage
inline size_t i2c_smem_bytes(int mc) {
    const int nz = mc > 0 ? mc : 1;
    return sizeof(float) * (size_t)I2C_STAGES * i2c_fields(nz) * I2C_THREADS;
}

template <int MC>
__global__ void __launch_bounds__(256, 2) k_interp_2d_cp(Geom gf, Geom gc, int nu, float a, float b,
                                                         SpaceOp<float> L,
                                                         const float *__restrict__ v,
                                                         const double *__restrict__ sigma,
                                                         const float *__restrict__ Xc,
                                                         int64_t xc_stride,
                                                         const double *__restrict__ yc,
                                                         float *__restrict__ x,
                                                         float *__restrict__ w, int kc,
                                                         const int *__restrict__ done) {
    if (done && *done) return;   // the same flag for every thread of the block
    constexpr int NZ = MC > 0 ? MC : 1;
    constexpr int SF = i2c_fields(NZ);
    extern __shared__ float i2c_ring[];   // [I2C_STAGES][SF][I2C_THREADS]
    __shared__ float s_w[NZ + 1];
    const int t = threadIdx.x + 32 * threadIdx.y;
    if (t == 0) s_w[0] = sigma ? (float)(*sigma) : 1.f;
    else if (MC > 0 && t <= MC) s_w[t] = (float)yc[t - 1];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int I = blockIdx.x * 32 + lane;
    const int J = blockIdx.y * 8 + threadIdx.y;
    const int nx = gf.nx, ny = gf.ny;
    const int64_t ldx = gf.ldx, cld = gc.ldx;
    const int i0 = 2 * I, j0 = 2 * J;
    if (j0 >= ny) return;   // the whole warp shares J; no block barrier follows
    const float sig = s_w[0];
    float ym[NZ];
#pragma unroll
    for (int m = 0; m < NZ; ++m) ym[m] = MC > 0 ? s_w[1 + m] : 1.f;
    const bool c0 = i0 < nx, c1 = i0 + 1 < nx, r1 = j0 + 1 < ny;
    const bool hd = c0 && j0 > 0, hu = c0 && j0 + 2 < ny;
    const bool cl = lane == 0 && i0 > 0 && i0 - 1 < nx, cr = lane == 31 && i0 + 2 < nx;
    const bool ce = cl || cr;
    const int64_t o0 = (int64_t)j0 * ldx + i0;   // fine offset of (2J, 2I) in a plane
    const int64_t oc = (int64_t)J * cld + I;      // coarse offset of (J, I)
    const int64_t oe = o0 + (cl ? -1 : 2);        // outside column of the first / last lane
    const int64_t oce = oc + (cl ? -1 : 1);
    const float *cx = L.x, *cy = L.y;
    const int i1 = i0 + 1, j1 = j0 + 1;
    const float xl0 = c0 ? cx[i0] : 0.f, xd0 = c0 ? cx[nx + i0] : 0.f, xu0 = c0 ? cx[2 * nx + i0] : 0.f;
    const float xl1 = c1 ? cx[i1] : 0.f, xd1 = c1 ? cx[nx + i1] : 0.f, xu1 = c1 ? cx[2 * nx + i1] : 0.f;
    const float yl0 = c0 ? cy[j0] : 0.f, yd0 = c0 ? cy[ny + j0] : 0.f, yu0 = c0 ? cy[2 * ny + j0] : 0.f;
    const float yl1 = (c0 && r1) ? cy[j1] : 0.f, yd1 = (c0 && r1) ? cy[ny + j1] : 0.f,
                yu1 = (c0 && r1) ? cy[2 * ny + j1] : 0.f;
    // ring fields of this thread: pairs of rows j0, j0+1, j0-1, j0+2, the two outer-column
    // values, then for each coarse direction the values of aggregates (J,I), (J-1,I), (J+1,I)
    // and the outer one
    auto field = [&](int stage, int f) -> float * {
        return i2c_ring + ((int64_t)stage * SF + f) * I2C_THREADS + t;
    };
    auto pair = [&](int stage, int f) -> float2 * {   // fields 2f, 2f+1 hold one float2 per thread
        return reinterpret_cast<float2 *>(i2c_ring + ((int64_t)stage * SF + 2 * f) * I2C_THREADS) + t;
    };
    auto issue = [&](int k, int K, int stage) {
        const float *vk = v + gf.guard + (int64_t)k * gf.plane;
        const float *zk = Xc + gc.guard + (int64_t)K * gc.plane;
        if (c0) cp_async8(pair(stage, 0), vk + o0);
        if (c0 && r1) cp_async8(pair(stage, 1), vk + o0 + ldx);
        if (hd) cp_async8(pair(stage, 2), vk + o0 - ldx);
        if (hu) cp_async8(pair(stage, 3), vk + o0 + 2 * ldx);
        if (ce) {
            cp_async4(field(stage, 8), vk + oe);
            if (r1) cp_async4(field(stage, 9), vk + oe + ldx);
        }
#pragma unroll
        for (int m = 0; m < NZ; ++m) {
            const float *zm = zk + (int64_t)m * xc_stride;
            if (c0) cp_async4(field(stage, 10 + 4 * m), zm + oc);
            if (hd) cp_async4(field(stage, 11 + 4 * m), zm + oc - cld);
            if (hu) cp_async4(field(stage, 12 + 4 * m), zm + oc + cld);
            if (ce) cp_async4(field(stage, 13 + 4 * m), zm + oce);
        }
        cp_async_commit();
    };
    auto comb = [&](int stage, int f) -> float {   // f: 0 own, 1 below, 2 above, 3 outer
        if (MC == 0) return *field(stage, 10 + f);
        float z = mul_rn(ym[0], *field(stage, 10 + f));
#pragma unroll
        for (int m = 1; m < NZ; ++m) z = fma_rn(ym[m], *field(stage, 10 + 4 * m + f), z);
        return z;
    };
    const int k0 = blockIdx.z * kc;
    const int k1 = min(k0 + kc, gf.nt + 1);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    // coarse block of fine step k: 0 for k = 0, (k-1)/nu + 1 otherwise; tracked for the step
    // being issued, two ahead of the step being computed
    int K = (kstart == 0) ? 0 : (kstart - 1) / nu + 1;
    int ph = (kstart == 0) ? nu - 1 : (kstart - 1) % nu;
    auto advance = [&]() {
        if (ph == nu - 1) {
            ++K;
            ph = 0;
        } else {
            ++ph;
        }
    };
    issue(kstart, K, 0);
    if (kstart + 1 < k1) {
        advance();
        issue(kstart + 1, K, 1);
    } else {
        cp_async_commit();
    }
    float p00 = 0.f, p01 = 0.f, p10 = 0.f, p11 = 0.f;   // x_{k-1}
    float L00 = 0.f, L01 = 0.f, L10 = 0.f, L11 = 0.f;   // L x_{k-1}
    int st = 0;   // stage of step k
    for (int k = kstart; k < k1; ++k) {
        if (k + 2 < k1) {
            advance();
            issue(k + 2, K, (st + 2) % I2C_STAGES);
        } else {
            cp_async_commit();
        }
        cp_async_wait<2>();   // this thread's copies of step k have landed
        const float2 A0 = *pair(st, 0), A1 = *pair(st, 1), QD = *pair(st, 2), QU = *pair(st, 3);
        const float ve0 = *field(st, 8), ve1 = *field(st, 9);
        const float zo = comb(st, 0), zd = comb(st, 1), zu = comb(st, 2), ze = comb(st, 3);
        const float x00 = c0 ? fma_rn(sig, A0.x, -zo) : 0.f;
        const float x01 = c1 ? fma_rn(sig, A0.y, -zo) : 0.f;
        const float x10 = (c0 && r1) ? fma_rn(sig, A1.x, -zo) : 0.f;
        const float x11 = (c1 && r1) ? fma_rn(sig, A1.y, -zo) : 0.f;
        const float d0 = hd ? fma_rn(sig, QD.x, -zd) : 0.f, d1 = (hd && c1) ? fma_rn(sig, QD.y, -zd) : 0.f;
        const float e0 = hu ? fma_rn(sig, QU.x, -zu) : 0.f, e1 = (hu && c1) ? fma_rn(sig, QU.y, -zu) : 0.f;
        float l0 = __shfl_up_sync(FULL, x01, 1), l1 = __shfl_up_sync(FULL, x11, 1);
        float q0 = __shfl_down_sync(FULL, x00, 1), q1 = __shfl_down_sync(FULL, x10, 1);
        const float xe0 = ce ? fma_rn(sig, ve0, -ze) : 0.f;
        const float xe1 = (ce && r1) ? fma_rn(sig, ve1, -ze) : 0.f;
        if (lane == 0) {
            l0 = xe0;
            l1 = xe1;
        }
        if (lane == 31) {
            q0 = xe0;
            q1 = xe1;
        }
        const float s00 = (xd0 * x00 + xl0 * l0 + xu0 * x01) + (yd0 * x00 + yl0 * d0 + yu0 * x10);
        const float s01 = (xd1 * x01 + xl1 * x00 + xu1 * q0) + (yd0 * x01 + yl0 * d1 + yu0 * x11);
        const float s10 = (xd0 * x10 + xl0 * l1 + xu0 * x11) + (yd1 * x10 + yl1 * x00 + yu1 * e0);
        const float s11 = (xd1 * x11 + xl1 * x10 + xu1 * q1) + (yd1 * x11 + yl1 * x01 + yu1 * e1);
        if (k >= k0 && c0) {
            auto wk = [&](float c, float Lc, float p, float Lp) -> float {
                return k == 0 ? c : (c - a * Lc) - (p + b * Lp);
            };
            const int64_t f0 = gf.guard + (int64_t)k * gf.plane + o0;
            st_pair_t<float>(x + f0, x00, x01);
            st_pair_t<float>(w + f0, wk(x00, s00, p00, L00), c1 ? wk(x01, s01, p01, L01) : 0.f);
            if (r1) {
                st_pair_t<float>(x + f0 + ldx, x10, x11);
                st_pair_t<float>(w + f0 + ldx, wk(x10, s10, p10, L10), c1 ? wk(x11, s11, p11, L11) : 0.f);
            }
        }
        p00 = x00; p01 = x01; p10 = x10; p11 = x11;
        L00 = s00; L01 = s01; L10 = s10; L11 = s11;
        st = (st + 1) % I2C_STAGES;
    }
    cp_async_wait<0>();   // no copy outlives the kernel
}

cudaError_t interp2d_set_attributes() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f, int mc) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)i2c_smem_bytes(mc));
        if (r != cudaSuccess) e = r;
    };
    set((const void *)k_interp_2d_cp<0>, 0);
    set((const void *)k_interp_2d_cp<1>, 1);
    set((const void *)k_interp_2d_cp<2>, 2);
    set((const void *)k_interp_2d_cp<3>, 3);
    set((const void *)k_interp_2d_cp<4>, 4);
    return e;
}

template <typename Tv, typename Tz, typename Tx, typename Tw, typename Tc>
void launch_interp(const Geom &gf, const Geom &gc, int nu, bool space, const Weights &w,
                   SpaceOp<Tc> L, const Tv *v, const double *sigma, const Tz *Xc, int mc,
                   int64_t xc_stride, const double *yc, Tx *x, Tw *wout, const int *done,
                   cudaStream_t s) {
    int kc = cap_kc(choose_kc(gf.npts(), gf.nt + 1), gf.nt + 1, gf.dim, gf.nx, gf.ny);
    int nch = (gf.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(gf.dim, gf.nx, gf.ny, nch);
    Tc a = (Tc)w.a, b = (Tc)w.b;
#define MK_INTERP(D, S)                                                                        \
    k_interp<D, S, Tv, Tz, Tx, Tw, Tc><<<l.grid, l.block, 0, s>>>(gf, gc, nu, a, b, L, v, sigma, \
                                                                  Xc, mc, xc_stride, yc, x, wout, \
                                                                  kc, done)
#define MK_INTERP1M(S, M)                                                                     \
    k_interp_1d<S, M, Tv, Tz, Tx, Tw, Tc><<<l.grid, l.block, 0, s>>>(gf, gc, nu, a, b, L, v,     \
                                                                     sigma, Xc, mc, xc_stride, yc, \
                                                                     x, wout, kc, done)
#define MK_INTERP1(S)                                                                         \
    do {                                                                                      \
        if (!yc) MK_INTERP1M(S, 0);                                                           \
        else if (mc == 1) MK_INTERP1M(S, 1);                                                  \
        else if (mc == 2) MK_INTERP1M(S, 2);                                                  \
        else MK_INTERP1M(S, -1);                                                              \
    } while (0)
    prof_begin(s);
    if (launch_interp_1d_tiled<Tv, Tz, Tx, Tw, Tc>(gf, gc, nu, space, w, L, v, sigma, Xc, mc,
                                                   xc_stride, yc, x, wout, done, s)) {
        // 1D, nu = 2: time-tiled kernel (transfer1d.cu)
    } else if (gf.dim == 1) {
        if (space) MK_INTERP1(true); else MK_INTERP1(false);
    } else if (std::is_same<Tc, float>::value && std::is_same<Tv, Tc>::value &&
               std::is_same<Tz, Tc>::value && std::is_same<Tx, Tc>::value &&
               std::is_same<Tw, Tc>::value && space && (!yc || (mc >= 1 && mc <= 4))) {
        // 2 x 2 aggregates in FP32 (the FP64 instances would spill registers):
        // aggregate-per-thread kernel walked in time;
        // chunks for one full wave of 2048 threads per SM, at least eight fine steps each
        // (the step before a chunk is formed again), at most 65535 chunks
        if constexpr (std::is_same<Tc, float>::value && std::is_same<Tv, Tc>::value &&
                      std::is_same<Tz, Tc>::value && std::is_same<Tx, Tc>::value &&
                      std::is_same<Tw, Tc>::value) {
            const int ncx = (gf.nx + 1) / 2, ncy = (gf.ny + 1) / 2;
            const int nsteps = gf.nt + 1;
            const int64_t want = (int64_t)g_num_sms * 2048;
            int64_t kt = ((int64_t)ncx * ncy * nsteps) / (want > 0 ? want : 1);
            if (kt < 8) kt = 8;
            if (kt > nsteps) kt = nsteps;
            while ((nsteps + kt - 1) / kt > 65535) ++kt;
            const int kct = (int)kt;
            const dim3 grid((ncx + 31) / 32, (ncy + 7) / 8, (nsteps + kct - 1) / kct), blk(32, 8, 1);
#define MK_I2T(M)                                                                                \
    k_interp_2d_cp<M><<<grid, blk, i2c_smem_bytes(M), s>>>(gf, gc, nu, a, b, L, v, sigma, Xc,       \
                                                           xc_stride, yc, x, wout, kct, done)
            if (!yc) MK_I2T(0);
            else if (mc == 1) MK_I2T(1);
            else if (mc == 2) MK_I2T(2);
            else if (mc == 3) MK_I2T(3);
            else MK_I2T(4);
#undef MK_I2T
        }
    } else {
        // 2D: x once per point, then w = A x from the stored x (the fused form evaluated x
        // again at each of the four stencil neighbours of every point)
        const dim3 g2 = grid_2d_points(gf), g4 = grid_2d_points4(gf), b2(32, 8, 1);
        if (space)
            k_interp_x2d<true, Tv, Tz, Tx><<<g4, b2, 0, s>>>(gf, gc, nu, v, sigma, Xc, mc, xc_stride,
                                                            yc, x, done);
        else
            k_interp_x2d<false, Tv, Tz, Tx><<<g4, b2, 0, s>>>(gf, gc, nu, v, sigma, Xc, mc,
                                                             xc_stride, yc, x, done);
        k_apply_2d<Tx, Tw, Tc><<<g2, b2, 0, s>>>(gf, a, b, L, x, wout, done);
        count_launch();
    }
#undef MK_INTERP
#undef MK_INTERP1
#undef MK_INTERP1M
    prof_end(s, PROF_INTERP, (double)gf.interior() * (sizeof(Tv) + sizeof(Tx) + sizeof(Tw)) +
                                 (double)mc * gc.interior() * sizeof(Tz));
    count_launch();
}

// ---------------------------------------------------------------------------------------
// Adjoint of Eq. (finesys).  A_h^T is block upper bidiagonal (psi, phi symmetric), so
// with y_j = lam_{nt+1-j} the system A_h^T lam = b becomes the forward system with
// right-hand side f_rev[0] = 0, f_rev[j] = b[nt+1-j] (then y_0 = 0).
// ---------------------------------------------------------------------------------------
__global__ void k_reverse_pack(Geom g, const double *__restrict__ b, double *__restrict__ f) {
    int64_t npts = g.npts();
    int64_t n = (int64_t)(g.nt + 1) * npts;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = e / npts;
        int64_t r = e - k * npts;
        int j = (int)(r / g.nx), i = (int)(r - (int64_t)j * g.nx);
        f[g.at((int)k, j, i)] = (k == 0) ? 0.0 : b[(g.nt + 1 - k) * npts + r];
    }
}

void launch_reverse_pack(const Geom &g, const double *dense, double *padded, cudaStream_t s) {
    k_reverse_pack<<<grid_for(g.interior(), 256), 256, 0, s>>>(g, dense, padded);
    count_launch();
}

// lam_k = y_{nt+1-k} (k >= 1), lam_{nt+1} = 0, lam_0 = b_0 + phi lam_1;
// dJ/dg_k = dt (theta lam_k + (1-theta) lam_{k+1}) (k >= 1), dJ/dg_0 = dt (1-theta) lam_1;
// dJ/dtau = (dt/tau) sum_{k>=1} lam_k^T L (theta u_k + (1-theta) u_{k-1}).
template <int DIM>
__global__ void __launch_bounds__(256) k_adjoint_grads(Geom g, double theta, double dt, double tau,
                                                       double bw, SpaceOp<double> L,
                                                       const double *__restrict__ y,
                                                       const double *__restrict__ b,
                                                       const double *__restrict__ upad,
                                                       double *__restrict__ lam,
                                                       double *__restrict__ gu0,
                                                       double *__restrict__ gg, int kc,
                                                       ReduceScratch rs, KState ks) {
    int i, j, chunk;
    point_index<DIM>(i, j, chunk);
    double acc = 0.0;
    if (i < g.nx && j < g.ny) {
        const int64_t npts = g.npts();
        const int64_t r = (int64_t)j * g.nx + i;
        int k0 = chunk * kc;
        int k1 = min(k0 + kc, g.nt + 1);
        double Luprev = 0.0;
        if (upad && k0 > 0) Luprev = lap_at<DIM, double>(upad, g.at(k0 - 1, j, i), i, j, g, L.x, L.y);
        for (int k = k0; k < k1; ++k) {
            double lk;
            if (k == 0) {
                int64_t i1 = g.at(g.nt, j, i);   // lam_1 = y_nt
                double l1 = y[i1];
                double Ll1 = lap_at<DIM, double>(y, i1, i, j, g, L.x, L.y);
                lk = b[r] + (l1 + bw * Ll1);
                if (gu0) gu0[r] = lk;
            } else {
                lk = y[g.at(g.nt + 1 - k, j, i)];
            }
            double lnext = (k + 1 <= g.nt) ? y[g.at(g.nt - k, j, i)] : 0.0;
            if (lam) lam[(int64_t)k * npts + r] = lk;
            if (gg) gg[(int64_t)k * npts + r] = (k == 0) ? dt * (1.0 - theta) * lnext
                                                         : dt * (theta * lk + (1.0 - theta) * lnext);
            if (upad) {
                double Lu = lap_at<DIM, double>(upad, g.at(k, j, i), i, j, g, L.x, L.y);
                if (k >= 1) acc += lk * (theta * Lu + (1.0 - theta) * Luprev);
                Luprev = Lu;
            }
        }
    }
    acc *= dt / tau;
    block_partial_and_finish(acc, rs, 0, ks, EPI_NONE);
}

void launch_adjoint_grads(const Geom &g, double theta, double dt, double tau, SpaceOp<double> L,
                          const double *y, const double *b, const double *upad, double *lam,
                          double *grad_u0, double *grad_g, const ReduceScratch &rs, KState ks,
                          cudaStream_t s) {
    int kc = cap_kc(choose_kc(g.npts(), g.nt + 1), g.nt + 1, g.dim, g.nx, g.ny);
    int nch = (g.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(g.dim, g.nx, g.ny, nch);
    double bw = (1.0 - theta) * dt;
    if (g.dim == 1)
        k_adjoint_grads<1><<<l.grid, l.block, 0, s>>>(g, theta, dt, tau, bw, L, y, b, upad, lam,
                                                      grad_u0, grad_g, kc, rs, ks);
    else
        k_adjoint_grads<2><<<l.grid, l.block, 0, s>>>(g, theta, dt, tau, bw, L, y, b, upad, lam,
                                                      grad_u0, grad_g, kc, rs, ks);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------------------
template void launch_pack<double, double>(const Geom &, const double *, double *, cudaStream_t);
template void launch_pack<double, float>(const Geom &, const double *, float *, cudaStream_t);
template void launch_unpack<double, double>(const Geom &, const double *, double *, cudaStream_t);
template void launch_unpack<float, double>(const Geom &, const float *, double *, cudaStream_t);
template void launch_pack<double, float2>(const Geom &, const double *, float2 *, cudaStream_t);
template void launch_unpack<float2, double>(const Geom &, const float2 *, double *, cudaStream_t);
template void launch_convert<double, float>(int64_t, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(int64_t, const float *, double *, cudaStream_t);

template void launch_apply<double, double, double>(const Geom &, const Weights &, SpaceOp<double>,
                                                   const double *, double *, cudaStream_t);
template void launch_apply<float, float, float>(const Geom &, const Weights &, SpaceOp<float>,
                                                const float *, float *, cudaStream_t);
template void launch_apply<float, double, double>(const Geom &, const Weights &, SpaceOp<double>,
                                                  const float *, double *, cudaStream_t);

template void launch_restrict<double, double, double>(const Geom &, const Geom &, int, bool,
                                                      const Weights &, SpaceOp<double>,
                                                      const double *, const double *, double *,
                                                      const ReduceScratch &, int, KState,
                                                      const int *, cudaStream_t);
template void launch_restrict<double, float, float>(const Geom &, const Geom &, int, bool,
                                                    const Weights &, SpaceOp<float>,
                                                    const double *, const double *, float *,
                                                    const ReduceScratch &, int, KState,
                                                    const int *, cudaStream_t);
// mixed, level 1 with the basis in double-float pairs
template void launch_restrict<float2, float, float>(const Geom &, const Geom &, int, bool,
                                                    const Weights &, SpaceOp<float>,
                                                    const float2 *, const double *, float *,
                                                    const ReduceScratch &, int, KState,
                                                    const int *, cudaStream_t);
template void launch_restrict<float, float, float>(const Geom &, const Geom &, int, bool,
                                                   const Weights &, SpaceOp<float>, const float *,
                                                   const double *, float *, const ReduceScratch &,
                                                   int, KState, const int *, cudaStream_t);

// FP64 throughout
template void launch_interp<double, double, double, double, double>(
    const Geom &, const Geom &, int, bool, const Weights &, SpaceOp<double>, const double *,
    const double *, const double *, int, int64_t, const double *, double *, double *,
    const int *, cudaStream_t);
// mixed, level 1: FP64 basis, FP32 coarse and x, FP64 w
template void launch_interp<double, float, float, double, double>(
    const Geom &, const Geom &, int, bool, const Weights &, SpaceOp<double>, const double *,
    const double *, const float *, int, int64_t, const double *, float *, double *,
    const int *, cudaStream_t);
// mixed, inner levels: FP32 throughout
template void launch_interp<float, float, float, float, float>(
    const Geom &, const Geom &, int, bool, const Weights &, SpaceOp<float>, const float *,
    const double *, const float *, int, int64_t, const double *, float *, float *, const int *,
    cudaStream_t);

}  // namespace mk
