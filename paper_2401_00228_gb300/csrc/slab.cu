// Coarsest-level solves and the sequential theta-march.
//
// The coarsest level is the perturbed, decoupled matrix of Sec. 3.3.2, Eq. (Qhtilde):
// block 0 is solved alone (x_0 = r_0) and the n_t steps split into n_cgs contiguous slabs
// whose first step drops its coupling to the previous step.  Each slab is an independent
// sequence of steps
//     (I - a L) x_k = r_k + (I + b L) x_{k-1},
// run by one CTA with the spatial vector kept in shared memory between steps.
//
// 1D: M = I - aL is a constant tridiagonal matrix, so parallel cyclic reduction (PCR)
//     needs only the right-hand side at run time: level l (stride s = 2^l) does
//       d_i <- d_i + alpha_i^l d_{i-s} + gamma_i^l d_{i+s},
//     and after ceil(log2 n) levels x_i = d_i / b_i.  The alpha/gamma/1/b tables are
//     computed once on the host in FP64.
// 2D: fast diagonalisation.  L = Lx (+) Ly with Lx = Sx Lx_diag Sx^{-1} (the tridiagonal
//     operators are similar to symmetric ones, so S is real), hence for a ny x nx array R
//       X = Sy [ (Sy^{-1} R Sx^{-T}) ./ (1 - a(lam_y_j + lam_x_i)) ] Sx^T.
//
// n_cgs = 0 keeps every coupling (one slab of all steps): the exact coarse solve and,
// on the fine level, the sequential theta-march of Eq. (timemarch).
#include "kernels.h"

namespace mk {

// ---------------------------------------------------------------------------------------
// 1D PCR slab kernel.  NT threads; each owns unknowns i = tid + u*NT (u < U).
// shared: buf0[npad], buf1[npad], xprev[npad + 2]
// ---------------------------------------------------------------------------------------
template <typename T, int U>
__global__ void __launch_bounds__(1024) k_slab_1d(Geom g, T b, SpaceOp<T> L,
                                                  const T *__restrict__ alpha,
                                                  const T *__restrict__ gamma,
                                                  const T *__restrict__ binv, int npad, int nlev,
                                                  int steps, int coupled,
                                                  const T *__restrict__ r, T *__restrict__ x,
                                                  const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ unsigned char smem_raw[];
    T *buf0 = reinterpret_cast<T *>(smem_raw);
    T *buf1 = buf0 + npad;
    T *xp = buf1 + npad;   // xp[i+1] = x_{k-1}[i]; xp[0] = xp[n+1..] = 0
    const int NT = blockDim.x;
    const int n = g.nx;
    const int tid = threadIdx.x;
    const int slab = blockIdx.x;
    const int kbeg = 1 + slab * steps;
    const T *lo = L.x, *di = L.x + n, *up = L.x + 2 * n;

    for (int i = tid; i < npad + 2; i += NT) xp[i] = (T)0;
    if (slab == 0)
        for (int i = tid; i < n; i += NT) x[g.at(0, 0, i)] = r[g.at(0, 0, i)];
    __syncthreads();
    if (coupled) {
        // the first step couples to block 0 (exact solve / march)
        for (int i = tid; i < n; i += NT) xp[i + 1] = r[g.at(0, 0, i)];
        __syncthreads();
    }
    // prefetch the first right-hand side
    T rnext[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        int i = tid + u * NT;
        rnext[u] = (i < n) ? r[g.at(kbeg, 0, i)] : (T)0;
    }
    for (int s = 0; s < steps; ++s) {
        const int k = kbeg + s;
        T rcur[U];
#pragma unroll
        for (int u = 0; u < U; ++u) rcur[u] = rnext[u];
        if (s + 1 < steps) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = tid + u * NT;
                rnext[u] = (i < n) ? r[g.at(k + 1, 0, i)] : (T)0;
            }
        }
        const bool first = (s == 0) && !coupled;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int i = tid + u * NT;
            T d = (T)0;
            if (i < n) {
                d = rcur[u];
                if (!first) {
                    T c = xp[i + 1];
                    T lx = di[i] * c + lo[i] * xp[i] + up[i] * xp[i + 2];
                    d = d + (c + b * lx);
                }
            }
            buf0[i] = d;
        }
        __syncthreads();
        T *src = buf0, *dst = buf1;
        for (int l = 0; l < nlev; ++l) {
            const int st = 1 << l;
            const T *al = alpha + (int64_t)l * npad;
            const T *ga = gamma + (int64_t)l * npad;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = tid + u * NT;
                T left = (i - st >= 0) ? src[i - st] : (T)0;
                T right = (i + st < npad) ? src[i + st] : (T)0;
                dst[i] = src[i] + al[i] * left + ga[i] * right;
            }
            __syncthreads();
            T *t = src;
            src = dst;
            dst = t;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int i = tid + u * NT;
            if (i < n) {
                T xi = src[i] * binv[i];
                x[g.at(k, 0, i)] = xi;
                xp[i + 1] = xi;
            }
        }
        __syncthreads();
    }
}

template <typename T>
static void slab_1d_launch(const Geom &g, double b, SpaceOp<T> L, const T *alpha, const T *gamma,
                           const T *binv, int npad, int nlev, int nslabs, int steps, int coupled,
                           const T *r, T *x, const int *done, cudaStream_t s) {
    int nt_threads = npad < 1024 ? npad : 1024;
    if (nt_threads < 32) nt_threads = 32;
    int U = (npad + nt_threads - 1) / nt_threads;
    size_t shm = sizeof(T) * (size_t)(3 * npad + 2);
    prof_begin(s);
    if (U == 1)
        k_slab_1d<T, 1><<<nslabs, nt_threads, shm, s>>>(g, (T)b, L, alpha, gamma, binv, npad, nlev,
                                                       steps, coupled, r, x, done);
    else if (U == 2)
        k_slab_1d<T, 2><<<nslabs, nt_threads, shm, s>>>(g, (T)b, L, alpha, gamma, binv, npad, nlev,
                                                       steps, coupled, r, x, done);
    else
        k_slab_1d<T, 4><<<nslabs, nt_threads, shm, s>>>(g, (T)b, L, alpha, gamma, binv, npad, nlev,
                                                       steps, coupled, r, x, done);
    prof_end(s, done ? PROF_SLAB : PROF_MARCH, 2.0 * sizeof(T) * (double)g.interior());
    count_launch();
}

// ---------------------------------------------------------------------------------------
// 1D, one warp per slab: partitioned (spike) solver for the constant tridiagonal I - aL.
// Lane p owns rows pU .. pU+U-1 (the system padded to 32U rows with identity rows):
//   1. right-hand side r_k + (I + bL) x_{k-1} from the lane's own x_{k-1} values and one
//      neighbour from each adjacent lane;
//   2. Thomas on the lane's U x U block (precomputed multipliers and pivots): y = M_p^{-1} d;
//   3. the interface unknowns (F_p, G_p) = (x[pU], x[pU+U-1]) satisfy a block-tridiagonal
//      system with 2x2 blocks, solved by block parallel cyclic reduction over the 32 lanes
//      in five shuffle steps (strides 1..16, precomputed multipliers);
//   4. x = y - A_p G_{p-1} v_p - C_p F_{p+1} w_p with the precomputed spikes v_p, w_p.
// No block barrier is needed.  Rows are read and written coalesced through a padded shared
// staging buffer, and the next right-hand side is prefetched during the current step.
// Tables: spike_tables() in setup.cpp (item-major, 32 lanes per item).
// ---------------------------------------------------------------------------------------
template <typename T, int U>
__global__ void __launch_bounds__(32) k_slab_1d_warp(Geom g, T b, const T *__restrict__ tab,
                                                     int steps, int coupled,
                                                     const T *__restrict__ r,
                                                     T *__restrict__ x,
                                                     const int *__restrict__ done) {
    if (done && *done) return;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int ITEMS = 8 * U + 46;
    extern __shared__ unsigned char smem_raw[];
    T *tb = reinterpret_cast<T *>(smem_raw);   // ITEMS x 32
    T *buf = tb + ITEMS * 32;                  // 32U values, one pad slot per 32
    const int lane = threadIdx.x;
    const int n = g.nx;
    const int slab = blockIdx.x;
    const int kbeg = 1 + slab * steps;
    for (int e = lane; e < ITEMS * 32; e += 32) tb[e] = tab[e];
    auto TB = [&](int item) -> T { return tb[item * 32 + lane]; };
    auto sidx = [](int e) { return e + (e >> 5); };
    T pre[U];
    auto load_row = [&](int k) {
        const T *row = r + g.guard + (int64_t)k * g.plane;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = q * 32 + lane;
            pre[q] = (e < n) ? row[e] : (T)0;
        }
    };
    auto stage = [&]() {
        __syncwarp();
#pragma unroll
        for (int q = 0; q < U; ++q) buf[sidx(q * 32 + lane)] = pre[q];
        __syncwarp();
    };
    T xp[U];
#pragma unroll
    for (int q = 0; q < U; ++q) xp[q] = (T)0;
    if (slab == 0 || coupled) {
        load_row(0);
        if (slab == 0) {
            T *row0 = x + g.guard;
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = q * 32 + lane;
                if (e < n) row0[e] = pre[q];
            }
        }
        if (coupled) {
            stage();
#pragma unroll
            for (int q = 0; q < U; ++q) xp[q] = buf[sidx(lane * U + q)];
        }
    }
    load_row(kbeg);
    for (int s = 0; s < steps; ++s) {
        const int k = kbeg + s;
        stage();
        if (s + 1 < steps) load_row(k + 1);
        const bool first = (s == 0) && !coupled;
        T xl = __shfl_up_sync(FULL, xp[U - 1], 1);
        T xr = __shfl_down_sync(FULL, xp[0], 1);
        if (lane == 0) xl = (T)0;
        if (lane == 31) xr = (T)0;
        T d[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            T rv = buf[sidx(lane * U + q)];
            if (!first) {
                const T left = q ? xp[q - 1] : xl;
                const T right = (q < U - 1) ? xp[q + 1] : xr;
                const T lx = TB(6 * U + q) * xp[q] + TB(5 * U + q) * left + TB(7 * U + q) * right;
                rv = rv + (xp[q] + b * lx);
            }
            d[q] = rv;
        }
        // Thomas on the lane's block
#pragma unroll
        for (int q = 1; q < U; ++q) d[q] -= TB(q) * d[q - 1];
        d[U - 1] *= TB(U + U - 1);
#pragma unroll
        for (int q = U - 2; q >= 0; --q) d[q] = (d[q] - TB(2 * U + q) * d[q + 1]) * TB(U + q);
        // interface unknowns: block PCR across the lanes
        T rF = d[0], rG = d[U - 1];
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int st = 1 << l;
            T lF = __shfl_up_sync(FULL, rF, st), lG = __shfl_up_sync(FULL, rG, st);
            T hF = __shfl_down_sync(FULL, rF, st), hG = __shfl_down_sync(FULL, rG, st);
            if (lane < st) {
                lF = (T)0;
                lG = (T)0;
            }
            if (lane + st >= 32) {
                hF = (T)0;
                hG = (T)0;
            }
            const int ia = 8 * U + 2 + 4 * l, ig = 8 * U + 22 + 4 * l;
            T nF = rF + TB(ia) * lF + TB(ia + 1) * lG + TB(ig) * hF + TB(ig + 1) * hG;
            T nG = rG + TB(ia + 2) * lF + TB(ia + 3) * lG + TB(ig + 2) * hF + TB(ig + 3) * hG;
            rF = nF;
            rG = nG;
        }
        const int idv = 8 * U + 42;
        const T F = TB(idv) * rF + TB(idv + 1) * rG;
        const T G = TB(idv + 2) * rF + TB(idv + 3) * rG;
        T Gm = __shfl_up_sync(FULL, G, 1), Fp = __shfl_down_sync(FULL, F, 1);
        if (lane == 0) Gm = (T)0;
        if (lane == 31) Fp = (T)0;
        const T cA = TB(8 * U) * Gm, cC = TB(8 * U + 1) * Fp;
#pragma unroll
        for (int q = 0; q < U; ++q) xp[q] = d[q] - cA * TB(3 * U + q) - cC * TB(4 * U + q);
        // write x_k coalesced
        __syncwarp();
#pragma unroll
        for (int q = 0; q < U; ++q) buf[sidx(lane * U + q)] = xp[q];
        __syncwarp();
        T *xrow = x + g.guard + (int64_t)k * g.plane;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = q * 32 + lane;
            if (e < n) xrow[e] = buf[sidx(e)];
        }
    }
}

int spike_block_size(int n) {
    int U = 1;
    while (32 * U < n) U *= 2;
    return U;
}

template <typename T>
size_t slab_warp_smem(int U) {
    return sizeof(T) * ((size_t)(8 * U + 46) * 32 + 32 * U + U);
}

template <typename T>
bool slab_warp_supported(int n) {
    const int U = spike_block_size(n);
    return sizeof(T) == 4 ? U <= 64 : U <= 32;
}

template <typename T>
void launch_slab_1d_warp(const Geom &g, double b, const T *tab, int U, int n_cgs, const T *r, T *x,
                         const int *done, cudaStream_t s, int cls) {
    const int nslabs = n_cgs <= 0 ? 1 : n_cgs;
    const int steps = n_cgs <= 0 ? g.nt : g.nt / n_cgs;
    const int coupled = n_cgs <= 0 ? 1 : 0;
    const size_t shm = slab_warp_smem<T>(U);
    prof_begin(s);
#define MK_SW(UU)                                                                              \
    case UU:                                                                                   \
        k_slab_1d_warp<T, UU><<<nslabs, 32, shm, s>>>(g, (T)b, tab, steps, coupled, r, x, done); \
        break
    switch (U) {
        MK_SW(1);
        MK_SW(2);
        MK_SW(4);
        MK_SW(8);
        MK_SW(16);
        MK_SW(32);
        default:
            if constexpr (sizeof(T) == 4)
                k_slab_1d_warp<T, 64><<<nslabs, 32, shm, s>>>(g, (T)b, tab, steps, coupled, r, x, done);
            break;
    }
#undef MK_SW
    prof_end(s, cls, 2.0 * sizeof(T) * (double)g.interior());
    count_launch();
}

template <typename T>
void launch_slab_1d(const Geom &g, double b, SpaceOp<T> L, const T *alpha, const T *gamma,
                    const T *binv, int npad, int nlev, int n_cgs, const T *r, T *x,
                    const int *done, cudaStream_t s) {
    if (n_cgs <= 0)
        slab_1d_launch<T>(g, b, L, alpha, gamma, binv, npad, nlev, 1, g.nt, 1, r, x, done, s);
    else
        slab_1d_launch<T>(g, b, L, alpha, gamma, binv, npad, nlev, n_cgs, g.nt / n_cgs, 0, r, x,
                          done, s);
}

void launch_march_1d(const Geom &g, double b, SpaceOp<double> L, const double *alpha,
                     const double *gamma, const double *binv, int npad, int nlev,
                     const double *f, double *u, cudaStream_t s) {
    slab_1d_launch<double>(g, b, L, alpha, gamma, binv, npad, nlev, 1, g.nt, 1, f, u, nullptr, s);
}

// ---------------------------------------------------------------------------------------
// 2D fast-diagonalisation slab kernel (nx, ny <= 64).
// shared: Sx, Sxi (nx*nx), Sy, Syi (ny*ny), lamx (nx), lamy (ny), A, B (ny*nx),
//         xp ((ny+2)*(nx+2)) previous step with a zero frame.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) k_slab_2d(Geom g, T a, T b, SpaceOp<T> L,
                                                  const T *__restrict__ Sx_g,
                                                  const T *__restrict__ Sxi_g,
                                                  const T *__restrict__ lamx_g,
                                                  const T *__restrict__ Sy_g,
                                                  const T *__restrict__ Syi_g,
                                                  const T *__restrict__ lamy_g, int steps,
                                                  int coupled, const T *__restrict__ r,
                                                  T *__restrict__ x,
                                                  const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.nx, ny = g.ny;
    const int nxy = nx * ny;
    T *Sx = reinterpret_cast<T *>(smem_raw);
    T *Sxi = Sx + nx * nx;
    T *Sy = Sxi + nx * nx;
    T *Syi = Sy + ny * ny;
    T *lamx = Syi + ny * ny;
    T *lamy = lamx + nx;
    T *A = lamy + ny;
    T *B = A + nxy;
    T *xp = B + nxy;
    const int fx = nx + 2;   // frame row length
    const int NT = blockDim.x, tid = threadIdx.x;
    const int slab = blockIdx.x;
    const int kbeg = 1 + slab * steps;
    const T *xlo = L.x, *xdi = L.x + nx, *xup = L.x + 2 * nx;
    const T *ylo = L.y, *ydi = L.y + ny, *yup = L.y + 2 * ny;

    for (int e = tid; e < nx * nx; e += NT) {
        Sx[e] = Sx_g[e];
        Sxi[e] = Sxi_g[e];
    }
    for (int e = tid; e < ny * ny; e += NT) {
        Sy[e] = Sy_g[e];
        Syi[e] = Syi_g[e];
    }
    for (int e = tid; e < nx; e += NT) lamx[e] = lamx_g[e];
    for (int e = tid; e < ny; e += NT) lamy[e] = lamy_g[e];
    for (int e = tid; e < (ny + 2) * fx; e += NT) xp[e] = (T)0;
    if (slab == 0)
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            x[g.at(0, j, i)] = r[g.at(0, j, i)];
        }
    __syncthreads();
    if (coupled) {
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            xp[(j + 1) * fx + i + 1] = r[g.at(0, j, i)];
        }
        __syncthreads();
    }
    for (int s = 0; s < steps; ++s) {
        const int k = kbeg + s;
        const bool first = (s == 0) && !coupled;
        // rhs -> A
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            T d = r[g.at(k, j, i)];
            if (!first) {
                const T *c = xp + (j + 1) * fx + (i + 1);
                T lx = xdi[i] * c[0] + xlo[i] * c[-1] + xup[i] * c[1];
                T ly = ydi[j] * c[0] + ylo[j] * c[-fx] + yup[j] * c[fx];
                d = d + (c[0] + b * (lx + ly));
            }
            A[e] = d;
        }
        __syncthreads();
        // B = Syi A   (y transform)
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            T acc = 0;
            for (int q = 0; q < ny; ++q) acc += Syi[j * ny + q] * A[q * nx + i];
            B[e] = acc;
        }
        __syncthreads();
        // A = (B Sxi^T) ./ (1 - a(lamy + lamx))
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            T acc = 0;
            for (int q = 0; q < nx; ++q) acc += B[j * nx + q] * Sxi[i * nx + q];
            A[e] = acc / ((T)1 - a * (lamy[j] + lamx[i]));
        }
        __syncthreads();
        // B = Sy A
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            T acc = 0;
            for (int q = 0; q < ny; ++q) acc += Sy[j * ny + q] * A[q * nx + i];
            B[e] = acc;
        }
        __syncthreads();
        // x = B Sx^T
        for (int e = tid; e < nxy; e += NT) {
            int j = e / nx, i = e - j * nx;
            T acc = 0;
            for (int q = 0; q < nx; ++q) acc += B[j * nx + q] * Sx[i * nx + q];
            x[g.at(k, j, i)] = acc;
            xp[(j + 1) * fx + i + 1] = acc;
        }
        __syncthreads();
    }
}

template <typename T>
static size_t slab_2d_smem(int nx, int ny) {
    return sizeof(T) * ((size_t)2 * nx * nx + 2 * ny * ny + nx + ny + 2 * nx * ny +
                        (size_t)(ny + 2) * (nx + 2));
}

template <typename T>
static void slab_2d_launch(const Geom &g, double a, double b, SpaceOp<T> L, const T *Sx,
                           const T *Sxi, const T *lamx, const T *Sy, const T *Syi, const T *lamy,
                           int nslabs, int steps, int coupled, const T *r, T *x, const int *done,
                           cudaStream_t s) {
    size_t shm = slab_2d_smem<T>(g.nx, g.ny);
    int threads = g.nx * g.ny;
    threads = ((threads + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    prof_begin(s);
    k_slab_2d<T><<<nslabs, threads, shm, s>>>(g, (T)a, (T)b, L, Sx, Sxi, lamx, Sy, Syi, lamy, steps,
                                              coupled, r, x, done);
    prof_end(s, done ? PROF_SLAB : PROF_MARCH, 2.0 * sizeof(T) * (double)g.interior());
    count_launch();
}

template <typename T>
void launch_slab_2d(const Geom &g, double a, double b, SpaceOp<T> L, const T *Sx, const T *Sxi,
                    const T *lamx, const T *Sy, const T *Syi, const T *lamy, int n_cgs,
                    const T *r, T *x, const int *done, cudaStream_t s) {
    if (n_cgs <= 0)
        slab_2d_launch<T>(g, a, b, L, Sx, Sxi, lamx, Sy, Syi, lamy, 1, g.nt, 1, r, x, done, s);
    else
        slab_2d_launch<T>(g, a, b, L, Sx, Sxi, lamx, Sy, Syi, lamy, n_cgs, g.nt / n_cgs, 0, r, x,
                          done, s);
}

void launch_march_2d(const Geom &g, double a, double b, SpaceOp<double> L, const double *Sx,
                     const double *Sxi, const double *lamx, const double *Sy, const double *Syi,
                     const double *lamy, const double *f, double *u, cudaStream_t s) {
    slab_2d_launch<double>(g, a, b, L, Sx, Sxi, lamx, Sy, Syi, lamy, 1, g.nt, 1, f, u, nullptr, s);
}

// Opt in to large dynamic shared memory once, before any launch or graph capture.
cudaError_t slab_set_attributes() {
    const int big = 200 * 1024;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        if (r != cudaSuccess) e = r;
    };
    set((const void *)k_slab_2d<float>);
    set((const void *)k_slab_2d<double>);
    set((const void *)k_slab_1d<float, 1>);
    set((const void *)k_slab_1d<float, 2>);
    set((const void *)k_slab_1d<float, 4>);
    set((const void *)k_slab_1d<double, 1>);
    set((const void *)k_slab_1d<double, 2>);
    set((const void *)k_slab_1d<double, 4>);
    set((const void *)k_slab_1d_warp<float, 1>);
    set((const void *)k_slab_1d_warp<float, 2>);
    set((const void *)k_slab_1d_warp<float, 4>);
    set((const void *)k_slab_1d_warp<float, 8>);
    set((const void *)k_slab_1d_warp<float, 16>);
    set((const void *)k_slab_1d_warp<float, 32>);
    set((const void *)k_slab_1d_warp<float, 64>);
    set((const void *)k_slab_1d_warp<double, 1>);
    set((const void *)k_slab_1d_warp<double, 2>);
    set((const void *)k_slab_1d_warp<double, 4>);
    set((const void *)k_slab_1d_warp<double, 8>);
    set((const void *)k_slab_1d_warp<double, 16>);
    set((const void *)k_slab_1d_warp<double, 32>);
    return e;
}

template void launch_slab_1d_warp<float>(const Geom &, double, const float *, int, int,
                                         const float *, float *, const int *, cudaStream_t, int);
template void launch_slab_1d_warp<double>(const Geom &, double, const double *, int, int,
                                          const double *, double *, const int *, cudaStream_t, int);
template bool slab_warp_supported<float>(int);
template bool slab_warp_supported<double>(int);
template void launch_slab_1d<double>(const Geom &, double, SpaceOp<double>, const double *,
                                     const double *, const double *, int, int, int,
                                     const double *, double *, const int *, cudaStream_t);
template void launch_slab_1d<float>(const Geom &, double, SpaceOp<float>, const float *,
                                    const float *, const float *, int, int, int, const float *,
                                    float *, const int *, cudaStream_t);
template void launch_slab_2d<double>(const Geom &, double, double, SpaceOp<double>,
                                     const double *, const double *, const double *,
                                     const double *, const double *, const double *, int,
                                     const double *, double *, const int *, cudaStream_t);
template void launch_slab_2d<float>(const Geom &, double, double, SpaceOp<float>, const float *,
                                    const float *, const float *, const float *, const float *,
                                    const float *, int, const float *, float *, const int *,
                                    cudaStream_t);

}  // namespace mk
