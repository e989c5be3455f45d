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
#include "scan.cuh"

namespace mk {

constexpr int SLAB_SMEM_LIMIT = 200 * 1024;   // dynamic shared memory of the slab kernels

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
// 1D partitioned (spike) slab solver for the constant tridiagonal I - aL, one CTA of
// P = 32*NW threads per slab.  Thread p owns rows pU .. pU+U-1 of the system padded to P*U
// rows (identity rows beyond n).  Per time step:
//   1. right-hand side r_k + (I + bL) x_{k-1} from the thread's own x_{k-1} values and one
//      neighbour on each side;
//   2. Thomas on the thread's U x U block (precomputed multipliers and pivots): y = M_p^{-1} d;
//   3. the interface unknowns (F_p, G_p) = (x[pU], x[pU+U-1]) satisfy a block-tridiagonal
//      system with 2x2 blocks, solved by block parallel cyclic reduction over the P threads
//      (strides 1..16 by warp shuffles, larger strides through shared memory);
//   4. x = y - A_p G_{p-1} v_p - C_p F_{p+1} w_p with the precomputed spikes v_p, w_p.
// The work per step is O(n) (Thomas) plus O(P log P) on the interfaces, against O(n log n)
// for plain PCR, and only log2(P) - 5 block barriers are on the critical path.  Rows are
// read and written coalesced through a padded shared staging buffer and the next
// right-hand side is prefetched during the current step.  Tables: spike_tables().
// ---------------------------------------------------------------------------------------
template <int NW>
struct SpikeLevels {
    static constexpr int value = NW == 1 ? 5 : NW == 2 ? 6 : NW == 4 ? 7 : 8;
};

template <typename T, int U, int NW>
__global__ void __launch_bounds__(32 * NW) k_slab_1d_spike(Geom g, T b, const T *__restrict__ tab,
                                                           int steps, int coupled,
                                                           const T *__restrict__ r,
                                                           T *__restrict__ x,
                                                           const int *__restrict__ done) {
    if (done && *done) return;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int P = 32 * NW;
    constexpr int NL = SpikeLevels<NW>::value;
    constexpr int ITEMS = 8 * U + 2 + 8 * NL + 4;
    constexpr int NBUF = P * U + (P * U) / 32;
    extern __shared__ unsigned char smem_raw[];
    T *tb = reinterpret_cast<T *>(smem_raw);   // ITEMS x P
    T *buf = tb + ITEMS * P;                   // staging, one pad slot per 32 values
    T *ifc = buf + NBUF;                       // interface exchange [2 buffers][F|G][P]
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int n = g.nx;
    const int slab = blockIdx.x;
    const int kbeg = 1 + slab * steps;
    for (int e = t; e < ITEMS * P; e += P) tb[e] = tab[e];
    auto TB = [&](int item) -> T { return tb[item * P + t]; };
    auto sidx = [](int e) { return e + (e >> 5); };
    T pre[U];
    auto load_row = [&](int k) {
        const T *row = r + g.guard + (int64_t)k * g.plane;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = q * P + t;
            pre[q] = (e < n) ? row[e] : (T)0;
        }
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
                const int e = q * P + t;
                if (e < n) row0[e] = pre[q];
            }
        }
        if (coupled) {
#pragma unroll
            for (int q = 0; q < U; ++q) buf[sidx(q * P + t)] = pre[q];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < U; ++q) xp[q] = buf[sidx(t * U + q)];
        }
    }
    __syncthreads();   // tables loaded; buf holds x_0 when coupled
    load_row(kbeg);
    int cur = 0;
    for (int s = 0; s < steps; ++s) {
        const int k = kbeg + s;
        const bool first = (s == 0) && !coupled;
        // neighbours of x_{k-1} across the thread's block boundaries (buf holds x_{k-1})
        T xl = (T)0, xr = (T)0;
        if (!first) {
            xl = (t > 0) ? buf[sidx(t * U - 1)] : (T)0;
            xr = (t < P - 1) ? buf[sidx(t * U + U)] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < U; ++q) buf[sidx(q * P + t)] = pre[q];
        __syncthreads();
        if (s + 1 < steps) load_row(k + 1);
        T d[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            T rv = buf[sidx(t * U + q)];
            if (!first) {
                const T left = q ? xp[q - 1] : xl;
                const T right = (q < U - 1) ? xp[q + 1] : xr;
                const T lx = TB(6 * U + q) * xp[q] + TB(5 * U + q) * left + TB(7 * U + q) * right;
                rv = rv + (xp[q] + b * lx);
            }
            d[q] = rv;
        }
        // Thomas on the thread's block
#pragma unroll
        for (int q = 1; q < U; ++q) d[q] -= TB(q) * d[q - 1];
        d[U - 1] *= TB(U + U - 1);
#pragma unroll
        for (int q = U - 2; q >= 0; --q) d[q] = (d[q] - TB(2 * U + q) * d[q + 1]) * TB(U + q);
        // interface unknowns: block PCR across the threads
        T rF = d[0], rG = d[U - 1];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int st = 1 << l;
            T lF, lG, hF, hG;
            if (st < 32) {
                lF = __shfl_up_sync(FULL, rF, st);
                lG = __shfl_up_sync(FULL, rG, st);
                hF = __shfl_down_sync(FULL, rF, st);
                hG = __shfl_down_sync(FULL, rG, st);
                // the shuffles stay inside a warp: partners in other warps come from
                // shared memory for the lanes at the warp edge
                if (NW > 1) {
                    T *fF = ifc + cur * 2 * P, *fG = fF + P;
                    fF[t] = rF;
                    fG[t] = rG;
                    __syncthreads();
                    if (lane < st) {
                        lF = (t - st >= 0) ? fF[t - st] : (T)0;
                        lG = (t - st >= 0) ? fG[t - st] : (T)0;
                    }
                    if (lane + st >= 32) {
                        hF = (t + st < P) ? fF[t + st] : (T)0;
                        hG = (t + st < P) ? fG[t + st] : (T)0;
                    }
                    cur ^= 1;
                } else {
                    if (lane < st) {
                        lF = (T)0;
                        lG = (T)0;
                    }
                    if (lane + st >= 32) {
                        hF = (T)0;
                        hG = (T)0;
                    }
                }
            } else {
                T *fF = ifc + cur * 2 * P, *fG = fF + P;
                fF[t] = rF;
                fG[t] = rG;
                __syncthreads();
                lF = (t - st >= 0) ? fF[t - st] : (T)0;
                lG = (t - st >= 0) ? fG[t - st] : (T)0;
                hF = (t + st < P) ? fF[t + st] : (T)0;
                hG = (t + st < P) ? fG[t + st] : (T)0;
                cur ^= 1;
            }
            const int ia = 8 * U + 2 + 4 * l, ig = 8 * U + 2 + 4 * NL + 4 * l;
            T nF = rF + TB(ia) * lF + TB(ia + 1) * lG + TB(ig) * hF + TB(ig + 1) * hG;
            T nG = rG + TB(ia + 2) * lF + TB(ia + 3) * lG + TB(ig + 2) * hF + TB(ig + 3) * hG;
            rF = nF;
            rG = nG;
        }
        const int idv = 8 * U + 2 + 8 * NL;
        const T F = TB(idv) * rF + TB(idv + 1) * rG;
        const T G = TB(idv + 2) * rF + TB(idv + 3) * rG;
        // neighbours' interface values
        T *fF = ifc + cur * 2 * P, *fG = fF + P;
        fF[t] = F;
        fG[t] = G;
        cur ^= 1;
        __syncthreads();
        const T Gm = (t > 0) ? fG[t - 1] : (T)0;
        const T Fp = (t < P - 1) ? fF[t + 1] : (T)0;
        const T cA = TB(8 * U) * Gm, cC = TB(8 * U + 1) * Fp;
#pragma unroll
        for (int q = 0; q < U; ++q) xp[q] = d[q] - cA * TB(3 * U + q) - cC * TB(4 * U + q);
        // write x_k coalesced (buf then keeps x_k for the next step's neighbours)
#pragma unroll
        for (int q = 0; q < U; ++q) buf[sidx(t * U + q)] = xp[q];
        __syncthreads();
        T *xrow = x + g.guard + (int64_t)k * g.plane;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = q * P + t;
            if (e < n) xrow[e] = buf[sidx(e)];
        }
    }
}

// (U, NW) for n unknowns: U rows per thread, NW warps per slab
void spike_shape(int n, bool fp64, int &U, int &NW) {
    if (n <= 256) {
        NW = 1;
        U = 1;
        while (32 * U < n) U *= 2;
    } else {
        NW = 4;
        U = 1;
        while (128 * U < n) U *= 2;
    }
    if (U > (fp64 ? 16 : 32)) U = 0;   // not supported: caller falls back to PCR
    // the tables and staging buffers must fit the dynamic shared memory the kernels are
    // configured for (slab_set_attributes); n = 2047 in FP64 does not
    if (U > 0) {
        const int P = 32 * NW;
        const int NL = NW == 1 ? 5 : NW == 2 ? 6 : NW == 4 ? 7 : 8;
        const size_t items = 8 * (size_t)U + 2 + 8 * (size_t)NL + 4;
        const size_t bytes = (fp64 ? 8 : 4) * (items * P + (size_t)P * U + (size_t)(P * U) / 32 + 4 * P);
        if (bytes > (size_t)SLAB_SMEM_LIMIT) U = 0;
    }
}

int spike_block_size(int n) {
    int U, NW;
    spike_shape(n, false, U, NW);
    return U;
}

template <typename T>
size_t slab_spike_smem(int U, int NW) {
    const int P = 32 * NW;
    const int NL = NW == 1 ? 5 : NW == 2 ? 6 : NW == 4 ? 7 : 8;
    const size_t items = 8 * U + 2 + 8 * NL + 4;
    return sizeof(T) * (items * P + (size_t)P * U + (size_t)(P * U) / 32 + 4 * P);
}

template <typename T>
bool slab_warp_supported(int n) {
    int U, NW;
    spike_shape(n, sizeof(T) == 8, U, NW);
    return U > 0;
}

// ---------------------------------------------------------------------------------------
// 2D slabs in the eigenbasis, all time rows at once.  With L = Lx (+) Ly and
// Lx = Sx diag(lamx) Sx^{-1}, Ly = Sy diag(lamy) Sy^{-1}, every mode m = (j, i) of a slab follows
//     xh_k = alpha_m xh_{k-1} + beta_m rh_k,  beta_m = 1/(1 - a lam_m), alpha_m = (1 + b lam_m) beta_m,
// lam_m = lamy_j + lamx_i, xh = 0 before the slab's first step (x_0 = r_0 before step 1 when the
// coupling is kept), where rh_k = Sy^{-1} R_k Sx^{-T} and X_k = Sy Xh_k Sx^T.  Three launches:
// forward transform of every row, recurrence per (mode, slab) in place, inverse transform.
// ---------------------------------------------------------------------------------------
constexpr int FDM_THREADS = 256;
constexpr int FDM_SHORT_SLAB = 32;   // longer slabs (and the coupled march) take the blocked scan

template <typename T>
__device__ __forceinline__ void fdm_product(const T *__restrict__ Mleft, const T *__restrict__ MrT,
                                            T *__restrict__ A, T *__restrict__ B, int nx, int ny) {
    // B = Mleft A (ny x ny times ny x nx), then A = B Mright^T with MrT[q][i] = Mright^T[q][i]
    // = Mright[i][q] (Mright nx x nx, kept transposed so that lanes of consecutive i read
    // consecutive words: no bank conflicts)
    const int nxy = nx * ny;
    for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) {
        const int j = e / nx, i = e - j * nx;
        T acc = 0;
        for (int q = 0; q < ny; ++q) acc += Mleft[j * ny + q] * A[q * nx + i];
        B[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) {
        const int j = e / nx, i = e - j * nx;
        T acc = 0;
        for (int q = 0; q < nx; ++q) acc += B[j * nx + q] * MrT[q * nx + i];
        A[e] = acc;
    }
    __syncthreads();
}

// rh[k] = Sy^{-1} R_k Sx^{-T} for k = k0 .. nt (one block per row)
template <typename T>
__global__ void __launch_bounds__(FDM_THREADS) k_fdm_forward(Geom g, const T *__restrict__ Sxi_g,
                                                             const T *__restrict__ Syi_g,
                                                             const T *__restrict__ r, T *__restrict__ rh,
                                                             int k0, const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    T *Sxi = reinterpret_cast<T *>(smem_raw);
    T *Syi = Sxi + nx * nx;
    T *A = Syi + ny * ny;
    T *B = A + nxy;
    const int k = k0 + blockIdx.x;
    for (int e = threadIdx.x; e < nx * nx; e += FDM_THREADS) Sxi[e] = Sxi_g[(e % nx) * nx + e / nx];
    for (int e = threadIdx.x; e < ny * ny; e += FDM_THREADS) Syi[e] = Syi_g[e];
    for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) {
        const int j = e / nx, i = e - j * nx;
        A[e] = r[g.at(k, j, i)];
    }
    __syncthreads();
    fdm_product(Syi, Sxi, A, B, nx, ny);
    T *out = rh + (int64_t)k * nxy;
    for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) out[e] = A[e];
}

// in place on rh: the scalar recurrence of every mode over every slab (thread = (mode, slab))
template <typename T>
__global__ void __launch_bounds__(FDM_THREADS) k_fdm_recurrence(int nx, int ny, T a, T b,
                                                                const T *__restrict__ lamx,
                                                                const T *__restrict__ lamy,
                                                                T *__restrict__ rh, int steps,
                                                                int coupled,
                                                                const int *__restrict__ done) {
    if (done && *done) return;
    const int nxy = nx * ny;
    const int m = blockIdx.x * FDM_THREADS + threadIdx.x;
    if (m >= nxy) return;
    const int j = m / nx, i = m - j * nx;
    const T lam = lamy[j] + lamx[i];
    const T beta = (T)1 / ((T)1 - a * lam);
    const T alpha = ((T)1 + b * lam) * beta;
    const int s0 = 1 + blockIdx.y * steps;
    T acc = coupled ? rh[m] : (T)0;   // coupled: x_0 = r_0, so xh_0 = rh_0
    T *p = rh + (int64_t)s0 * nxy + m;
    for (int q = 0; q < steps; ++q) {
        acc = alpha * acc + beta * p[(int64_t)q * nxy];
        p[(int64_t)q * nxy] = acc;
    }
}

// X_k = Sy Xh_k Sx^T into the padded layout (k >= 1); block 0 copies x_0 = r_0
template <typename T>
__global__ void __launch_bounds__(FDM_THREADS) k_fdm_inverse(Geom g, const T *__restrict__ Sx_g,
                                                             const T *__restrict__ Sy_g,
                                                             const T *__restrict__ r,
                                                             const T *__restrict__ xh,
                                                             T *__restrict__ x,
                                                             const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    const int k = blockIdx.x;
    if (k == 0) {
        for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) {
            const int j = e / nx, i = e - j * nx;
            x[g.at(0, j, i)] = r[g.at(0, j, i)];
        }
        return;
    }
    T *Sx = reinterpret_cast<T *>(smem_raw);
    T *Sy = Sx + nx * nx;
    T *A = Sy + ny * ny;
    T *B = A + nxy;
    for (int e = threadIdx.x; e < nx * nx; e += FDM_THREADS) Sx[e] = Sx_g[(e % nx) * nx + e / nx];
    for (int e = threadIdx.x; e < ny * ny; e += FDM_THREADS) Sy[e] = Sy_g[e];
    const T *in = xh + (int64_t)k * nxy;
    for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) A[e] = in[e];
    __syncthreads();
    fdm_product(Sy, Sx, A, B, nx, ny);
    for (int e = threadIdx.x; e < nxy; e += FDM_THREADS) {
        const int j = e / nx, i = e - j * nx;
        x[g.at(k, j, i)] = A[e];
    }
}

template <typename T>
size_t fdm_smem_bytes(int nx, int ny) {
    return sizeof(T) * ((size_t)nx * nx + (size_t)ny * ny + 2 * (size_t)nx * ny);
}

template <typename T>
void launch_slab_2d_fdm(const Geom &g, double a, double b, const T *Sx, const T *Sxi,
                        const T *lamx, const T *Sy, const T *Syi, const T *lamy, int n_cgs,
                        T *rh, const T *r, T *x, const int *done, cudaStream_t s) {
    const int coupled = n_cgs <= 0 ? 1 : 0;
    const int nslabs = coupled ? 1 : n_cgs;
    const int steps = coupled ? g.nt : g.nt / n_cgs;
    const int nxy = g.nx * g.ny;
    const size_t shm = fdm_smem_bytes<T>(g.nx, g.ny);
    prof_begin(s);
    // row 0 is transformed only when the coupling to x_0 is kept
    const int k0 = coupled ? 0 : 1;
    k_fdm_forward<T><<<g.nt + 1 - k0, FDM_THREADS, shm, s>>>(g, Sxi, Syi, r, rh, k0, done);
    if (!coupled && steps <= FDM_SHORT_SLAB)
        k_fdm_recurrence<T><<<dim3((nxy + FDM_THREADS - 1) / FDM_THREADS, nslabs), FDM_THREADS, 0, s>>>(
            g.nx, g.ny, (T)a, (T)b, lamx, lamy, rh, steps, coupled, done);
    else   // long slabs and the coupled march: blocked scan over time
        launch_mode_scan<T>(nxy, rh, nxy, ModeEig2D<T>{lamx, lamy, g.nx, (T)a, (T)b}, n_cgs, g.nt,
                            done, s);
    k_fdm_inverse<T><<<g.nt + 1, FDM_THREADS, shm, s>>>(g, Sx, Sy, r, rh, x, done);
    prof_end(s, PROF_SLAB, 2.0 * sizeof(T) * (double)g.interior());
    count_launch(3);
}

template void launch_slab_2d_fdm<float>(const Geom &, double, double, const float *, const float *,
                                        const float *, const float *, const float *, const float *,
                                        int, float *, const float *, float *, const int *,
                                        cudaStream_t);
template void launch_slab_2d_fdm<double>(const Geom &, double, double, const double *,
                                         const double *, const double *, const double *,
                                         const double *, const double *, int, double *,
                                         const double *, double *, const int *, cudaStream_t);

template <typename T>
void launch_slab_1d_warp(const Geom &g, double b, const T *tab, int U, int n_cgs, const T *r, T *x,
                         const int *done, cudaStream_t s, int cls) {
    int Uc, NW;
    spike_shape(g.nx, sizeof(T) == 8, Uc, NW);
    (void)U;
    const int nslabs = n_cgs <= 0 ? 1 : n_cgs;
    const int steps = n_cgs <= 0 ? g.nt : g.nt / n_cgs;
    const int coupled = n_cgs <= 0 ? 1 : 0;
    const size_t shm = slab_spike_smem<T>(Uc, NW);
    prof_begin(s);
#define MK_SP(UU, WW)                                                                                  \
    if (Uc == UU && NW == WW)                                                                          \
        k_slab_1d_spike<T, UU, WW><<<nslabs, 32 * WW, shm, s>>>(g, (T)b, tab, steps, coupled, r, x, done)
    MK_SP(1, 1);
    MK_SP(2, 1);
    MK_SP(4, 1);
    MK_SP(8, 1);
    MK_SP(4, 4);
    MK_SP(8, 4);
    MK_SP(16, 4);
    if constexpr (sizeof(T) == 4) {
        MK_SP(32, 4);
    }
#undef MK_SP
    prof_end(s, cls, 2.0 * sizeof(T) * (double)g.interior());
    count_launch();
}

int spike_threads(int n) {
    int U, NW;
    spike_shape(n, false, U, NW);
    return 32 * NW;
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
        // transposed ([q][i] = S[i][q]): the products below read consecutive words across lanes
        const int et = (e % nx) * nx + e / nx;
        Sx[e] = Sx_g[et];
        Sxi[e] = Sxi_g[et];
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
            for (int q = 0; q < nx; ++q) acc += B[j * nx + q] * Sxi[q * nx + i];
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
            for (int q = 0; q < nx; ++q) acc += B[j * nx + q] * Sx[q * nx + i];
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

// Opt in to large dynamic shared memory once, before any launch or graph capture.
cudaError_t slab_set_attributes() {
    const int big = SLAB_SMEM_LIMIT;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        if (r != cudaSuccess) e = r;
    };
    set((const void *)k_slab_2d<float>);
    set((const void *)k_slab_2d<double>);
    set((const void *)k_fdm_forward<float>);
    set((const void *)k_fdm_forward<double>);
    set((const void *)k_fdm_inverse<float>);
    set((const void *)k_fdm_inverse<double>);
    set((const void *)k_slab_1d<float, 1>);
    set((const void *)k_slab_1d<float, 2>);
    set((const void *)k_slab_1d<float, 4>);
    set((const void *)k_slab_1d<double, 1>);
    set((const void *)k_slab_1d<double, 2>);
    set((const void *)k_slab_1d<double, 4>);
    set((const void *)k_slab_1d_spike<float, 1, 1>);
    set((const void *)k_slab_1d_spike<float, 2, 1>);
    set((const void *)k_slab_1d_spike<float, 4, 1>);
    set((const void *)k_slab_1d_spike<float, 8, 1>);
    set((const void *)k_slab_1d_spike<float, 4, 4>);
    set((const void *)k_slab_1d_spike<float, 8, 4>);
    set((const void *)k_slab_1d_spike<float, 16, 4>);
    set((const void *)k_slab_1d_spike<float, 32, 4>);
    set((const void *)k_slab_1d_spike<double, 1, 1>);
    set((const void *)k_slab_1d_spike<double, 2, 1>);
    set((const void *)k_slab_1d_spike<double, 4, 1>);
    set((const void *)k_slab_1d_spike<double, 8, 1>);
    set((const void *)k_slab_1d_spike<double, 4, 4>);
    set((const void *)k_slab_1d_spike<double, 8, 4>);
    set((const void *)k_slab_1d_spike<double, 16, 4>);
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
