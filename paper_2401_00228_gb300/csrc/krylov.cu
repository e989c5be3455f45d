// Krylov kernels of FGMRES (Algorithm 2): Arnoldi orthogonalisation by classical
// Gram-Schmidt (one pass, and a second pass when the norm drops by more than 1/sqrt(2)),
// the Hessenberg least-squares problem by Givens rotations, and the solution update
// u = u_0 + X_J y_J.
//
// The basis is stored unnormalised: v_i = sigma_i V_i with sigma_i = 1/||V_i|| kept on the
// device, so no separate scaling pass is needed.  Every scalar of the process (H, Givens
// rotations, y, flags) lives on the device and is updated by the last block of the
// reduction that produces it, so a whole restart cycle runs without a host round trip.
#include "kernels.h"
#include "reduce.cuh"

namespace mk {

constexpr int KR_THREADS = 256;
constexpr int KR_WARPS = KR_THREADS / 32;
constexpr int MD_EPT = 16;                       // elements per thread per tile
constexpr int MD_TILE = KR_THREADS * MD_EPT;

// Warp-per-slot sum of the partials of nslots reductions; fixed order.
__device__ __forceinline__ void finish_slots(const double *part, int max_blocks, int nslots,
                                             int nb, double *out_smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = warp; t < nslots; t += KR_WARPS) {
        const volatile double *p = part + (int64_t)t * max_blocks;
        double acc = 0.0;
        for (int b = lane; b < nb; b += 32) acc += p[b];
        acc = warp_sum(acc);
        if (lane == 0) out_smem[t] = acc;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------
// multidot: d_i = <W, V_i>, i = 0..j ; first pass also ||W||^2.
// ---------------------------------------------------------------------------------------
template <typename TW, typename TV>
__global__ void __launch_bounds__(KR_THREADS) k_multidot(int64_t len, const TW *__restrict__ W,
                                                         const TV *__restrict__ V,
                                                         int64_t vstride, int j,
                                                         ReduceScratch rs, KState ks, int second,
                                                         const int *__restrict__ done) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    extern __shared__ double smem[];
    const int nv = j + 1;
    const int nslots = second ? nv : nv + 1;
    double *acc = smem;                      // [nslots][KR_WARPS]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < nslots * KR_WARPS; t += KR_THREADS) acc[t] = 0.0;
    __syncthreads();
    // arithmetic in the storage type (FP32 for the inner levels of the mixed cycle); the
    // per-warp results are accumulated across tiles in FP64
    using Ta = TV;
    const TW *src = second ? (const TW *)(V + (int64_t)(j + 1) * vstride) : W;
    for (int64_t base = (int64_t)blockIdx.x * MD_TILE; base < len;
         base += (int64_t)gridDim.x * MD_TILE) {
        Ta w[MD_EPT];
#pragma unroll
        for (int q = 0; q < MD_EPT; ++q) {
            int64_t e = base + threadIdx.x + q * KR_THREADS;
            w[q] = (e < len) ? (Ta)src[e] : (Ta)0;
        }
        if (!second) {
            Ta s = 0;
#pragma unroll
            for (int q = 0; q < MD_EPT; ++q) s += w[q] * w[q];
            s = warp_sum_t(s);
            if (lane == 0) acc[nv * KR_WARPS + warp] += (double)s;
        }
        for (int i = 0; i < nv; ++i) {
            const TV *vi = V + (int64_t)i * vstride;
            Ta s = 0;
#pragma unroll
            for (int q = 0; q < MD_EPT; ++q) {
                int64_t e = base + threadIdx.x + q * KR_THREADS;
                Ta vv = (e < len) ? vi[e] : (Ta)0;
                s += w[q] * vv;
            }
            s = warp_sum_t(s);
            if (lane == 0) acc[i * KR_WARPS + warp] += (double)s;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nslots; t += KR_THREADS) {
        double s = 0.0;
        for (int w2 = 0; w2 < KR_WARPS; ++w2) s += acc[t * KR_WARPS + w2];
        rs.partials[(int64_t)t * rs.max_blocks + blockIdx.x] = s;
    }
    if (last_block_ticket(rs.counter)) {
        double *res = smem;  // reuse
        finish_slots(rs.partials, rs.max_blocks, nslots, gridDim.x, res);
        if (threadIdx.x == 0) {
            double *H = ks.H() + (int64_t)j * (ks.m + 1);
            for (int i = 0; i < nv; ++i) {
                double hc = ks.sigma()[i] * res[i];
                ks.tmp()[i] = hc;
                H[i] = second ? H[i] + hc : hc;
            }
            if (!second) ks.misc()[2] = res[nv];
            rs.counter[0] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Givens least squares helpers (one thread).
// ---------------------------------------------------------------------------------------
__device__ void givens_solve(double *R, int ld, int n, double beta, double *gg, double *y,
                             double *res) {
    // least squares min || beta e1 - H y ||, H (n+1) x n (column-major, leading dim ld),
    // rotated in place into R; gg receives the rotated right-hand side (n+1 entries)
    for (int r = 0; r <= n; ++r) gg[r] = 0.0;
    gg[0] = beta;
    for (int c = 0; c < n; ++c) {
        double a = R[c + c * ld], b = R[c + 1 + c * ld];
        double rr = sqrt(a * a + b * b);
        double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
        for (int k = c; k < n; ++k) {
            double t1 = R[c + k * ld], t2 = R[c + 1 + k * ld];
            R[c + k * ld] = cs * t1 + sn * t2;
            R[c + 1 + k * ld] = -sn * t1 + cs * t2;
        }
        double t1 = gg[c], t2 = gg[c + 1];
        gg[c] = cs * t1 + sn * t2;
        gg[c + 1] = -sn * t1 + cs * t2;
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = gg[c];
        for (int k = c + 1; k < n; ++k) s -= R[c + k * ld] * y[k];
        double d = R[c + c * ld];
        y[c] = (fabs(d) > 0.0) ? s / d : 0.0;
    }
    if (res) *res = fabs(gg[n]);
}

// ---------------------------------------------------------------------------------------
// update: V_{j+1} = src - sum_i c_i V_i, c_i = tmp_i sigma_i ; ||.||^2 ; epilogue.
// ---------------------------------------------------------------------------------------
__device__ void update_epilogue(double nrm2, KState ks, int j, int mode, int second) {
    double nrm = sqrt(nrm2);
    double *misc = ks.misc();
    const int m = ks.m;
    if (!isfinite(nrm)) {
        ks.flags[3] = 1;
        ks.flags[0] = 1;
        ks.flags[1] = 0;
        return;
    }
    if (!second && ((mode & UPD_REORTH_ALWAYS) ||
                    ((mode & UPD_REORTH) && nrm < 0.70710678118654752 * sqrt(misc[2])))) {
        ks.flags[2] = 1;  // a second Gram-Schmidt pass follows
        return;
    }
    ks.flags[2] = 0;
    double *H = ks.H() + (int64_t)j * (m + 1);
    H[j + 1] = nrm;
    ks.sigma()[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (mode & UPD_GIVENS) {
        double *cs = ks.cs(), *sn = ks.sn(), *g = ks.g();
        for (int i = 0; i < j; ++i) {
            double t = cs[i] * H[i] + sn[i] * H[i + 1];
            H[i + 1] = -sn[i] * H[i] + cs[i] * H[i + 1];
            H[i] = t;
        }
        double a = H[j], b = H[j + 1];
        double r = sqrt(a * a + b * b);
        double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
        H[j] = r;
        H[j + 1] = 0.0;
        cs[j] = c;
        sn[j] = s;
        g[j + 1] = -s * g[j];
        g[j] = c * g[j];
        double est = fabs(g[j + 1]);
        misc[6] = est;
        ks.flags[4] += 1;
        bool conv = (est <= misc[1]) || (nrm == 0.0);
        if (conv || j == m - 1) {
            int jf = j + 1;
            ks.flags[1] = jf;
            double *y = ks.y();
            for (int c2 = jf - 1; c2 >= 0; --c2) {
                double sacc = g[c2];
                for (int k = c2 + 1; k < jf; ++k) sacc -= ks.H()[c2 + (int64_t)k * (m + 1)] * y[k];
                double d = ks.H()[c2 + (int64_t)c2 * (m + 1)];
                y[c2] = (fabs(d) > 0.0) ? sacc / d : 0.0;
            }
            if (conv) ks.flags[0] = 1;
        }
    } else if (mode & UPD_INNER_LSQ) {
        if (j == m - 1) givens_solve(ks.H(), m + 1, m, misc[0], ks.g(), ks.y(), nullptr);
    }
}

template <typename TW, typename TV>
__global__ void __launch_bounds__(KR_THREADS) k_update(int64_t len, const TW *__restrict__ W,
                                                       TV *__restrict__ V, int64_t vstride,
                                                       int j, int write_next, ReduceScratch rs,
                                                       KState ks, int mode, int second,
                                                       const int *__restrict__ done) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    // arithmetic in the storage type (FP32 on the inner levels of the mixed cycle)
    using Ta = TV;
    __shared__ Ta c[MK_MAX_RESTART + 1];
    const int nv = j + 1;
    for (int i = threadIdx.x; i < nv; i += KR_THREADS) c[i] = (Ta)(ks.tmp()[i] * ks.sigma()[i]);
    __syncthreads();
    TV *out = V + (int64_t)(j + 1) * vstride;
    Ta acc = 0;
    for (int64_t e = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * KR_THREADS) {
        Ta val = second ? (Ta)out[e] : (Ta)W[e];
        for (int i = 0; i < nv; ++i) val -= c[i] * (Ta)V[(int64_t)i * vstride + e];
        if (write_next) out[e] = (TV)val;
        acc += val * val;
    }
    double bs = block_sum((double)acc);
    if (threadIdx.x == 0) rs.partials[blockIdx.x] = bs;
    if (last_block_ticket(rs.counter)) {
        double tot = sum_partials(rs.partials, gridDim.x);
        if (threadIdx.x == 0) {
            update_epilogue(tot, ks, j, mode, second);
            rs.counter[0] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// combine: u += sum_{i < jf} y_i X_i
// ---------------------------------------------------------------------------------------
template <typename TX>
__global__ void __launch_bounds__(KR_THREADS) k_combine(int64_t len, double *__restrict__ u,
                                                        const TX *__restrict__ X,
                                                        int64_t xstride, KState ks) {
    __shared__ double y[MK_MAX_RESTART];
    const int jf = ks.flags[1];
    if (jf <= 0 || ks.flags[3]) return;
    for (int i = threadIdx.x; i < jf; i += KR_THREADS) y[i] = ks.y()[i];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * KR_THREADS) {
        double acc = u[e];
        for (int i = 0; i < jf; ++i) acc += y[i] * (double)X[(int64_t)i * xstride + e];
        u[e] = acc;
    }
}

__global__ void k_lsq(int j, double *H, double beta, double *gg, double *y, double *res) {
    if (threadIdx.x == 0 && blockIdx.x == 0) givens_solve(H, j + 1, j, beta, gg, y, res);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
static int krylov_grid(int64_t len, int64_t per_block) {
    int64_t g = (len + per_block - 1) / per_block;
    int64_t cap = (int64_t)g_num_sms * 4;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename TW, typename TV>
void launch_multidot(int64_t len, const TW *W, const TV *V, int64_t vstride, int j,
                     const ReduceScratch &rs, KState ks, bool second_pass, const int *done,
                     cudaStream_t s) {
    int grid = krylov_grid(len, MD_TILE);
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    size_t shm = sizeof(double) * (size_t)(j + 2) * KR_WARPS;
    if (shm < sizeof(double) * (size_t)(j + 2)) shm = sizeof(double) * (size_t)(j + 2);
    prof_begin(s);
    k_multidot<TW, TV><<<grid, KR_THREADS, shm, s>>>(len, W, V, vstride, j, rs, ks,
                                                      second_pass ? 1 : 0, done);
    prof_end(s, PROF_MULTIDOT, (double)(j + 2) * alg_n * sizeof(TV));
    count_launch();
}

template <typename TW, typename TV>
void launch_update(int64_t len, const TW *W, TV *V, int64_t vstride, int j, bool write_next,
                   const ReduceScratch &rs, KState ks, int mode, bool second_pass,
                   const int *done, cudaStream_t s) {
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    int grid = krylov_grid(len, (int64_t)KR_THREADS * 8);
    prof_begin(s);
    k_update<TW, TV><<<grid, KR_THREADS, 0, s>>>(len, W, V, vstride, j, write_next ? 1 : 0, rs,
                                                  ks, mode, second_pass ? 1 : 0, done);
    prof_end(s, PROF_UPDATE, (double)(j + 2 + (write_next ? 1 : 0)) * alg_n * sizeof(TV));
    count_launch();
}

template <typename TX>
void launch_combine(int64_t len, double *u, const TX *X, int64_t xstride, KState ks,
                    cudaStream_t s) {
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    int grid = krylov_grid(len, (int64_t)KR_THREADS * 8);
    prof_begin(s);
    k_combine<TX><<<grid, KR_THREADS, 0, s>>>(len, u, X, xstride, ks);
    prof_end(s, PROF_COMBINE, (double)alg_n * (16.0 + (double)ks.m * sizeof(TX)));
    count_launch();
}

void launch_lsq(int j, double *H, double beta, double *gg, double *y, double *res,
                cudaStream_t s) {
    k_lsq<<<1, 32, 0, s>>>(j, H, beta, gg, y, res);
    count_launch();
}

template void launch_multidot<double, double>(int64_t, const double *, const double *, int64_t,
                                              int, const ReduceScratch &, KState, bool,
                                              const int *, cudaStream_t);
template void launch_multidot<float, float>(int64_t, const float *, const float *, int64_t, int,
                                            const ReduceScratch &, KState, bool, const int *,
                                            cudaStream_t);
template void launch_update<double, double>(int64_t, const double *, double *, int64_t, int, bool,
                                            const ReduceScratch &, KState, int, bool,
                                            const int *, cudaStream_t);
template void launch_update<float, float>(int64_t, const float *, float *, int64_t, int, bool,
                                          const ReduceScratch &, KState, int, bool, const int *,
                                          cudaStream_t);
template void launch_combine<double>(int64_t, double *, const double *, int64_t, KState,
                                     cudaStream_t);
template void launch_combine<float>(int64_t, double *, const float *, int64_t, KState,
                                    cudaStream_t);

}  // namespace mk
