// Coarsest decoupled slabs (Sec. 3.3.2, Eq. (Qhtilde)) for a uniform 1D operator
// L = c tridiag(1, -2, 1) with zero Dirichlet ends, by sine-transform diagonalisation.
//
// L = S diag(lam) S^{-1} with S_ij = sin(pi (i+1)(j+1)/(n+1)), S^{-1} = 2/(n+1) S and
// lam_j = -4c sin^2(pi (j+1) / (2(n+1))).  In that basis every slab step
//     (I - a L) x_k = r_k + (I + b L) x_{k-1}
// is a scalar recurrence per mode, xh_k = alpha_j xh_{k-1} + beta_j rh_k with
// beta_j = 1/(1 - a lam_j), alpha_j = (1 + b lam_j) beta_j, and xh = 0 before the first step
// of each slab (the dropped coupling).  So the solve is
//     rh = DST(r)  per row;   xh_k = alpha xh_{k-1} + beta rh_k  per mode and slab;
//     x = 2/(n+1) DST(xh)  per row;   x_0 = r_0.  The rows are independent, so all n_t + 1 rows
// run at once instead of s sequential tridiagonal solves per slab.  This is the fast form of
// the diagonalisation the 2D coarsest solve uses.
//
// DST-I through a complex FFT of length N2 = 2(n+1), two rows per transform: the odd extension
//     y_0 = 0, y_m = v_{m-1} (1 <= m <= n), y_{n+1} = 0, y_{N2-m} = -v_{m-1}
// has Y_m = -2i sum_j v_j sin(pi m (j+1)/(n+1)), so DST(v)_j = -Im(Y_{j+1}) / 2.  The FFT is
// the shared-memory Stockham FFT of dst_fft.cuh.
// Three launches: forward transform of every row, the per-mode recurrence over each slab
// (in place on the transformed rows; a thread walks a short slab, longer slabs and the
// coupled march over all steps, n_cgs = 0, take the blocked scan of scan.cuh), inverse
// transform of every row.
#include "kernels.h"
#include "scan.cuh"
#include "dst_fft.cuh"

namespace mk {

namespace {

using namespace dstfft;

// rh[k][j] = DST(r_k)_j for every row k = k0..nt (k0 = 0 when the coupling to x_0 is kept).
// Two rows per FFT: the odd extension of a real row has a purely imaginary transform
// (Y = -2i S), so with row k in the real and row k+1 in the imaginary part of the input,
// Y = -2i S_k + 2 S_{k+1}: S_k = -Im(Y)/2 and S_{k+1} = Re(Y)/2.  Grid: one block per pair.
__global__ void __launch_bounds__(DST_THREADS) k_dst_forward(Geom g, const float *__restrict__ r,
                                                              float *__restrict__ rh, int ldd,
                                                              const float2 *__restrict__ tw,
                                                              int N2, int logN2,
                                                              int k0,
                                                              const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ float2 sm_dst[];
    float2 *a = sm_dst;
    const int k = k0 + 2 * blockIdx.x;
    const bool two = k + 1 <= g.nt;
    const int n = g.nx, N = n + 1;
    const float *row = r + g.guard + (int64_t)k * g.plane;
    const float *row2 = row + g.plane;
    for (int m = threadIdx.x; m < N2; m += DST_THREADS) {
        float v = 0.f, w = 0.f;
        if (m > 0 && m < N) {
            v = row[m - 1];
            if (two) w = row2[m - 1];
        } else if (m > N) {
            v = -row[N2 - m - 1];
            if (two) w = -row2[N2 - m - 1];
        }
        a[pad(m)] = make_float2(v, w);
    }
    __syncthreads();
    fft_smem(a, N2, logN2, tw);
    float *out = rh + (int64_t)k * ldd;
    for (int j = threadIdx.x; j < n; j += DST_THREADS) {
        const float2 y = a[pad(j + 1)];
        out[j] = -0.5f * y.y;
        if (two) out[ldd + j] = 0.5f * y.x;
    }
}

// In place on rh: xh_k = alpha_j xh_{k-1} + beta_j rh_k over each slab, xh = 0 before its
// first step.  Short slabs: one thread per (mode, slab) walks the slab's steps.  Grid:
// (modes / 128, slabs); the slab's rows are loaded 8 at a time.
constexpr int REC_THREADS = 128;
constexpr int DST_SHORT_SLAB = 32;   // longer slabs (and the coupled march) take the blocked scan
__global__ void __launch_bounds__(REC_THREADS) k_dst_recurrence(int n, float *__restrict__ rh, int ldd,
                                                                const float *__restrict__ alpha,
                                                                const float *__restrict__ beta,
                                                                int steps,
                                                                const int *__restrict__ done) {
    if (done && *done) return;
    const int j = blockIdx.x * REC_THREADS + threadIdx.x;
    if (j >= n) return;
    const int s0 = 1 + blockIdx.y * steps;
    const float al = alpha[j], be = beta[j];
    float acc = 0.f;
    float *p = rh + (int64_t)s0 * ldd + j;
    int i = 0;
    for (; i + 8 <= steps; i += 8) {
        float t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = p[(int64_t)(i + q) * ldd];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc = al * acc + be * t[q];
            p[(int64_t)(i + q) * ldd] = acc;
        }
    }
    for (; i < steps; ++i) {
        acc = al * acc + be * p[(int64_t)i * ldd];
        p[(int64_t)i * ldd] = acc;
    }
}

// x_k = 2/(n+1) DST(xh_k), k = 1..nt, two rows per FFT as in k_dst_forward; block 0 also
// copies x_0 = r_0.
__global__ void __launch_bounds__(DST_THREADS) k_dst_inverse(Geom g, const float *__restrict__ r,
                                                              const float *__restrict__ xh, int ldd,
                                                              const float2 *__restrict__ tw,
                                                              int N2, int logN2,
                                                              float *__restrict__ x,
                                                              const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ float2 sm_dst[];
    float2 *a = sm_dst;
    const int n = g.nx, N = n + 1;
    if (blockIdx.x == 0) {
        const float *r0 = r + g.guard;
        float *x0 = x + g.guard;
        for (int i = threadIdx.x; i < n; i += DST_THREADS) x0[i] = r0[i];
    }
    const int k = 1 + 2 * blockIdx.x;
    const bool two = k + 1 <= g.nt;
    const float *in = xh + (int64_t)k * ldd;
    for (int m = threadIdx.x; m < N2; m += DST_THREADS) {
        float v = 0.f, w = 0.f;
        if (m > 0 && m < N) {
            v = in[m - 1];
            if (two) w = in[ldd + m - 1];
        } else if (m > N) {
            v = -in[N2 - m - 1];
            if (two) w = -in[ldd + N2 - m - 1];
        }
        a[pad(m)] = make_float2(v, w);
    }
    __syncthreads();
    fft_smem(a, N2, logN2, tw);
    const float sc = 1.f / (float)N;
    float *xrow = x + g.guard + (int64_t)k * g.plane;
    for (int i = threadIdx.x; i < n; i += DST_THREADS) {
        const float2 y = a[pad(i + 1)];
        xrow[i] = -sc * y.y;
        if (two) xrow[g.plane + i] = sc * y.x;
    }
}

}  // namespace

int dst_transform_size(int n) {
    const int N2 = 2 * (n + 1);
    if (n < 1 || N2 > 4096 || (N2 & (N2 - 1)) != 0) return 0;
    return N2;
}

size_t dst_smem_bytes(int N2) { return sizeof(float2) * ((size_t)N2 + (size_t)N2 / 32 + 1); }

cudaError_t dst_set_attributes() {
    const int mx = (int)dst_smem_bytes(4096);
    cudaError_t e = cudaFuncSetAttribute(k_dst_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dst_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

void launch_slab_1d_dst(const Geom &g, const float *tab, const float2 *tw, int N2, int n_cgs,
                        float *rh, int ldd, const float *r, float *x, const int *done,
                        cudaStream_t s) {
    int logN2 = 0;
    while ((1 << logN2) < N2) ++logN2;
    const int coupled = n_cgs <= 0 ? 1 : 0;
    const int steps = coupled ? g.nt : g.nt / n_cgs;
    const int k0 = coupled ? 0 : 1;   // row 0 is transformed only when its coupling is kept
    const size_t shm = dst_smem_bytes(N2);
    prof_begin(s);
    k_dst_forward<<<(g.nt + 2 - k0) / 2, DST_THREADS, shm, s>>>(g, r, rh, ldd, tw, N2, logN2, k0, done);
    if (!coupled && steps <= DST_SHORT_SLAB)
        k_dst_recurrence<<<dim3((g.nx + REC_THREADS - 1) / REC_THREADS, n_cgs), REC_THREADS, 0, s>>>(
            g.nx, rh, ldd, tab, tab + g.nx, steps, done);
    else
        launch_mode_scan<float>(g.nx, rh, ldd, ModeTable<float>{tab, tab + g.nx}, n_cgs, g.nt, done, s);
    k_dst_inverse<<<(g.nt + 1) / 2, DST_THREADS, shm, s>>>(g, r, rh, ldd, tw, N2, logN2, x, done);
    prof_end(s, PROF_SLAB, 2.0 * sizeof(float) * (double)g.interior());
    count_launch(3);
}

}  // namespace mk
