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
// DST-I through a complex FFT of length N2 = 2(n+1): the odd extension
//     y_0 = 0, y_m = v_{m-1} (1 <= m <= n), y_{n+1} = 0, y_{N2-m} = -v_{m-1}
// has Y_m = -2i sum_j v_j sin(pi m (j+1)/(n+1)), so DST(v)_j = -Im(Y_{j+1}) / 2.  The FFT is
// the Stockham auto-sort form (natural order in and out) with radix-8 passes and one final
// radix-4 or radix-2 pass: each thread keeps its butterfly groups in registers between two
// barriers, the twiddles of each pass come from a table computed once on the host (a
// thread's R-1 factors are contiguous), and the shared array has one pad slot per 32
// elements so that the strided stores of the early passes spread over the banks.
// Three launches: forward transform of every row, the per-mode recurrence over each slab
// (in place on the transformed rows; a thread walks a short slab, longer slabs and the
// coupled march over all steps, n_cgs = 0, take the blocked scan of scan.cuh), inverse
// transform of every row.
#include "kernels.h"
#include "scan.cuh"

namespace mk {

namespace {

constexpr int DST_THREADS = 256;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }   // a * (-i)
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

__device__ __forceinline__ void dft2(float2 *v) {
    const float2 t = csub(v[0], v[1]);
    v[0] = cadd(v[0], v[1]);
    v[1] = t;
}
__device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3) {
    const float2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = cmi(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}
// forward DFT of size 8 as two size-4 DFTs of the even and odd entries
__device__ __forceinline__ void dft8(float2 *v) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    const float c = 0.70710678118654752f;
    const float2 w1 = make_float2(c * (o1.x + o1.y), c * (o1.y - o1.x));    // o1 e^{-i pi/4}
    const float2 w2 = cmi(o2);                                               // o2 e^{-i pi/2}
    const float2 w3 = make_float2(c * (o3.y - o3.x), -c * (o3.x + o3.y));   // o3 e^{-3i pi/4}
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1);
    v[5] = csub(e1, w1);
    v[2] = cadd(e2, w2);
    v[6] = csub(e2, w2);
    v[3] = cadd(e3, w3);
    v[7] = csub(e3, w3);
}

// One Stockham pass of radix R over a[] (padded indices), current span Ns; tw holds the
// pass's twiddles exp(-2 pi i k r / (Ns R)) at k (R-1) + r - 1 (k < Ns, 1 <= r < R).
template <int R>
__device__ __forceinline__ void stockham_pass(float2 *a, int N, int Ns, const float2 *__restrict__ tw) {
    constexpr int G = 2;   // groups per thread: N / R <= 2 * DST_THREADS for N <= 4096
    const int ngroups = N / R;
    float2 v[G][R];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = threadIdx.x + g * DST_THREADS;
        if (j < ngroups) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[g][r] = a[pad(j + r * ngroups)];
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                const float2 *t = tw + k * (R - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) v[g][r] = cmul(v[g][r], __ldg(t + r - 1));
            }
            if (R == 8) dft8(v[g]);
            else if (R == 4) dft4(v[g][0], v[g][1], v[g][2], v[g][3]);
            else dft2(v[g]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = threadIdx.x + g * DST_THREADS;
        if (j < ngroups) {
            const int k = j & (Ns - 1);
            const int d = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) a[pad(d + r * Ns)] = v[g][r];
        }
    }
    __syncthreads();
}

// In-place forward FFT of a[] (natural order, padded indices), N = 2^logN <= 4096; the
// passes' twiddle tables follow each other in tw (a pass of span Ns and radix R uses
// Ns (R - 1) entries).
__device__ __forceinline__ void fft_smem(float2 *a, int N, int logN, const float2 *__restrict__ tw) {
    int Ns = 1, p = logN;
    while (p >= 3) {
        stockham_pass<8>(a, N, Ns, tw);
        tw += Ns * 7;
        Ns *= 8;
        p -= 3;
    }
    if (p == 2) stockham_pass<4>(a, N, Ns, tw);
    else if (p == 1) stockham_pass<2>(a, N, Ns, tw);
}

// rh[k][j] = DST(r_k)_j for every row k = k0..nt (k0 = 0 when the coupling to x_0 is kept).
// Grid: one block per row.
__global__ void __launch_bounds__(DST_THREADS) k_dst_forward(Geom g, const float *__restrict__ r,
                                                              float *__restrict__ rh, int ldd,
                                                              const float2 *__restrict__ tw,
                                                              int N2, int logN2,
                                                              int k0,
                                                              const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ float2 sm_dst[];
    float2 *a = sm_dst;
    const int k = blockIdx.x + k0;
    const int n = g.nx, N = n + 1;
    const float *row = r + g.guard + (int64_t)k * g.plane;
    for (int m = threadIdx.x; m < N2; m += DST_THREADS) {
        float v = 0.f;
        if (m > 0 && m < N) v = row[m - 1];
        else if (m > N) v = -row[N2 - m - 1];
        a[pad(m)] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft_smem(a, N2, logN2, tw);
    float *out = rh + (int64_t)k * ldd;
    for (int j = threadIdx.x; j < n; j += DST_THREADS) out[j] = -0.5f * a[pad(j + 1)].y;
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

// x_k = 2/(n+1) DST(xh_k), k = 1..nt; block 0 copies x_0 = r_0.
__global__ void __launch_bounds__(DST_THREADS) k_dst_inverse(Geom g, const float *__restrict__ r,
                                                              const float *__restrict__ xh, int ldd,
                                                              const float2 *__restrict__ tw,
                                                              int N2, int logN2,
                                                              float *__restrict__ x,
                                                              const int *__restrict__ done) {
    if (done && *done) return;
    extern __shared__ float2 sm_dst[];
    float2 *a = sm_dst;
    const int k = blockIdx.x;
    const int n = g.nx, N = n + 1;
    float *xrow = x + g.guard + (int64_t)k * g.plane;
    if (k == 0) {
        const float *r0 = r + g.guard;
        for (int i = threadIdx.x; i < n; i += DST_THREADS) xrow[i] = r0[i];
        return;
    }
    const float *in = xh + (int64_t)k * ldd;
    for (int m = threadIdx.x; m < N2; m += DST_THREADS) {
        float v = 0.f;
        if (m > 0 && m < N) v = in[m - 1];
        else if (m > N) v = -in[N2 - m - 1];
        a[pad(m)] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft_smem(a, N2, logN2, tw);
    const float sc = -1.f / (float)N;
    for (int i = threadIdx.x; i < n; i += DST_THREADS) xrow[i] = sc * a[pad(i + 1)].y;
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
    k_dst_forward<<<g.nt + 1 - k0, DST_THREADS, shm, s>>>(g, r, rh, ldd, tw, N2, logN2, k0, done);
    if (!coupled && steps <= DST_SHORT_SLAB)
        k_dst_recurrence<<<dim3((g.nx + REC_THREADS - 1) / REC_THREADS, n_cgs), REC_THREADS, 0, s>>>(
            g.nx, rh, ldd, tab, tab + g.nx, steps, done);
    else
        launch_mode_scan<float>(g.nx, rh, ldd, ModeTable<float>{tab, tab + g.nx}, n_cgs, g.nt, done, s);
    k_dst_inverse<<<g.nt + 1, DST_THREADS, shm, s>>>(g, r, rh, ldd, tw, N2, logN2, x, done);
    prof_end(s, PROF_SLAB, 2.0 * sizeof(float) * (double)g.interior());
    count_launch(3);
}

}  // namespace mk
