// Allocation-free fine-level residual: r = f - A_h u of the all-at-once system
// (Eq. (finesys)) together with ||r||_2 and the per-step norms ||r_k||_2.
//
// The block partial sums of the norm reduction live in a fixed-size array in static
// device memory instead of a buffer obtained from cudaMalloc, so a call allocates
// nothing.  Its address is looked up once per device with cudaGetSymbolAddress.
//
// Operator (dense (n_t+1) x n layout, n = nx*ny, zero Dirichlet boundaries):
//   r_0 = f_0 - u_0,
//   r_k = f_k - [(u_k - a L u_k) - (u_{k-1} + b L u_{k-1})],  a = theta dt, b = (1-theta) dt,
//   (L v)_{j,i} = cx (v_{j,i-1} - 2 v_{j,i} + v_{j,i+1}) + cy (v_{j-1,i} - 2 v_{j,i} + v_{j+1,i}),
//   cx = tau / hx^2, cy = tau / hy^2 (cy = 0 in 1D), out-of-range neighbours read as 0.
#include <math.h>

#include <mutex>

#include "solver.h"

namespace mk {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 8;
constexpr int NA_CHUNK = NA_THREADS * NA_PER_THREAD;   // spatial points per block
static_assert(NA_CHUNK == MK_NOALLOC_CHUNK, "chunk size of the header");

// Sum of squares of one block's residuals; the block of time step k and chunk c
// writes slot k * chunks + c.  No slot needs an initial value.
static __device__ __align__(256) double g_na_partials[MK_NOALLOC_MAX_PARTIALS];
// Arrival counter of the last-block reduction.  It must be zero when a launch starts:
// static device memory is zero when the module is loaded, and the last block of every
// launch stores zero again.
static __device__ __align__(256) unsigned g_na_ticket;

struct NaSlots {
    double *partials = nullptr;
    unsigned *ticket = nullptr;
};
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
NaSlots g_na_slots[NA_MAX_DEVICES];

// Device addresses of the scratch on the current device (looked up on first use).
cudaError_t na_slots(NaSlots &out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaSlots &sl = g_na_slots[dev];
    if (!sl.partials) {
        void *p = nullptr, *t = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&t, g_na_ticket);
        if (e != cudaSuccess) return e;
        sl.partials = static_cast<double *>(p);
        sl.ticket = static_cast<unsigned *>(t);
    }
    out = sl;
    return cudaSuccess;
}

__device__ __forceinline__ double na_lap(const double *__restrict__ v, int64_t p, int i, int j,
                                         int nx, int ny, double cx, double cy) {
    const double c = v[p];
    double s = cx * (((i > 0) ? v[p - 1] : 0.0) - 2.0 * c + ((i + 1 < nx) ? v[p + 1] : 0.0));
    if (ny > 1)
        s += cy * (((j > 0) ? v[p - nx] : 0.0) - 2.0 * c + ((j + 1 < ny) ? v[p + nx] : 0.0));
    return s;
}

// Fixed-order block sum (warp shuffles, then the warp sums in warp order).
__device__ __forceinline__ double na_block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w];
    __syncthreads();
    return t;   // valid in thread 0
}

// One block per (time step k, chunk c of NA_CHUNK spatial points); grid = (nt+1) * chunks.
__global__ void __launch_bounds__(NA_THREADS)
k_residual_noalloc(int nx, int ny, int nt, int chunks, double a, double b, double cx, double cy,
                   const double *__restrict__ f, const double *__restrict__ u,
                   double *__restrict__ r, double *partials, unsigned *ticket,
                   double *rnorm, double *rnorm_steps) {
    __shared__ double sh[NA_THREADS / 32];
    __shared__ int s_last;
    const int64_t n = (int64_t)nx * ny;
    const int k = blockIdx.x / chunks;
    const int c = blockIdx.x - k * chunks;
    const double *fk = f + (int64_t)k * n;
    const double *uk = u + (int64_t)k * n;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < NA_PER_THREAD; ++q) {
        const int64_t p = (int64_t)c * NA_CHUNK + q * NA_THREADS + threadIdx.x;
        if (p < n) {
            double res;
            if (k == 0) {
                res = fk[p] - uk[p];
            } else {
                const int j = (int)(p / nx), i = (int)(p - (int64_t)j * nx);
                const double *um = uk - n;
                const double lk = na_lap(uk, p, i, j, nx, ny, cx, cy);
                const double lm = na_lap(um, p, i, j, nx, ny, cx, cy);
                res = fk[p] - ((uk[p] - a * lk) - (um[p] + b * lm));
            }
            if (r) r[(int64_t)k * n + p] = res;
            acc += res * res;
        }
    }
    const double bsum = na_block_sum(acc, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bsum;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Last block: per-step sums over the chunks in chunk order, then the total over
    // the steps (thread t takes steps t, t + 256, ...), in a fixed order.
    double tot = 0.0;
    for (int kk = threadIdx.x; kk <= nt; kk += NA_THREADS) {
        double sk = 0.0;
        for (int cc = 0; cc < chunks; ++cc) sk += __ldcg(partials + (int64_t)kk * chunks + cc);
        if (rnorm_steps) rnorm_steps[kk] = sqrt(sk);
        tot += sk;
    }
    const double total = na_block_sum(tot, sh);
    if (threadIdx.x == 0) {
        *rnorm = sqrt(total);
        *ticket = 0u;
    }
}

}  // namespace

int64_t noalloc_partials_needed(const Problem &P) {
    const int64_t n = (int64_t)P.nx * P.ny;
    return (int64_t)(P.nt + 1) * ((n + NA_CHUNK - 1) / NA_CHUNK);
}

mk_status residual_noalloc(const Problem &P, const double *f, const double *u, double *r,
                           double *rnorm, double *rnorm_steps, cudaStream_t s) {
    const int64_t need = noalloc_partials_needed(P);
    if (need > MK_NOALLOC_MAX_PARTIALS) return MK_ERR_TOO_LARGE;
    NaSlots sl;
    cudaError_t e = na_slots(sl);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MK_ERR_CUDA;
    }
    const int64_t n = (int64_t)P.nx * P.ny;
    const int chunks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    const double hx = 1.0 / (P.nx + 1);
    const double cx = P.tau / (hx * hx);
    double cy = 0.0;
    if (P.dim == 2) {
        const double hy = 1.0 / (P.ny + 1);
        cy = P.tau / (hy * hy);
    }
    const double a = P.theta * P.dt, b = (1.0 - P.theta) * P.dt;
    k_residual_noalloc<<<(unsigned)need, NA_THREADS, 0, s>>>(
        P.nx, P.dim == 2 ? P.ny : 1, P.nt, chunks, a, b, cx, cy, f, u, r, sl.partials, sl.ticket,
        rnorm, rnorm_steps);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MK_ERR_CUDA;
    }
    return MK_OK;
}

}  // namespace mk
