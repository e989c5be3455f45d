// Sequential theta-march of a 2D problem on the GPU (the baseline of Eq. (timemarch)): for
// k = 1 .. n_t,
//     (I - a L) u_k = f_k + (I + b L) u_{k-1},   a = theta dt, b = (1 - theta) dt,
// with L = cx tridiag_x(1, -2, 1) (+) cy tridiag_y(1, -2, 1) (the fine level's uniform FD
// Laplacian, zero Dirichlet).  Every step is a fast Poisson-type solve by the 2D sine transform:
//     rhat = S_y S_x rhs,   uhat = rhat / (1 - a (lamx_i + lamy_j)),   u = (2/(nx+1))(2/(ny+1)) S_y S_x uhat,
// S_x the DST-I of length nx (lamx_i = -4 cx sin^2(pi (i+1) / (2(nx+1)))).  Three launches per
// step (rows: stencil + DST in x; columns: DST in y, divide, inverse DST in y; rows: inverse DST
// in x), all in FP64; the time loop stays sequential.
//
// When n + 1 is a power of two, the DST-I runs through a complex FFT of length N2 = 2(n+1);
// otherwise (n <= MARCH2D_DENSE_MAX) as a dense product with the sine matrix.  The odd extension
//     y_0 = 0, y_m = v_{m-1} (1 <= m <= n), y_{n+1} = 0, y_{N2-m} = -v_{m-1}
// has Y_m = -2i sum_j v_j sin(pi m (j+1)/(n+1)), so DST(v)_j = -Im(Y_{j+1}) / 2.  The FFT is the
// Stockham auto-sort form with radix-8 passes and one radix-4 or radix-2 pass, twiddles from a
// table computed once on the host, one pad slot per 32 elements of shared memory.
#include "kernels.h"

namespace mk {

namespace {

constexpr int M2_THREADS = 256;

__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmi(double2 a) { return make_double2(a.y, -a.x); }   // a * (-i)
__device__ __forceinline__ int zpad(int i) { return i + (i >> 5); }

__device__ __forceinline__ void zdft4(double2 &v0, double2 &v1, double2 &v2, double2 &v3) {
    const double2 t0 = zadd(v0, v2), t1 = zsub(v0, v2), t2 = zadd(v1, v3), t3 = zmi(zsub(v1, v3));
    v0 = zadd(t0, t2);
    v2 = zsub(t0, t2);
    v1 = zadd(t1, t3);
    v3 = zsub(t1, t3);
}
__device__ __forceinline__ void zdft8(double2 *v) {
    double2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    zdft4(e0, e1, e2, e3);
    zdft4(o0, o1, o2, o3);
    const double c = 0.70710678118654752440;
    const double2 w1 = make_double2(c * (o1.x + o1.y), c * (o1.y - o1.x));
    const double2 w2 = zmi(o2);
    const double2 w3 = make_double2(c * (o3.y - o3.x), -c * (o3.x + o3.y));
    v[0] = zadd(e0, o0);
    v[4] = zsub(e0, o0);
    v[1] = zadd(e1, w1);
    v[5] = zsub(e1, w1);
    v[2] = zadd(e2, w2);
    v[6] = zsub(e2, w2);
    v[3] = zadd(e3, w3);
    v[7] = zsub(e3, w3);
}

template <int R>
__device__ __forceinline__ void zpass(double2 *a, int N, int Ns, const double2 *__restrict__ tw) {
    constexpr int G = 2;   // groups per thread: N / R <= 2 * M2_THREADS for N <= 4096
    const int ngroups = N / R;
    double2 v[G][R];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = threadIdx.x + g * M2_THREADS;
        if (j < ngroups) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[g][r] = a[zpad(j + r * ngroups)];
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                const double2 *t = tw + k * (R - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) v[g][r] = zmul(v[g][r], t[r - 1]);
            }
            if (R == 8) {
                zdft8(v[g]);
            } else if (R == 4) {
                zdft4(v[g][0], v[g][1], v[g][2], v[g][3]);
            } else {
                const double2 t = zsub(v[g][0], v[g][1]);
                v[g][0] = zadd(v[g][0], v[g][1]);
                v[g][1] = t;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = threadIdx.x + g * M2_THREADS;
        if (j < ngroups) {
            const int k = j & (Ns - 1);
            const int d = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) a[zpad(d + r * Ns)] = v[g][r];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void zfft(double2 *a, int N, int logN, const double2 *__restrict__ tw) {
    int Ns = 1, p = logN;
    while (p >= 3) {
        zpass<8>(a, N, Ns, tw);
        tw += Ns * 7;
        Ns *= 8;
        p -= 3;
    }
    if (p == 2) zpass<4>(a, N, Ns, tw);
    else if (p == 1) zpass<2>(a, N, Ns, tw);
}

// DST-I of the n values get(m), m = 0..n-1, into put(j, value), j = 0..n-1.  With S non-null
// (n + 1 not a power of two) the transform is the dense product with the symmetric matrix
// S[m][j] = sin(pi (m+1)(j+1) / (n+1)), one output per thread, v staged in shared memory.
template <typename Get, typename Put>
__device__ __forceinline__ void zdst(double2 *a, int n, int N2, int logN2, const double2 *tw,
                                     const double *__restrict__ S, Get get, Put put) {
    if (S) {
        double *v = reinterpret_cast<double *>(a);
        for (int m = threadIdx.x; m < n; m += M2_THREADS) v[m] = get(m);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += M2_THREADS) {
            double acc = 0.0;
            for (int m = 0; m < n; ++m) acc = fma(S[(int64_t)m * n + j], v[m], acc);
            put(j, acc);
        }
        __syncthreads();
        return;
    }
    const int N = n + 1;
    for (int m = threadIdx.x; m < N2; m += M2_THREADS) {
        double v = 0.0;
        if (m > 0 && m < N) v = get(m - 1);
        else if (m > N) v = -get(N2 - m - 1);
        a[zpad(m)] = make_double2(v, 0.0);
    }
    __syncthreads();
    zfft(a, N2, logN2, tw);
    for (int j = threadIdx.x; j < n; j += M2_THREADS) put(j, -0.5 * a[zpad(j + 1)].y);
    __syncthreads();
}

struct March2D {
    Geom g;
    double b, cx, cy;
    int N2x, logx, N2y, logy;
    const double *Sx, *Sy;   // dense transforms (null: FFT)
};

// rows j: t1[j][:] = DST_x(f_k + u_{k-1} + b L u_{k-1})[j][:]
__global__ void __launch_bounds__(M2_THREADS) k_march2d_rows(March2D M, int k,
                                                              const double *__restrict__ f,
                                                              const double *__restrict__ u,
                                                              double *__restrict__ t1,
                                                              const double2 *__restrict__ twx) {
    extern __shared__ double2 zs[];
    const Geom &g = M.g;
    const int j = blockIdx.x;
    const int64_t base = g.at(k, j, 0), prev = g.at(k - 1, j, 0);
    auto get = [&](int i) -> double {
        const int64_t p = prev + i;
        const double c = u[p];
        const double lx = u[p - 1] - 2.0 * c + u[p + 1];
        const double ly = u[p - g.ldx] - 2.0 * c + u[p + g.ldx];
        return f[base + i] + (c + M.b * (M.cx * lx + M.cy * ly));
    };
    auto put = [&](int i, double v) { t1[(int64_t)j * g.nx + i] = v; };
    zdst(zs, g.nx, M.N2x, M.logx, twx, M.Sx, get, put);
}

// columns i: t1[:][i] <- S_y^{-1}-scaled solve in the eigenbasis, back through S_y
__global__ void __launch_bounds__(M2_THREADS) k_march2d_cols(March2D M, double a,
                                                              double *__restrict__ t1,
                                                              const double *__restrict__ lamx,
                                                              const double *__restrict__ lamy,
                                                              const double2 *__restrict__ twy) {
    extern __shared__ double2 zs[];
    const Geom &g = M.g;
    const int i = blockIdx.x;
    const double lx = lamx[i];
    auto get = [&](int j) -> double { return t1[(int64_t)j * g.nx + i]; };
    auto put_div = [&](int j, double v) {
        t1[(int64_t)j * g.nx + i] = v / (1.0 - a * (lx + lamy[j]));
    };
    zdst(zs, g.ny, M.N2y, M.logy, twy, M.Sy, get, put_div);
    auto put = [&](int j, double v) { t1[(int64_t)j * g.nx + i] = v; };
    zdst(zs, g.ny, M.N2y, M.logy, twy, M.Sy, get, put);
}

// rows j: u_k[j][:] = (4 / ((nx+1)(ny+1))) DST_x(t1[j][:])
__global__ void __launch_bounds__(M2_THREADS) k_march2d_out(March2D M, int k,
                                                             const double *__restrict__ t1,
                                                             double *__restrict__ u,
                                                             const double2 *__restrict__ twx) {
    extern __shared__ double2 zs[];
    const Geom &g = M.g;
    const int j = blockIdx.x;
    const double sc = 4.0 / ((double)(g.nx + 1) * (double)(g.ny + 1));
    auto get = [&](int i) -> double { return t1[(int64_t)j * g.nx + i]; };
    const int64_t base = g.at(k, j, 0);
    auto put = [&](int i, double v) { u[base + i] = sc * v; };
    zdst(zs, g.nx, M.N2x, M.logx, twx, M.Sx, get, put);
}

}  // namespace

int march2d_transform_size(int n) {
    const int N2 = 2 * (n + 1);
    if (n < 1 || N2 > 4096 || (N2 & (N2 - 1)) != 0) return 0;
    return N2;
}

size_t march2d_smem_bytes(int N2) { return sizeof(double2) * ((size_t)N2 + (size_t)N2 / 32 + 1); }

static size_t march2d_smem_for(int n) {
    const int N2 = march2d_transform_size(n);
    return N2 ? march2d_smem_bytes(N2) : sizeof(double) * (size_t)n;
}

cudaError_t march2d_set_attributes() {
    const int mx = (int)march2d_smem_bytes(4096);
    cudaError_t e = cudaFuncSetAttribute(k_march2d_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_march2d_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_march2d_out, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

void launch_march_2d_dst(const Geom &g, double a, double b, double cx, double cy,
                         const double *lamx, const double *lamy, const double2 *twx,
                         const double2 *twy, const double *Sx, const double *Sy, const double *f,
                         double *u, double *t1, cudaStream_t s) {
    March2D M;
    M.g = g;
    M.b = b;
    M.cx = cx;
    M.cy = cy;
    M.N2x = march2d_transform_size(g.nx);
    M.N2y = march2d_transform_size(g.ny);
    M.logx = 0;
    while ((1 << M.logx) < M.N2x) ++M.logx;
    M.logy = 0;
    while ((1 << M.logy) < M.N2y) ++M.logy;
    M.Sx = M.N2x ? nullptr : Sx;
    M.Sy = M.N2y ? nullptr : Sy;
    const size_t shx = march2d_smem_for(g.nx), shy = march2d_smem_for(g.ny);
    prof_begin(s);
    for (int k = 1; k <= g.nt; ++k) {
        k_march2d_rows<<<g.ny, M2_THREADS, shx, s>>>(M, k, f, u, t1, twx);
        k_march2d_cols<<<g.nx, M2_THREADS, shy, s>>>(M, a, t1, lamx, lamy, twy);
        k_march2d_out<<<g.ny, M2_THREADS, shx, s>>>(M, k, t1, u, twx);
    }
    prof_end(s, PROF_MARCH, 3.0 * 8.0 * (double)g.interior());
    count_launch(3 * g.nt);
}

}  // namespace mk
