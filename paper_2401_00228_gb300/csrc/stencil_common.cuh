// Helpers shared by the space-time stencil kernels (see stencil.cu).
#pragma once

#include "kernels.h"
#include "rounding.cuh"

namespace mk {

// ---------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------
// load an element in the arithmetic type; a double-float pair (float2) is read as its
// leading float (the value rounded to FP32)
// conversions used by the layout kernels; a double becomes a double-float pair (hi, lo)
template <typename Td, typename Ts>
__device__ __forceinline__ Td cvt_to(Ts v) {
    return (Td)v;
}
template <>
__device__ __forceinline__ float2 cvt_to<float2, double>(double v) {
    float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
template <>
__device__ __forceinline__ double cvt_to<double, float2>(float2 v) {
    return (double)v.x + (double)v.y;
}

// A device FP64 scalar (may be null: 1) in the arithmetic type, converted once per block: a
// double -> float conversion issues at GB300's FP64 rate, so per thread it costs as much as
// the rest of a short kernel's arithmetic.  Every thread of the block must call it.
template <typename T>
__device__ __forceinline__ T block_scalar(const double *p) {
    __shared__ T s_scalar;
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) s_scalar = p ? (T)(*p) : (T)1;
    __syncthreads();
    return s_scalar;
}

template <typename Tc, typename T>
__device__ __forceinline__ Tc ldv(const T *__restrict__ p, int64_t i) {
    return (Tc)p[i];
}
template <>
__device__ __forceinline__ float ldv<float, float2>(const float2 *__restrict__ p, int64_t i) {
    return p[i].x;
}

template <int DIM, typename Tc, typename Tin>
__device__ __forceinline__ Tc lap_at(const Tin *__restrict__ x, int64_t idx, int i, int j,
                                     const Geom &g, const Tc *__restrict__ cx,
                                     const Tc *__restrict__ cy) {
    Tc v = ldv<Tc>(x, idx);
    Tc s = cx[g.nx + i] * v + cx[i] * ldv<Tc>(x, idx - 1) + cx[2 * g.nx + i] * ldv<Tc>(x, idx + 1);
    if (DIM == 2) {
        Tc sy = cy[g.ny + j] * v + cy[j] * ldv<Tc>(x, idx - g.ldx) + cy[2 * g.ny + j] * ldv<Tc>(x, idx + g.ldx);
        s = s + sy;
    }
    return s;
}

static inline int choose_kc(int64_t npts, int nsteps) {
    // enough threads to fill the GPU a few times over; at most 32 steps per thread, and
    // never more than 60000 blocks in a launch (the reduction partials hold 65536)
    int64_t target = (int64_t)g_num_sms * 2048;
    int64_t kc = (npts * nsteps) / (target > 0 ? target : 1);
    if (kc < 1) kc = 1;
    if (kc > 32) kc = 32;
    int64_t blocks_per_chunk = (npts + 255) / 256 + 1;
    while (blocks_per_chunk * ((nsteps + kc - 1) / kc) > 60000) ++kc;
    return (int)kc;
}

struct Launch2 {
    dim3 grid, block;
};

// thread -> spatial point (i, j); block/grid cover (nx, ny) x chunks
static inline Launch2 point_launch(int dim, int nx, int ny, int nchunks) {
    Launch2 L;
    if (dim == 1) {
        int bx = nx >= 256 ? 256 : ((nx + 31) / 32) * 32;
        L.block = dim3(bx, 1, 1);
        L.grid = dim3((nx + bx - 1) / bx, nchunks, 1);
    } else {
        L.block = dim3(32, 8, 1);
        L.grid = dim3((nx + 31) / 32, (ny + 7) / 8, nchunks);
    }
    return L;
}

// Smallest chunk depth >= kc for which the point_launch grid over nsteps steps has at most
// 60000 blocks (the reduction partials hold 65536; this also keeps a 2D grid's z extent in
// range).  choose_kc estimates the blocks per chunk from the point count, which undercounts
// thin 2D grids (32 x 8 blocks); this counts them exactly.
static inline int cap_kc(int kc, int nsteps, int dim, int nx, int ny) {
    const Launch2 one = point_launch(dim, nx, ny, 1);
    const int64_t per = (int64_t)one.grid.x * one.grid.y;
    if (kc < 1) kc = 1;
    const int64_t need = (per * (int64_t)nsteps + 59999) / 60000;
    if (need > kc) kc = (int)need;
    while (per * (((int64_t)nsteps + kc - 1) / kc) > 60000) ++kc;
    return kc;
}

template <int DIM>
__device__ __forceinline__ bool point_index(int &i, int &j, int &chunk) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    if (DIM == 1) {
        j = 0;
        chunk = blockIdx.y;
    } else {
        j = blockIdx.y * blockDim.y + threadIdx.y;
        chunk = blockIdx.z;
    }
    return true;
}


// 2D interpolation + correction, element-wise: x_k = sigma v_k - (Z vt)_{K(k)}, K(0) = 0,
// K(k) = (k-1)/nu + 1, vt = sum_m y_m Xc_m (Xc itself when yc is null); aggregates of Z are
// 2 x 2 with SPACE.  A thread takes four consecutive points of one row (16-byte stores of x,
// 16-byte loads of v); blocks are 32 x 8 threads over (i / 4, j), blockIdx.z = k.  Each x is
// formed once; w = A x follows in a separate stencil kernel that reads x back.  A row holds
// ldx >= nx + 1 elements with ldx a multiple of 8, so the four points of a thread whose first
// point is interior stay inside the row (points beyond nx are written as 0, the padding).
template <typename Tv, typename Tx>
__device__ __forceinline__ Tx x2d_vload(const Tv *p) { return (Tx)*p; }
template <>
__device__ __forceinline__ float x2d_vload<float2, float>(const float2 *p) { return p->x; }

// the four values v[0..3] (16-byte aligned: the first point's index is a multiple of 4) as
// the arithmetic type; a double-float element contributes its leading float
template <typename Tv, typename Tx>
__device__ __forceinline__ void x2d_vload4(const Tv *p, Tx (&o)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = x2d_vload<Tv, Tx>(p + q);
}
template <>
__device__ __forceinline__ void x2d_vload4<float2, float>(const float2 *p, float (&o)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 2);
    o[0] = a.x; o[1] = a.z; o[2] = b.x; o[3] = b.z;
}
template <>
__device__ __forceinline__ void x2d_vload4<float, float>(const float *p, float (&o)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
template <typename Tx>
__device__ __forceinline__ void x2d_store4(Tx *p, const Tx (&o)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = o[q];
}
template <>
__device__ __forceinline__ void x2d_store4<float>(float *p, const float (&o)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
}

template <bool SPACE, typename Tv, typename Tz, typename Tx>
__global__ void __launch_bounds__(256) k_interp_x2d(Geom gf, Geom gc, int nu,
                                                    const Tv *__restrict__ v,
                                                    const double *__restrict__ sigma,
                                                    const Tz *__restrict__ Xc, int mc,
                                                    int64_t xc_stride,
                                                    const double *__restrict__ yc,
                                                    Tx *__restrict__ x,
                                                    const int *__restrict__ done) {
    if (done && *done) return;   // the same flag for every thread of the block
    // sigma and the coarse weights y_m, converted once per block (a double -> float
    // conversion issues at the FP64 rate)
    __shared__ Tx s_w[MK_MAX_INNER + 1];
    const int nm = yc ? (mc < MK_MAX_INNER ? mc : MK_MAX_INNER) : 0;
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    if (t == 0) s_w[0] = sigma ? (Tx)(*sigma) : (Tx)1;
    else if (t <= nm) s_w[t] = (Tx)yc[t - 1];
    __syncthreads();
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i0 >= gf.nx || j >= gf.ny) return;
    const int K = (k == 0) ? 0 : (k - 1) / nu + 1;
    const int J = SPACE ? (j >> 1) : j;
    const Tz *crow = Xc + gc.at(K, J, 0);
    const Tx sig = s_w[0];
    const int64_t idx = gf.at(k, j, i0);
    Tx vin[4], out[4];
    x2d_vload4<Tv, Tx>(v + idx, vin);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + p;
        const int I = SPACE ? (i >> 1) : i;
        Tx zt = (Tx)0;
        if (i < gf.nx) {
            if (!yc) {
                zt = (Tx)crow[I];
            } else {
                for (int m = 0; m < nm; ++m) zt = fma_rn(s_w[1 + m], (Tx)crow[I + m * xc_stride], zt);
            }
        }
        out[p] = (i < gf.nx) ? fma_rn(sig, vin[p], -zt) : (Tx)0;
    }
    x2d_store4<Tx>(x + idx, out);
}

// one point per thread (32 x 8 blocks) / four points per thread (k_interp_x2d)
inline dim3 grid_2d_points(const Geom &g) {
    return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nt + 1);
}
inline dim3 grid_2d_points4(const Geom &g) {
    return dim3((g.nx + 127) / 128, (g.ny + 7) / 8, g.nt + 1);
}

static inline int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)g_num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace mk
