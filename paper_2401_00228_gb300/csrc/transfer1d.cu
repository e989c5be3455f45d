// Time-tiled 1D transfer kernels for time coarsening factor nu = 2:
//   * restriction with shift, vhat = sigma Y^T (A v - mu v)   (Sec. 3.1 substeps 4.1-4.2),
//   * interpolation + correction + matvec, x = sigma v - Z vt, w = A x
//     (substeps 4.4-4.5 fused with step 5 of Algorithm 2),
// with optional pair agglomeration in space (Case 2 "TS", Eqs. (constructZ)/(constructY)).
//
// Each thread owns four consecutive spatial points and a chunk of KC output time steps.
// Every row the chunk needs is loaded before any is used (16-byte vector loads), so a thread
// keeps 2 KC + 1 (restriction) or KC + 1 (interpolation) independent loads in flight rather
// than walking the time axis one dependent load at a time; the x_{k-1} row and its Laplacian
// stay in registers.  Spatial neighbours come from the adjacent lanes by warp shuffles; the
// two warp-edge lanes load theirs directly.  A thread's four points start at a multiple of 4
// and the padded row length is a multiple of 8, so a thread that owns an interior point
// never reads past the end of its row; points beyond n_x are the zero padding.
#include "kernels.h"
#include "reduce.cuh"
#include "stencil_common.cuh"
#include "df64.cuh"

namespace mk {

namespace {

constexpr int TT = 128;   // threads per block
constexpr int PT = 4;     // spatial points per thread
constexpr unsigned FULL = 0xffffffffu;

// ---- loads of 4 (or 2) consecutive elements, converted to the arithmetic type --------------
template <typename Tc>
__device__ __forceinline__ void ld4(const float *p, Tc (&o)[4]) {
    const float4 f = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = (Tc)f.x; o[1] = (Tc)f.y; o[2] = (Tc)f.z; o[3] = (Tc)f.w;
}
template <typename Tc>
__device__ __forceinline__ void ld4(const double *p, Tc (&o)[4]) {
    const double2 u = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 w = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = (Tc)u.x; o[1] = (Tc)u.y; o[2] = (Tc)w.x; o[3] = (Tc)w.y;
}
// a double-float pair is read as its leading float (the value rounded to FP32)
template <typename Tc>
__device__ __forceinline__ void ld4(const float2 *p, Tc (&o)[4]) {
    const float4 u = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 w = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    o[0] = (Tc)u.x; o[1] = (Tc)u.z; o[2] = (Tc)w.x; o[3] = (Tc)w.z;
}
template <typename Tc>
__device__ __forceinline__ void ld2(const float *p, Tc (&o)[2]) {
    const float2 f = __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = (Tc)f.x; o[1] = (Tc)f.y;
}
template <typename Tc>
__device__ __forceinline__ void ld2(const double *p, Tc (&o)[2]) {
    const double2 f = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = (Tc)f.x; o[1] = (Tc)f.y;
}
template <typename Tc, typename T>
__device__ __forceinline__ Tc ld1(const T *p) { return (Tc)__ldg(p); }
template <>
__device__ __forceinline__ float ld1<float, float2>(const float2 *p) { return __ldg(p).x; }
template <>
__device__ __forceinline__ double ld1<double, float2>(const float2 *p) { return (double)__ldg(p).x; }

// ---- stores ----------------------------------------------------------------------------------
template <typename Tc>
__device__ __forceinline__ void st4(float *p, const Tc (&o)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
}
template <typename Tc>
__device__ __forceinline__ void st4(double *p, const Tc (&o)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2((double)o[0], (double)o[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2((double)o[2], (double)o[3]);
}
template <typename Tc>
__device__ __forceinline__ void st2(float *p, const Tc (&o)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2((float)o[0], (float)o[1]);
}
template <typename Tc>
__device__ __forceinline__ void st2(double *p, const Tc (&o)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2((double)o[0], (double)o[1]);
}

// Laplacian of a thread's four points; left/right are the values just outside them.
template <typename Tc>
__device__ __forceinline__ void lap4(const Tc (&c)[4], Tc left, Tc right, const Tc (&lo)[4],
                                     const Tc (&di)[4], const Tc (&up)[4], Tc (&l)[4]) {
    l[0] = di[0] * c[0] + lo[0] * left + up[0] * c[1];
    l[1] = di[1] * c[1] + lo[1] * c[0] + up[1] * c[2];
    l[2] = di[2] * c[2] + lo[2] * c[1] + up[2] * c[3];
    l[3] = di[3] * c[3] + lo[3] * c[2] + up[3] * right;
}

template <typename Tc>
__device__ __forceinline__ void load_coefs(const Tc *cx, int nf, int i0, Tc (&lo)[4], Tc (&di)[4],
                                           Tc (&up)[4]) {
#pragma unroll
    for (int p = 0; p < PT; ++p) {
        const int i = i0 + p;
        const bool in = i < nf;
        lo[p] = in ? cx[i] : (Tc)0;
        di[p] = in ? cx[nf + i] : (Tc)0;
        up[p] = in ? cx[2 * nf + i] : (Tc)0;
    }
}

// ---------------------------------------------------------------------------------------
// Restriction.  Chunk of coarse steps K0 .. K0+KC-1 reads fine rows 2(K0-1) .. 2(K0-1)+2KC
// (row r is fine step 2(K0-1)+r; the first chunk starts at -2, rows that do not exist read 0).
//   K = 0:  vhat_0 = sigma Y^T (v_0 - mu v_0)
//   K >= 1: vhat_K = sigma Y^T sum_{st=1,2} [(A v)_{2(K-1)+st} - mu v_{2(K-1)+st}]
// ---------------------------------------------------------------------------------------
template <bool SPACE, int KC, typename Tin, typename Tout, typename Tc>
__global__ void __launch_bounds__(TT) k_restrict_1d_t(Geom gf, Geom gc, Tc a, Tc b, Tc mu,
                                                      SpaceOp<Tc> L, const Tin *__restrict__ v,
                                                      const double *__restrict__ sigma,
                                                      Tout *__restrict__ vhat, ReduceScratch rs,
                                                      int slot, KState ks,
                                                      const int *__restrict__ done) {
    if (done && *done) return;
    constexpr int R = 2 * KC + 1;
    const int lane = threadIdx.x & 31;
    const int i0 = PT * (blockIdx.x * TT + threadIdx.x);
    const int nf = gf.nx;
    const bool act = i0 < nf;
    const int K0 = blockIdx.y * KC;
    const int kb = 2 * (K0 - 1);
    Tc c[R][PT], eL[R], eR[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int kf = kb + r;
        const bool ok = act && kf >= 0 && kf <= gf.nt;
        const Tin *row = v + gf.guard + (int64_t)(ok ? kf : 0) * gf.plane;
        if (ok) {
            ld4(row + i0, c[r]);
        } else {
#pragma unroll
            for (int p = 0; p < PT; ++p) c[r][p] = (Tc)0;
        }
        eL[r] = (ok && lane == 0 && i0 > 0) ? ld1<Tc>(row + i0 - 1) : (Tc)0;
        eR[r] = (ok && lane == 31 && i0 + PT < nf) ? ld1<Tc>(row + i0 + PT) : (Tc)0;
    }
    Tc lo[PT], di[PT], up[PT];
    load_coefs(L.x, nf, i0, lo, di, up);
    auto lap = [&](int r, Tc (&l)[PT]) {
        Tc left = __shfl_up_sync(FULL, c[r][PT - 1], 1);
        Tc right = __shfl_down_sync(FULL, c[r][0], 1);
        if (lane == 0) left = eL[r];
        if (lane == 31) right = eR[r];
        lap4(c[r], left, right, lo, di, up, l);
    };
    const Tc scale = block_scalar<Tc>(sigma);
    const int nK = gc.nt + 1 - K0;
    // the norm of vhat for the next level's beta: summed per thread and per warp in the
    // arithmetic type (FP64 per element would run at the FP64 rate, 1/58 of FP32 here), in FP64
    // across warps
    Tc acc2 = (Tc)0;
    Tc lp[PT];
    lap(0, lp);
#pragma unroll
    for (int q = 0; q < KC; ++q) {
        Tc l1[PT], l2[PT];
        lap(2 * q + 1, l1);
        lap(2 * q + 2, l2);
        Tc t1[PT], t2[PT];   // (A v - mu v) at the two fine steps of coarse step K0 + q
#pragma unroll
        for (int p = 0; p < PT; ++p) {
            if (K0 + q == 0) {
                t1[p] = c[2][p] - mu * c[2][p];
                t2[p] = (Tc)0;
            } else {
                const Tc av1 = (c[2 * q + 1][p] - a * l1[p]) - (c[2 * q][p] + b * lp[p]);
                const Tc av2 = (c[2 * q + 2][p] - a * l2[p]) - (c[2 * q + 1][p] + b * l1[p]);
                t1[p] = av1 - mu * c[2 * q + 1][p];
                t2[p] = av2 - mu * c[2 * q + 2][p];
            }
            lp[p] = l2[p];
        }
        if (q < nK && act) {
            const int K = K0 + q;
            if (SPACE) {
                Tc o[2];
#pragma unroll
                for (int P = 0; P < 2; ++P) {
                    const int I = i0 / 2 + P;
                    Tc sum = (K == 0) ? (t1[2 * P] + t1[2 * P + 1])
                                      : (((t1[2 * P] + t1[2 * P + 1]) + t2[2 * P]) + t2[2 * P + 1]);
                    const Tc inv = (2 * I + 1 < nf) ? (Tc)0.5 : (Tc)1;
                    o[P] = (I < gc.nx) ? scale * (sum * inv) : (Tc)0;
                    acc2 += o[P] * o[P];
                }
                st2(vhat + gc.guard + (int64_t)K * gc.plane + i0 / 2, o);
            } else {
                Tc o[PT];
#pragma unroll
                for (int p = 0; p < PT; ++p) {
                    Tc sum = (K == 0) ? t1[p] : t1[p] + t2[p];
                    o[p] = (i0 + p < nf) ? scale * sum : (Tc)0;
                    acc2 += o[p] * o[p];
                }
                st4(vhat + gc.guard + (int64_t)K * gc.plane + i0, o);
            }
        }
    }
    if (ks.d) block_partial_and_finish_t(acc2, rs, slot, ks, EPI_BETA);
}

// ---------------------------------------------------------------------------------------
// Interpolation + correction + matvec.  Chunk of fine steps k0 .. k0+KC-1 (KC even, so k0
// is even) uses fine rows k0-1 .. k0+KC-1 (row r is step k0-1+r) and coarse rows
// k0/2 .. k0/2+KC/2: the coarse block of fine step k0-1+r is k0/2 + r/2.
//   x_k = sigma v_k - (Z vt)_k,  vt = sum_m y_m Xc_m (or Xc itself when yc is null),
//   w_0 = x_0,  w_k = (x_k - a L x_k) - (x_{k-1} + b L x_{k-1}).
// ---------------------------------------------------------------------------------------
template <bool SPACE, int MC, int KC, typename Tz, typename Tx>
struct CoarseRows {
    static constexpr int RC = KC / 2 + 1;
    static constexpr int PC = SPACE ? PT / 2 : PT;
    static constexpr int NY = MC > 0 ? MC : MK_MAX_INNER;
    Tx z[RC][PC], zl[RC], zr[RC];

    // z = sum_m y_m Xc_m at the thread's coarse points (and the edge neighbours)
    __device__ __forceinline__ void load(const Geom &gc, const Tz *__restrict__ Xc, int mc,
                                         int64_t xc_stride, const Tx (&y)[NY], int Kb, int i0,
                                         int nf, bool act, int lane) {
        const int I0 = SPACE ? i0 / 2 : i0;
        const int Il = SPACE ? I0 - 1 : i0 - 1;       // coarse point of fine i0 - 1
        const int Ir = SPACE ? I0 + 2 : i0 + PT;      // coarse point of fine i0 + 4
        const bool wl = act && lane == 0 && i0 > 0;
        const bool wr = act && lane == 31 && i0 + PT < nf;
#pragma unroll
        for (int rc = 0; rc < RC; ++rc) {
            const int K = Kb + rc;
            const bool ok = act && K <= gc.nt;
            const Tz *crow = Xc + gc.guard + (int64_t)(ok ? K : 0) * gc.plane;
#pragma unroll
            for (int p = 0; p < PC; ++p) z[rc][p] = (Tx)0;
            zl[rc] = (Tx)0;
            zr[rc] = (Tx)0;
            if (!ok) continue;
            constexpr int NM = MC == 0 ? 1 : NY;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                if (MC < 0 && m >= mc) break;
                const Tz *cm = crow + (int64_t)m * xc_stride;
                const Tx ym = (MC == 0) ? (Tx)1 : y[m];
                Tx t[PC];
                if constexpr (PC == 4) ld4(cm + I0, t);
                else ld2(cm + I0, t);
#pragma unroll
                for (int p = 0; p < PC; ++p) z[rc][p] = (m == 0) ? mul_rn(ym, t[p]) : fma_rn(ym, t[p], z[rc][p]);
                if (wl) zl[rc] = (m == 0) ? mul_rn(ym, ld1<Tx>(cm + Il)) : fma_rn(ym, ld1<Tx>(cm + Il), zl[rc]);
                if (wr) zr[rc] = (m == 0) ? mul_rn(ym, ld1<Tx>(cm + Ir)) : fma_rn(ym, ld1<Tx>(cm + Ir), zr[rc]);
            }
        }
    }
};

template <bool SPACE, int MC, int KC, typename Tv, typename Tz, typename Tx, typename Tw,
          typename Tc>
__global__ void __launch_bounds__(TT) k_interp_1d_t(Geom gf, Geom gc, Tc a, Tc b, SpaceOp<Tc> L,
                                                    const Tv *__restrict__ v,
                                                    const double *__restrict__ sigma,
                                                    const Tz *__restrict__ Xc, int mc,
                                                    int64_t xc_stride,
                                                    const double *__restrict__ yc,
                                                    Tx *__restrict__ xout, Tw *__restrict__ wout,
                                                    const int *__restrict__ done) {
    if (done && *done) return;
    constexpr int R = KC + 1;
    using CR = CoarseRows<SPACE, MC, KC, Tz, Tx>;
    const int lane = threadIdx.x & 31;
    const int i0 = PT * (blockIdx.x * TT + threadIdx.x);
    const int nf = gf.nx;
    const bool act = i0 < nf;
    const int k0 = blockIdx.y * KC;
    // sigma and the coarse weights, converted once per block
    __shared__ Tx s_w[CR::NY + 1];
    if (threadIdx.x == 0) s_w[0] = sigma ? (Tx)(*sigma) : (Tx)1;
    else if (threadIdx.x <= CR::NY)
        s_w[threadIdx.x] = (yc && (int)threadIdx.x - 1 < mc) ? (Tx)yc[threadIdx.x - 1] : (Tx)0;
    __syncthreads();
    Tx y[CR::NY];
#pragma unroll
    for (int m = 0; m < CR::NY; ++m) y[m] = s_w[1 + m];
    const Tx sig = s_w[0];
    // fine rows
    Tx vv[R][PT], vl[R], vr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = k0 - 1 + r;
        const bool ok = act && k >= 0 && k <= gf.nt;
        const Tv *row = v + gf.guard + (int64_t)(ok ? k : 0) * gf.plane;
        if (ok) {
            ld4(row + i0, vv[r]);
        } else {
#pragma unroll
            for (int p = 0; p < PT; ++p) vv[r][p] = (Tx)0;
        }
        vl[r] = (ok && lane == 0 && i0 > 0) ? ld1<Tx>(row + i0 - 1) : (Tx)0;
        vr[r] = (ok && lane == 31 && i0 + PT < nf) ? ld1<Tx>(row + i0 + PT) : (Tx)0;
    }
    CR cr;
    cr.load(gc, Xc, mc, xc_stride, y, k0 / 2, i0, nf, act, lane);
    Tc lo[PT], di[PT], up[PT];
    load_coefs(L.x, nf, i0, lo, di, up);
    Tc xp[PT], lxp[PT];   // x and L x of the previous row
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = k0 - 1 + r;
        const bool ok = k >= 0 && k <= gf.nt;
        Tx x[PT];
#pragma unroll
        for (int p = 0; p < PT; ++p)
            x[p] = (ok && i0 + p < nf) ? fma_rn(sig, vv[r][p], -cr.z[r / 2][SPACE ? p / 2 : p]) : (Tx)0;
        Tx xl = __shfl_up_sync(FULL, x[PT - 1], 1), xr = __shfl_down_sync(FULL, x[0], 1);
        if (lane == 0) xl = (ok && i0 > 0) ? fma_rn(sig, vl[r], -cr.zl[r / 2]) : (Tx)0;
        if (lane == 31) xr = (ok && i0 + PT < nf) ? fma_rn(sig, vr[r], -cr.zr[r / 2]) : (Tx)0;
        Tc xc[PT], lx[PT];
#pragma unroll
        for (int p = 0; p < PT; ++p) xc[p] = (Tc)x[p];
        lap4(xc, (Tc)xl, (Tc)xr, lo, di, up, lx);
        if (r > 0 && ok && act) {
            Tc w[PT];
#pragma unroll
            for (int p = 0; p < PT; ++p)
                w[p] = (k == 0) ? xc[p] : (xc[p] - a * lx[p]) - (xp[p] + b * lxp[p]);
            const int64_t idx = gf.guard + (int64_t)k * gf.plane + i0;
            st4(xout + idx, x);
            st4(wout + idx, w);
        }
#pragma unroll
        for (int p = 0; p < PT; ++p) {
            xp[p] = xc[p];
            lxp[p] = lx[p];
        }
    }
}

// Mixed level 1: v is a double-float basis vector (read as its FP32 rounding), x is FP32
// and w = A x is formed in double-float from double-float coefficient rows a*L and b*L, so
// the FP32 x enters the FP64-accurate Arnoldi with only the rounding of the product terms.
// UNIFORM: L = c tridiag(1, -2, 1) (the fine level), a L x = (a c) (x_{i-1} - 2 x_i + x_{i+1})
// with the bracket exact and one double-float product (ca[0], cb[0] hold a c and b c);
// HAS_B = false drops the (I + b L) x_{k-1} stencil (theta = 1).
template <bool SPACE, int MC, int KC, bool UNIFORM, bool HAS_B>
__global__ void __launch_bounds__(TT) k_interp_df_1d_t(Geom gf, Geom gc,
                                                       const float2 *__restrict__ ca,
                                                       const float2 *__restrict__ cb, int has_b,
                                                       const float2 *__restrict__ v,
                                                       const double *__restrict__ sigma,
                                                       const float *__restrict__ Xc, int mc,
                                                       int64_t xc_stride,
                                                       const double *__restrict__ yc,
                                                       float *__restrict__ xout,
                                                       float2 *__restrict__ wout,
                                                       const int *__restrict__ done) {
    if (done && *done) return;
    constexpr int R = KC + 1;
    using CR = CoarseRows<SPACE, MC, KC, float, float>;
    const int lane = threadIdx.x & 31;
    const int i0 = PT * (blockIdx.x * TT + threadIdx.x);
    const int nf = gf.nx;
    const bool act = i0 < nf;
    const int k0 = blockIdx.y * KC;
    // sigma and the coarse weights, converted from FP64 once per block
    __shared__ float s_w[CR::NY + 1];
    if (threadIdx.x == 0) s_w[0] = sigma ? (float)(*sigma) : 1.f;
    else if (threadIdx.x <= CR::NY)
        s_w[threadIdx.x] = (yc && (int)threadIdx.x - 1 < mc) ? (float)yc[threadIdx.x - 1] : 0.f;
    __syncthreads();
    float y[CR::NY];
#pragma unroll
    for (int m = 0; m < CR::NY; ++m) y[m] = s_w[1 + m];
    const float sig = s_w[0];
    float vv[R][PT], vl[R], vr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = k0 - 1 + r;
        const bool ok = act && k >= 0 && k <= gf.nt;
        const float2 *row = v + gf.guard + (int64_t)(ok ? k : 0) * gf.plane;
        if (ok) {
            ld4(row + i0, vv[r]);
        } else {
#pragma unroll
            for (int p = 0; p < PT; ++p) vv[r][p] = 0.f;
        }
        vl[r] = (ok && lane == 0 && i0 > 0) ? ld1<float>(row + i0 - 1) : 0.f;
        vr[r] = (ok && lane == 31 && i0 + PT < nf) ? ld1<float>(row + i0 + PT) : 0.f;
    }
    CR cr;
    cr.load(gc, Xc, mc, xc_stride, y, k0 / 2, i0, nf, act, lane);
    const df z = {0.f, 0.f};
    (void)has_b;
    df alo[UNIFORM ? 1 : PT], adi[UNIFORM ? 1 : PT], aup[UNIFORM ? 1 : PT];
    df blo[UNIFORM || !HAS_B ? 1 : PT], bdi[UNIFORM || !HAS_B ? 1 : PT], bup[UNIFORM || !HAS_B ? 1 : PT];
    df ac = z, bc = z;
    if constexpr (UNIFORM) {
        ac = df_unpack(ca[0]);
        if constexpr (HAS_B) bc = df_unpack(cb[0]);
    } else {
#pragma unroll
        for (int p = 0; p < PT; ++p) {
            const int i = i0 + p;
            const bool in = i < nf;
            alo[p] = in ? df_unpack(ca[i]) : z;
            adi[p] = in ? df_unpack(ca[nf + i]) : z;
            aup[p] = in ? df_unpack(ca[2 * nf + i]) : z;
            if constexpr (HAS_B) {
                blo[p] = in ? df_unpack(cb[i]) : z;
                bdi[p] = in ? df_unpack(cb[nf + i]) : z;
                bup[p] = in ? df_unpack(cb[2 * nf + i]) : z;
            }
        }
    }
    float xp[PT];
    df bLp[PT];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = k0 - 1 + r;
        const bool ok = k >= 0 && k <= gf.nt;
        float x[PT];
#pragma unroll
        for (int p = 0; p < PT; ++p)
            x[p] = (ok && i0 + p < nf) ? fma_rn(sig, vv[r][p], -cr.z[r / 2][SPACE ? p / 2 : p]) : 0.f;
        float xl = __shfl_up_sync(FULL, x[PT - 1], 1), xr = __shfl_down_sync(FULL, x[0], 1);
        if (lane == 0) xl = (ok && i0 > 0) ? fma_rn(sig, vl[r], -cr.zl[r / 2]) : 0.f;
        if (lane == 31) xr = (ok && i0 + PT < nf) ? fma_rn(sig, vr[r], -cr.zr[r / 2]) : 0.f;
        df aL[PT], bL[PT];
#pragma unroll
        for (int p = 0; p < PT; ++p) {
            const float left = p == 0 ? xl : x[p - 1];
            const float right = p == PT - 1 ? xr : x[p + 1];
            if constexpr (UNIFORM) {
                // points beyond n_x have x = 0 and neighbours 0 or x_{n-1}: mask them
                const df t = lap3_exact(left, x[p], right);
                const bool in = i0 + p < nf;
                aL[p] = in ? df_mul(ac, t) : z;
                bL[p] = (HAS_B && in) ? df_mul(bc, t) : z;
            } else {
                aL[p] = df_add(df_add(df_mul_f(adi[p], x[p]), df_mul_f(alo[p], left)),
                               df_mul_f(aup[p], right));
                if constexpr (HAS_B)
                    bL[p] = df_add(df_add(df_mul_f(bdi[p], x[p]), df_mul_f(blo[p], left)),
                                   df_mul_f(bup[p], right));
                else
                    bL[p] = z;
            }
        }
        if (r > 0 && ok && act) {
            float2 w[PT];
#pragma unroll
            for (int p = 0; p < PT; ++p) {
                const df wk = (k == 0) ? df_from_float(x[p])
                                       : df_sub(df_sub(df_from_sum(x[p], -xp[p]), aL[p]), bLp[p]);
                w[p] = df_pack(wk);
            }
            const int64_t idx = gf.guard + (int64_t)k * gf.plane + i0;
            st4(xout + idx, x);
            float4 *wo = reinterpret_cast<float4 *>(wout + idx);
            wo[0] = make_float4(w[0].x, w[0].y, w[1].x, w[1].y);
            wo[1] = make_float4(w[2].x, w[2].y, w[3].x, w[3].y);
        }
#pragma unroll
        for (int p = 0; p < PT; ++p) {
            xp[p] = x[p];
            bLp[p] = bL[p];
        }
    }
}

// Steps per thread: the largest of {4, 2, 1} (interpolation {4, 2}) that still launches
// eight 4-warp blocks per SM.  These kernels are latency-bound chains of loads, shuffles
// and FMAs; fewer steps per thread and more resident warps hide the latency better than
// longer chains do (measured: at 13 resident warps per SM, KC = 4 ran twice as long as
// KC = 2 on the same number of blocks).
inline int tiled_kc(int xb, int rows, bool allow1) {
    int kc = 4;
    const int lo = allow1 ? 1 : 2;
    while (kc > lo && (int64_t)xb * ((rows + kc - 1) / kc) < 8 * (int64_t)g_num_sms) kc /= 2;
    return kc;
}

// tile depths chosen by the autotuner for the level being enqueued (0: heuristic)
thread_local int t_kc_restrict = 0;
thread_local int t_kc_interp = 0;

}  // namespace

void set_tile_hint(int kc_restrict, int kc_interp) {
    t_kc_restrict = kc_restrict;
    t_kc_interp = kc_interp;
}

template <typename Tin, typename Tout, typename Tc>
bool launch_restrict_1d_tiled(const Geom &gf, const Geom &gc, int nu, bool space,
                              const Weights &w, SpaceOp<Tc> L, const Tin *v, const double *sigma,
                              Tout *vhat, const ReduceScratch &rs, int slot, KState ks_c,
                              const int *done, cudaStream_t s) {
    if (gf.dim != 1 || nu != 2) return false;
    const int xb = (gf.nx + TT * PT - 1) / (TT * PT);
    const int rows = gc.nt + 1;
    const int h = t_kc_restrict;
    const int kc = (h == 1 || h == 2 || h == 4 || h == 8) ? h : tiled_kc(xb, rows, true);
    const int yb = (rows + kc - 1) / kc;
    if (ks_c.d && (int64_t)xb * yb > rs.max_blocks) return false;
    const dim3 grid(xb, yb);
    const Tc a = (Tc)w.a, b = (Tc)w.b, mu = (Tc)w.mu;
#define MK_RT(S, K)                                                                       \
    k_restrict_1d_t<S, K, Tin, Tout, Tc><<<grid, TT, 0, s>>>(gf, gc, a, b, mu, L, v, sigma, \
                                                             vhat, rs, slot, ks_c, done)
    if (space) {
        if (kc == 8) MK_RT(true, 8); else if (kc == 4) MK_RT(true, 4); else if (kc == 2) MK_RT(true, 2); else MK_RT(true, 1);
    } else {
        if (kc == 8) MK_RT(false, 8); else if (kc == 4) MK_RT(false, 4); else if (kc == 2) MK_RT(false, 2); else MK_RT(false, 1);
    }
#undef MK_RT
    return true;
}

template <typename Tv, typename Tz, typename Tx, typename Tw, typename Tc>
bool launch_interp_1d_tiled(const Geom &gf, const Geom &gc, int nu, bool space, const Weights &w,
                            SpaceOp<Tc> L, const Tv *v, const double *sigma, const Tz *Xc,
                            int mc, int64_t xc_stride, const double *yc, Tx *x, Tw *wout,
                            const int *done, cudaStream_t s) {
    if (gf.dim != 1 || nu != 2) return false;
    const int xb = (gf.nx + TT * PT - 1) / (TT * PT);
    const int rows = gf.nt + 1;
    const int h = t_kc_interp;
    const int kc = (h == 2 || h == 4) ? h : tiled_kc(xb, rows, false);
    const dim3 grid(xb, (rows + kc - 1) / kc);
    const Tc a = (Tc)w.a, b = (Tc)w.b;
#define MK_IT(S, M, K)                                                                        \
    k_interp_1d_t<S, M, K, Tv, Tz, Tx, Tw, Tc><<<grid, TT, 0, s>>>(gf, gc, a, b, L, v, sigma,   \
                                                                   Xc, mc, xc_stride, yc, x,  \
                                                                   wout, done)
#define MK_IT_K(S, M) \
    do { if (kc == 4) MK_IT(S, M, 4); else MK_IT(S, M, 2); } while (0)
#define MK_IT_M(S)                                       \
    do {                                                 \
        if (!yc) MK_IT_K(S, 0);                          \
        else if (mc == 1) MK_IT_K(S, 1);                 \
        else if (mc == 2) MK_IT_K(S, 2);                 \
        else MK_IT_K(S, -1);                             \
    } while (0)
    if (space) MK_IT_M(true); else MK_IT_M(false);
#undef MK_IT_M
#undef MK_IT_K
#undef MK_IT
    return true;
}

bool launch_interp_df_1d_tiled(const Geom &gf, const Geom &gc, int nu, bool space,
                               const float2 *ca, const float2 *cb, bool has_b, const float2 *v,
                               const double *sigma, const float *Xc, int mc, int64_t xc_stride,
                               const double *yc, float *x, float2 *wout, const int *done,
                               cudaStream_t s, const float2 *uniform_ab) {
    if (gf.dim != 1 || nu != 2) return false;
    const int xb = (gf.nx + TT * PT - 1) / (TT * PT);
    const int rows = gf.nt + 1;
    const int h = t_kc_interp;
    const int kc = (h == 2 || h == 4) ? h : tiled_kc(xb, rows, false);
    const dim3 grid(xb, (rows + kc - 1) / kc);
    const int hb = has_b ? 1 : 0;
    // uniform fine-level operator: ca[0], cb[0] of the kernel are a c and b c
    const bool uni = uniform_ab != nullptr;
    const float2 *ka = uni ? uniform_ab : ca, *kb = uni ? uniform_ab + 1 : cb;
#define MK_ID(S, M, K)                                                                        \
    do {                                                                                      \
        if (uni && hb)                                                                        \
            k_interp_df_1d_t<S, M, K, true, true><<<grid, TT, 0, s>>>(                        \
                gf, gc, ka, kb, hb, v, sigma, Xc, mc, xc_stride, yc, x, wout, done);          \
        else if (uni)                                                                         \
            k_interp_df_1d_t<S, M, K, true, false><<<grid, TT, 0, s>>>(                       \
                gf, gc, ka, kb, hb, v, sigma, Xc, mc, xc_stride, yc, x, wout, done);          \
        else if (hb)                                                                          \
            k_interp_df_1d_t<S, M, K, false, true><<<grid, TT, 0, s>>>(                       \
                gf, gc, ka, kb, hb, v, sigma, Xc, mc, xc_stride, yc, x, wout, done);          \
        else                                                                                  \
            k_interp_df_1d_t<S, M, K, false, false><<<grid, TT, 0, s>>>(                      \
                gf, gc, ka, kb, hb, v, sigma, Xc, mc, xc_stride, yc, x, wout, done);          \
    } while (0)
#define MK_ID_K(S, M) \
    do { if (kc == 4) MK_ID(S, M, 4); else MK_ID(S, M, 2); } while (0)
#define MK_ID_M(S)                                       \
    do {                                                 \
        if (!yc) MK_ID_K(S, 0);                          \
        else if (mc == 1) MK_ID_K(S, 1);                 \
        else if (mc == 2) MK_ID_K(S, 2);                 \
        else MK_ID_K(S, -1);                             \
    } while (0)
    if (space) MK_ID_M(true); else MK_ID_M(false);
#undef MK_ID_M
#undef MK_ID_K
#undef MK_ID
    return true;
}

#define MK_INST_R(Tin, Tout, Tc)                                                               \
    template bool launch_restrict_1d_tiled<Tin, Tout, Tc>(                                     \
        const Geom &, const Geom &, int, bool, const Weights &, SpaceOp<Tc>, const Tin *,      \
        const double *, Tout *, const ReduceScratch &, int, KState, const int *, cudaStream_t);
MK_INST_R(double, double, double)
MK_INST_R(double, float, float)
MK_INST_R(float2, float, float)
MK_INST_R(float, float, float)
#undef MK_INST_R

#define MK_INST_I(Tv, Tz, Tx, Tw, Tc)                                                          \
    template bool launch_interp_1d_tiled<Tv, Tz, Tx, Tw, Tc>(                                  \
        const Geom &, const Geom &, int, bool, const Weights &, SpaceOp<Tc>, const Tv *,       \
        const double *, const Tz *, int, int64_t, const double *, Tx *, Tw *, const int *,     \
        cudaStream_t);
MK_INST_I(double, double, double, double, double)
MK_INST_I(double, float, float, double, double)
MK_INST_I(float, float, float, float, float)
#undef MK_INST_I

}  // namespace mk
