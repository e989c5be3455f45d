// Level-1 kernels of the mixed-precision solve with the FGMRES basis in double-float pairs
// (see df64.cuh): the Arnoldi orthogonalisation of Algorithm 2 (classical Gram-Schmidt:
// multidot and update), the fused interpolation-correction-matvec of substeps 4.4-4.5 and
// step 5 with w = A x evaluated in double-float, and the true residual r = f - A u (FP64
// arithmetic, stored as a pair).  Storage is 8 bytes per element as in FP64, but the
// arithmetic runs on the FP32 pipe, so these kernels are bound by HBM rather than by
// GB300's FP64 rate.
#include "df64.cuh"
#include "kernels.h"
#include "krylov_epilogue.cuh"
#include "reduce.cuh"
#include "stencil_common.cuh"

namespace mk {

constexpr int DF_THREADS = 256;
constexpr int DF_WARPS = DF_THREADS / 32;
constexpr int DF_EPT = 16;
constexpr int DF_TILE = DF_THREADS * DF_EPT;

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df w;
        w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

// ---------------------------------------------------------------------------------------
// K2: r = f - A u in FP64; r stored as a double-float pair (the basis vector V_0 of the mixed
// solve) or rounded to FP32 (the FP32 level-1 basis)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void store_r(float2 *r, int64_t idx, double v) { r[idx] = df_pack(df_from_double(v)); }
__device__ __forceinline__ void store_r(float *r, int64_t idx, double v) { r[idx] = (float)v; }

template <int DIM, typename Tr>
__global__ void __launch_bounds__(256) k_residual_df(Geom g, double a, double b, SpaceOp<double> L,
                                                     const double *__restrict__ f,
                                                     const double *__restrict__ u,
                                                     Tr *__restrict__ r, int kc,
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
            store_r(r, idx, rv);
            acc += rv * rv;
            prev = cur;
            Lprev = Lc;
        }
    }
    block_partial_and_finish(acc, rs, slot, ks, epi);
}

template <typename Tr>
static void launch_residual_t(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                              const double *u, Tr *r, const ReduceScratch &rs, int slot, KState ks,
                              int epi, cudaStream_t s) {
    int kc = cap_kc(choose_kc(g.npts(), g.nt + 1), g.nt + 1, g.dim, g.nx, g.ny);
    int nch = (g.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(g.dim, g.nx, g.ny, nch);
    prof_begin(s);
    if (g.dim == 1)
        k_residual_df<1, Tr><<<l.grid, l.block, 0, s>>>(g, w.a, w.b, L, f, u, r, kc, rs, slot, ks, epi);
    else
        k_residual_df<2, Tr><<<l.grid, l.block, 0, s>>>(g, w.a, w.b, L, f, u, r, kc, rs, slot, ks, epi);
    prof_end(s, PROF_RESIDUAL, (double)g.interior() * (16.0 + sizeof(Tr)));
    count_launch();
}

void launch_residual_df(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                        const double *u, float2 *r, const ReduceScratch &rs, int slot, KState ks,
                        int epi, cudaStream_t s) {
    launch_residual_t<float2>(g, w, L, f, u, r, rs, slot, ks, epi, s);
}

void launch_residual_f32(const Geom &g, const Weights &w, SpaceOp<double> L, const double *f,
                         const double *u, float *r, const ReduceScratch &rs, int slot, KState ks,
                         int epi, cudaStream_t s) {
    launch_residual_t<float>(g, w, L, f, u, r, rs, slot, ks, epi, s);
}

// ---------------------------------------------------------------------------------------
// K4 (level 1, mixed): x = sigma v - Z vt in FP32, w = A x in double-float.
//   v: basis vector (pairs; its leading float is used), Xc: coarse FGMRES directions
//   (FP32) combined with yc on the fly.  The spatial operator enters as per-index
//   double-float coefficients a*L and b*L: aL = [lo|di|up] (x) then (y).
// ---------------------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ df lap_df(const float2 *__restrict__ cx, const float2 *__restrict__ cy,
                                     int nx, int ny, int i, int j, float c, float l, float r,
                                     float d, float u) {
    df s = df_mul_f(df_unpack(cx[nx + i]), c);
    s = df_add(s, df_mul_f(df_unpack(cx[i]), l));
    s = df_add(s, df_mul_f(df_unpack(cx[2 * nx + i]), r));
    if (DIM == 2) {
        s = df_add(s, df_mul_f(df_unpack(cy[ny + j]), c));
        s = df_add(s, df_mul_f(df_unpack(cy[j]), d));
        s = df_add(s, df_mul_f(df_unpack(cy[2 * ny + j]), u));
    }
    return s;
}

// w = A x in double-float, element-wise in 2D, for FP32 x (32 x 8 x 1 blocks over (i, j, k)):
// w_0 = x_0, w_k = (x_k - x_{k-1}) - a L x_k - b L x_{k-1} with double-float a L, b L rows.
__global__ void __launch_bounds__(256) k_apply_df_2d(Geom g, const float2 *__restrict__ ca,
                                                     const float2 *__restrict__ cb, int has_b,
                                                     const float *__restrict__ x,
                                                     float2 *__restrict__ w,
                                                     const int *__restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t idx = g.at(k, j, i);
    const float c = x[idx];
    df r;
    if (k == 0) {
        r = df_from_float(c);
    } else {
        const float2 *cax = ca, *cay = ca + 3 * g.nx;
        const df aL = lap_df<2>(cax, cay, g.nx, g.ny, i, j, c, x[idx - 1], x[idx + 1],
                                x[idx - g.ldx], x[idx + g.ldx]);
        const int64_t ip = idx - g.plane;
        const float p = x[ip];
        r = df_sub(df_from_sum(c, -p), aL);
        if (has_b) {
            const float2 *cbx = cb, *cby = cb + 3 * g.nx;
            r = df_sub(r, lap_df<2>(cbx, cby, g.nx, g.ny, i, j, p, x[ip - 1], x[ip + 1],
                                    x[ip - g.ldx], x[ip + g.ldx]));
        }
    }
    w[idx] = df_pack(r);
}

// The same for L = cx tridiag_x(1,-2,1) (+) cy tridiag_y(1,-2,1) (the fine level): each bracket
// exact, one double-float product per direction.  u = [a cx, b cx, a cy, b cy].
template <bool HAS_B>
__global__ void __launch_bounds__(256) k_apply_df_2d_uni(Geom g, const float2 *__restrict__ u,
                                                         const float *__restrict__ x,
                                                         float2 *__restrict__ w,
                                                         const int *__restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t idx = g.at(k, j, i);
    const float c = x[idx];
    df r;
    if (k == 0) {
        r = df_from_float(c);
    } else {
        const df acx = df_unpack(u[0]), acy = df_unpack(u[2]);
        const df aL = df_add(df_mul(acx, lap3_exact(x[idx - 1], c, x[idx + 1])),
                             df_mul(acy, lap3_exact(x[idx - g.ldx], c, x[idx + g.ldx])));
        const int64_t ip = idx - g.plane;
        const float p = x[ip];
        r = df_sub(df_from_sum(c, -p), aL);
        if (HAS_B) {
            const df bcx = df_unpack(u[1]), bcy = df_unpack(u[3]);
            r = df_sub(r, df_add(df_mul(bcx, lap3_exact(x[ip - 1], p, x[ip + 1])),
                                 df_mul(bcy, lap3_exact(x[ip - g.ldx], p, x[ip + g.ldx]))));
        }
    }
    w[idx] = df_pack(r);
}

// The same for cx == cy (a square grid): one five-point bracket per plane and one
// double-float product per time weight.  u = [a c, b c, a c, b c].
template <bool HAS_B>
__global__ void __launch_bounds__(256) k_apply_df_2d_sq(Geom g, const float2 *__restrict__ u,
                                                        const float *__restrict__ x,
                                                        float2 *__restrict__ w,
                                                        const int *__restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t idx = g.at(k, j, i);
    const float c = x[idx];
    df r;
    if (k == 0) {
        r = df_from_float(c);
    } else {
        const int64_t ip = idx - g.plane;
        const float p = x[ip];
        const df aL = df_mul(df_unpack(u[0]), lap5_df(x[idx - 1], x[idx + 1], x[idx - g.ldx],
                                                      x[idx + g.ldx], c));
        r = df_sub(df_from_sum(c, -p), aL);
        if (HAS_B)
            r = df_sub(r, df_mul(df_unpack(u[1]), lap5_df(x[ip - 1], x[ip + 1], x[ip - g.ldx],
                                                          x[ip + g.ldx], p)));
    }
    w[idx] = df_pack(r);
}

// 1D specialisation: x once per point, neighbours from the adjacent lanes, the point's
// double-float coefficients held in registers, row pointers and the coarse block index
// advanced once per step, the coarse combination specialised on its size MC (see the FP32
// version in stencil.cu).
template <bool SPACE, int MC>
__global__ void __launch_bounds__(256) k_interp_df_1d(Geom gf, Geom gc, int nu,
                                                      const float2 *__restrict__ ca,
                                                      const float2 *__restrict__ cb, int has_b,
                                                      const float2 *__restrict__ v,
                                                      const double *__restrict__ sigma,
                                                      const float *__restrict__ Xc, int mc,
                                                      int64_t xc_stride,
                                                      const double *__restrict__ yc,
                                                      float *__restrict__ xout,
                                                      float2 *__restrict__ wout, int kc,
                                                      const int *__restrict__ done) {
    if (done && *done) return;
    const unsigned FULL = 0xffffffffu;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int nx = gf.nx;
    const bool act = i < nx;
    const float sig = sigma ? (float)(*sigma) : 1.f;
    constexpr int NY = MC > 0 ? MC : MK_MAX_INNER;
    float y[NY];
#pragma unroll
    for (int m = 0; m < NY; ++m) y[m] = (yc && m < mc) ? (float)yc[m] : 0.f;
    const df z = {0.f, 0.f};
    const df alo = act ? df_unpack(ca[i]) : z, adi = act ? df_unpack(ca[nx + i]) : z,
             aup = act ? df_unpack(ca[2 * nx + i]) : z;
    const df blo = (act && has_b) ? df_unpack(cb[i]) : z,
             bdi = (act && has_b) ? df_unpack(cb[nx + i]) : z,
             bup = (act && has_b) ? df_unpack(cb[2 * nx + i]) : z;
    auto xval = [&](const float2 *vr, const float *zr, int ii) -> float {
        if (ii < 0 || ii >= nx) return 0.f;
        const float *zp = zr + (SPACE ? (ii >> 1) : ii);
        float zt;
        if (MC == 0) {
            zt = zp[0];
        } else if (MC == 1) {
            zt = mul_rn(y[0], zp[0]);
        } else if (MC == 2) {
            zt = fma_rn(y[NY > 1 ? 1 : 0], zp[xc_stride], mul_rn(y[0], zp[0]));
        } else {
            zt = 0.f;
#pragma unroll
            for (int m = 0; m < NY; ++m)
                if (m < mc) zt = fma_rn(y[m], zp[m * xc_stride], zt);
        }
        return fma_rn(sig, vr[ii].x, -zt);
    };
    const int k0 = blockIdx.y * kc;
    const int k1 = min(k0 + kc, gf.nt + 1);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    int K = (kstart == 0) ? 0 : (kstart - 1) / nu + 1;
    int ph = (kstart == 0) ? nu - 1 : (kstart - 1) % nu;
    float prev = 0.f;
    df bLprev = z;
    for (int k = kstart; k < k1; ++k) {
        if (k > kstart) {
            if (ph == nu - 1) {
                ++K;
                ph = 0;
            } else {
                ++ph;
            }
        }
        const float2 *vr = v + gf.guard + (int64_t)k * gf.plane;
        const float *zr = Xc + gc.guard + (int64_t)K * gc.plane;
        float c = xval(vr, zr, i);
        float l = __shfl_up_sync(FULL, c, 1), r = __shfl_down_sync(FULL, c, 1);
        if (lane == 0) l = xval(vr, zr, i - 1);
        if (lane == 31) r = xval(vr, zr, i + 1);
        df aL = df_add(df_add(df_mul_f(adi, c), df_mul_f(alo, l)), df_mul_f(aup, r));
        df bL = has_b ? df_add(df_add(df_mul_f(bdi, c), df_mul_f(blo, l)), df_mul_f(bup, r)) : z;
        if (k >= k0) {
            df w = (k == 0) ? df_from_float(c) : df_sub(df_sub(df_from_sum(c, -prev), aL), bLprev);
            if (act) {
                int64_t idx = gf.guard + (int64_t)k * gf.plane + i;
                xout[idx] = c;
                wout[idx] = df_pack(w);
            }
        }
        prev = c;
        bLprev = bL;
    }
}

// 2D K4 in double-float with 2 x 2 aggregates and a uniform fine operator, walked in time.
// A thread owns the aggregate (I, J): the fine points (2I, 2I+1) x (2J, 2J+1), which share
// one coarse value (Z vt)_{K(k)}.  Per fine step it forms x at those four points and at the
// two points of each adjacent row (2J-1 and 2J+2, from the aggregates J-1 and J+1); the
// columns 2I-1 and 2I+2 come from the neighbouring lanes by warp shuffles (the first and
// last lane form them itself).  The five-point sums S(x_{k-1}) stay in registers from the
// previous step, so x and w are written once per point and v is read once per point from
// HBM (the adjacent rows are the neighbouring threads' rows, served by the caches).  The
// global loads of step k+1 are issued before step k is computed.
//   w_0 = x_0,  w_k = (x_k - x_{k-1}) - [a c S(x_k) + b c S(x_{k-1})]    (SQ: cx = cy = c)
//   w_k = (x_k - x_{k-1}) - [a cx Sx(x_k) + b cx Sx(x_{k-1})] - [a cy Sy(x_k) + b cy Sy(x_{k-1})]
// in double-float (lap5_pair / lap3_exact, df_dot2, df_diff_sub); u = [a cx, b cx, a cy, b cy].
// MC: number of coarse directions combined, vt = sum_m y_m Xc_m (0: Xc itself).
// Row starts are multiples of eight elements and i0 is even, so the paired accesses are
// 16-byte (v, w) and 8-byte (x) aligned; a row is read only where it is interior.
__device__ __forceinline__ float4 ld_df_pair(const float2 *p) {
    return *reinterpret_cast<const float4 *>(p);
}

template <bool SQ, bool HAS_B, int MC>
__global__ void __launch_bounds__(256, 2) k_interp_df_2d_ts(Geom gf, Geom gc, int nu,
                                                            const float2 *__restrict__ u,
                                                            const float2 *__restrict__ v,
                                                            const double *__restrict__ sigma,
                                                            const float *__restrict__ Xc,
                                                            int64_t xc_stride,
                                                            const double *__restrict__ yc,
                                                            float *__restrict__ x,
                                                            float2 *__restrict__ w, int kc,
                                                            const int *__restrict__ done) {
    if (done && *done) return;   // the same flag for every thread of the block
    constexpr int NZ = MC > 0 ? MC : 1;
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
    if (j0 >= ny) return;   // the whole warp shares J
    const float sig = s_w[0];
    float ym[NZ];
#pragma unroll
    for (int m = 0; m < NZ; ++m) ym[m] = MC > 0 ? s_w[1 + m] : 1.f;
    const bool c0 = i0 < nx, c1 = i0 + 1 < nx, r1 = j0 + 1 < ny;
    const bool hd = c0 && j0 > 0, hu = c0 && j0 + 2 < ny;
    const bool cl = lane == 0 && i0 > 0 && i0 - 1 < nx, cr = lane == 31 && i0 + 2 < nx;
    const int64_t o0 = (int64_t)j0 * ldx + i0;   // fine offset of (2J, 2I) in a plane
    const int64_t oc = (int64_t)J * cld + I;      // coarse offset of (J, I)
    const int64_t oe = o0 + (cl ? -1 : 2);        // outside column of the first / last lane
    const int64_t oce = oc + (cl ? -1 : 1);
    const df ua = df_unpack(u[0]), ub = df_unpack(u[1]);
    const df uay = df_unpack(u[2]), uby = df_unpack(u[3]);
    // raw loads of one step
    const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 A0 = Z4, A1 = Z4, QD = Z4, QU = Z4;
    float ZO[NZ], ZD[NZ], ZU[NZ], ZE[NZ], VE0 = 0.f, VE1 = 0.f;
    auto load = [&](int k, int K) {
        const float2 *vk = v + gf.guard + (int64_t)k * gf.plane;
        const float *zk = Xc + gc.guard + (int64_t)K * gc.plane;
        A0 = c0 ? ld_df_pair(vk + o0) : Z4;
        A1 = (c0 && r1) ? ld_df_pair(vk + o0 + ldx) : Z4;
        QD = hd ? ld_df_pair(vk + o0 - ldx) : Z4;
        QU = hu ? ld_df_pair(vk + o0 + 2 * ldx) : Z4;
#pragma unroll
        for (int m = 0; m < NZ; ++m) {
            const float *zm = zk + (int64_t)m * xc_stride;
            ZO[m] = c0 ? zm[oc] : 0.f;
            ZD[m] = hd ? zm[oc - cld] : 0.f;
            ZU[m] = hu ? zm[oc + cld] : 0.f;
            ZE[m] = (cl || cr) ? zm[oce] : 0.f;
        }
        VE0 = (cl || cr) ? vk[oe].x : 0.f;
        VE1 = ((cl || cr) && r1) ? vk[oe + ldx].x : 0.f;
    };
    // (Z vt) from the raw coarse values
    auto comb = [&](const float (&zr)[NZ]) -> float {
        if (MC == 0) return zr[0];
        float z = mul_rn(ym[0], zr[0]);
#pragma unroll
        for (int m = 1; m < NZ; ++m) z = fma_rn(ym[m], zr[m], z);
        return z;
    };
    const int k0 = blockIdx.z * kc;
    const int k1 = min(k0 + kc, gf.nt + 1);
    const int kstart = k0 > 0 ? k0 - 1 : 0;
    // coarse block of fine step k: 0 for k = 0, (k-1)/nu + 1 otherwise (tracked incrementally)
    int K = (kstart == 0) ? 0 : (kstart - 1) / nu + 1;
    int ph = (kstart == 0) ? nu - 1 : (kstart - 1) % nu;
    float p00 = 0.f, p01 = 0.f, p10 = 0.f, p11 = 0.f;   // x_{k-1}
    // S(x_{k-1}) (SQ), or Sx and Sy
    df s00 = {0.f, 0.f}, s01 = s00, s10 = s00, s11 = s00;
    df y00 = s00, y01 = s00, y10 = s00, y11 = s00;
    load(kstart, K);
    for (int k = kstart; k < k1; ++k) {
        const float4 a0 = A0, a1 = A1, qd = QD, qu = QU;
        const float zo = comb(ZO), zd = comb(ZD), zu = comb(ZU), ze = comb(ZE);
        const float ve0 = VE0, ve1 = VE1;
        if (k + 1 < k1) {
            if (ph == nu - 1) {
                ++K;
                ph = 0;
            } else {
                ++ph;
            }
            load(k + 1, K);
        }
        const float x00 = c0 ? fma_rn(sig, a0.x, -zo) : 0.f;
        const float x01 = c1 ? fma_rn(sig, a0.z, -zo) : 0.f;
        const float x10 = (c0 && r1) ? fma_rn(sig, a1.x, -zo) : 0.f;
        const float x11 = (c1 && r1) ? fma_rn(sig, a1.z, -zo) : 0.f;
        const float d0 = hd ? fma_rn(sig, qd.x, -zd) : 0.f, d1 = (hd && c1) ? fma_rn(sig, qd.z, -zd) : 0.f;
        const float e0 = hu ? fma_rn(sig, qu.x, -zu) : 0.f, e1 = (hu && c1) ? fma_rn(sig, qu.z, -zu) : 0.f;
        float l0 = __shfl_up_sync(FULL, x01, 1), l1 = __shfl_up_sync(FULL, x11, 1);
        float q0 = __shfl_down_sync(FULL, x00, 1), q1 = __shfl_down_sync(FULL, x10, 1);
        const float xe0 = (cl || cr) ? fma_rn(sig, ve0, -ze) : 0.f;
        const float xe1 = ((cl || cr) && r1) ? fma_rn(sig, ve1, -ze) : 0.f;
        if (lane == 0) {
            l0 = xe0;
            l1 = xe1;
        }
        if (lane == 31) {
            q0 = xe0;
            q1 = xe1;
        }
        // stencil (left, right, down, up, centre) at the four points
        df S00, S01, S10, S11, Y00, Y01, Y10, Y11;
        if (SQ) {
            S00 = lap5_pair(l0, x01, d0, x10, x00);
            S01 = lap5_pair(x00, q0, d1, x11, x01);
            S10 = lap5_pair(l1, x11, x00, e0, x10);
            S11 = lap5_pair(x10, q1, x01, e1, x11);
        } else {
            S00 = lap3_exact(l0, x00, x01); Y00 = lap3_exact(d0, x00, x10);
            S01 = lap3_exact(x00, x01, q0); Y01 = lap3_exact(d1, x01, x11);
            S10 = lap3_exact(l1, x10, x11); Y10 = lap3_exact(x00, x10, e0);
            S11 = lap3_exact(x10, x11, q1); Y11 = lap3_exact(x01, x11, e1);
        }
        if (k >= k0 && c0) {
            auto wk = [&](float c, float p, df S, df Sp, df Y, df Yp) -> df {
                if (k == 0) return df_from_float(c);
                df D;
                if (SQ) {
                    D = HAS_B ? df_dot2(ua, S, ub, Sp) : df_dot1(ua, S);
                } else {
                    const df dx = HAS_B ? df_dot2(ua, S, ub, Sp) : df_dot1(ua, S);
                    const df dy = HAS_B ? df_dot2(uay, Y, uby, Yp) : df_dot1(uay, Y);
                    D = df_add(fast_two_sum(dx.hi, dx.lo), fast_two_sum(dy.hi, dy.lo));
                }
                return df_diff_sub(c, p, D);
            };
            const int64_t f0 = gf.guard + (int64_t)k * gf.plane + o0;
            const df w00 = wk(x00, p00, S00, s00, Y00, y00);
            const df w01 = c1 ? wk(x01, p01, S01, s01, Y01, y01) : df{0.f, 0.f};
            *reinterpret_cast<float2 *>(x + f0) = make_float2(x00, x01);
            *reinterpret_cast<float4 *>(w + f0) = make_float4(w00.hi, w00.lo, w01.hi, w01.lo);
            if (r1) {
                const df w10 = wk(x10, p10, S10, s10, Y10, y10);
                const df w11 = c1 ? wk(x11, p11, S11, s11, Y11, y11) : df{0.f, 0.f};
                *reinterpret_cast<float2 *>(x + f0 + ldx) = make_float2(x10, x11);
                *reinterpret_cast<float4 *>(w + f0 + ldx) = make_float4(w10.hi, w10.lo, w11.hi, w11.lo);
            }
        }
        p00 = x00; p01 = x01; p10 = x10; p11 = x11;
        if (HAS_B) {
            s00 = S00; s01 = S01; s10 = S10; s11 = S11;
            if (!SQ) {
                y00 = Y00; y01 = Y01; y10 = Y10; y11 = Y11;
            }
        }
    }
}

void launch_interp_df(const Geom &gf, const Geom &gc, int nu, bool space, const float2 *ca,
                      const float2 *cb, bool has_b, const float2 *v, const double *sigma,
                      const float *Xc, int mc, int64_t xc_stride, const double *yc, float *x,
                      float2 *wout, const int *done, cudaStream_t s, const float2 *uniform_ab,
                      bool uniform_square) {
    int kc = cap_kc(choose_kc(gf.npts(), gf.nt + 1), gf.nt + 1, gf.dim, gf.nx, gf.ny);
    int nch = (gf.nt + 1 + kc - 1) / kc;
    Launch2 l = point_launch(gf.dim, gf.nx, gf.ny, nch);
    const int hb = has_b ? 1 : 0;
#define MK_IDF1M(S, M)                                                                        \
    k_interp_df_1d<S, M><<<l.grid, l.block, 0, s>>>(gf, gc, nu, ca, cb, hb, v, sigma, Xc, mc, \
                                                    xc_stride, yc, x, wout, kc, done)
#define MK_IDF1(S)                                                                            \
    do {                                                                                      \
        if (!yc) MK_IDF1M(S, 0);                                                              \
        else if (mc == 1) MK_IDF1M(S, 1);                                                     \
        else if (mc == 2) MK_IDF1M(S, 2);                                                     \
        else MK_IDF1M(S, -1);                                                                 \
    } while (0)
    prof_begin(s);
    if (launch_interp_df_1d_tiled(gf, gc, nu, space, ca, cb, has_b, v, sigma, Xc, mc, xc_stride,
                                  yc, x, wout, done, s, uniform_ab)) {
        // 1D, nu = 2: time-tiled kernel (transfer1d.cu)
    } else if (gf.dim == 1) {
        if (space) MK_IDF1(true); else MK_IDF1(false);
    } else if (space && uniform_ab && (!yc || (mc >= 1 && mc <= 4))) {
        // 2 x 2 agglomeration, uniform operator: aggregate-per-thread kernel walked in time;
        // chunks for one full wave of 2048 threads per SM, at least eight fine steps each
        // (the step before a chunk is formed again), at most 65535 chunks
        const int ncx = (gf.nx + 1) / 2, ncy = (gf.ny + 1) / 2;
        const int nsteps = gf.nt + 1;
        const int64_t want = (int64_t)g_num_sms * 2048;
        int64_t kt = ((int64_t)ncx * ncy * nsteps) / (want > 0 ? want : 1);
        if (kt < 8) kt = 8;
        if (kt > nsteps) kt = nsteps;
        while ((nsteps + kt - 1) / kt > 65535) ++kt;
        const int kct = (int)kt;
        const dim3 grid((ncx + 31) / 32, (ncy + 7) / 8, (nsteps + kct - 1) / kct), blk(32, 8, 1);
#define MK_IDF2M(SQ, HB, M)                                                                     \
    k_interp_df_2d_ts<SQ, HB, M><<<grid, blk, 0, s>>>(gf, gc, nu, uniform_ab, v, sigma, Xc,      \
                                                      xc_stride, yc, x, wout, kct, done)
#define MK_IDF2(SQ, HB)                                                                         \
    do {                                                                                        \
        if (!yc) MK_IDF2M(SQ, HB, 0);                                                           \
        else if (mc == 1) MK_IDF2M(SQ, HB, 1);                                                  \
        else if (mc == 2) MK_IDF2M(SQ, HB, 2);                                                  \
        else if (mc == 3) MK_IDF2M(SQ, HB, 3);                                                  \
        else MK_IDF2M(SQ, HB, 4);                                                               \
    } while (0)
        if (uniform_square) {
            if (hb) MK_IDF2(true, true); else MK_IDF2(true, false);
        } else {
            if (hb) MK_IDF2(false, true); else MK_IDF2(false, false);
        }
#undef MK_IDF2
#undef MK_IDF2M
    } else {
        // 2D: x once per point, then w = A x in double-float from the stored x
        const dim3 g2 = grid_2d_points(gf), g4 = grid_2d_points4(gf), b2(32, 8, 1);
        if (space)
            k_interp_x2d<true, float2, float, float><<<g4, b2, 0, s>>>(gf, gc, nu, v, sigma, Xc, mc,
                                                                      xc_stride, yc, x, done);
        else
            k_interp_x2d<false, float2, float, float><<<g4, b2, 0, s>>>(gf, gc, nu, v, sigma, Xc, mc,
                                                                       xc_stride, yc, x, done);
        if (uniform_ab && uniform_square && hb)
            k_apply_df_2d_sq<true><<<g2, b2, 0, s>>>(gf, uniform_ab, x, wout, done);
        else if (uniform_ab && uniform_square)
            k_apply_df_2d_sq<false><<<g2, b2, 0, s>>>(gf, uniform_ab, x, wout, done);
        else if (uniform_ab && hb) k_apply_df_2d_uni<true><<<g2, b2, 0, s>>>(gf, uniform_ab, x, wout, done);
        else if (uniform_ab) k_apply_df_2d_uni<false><<<g2, b2, 0, s>>>(gf, uniform_ab, x, wout, done);
        else k_apply_df_2d<<<g2, b2, 0, s>>>(gf, ca, cb, hb, x, wout, done);
        count_launch();
    }
#undef MK_IDF1
#undef MK_IDF1M
    prof_end(s, PROF_INTERP, (double)gf.interior() * (8.0 + 4.0 + 8.0) + (double)mc * gc.interior() * 4.0);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// Arnoldi with double-float vectors (first and second classical Gram-Schmidt pass).
// multidot: d_i = <W, V_i> (i <= j) and, on the first pass, ||W||^2.
//
// Compensated dot product (the "Dot2" scheme of Ogita, Rump and Oishi): each product is
// split exactly by TwoProduct, the high parts are summed with TwoSum and every rounding
// error goes into a float compensation, so the dependent chain per element is a single
// addition.  Two basis vectors are processed per sweep with independent accumulators, and
// the W tile is re-read from L1 instead of being held in registers.  Vector lengths are a
// whole number of tiles (padding is zero), so the sweep has no bounds checks.
// ---------------------------------------------------------------------------------------
struct Dot2 {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
    // accumulate (ah + al)(bh + bl) without the al*bl term
    __device__ __forceinline__ void add(float2 a, float2 b) {
        df p = two_prod(a.x, b.x);
        float low = fmaf(a.x, b.y, fmaf(a.y, b.x, p.lo));
        df t = two_sum(s, p.hi);
        s = t.hi;
        c += t.lo + low;
    }
    __device__ __forceinline__ df value() const { return fast_two_sum(s, c); }
};

__global__ void __launch_bounds__(DF_THREADS) k_multidot_df(int64_t len, const float2 *__restrict__ W,
                                                            const float2 *__restrict__ V,
                                                            int64_t vstride, int j,
                                                            ReduceScratch rs, KState ks,
                                                            int second,
                                                            const int *__restrict__ done) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    extern __shared__ double smem_md[];
    const int nv = j + 1;
    const int nslots = second ? nv : nv + 1;
    double *acc = smem_md;                      // [nslots][DF_WARPS]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < nslots * DF_WARPS; t += DF_THREADS) acc[t] = 0.0;
    __syncthreads();
    const float2 *src = second ? V + (int64_t)(j + 1) * vstride : W;
    for (int64_t base = (int64_t)blockIdx.x * DF_TILE + threadIdx.x; base < len;
         base += (int64_t)gridDim.x * DF_TILE) {
        if (!second) {
            Dot2 d0, d1;
            d0.init();
            d1.init();
#pragma unroll
            for (int q = 0; q < DF_EPT; q += 2) {
                float2 w0 = src[base + q * DF_THREADS], w1 = src[base + (q + 1) * DF_THREADS];
                d0.add(w0, w0);
                d1.add(w1, w1);
            }
            df r = warp_sum_df(df_add(d0.value(), d1.value()));
            if (lane == 0) acc[nv * DF_WARPS + warp] += df_to_double(r);
        }
        for (int i = 0; i < nv; i += 2) {
            const bool pair = (i + 1 < nv);
            const float2 *va = V + (int64_t)i * vstride;
            const float2 *vb = pair ? va + vstride : va;
            Dot2 a0, a1, b0, b1;
            a0.init();
            a1.init();
            b0.init();
            b1.init();
#pragma unroll
            for (int q = 0; q < DF_EPT; q += 2) {
                const int64_t e0 = base + q * DF_THREADS, e1 = e0 + DF_THREADS;
                float2 w0 = src[e0], w1 = src[e1];
                float2 x0 = va[e0], x1 = va[e1];
                float2 y0 = vb[e0], y1 = vb[e1];
                a0.add(w0, x0);
                a1.add(w1, x1);
                b0.add(w0, y0);
                b1.add(w1, y1);
            }
            df ra = warp_sum_df(df_add(a0.value(), a1.value()));
            df rb = warp_sum_df(df_add(b0.value(), b1.value()));
            if (lane == 0) {
                acc[i * DF_WARPS + warp] += df_to_double(ra);
                if (pair) acc[(i + 1) * DF_WARPS + warp] += df_to_double(rb);
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nslots; t += DF_THREADS) {
        double s = 0.0;
        for (int w2 = 0; w2 < DF_WARPS; ++w2) s += acc[t * DF_WARPS + w2];
        rs.partials[(int64_t)t * rs.max_blocks + blockIdx.x] = s;
    }
    if (last_block_ticket(rs.counter, (int)threadIdx.x < nslots)) {
        const int lane2 = threadIdx.x & 31, warp2 = threadIdx.x >> 5;
        double *res = smem_md;
        for (int t = warp2; t < nslots; t += DF_WARPS) {
            const double *p = rs.partials + (int64_t)t * rs.max_blocks;
            double a = 0.0;
#pragma unroll 8
            for (int b = lane2; b < (int)gridDim.x; b += 32) a += __ldcg(p + b);
            a = warp_sum(a);
            if (lane2 == 0) res[t] = a;
        }
        __syncthreads();
        {
            double *H = ks.H() + (int64_t)j * (ks.m + 1);
            for (int i = threadIdx.x; i < nv; i += blockDim.x) {
                const double hc = ks.sigma()[i] * res[i];
                ks.tmp()[i] = hc;
                H[i] = second ? H[i] + hc : hc;
            }
            if (threadIdx.x == 0) {
                if (!second) ks.misc()[2] = res[nv];
                rs.counter[0] = 0u;
            }
        }
    }
}

// update: V_{j+1} = src - sum_i c_i V_i, c_i = tmp_i sigma_i, ||.||^2, epilogue
__global__ void __launch_bounds__(DF_THREADS) k_update_df(int64_t len, const float2 *__restrict__ W,
                                                          float2 *__restrict__ V, int64_t vstride,
                                                          int j, ReduceScratch rs, KState ks,
                                                          int mode, int second,
                                                          const int *__restrict__ done) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    __shared__ float2 c[MK_MAX_RESTART + 1];
    const int nv = j + 1;
    for (int i = threadIdx.x; i < nv; i += DF_THREADS)
        c[i] = df_pack(df_from_double(ks.tmp()[i] * ks.sigma()[i]));
    __syncthreads();
    float2 *out = V + (int64_t)(j + 1) * vstride;
    df acc = {0.f, 0.f};
    for (int64_t e = (int64_t)blockIdx.x * DF_THREADS + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * DF_THREADS) {
        df val = df_unpack(second ? out[e] : W[e]);
        for (int i = 0; i < nv; ++i)
            val = df_sub(val, df_mul(df_unpack(c[i]), df_unpack(V[(int64_t)i * vstride + e])));
        out[e] = df_pack(val);
        df p = two_prod(val.hi, val.hi);
        p.lo = fmaf(2.f * val.hi, val.lo, p.lo);
        acc = df_add(acc, p);
    }
    double bs = block_sum(df_to_double(acc));
    if (threadIdx.x == 0) rs.partials[blockIdx.x] = bs;
    if (last_block_ticket(rs.counter, threadIdx.x == 0)) {
        double tot = sum_partials(rs.partials, gridDim.x);
        update_epilogue_block(tot, ks, j, mode, second);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
    }
}

static int df_grid(int64_t len, int64_t per_block) {
    int64_t g = (len + per_block - 1) / per_block;
    int64_t cap = (int64_t)g_num_sms * 4;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// u += sum_{i < jf} y_i X_i with FP32 X: y_i split into double-float once per block, each
// term y_i X_i formed and summed in double-float on the FP32 pipe, one FP64 add per element.
// aug (recycled corrections, may be null): the cycle's correction sum y_i X_i is also stored,
// rounded to FP32, in ring slot flags[5] mod augk.
__global__ void __launch_bounds__(DF_THREADS) k_combine_df(int64_t len, double *__restrict__ u,
                                                           const float *__restrict__ X,
                                                           int64_t xstride, KState ks,
                                                           float *__restrict__ aug, int augk) {
    __shared__ float2 y[MK_MAX_RESTART];
    const int jf = ks.flags[1];
    if (jf <= 0 || ks.flags[3]) return;
    for (int i = threadIdx.x; i < jf; i += DF_THREADS) y[i] = df_pack(df_from_double(ks.y()[i]));
    __syncthreads();
    float *d = aug ? aug + (int64_t)(ks.flags[5] % augk) * xstride : nullptr;
    for (int64_t e = (int64_t)blockIdx.x * DF_THREADS + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * DF_THREADS) {
        df acc = {0.f, 0.f};
#pragma unroll 4
        for (int i = 0; i < jf; ++i) acc = df_add(acc, df_mul_f(df_unpack(y[i]), X[(int64_t)i * xstride + e]));
        const double c = df_to_double(acc);
        u[e] += c;
        if (d) d[e] = (float)c;
    }
}

// w (double-float pairs) from the FP64 values stored in the same 8 bytes, in place.
__global__ void k_f64_to_df(int64_t len, void *w) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double v = reinterpret_cast<const double *>(w)[e];
        reinterpret_cast<float2 *>(w)[e] = df_pack(df_from_double(v));
    }
}

void launch_f64_to_df(int64_t len, void *w, const int *done, cudaStream_t s) {
    (void)done;
    k_f64_to_df<<<df_grid(len, (int64_t)DF_THREADS * 8), DF_THREADS, 0, s>>>(len, w);
    count_launch();
}

void launch_combine_df(int64_t len, double *u, const float *X, int64_t xstride, KState ks,
                       cudaStream_t s, float *aug, int augk) {
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    // one element per thread: each element is a dependent chain of jf double-float terms, so
    // independent chains (threads), not a grid-stride loop, hide its latency
    const int64_t grid = (len + DF_THREADS - 1) / DF_THREADS;
    prof_begin(s);
    k_combine_df<<<(unsigned)grid, DF_THREADS, 0, s>>>(len, u, X, xstride, ks, aug, augk);
    prof_end(s, PROF_COMBINE, (double)alg_n * (16.0 + (double)ks.m * sizeof(float)));
    count_launch();
}

void launch_multidot_df(int64_t len, const float2 *W, const float2 *V, int64_t vstride, int j,
                        const ReduceScratch &rs, KState ks, bool second_pass, const int *done,
                        cudaStream_t s) {
    int grid = df_grid(len, DF_TILE);
    size_t shm = sizeof(double) * (size_t)(j + 2) * DF_WARPS;
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    prof_begin(s);
    k_multidot_df<<<grid, DF_THREADS, shm, s>>>(len, W, V, vstride, j, rs, ks, second_pass ? 1 : 0,
                                                done);
    prof_end(s, PROF_MULTIDOT, (double)(j + 2) * alg_n * 8.0);
    count_launch();
}

void launch_update_df(int64_t len, const float2 *W, float2 *V, int64_t vstride, int j,
                      const ReduceScratch &rs, KState ks, int mode, bool second_pass,
                      const int *done, cudaStream_t s) {
    int grid = df_grid(len, (int64_t)DF_THREADS * 8);
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    prof_begin(s);
    k_update_df<<<grid, DF_THREADS, 0, s>>>(len, W, V, vstride, j, rs, ks, mode,
                                            second_pass ? 1 : 0, done);
    prof_end(s, PROF_UPDATE, (double)(j + 3) * alg_n * 8.0);
    count_launch();
}

}  // namespace mk
