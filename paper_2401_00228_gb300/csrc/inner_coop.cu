// The inner levels of the 1D mixed-precision MK cycle (Sec. 4.1 recursion: fixed-m FGMRES on
// every intermediate level, Sec. 3.1 substeps 4.1-4.5 between consecutive levels, the
// decoupled or coupled coarsest level of Sec. 3.3 by the sine transform) in ONE cooperative
// kernel per outer iteration.
//
// On these levels the vectors are 2-17 MB and stay in L2; launched one kernel per step, every
// restriction, interpolation, dot product and update waits for its own launch, its last
// block's reduction tail and the next launch, so the inner levels run far below the memory
// rate.  Here every block of a cooperative launch (all co-resident) walks the same sequence
// of phases, separated by grid-wide barriers:
//   restriction of V_l[j] (shifted residual, Y^T of nu = 2)  -> level l+1 right-hand side,
//   recursion (inner FGMRES of level l+1) or the coarsest sine-transform solve,
//   interpolation + correction + matvec: X_l[j] = sigma_j V_l[j] - Z sum_m y_m X_{l+1,m},
//   W = A_l X_l[j],
//   classical Gram-Schmidt: dot products <W, V_i>, then V_{j+1} = W - sum_i h_ij V_i,
//   and on the last iteration the small least-squares problem for y_l.
// Every reduction is two-stage: one partial per block, then after the barrier EVERY block
// adds the partials in the same fixed order and runs the same small epilogue (Hessenberg
// column, norms, Givens least squares) on its own shared-memory copy of the level state, so
// all blocks hold bitwise identical scalars without a second barrier; block 0 also writes
// them to the level's device state.  Data written inside the kernel by other blocks is read
// through L2 (ld.global.cg).  The arithmetic of each phase is that of the separate kernels
// (FP32 vectors and stencils, FP64 reductions and epilogues).
#include <cooperative_groups.h>

#include "kernels.h"
#include "reduce.cuh"
#include "rounding.cuh"
#include "dst_fft.cuh"
#include "scan.cuh"
#include "krylov_epilogue.cuh"

namespace cg = cooperative_groups;

namespace mk {

namespace {

constexpr int CT = 256;          // threads per block (the FFT's block size)
constexpr int CWARPS = CT / 32;
constexpr int NSLOT = MK_MAX_INNER + 2;

__device__ __forceinline__ float4 ldcg4(const float *p) {
    return __ldcg(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ void st4f(float *p, const float (&o)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
}

// Small FGMRES state of one level, one copy per block.
struct LvState {
    double sigma[MK_MAX_INNER + 1];
    double H[(MK_MAX_INNER + 1) * MK_MAX_INNER];   // column-major, leading dim m+1
    double tmp[MK_MAX_INNER + 1];
    double y[MK_MAX_INNER];
    double beta;
};

// partials[s * maxb + block] = block sum of v[s], s < ns.  red: CWARPS * NSLOT doubles.
__device__ __forceinline__ void put_partials(const double (&v)[NSLOT], int ns, double *partials,
                                             int maxb, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        if (s < ns) {
            const double t = warp_sum(v[s]);
            if (lane == 0) red[s * CWARPS + warp] = t;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < ns) {
        double t = 0.0;
        for (int w = 0; w < CWARPS; ++w) t += red[threadIdx.x * CWARPS + w];
        partials[(int64_t)threadIdx.x * maxb + blockIdx.x] = t;
    }
    __syncthreads();
}

// out[s] = sum over blocks of partials[s][b], in the same order in every block.
__device__ __forceinline__ void grid_totals(const double *partials, int maxb, int ns, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = warp; s < ns; s += CWARPS) {
        // up to 32 partials per lane, loaded together, then added in block order
        const double *p = partials + (int64_t)s * maxb;
        double t[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int b = lane + 32 * q;
            t[q] = (b < (int)gridDim.x) ? __ldcg(p + b) : 0.0;
        }
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 32; ++q) acc += t[q];
        acc = warp_sum(acc);
        if (lane == 0) out[s] = acc;
    }
    __syncthreads();
}

// Laplacian of four consecutive points with the values just outside them (the order of the
// separate kernels' lap4).
__device__ __forceinline__ void lap4c(const float (&c)[4], float left, float right, const float (&lo)[4],
                                      const float (&di)[4], const float (&up)[4], float (&l)[4]) {
    l[0] = di[0] * c[0] + lo[0] * left + up[0] * c[1];
    l[1] = di[1] * c[1] + lo[1] * c[0] + up[1] * c[2];
    l[2] = di[2] * c[2] + lo[2] * c[1] + up[2] * c[3];
    l[3] = di[3] * c[3] + lo[3] * c[2] + up[3] * right;
}

__device__ __forceinline__ void coefs4(const float *L, int nf, int i0, float (&lo)[4], float (&di)[4],
                                       float (&up)[4]) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + p;
        const bool in = i < nf;
        lo[p] = in ? L[i] : 0.f;
        di[p] = in ? L[nf + i] : 0.f;
        up[p] = in ? L[2 * nf + i] : 0.f;
    }
}

// Row k of v at points i0..i0+3 and the two outside neighbours (zero beyond the boundary;
// the padding of the layout is zero, so i0 - 1 = -1 reads 0).
__device__ __forceinline__ void row4(const Geom &g, const float *v, int k, int i0, float (&c)[4],
                                     float &l, float &r) {
    const float *rp = v + g.guard + (int64_t)k * g.plane;
    const float4 q = ldcg4(rp + i0);
    c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
    l = __ldcg(rp + i0 - 1);
    r = (i0 + 4 < g.nx) ? __ldcg(rp + i0 + 4) : 0.f;
}

// ---- 4.1-4.2: vhat = sigma Y^T (A v - mu v), nu = 2, no space agglomeration ----------------
// One item = one coarse step K and four points.  Returns the thread's sum of vhat^2.
__device__ __noinline__ double restrict_phase(const CoopLevel &F, const Geom &gc, const float *v, float sig,
                                 float *out) {
    const int nf = F.g.nx, ng = (nf + 3) / 4;
    const int64_t items = (int64_t)(gc.nt + 1) * ng;
    const float a = F.a, b = F.b, mu = F.mu;
    float acc = 0.f;   // per-thread sum in FP32 (FP64 only across threads)
    for (int64_t t = (int64_t)blockIdx.x * CT + threadIdx.x; t < items; t += (int64_t)gridDim.x * CT) {
        const int K = (int)(t / ng);
        const int i0 = 4 * (int)(t - (int64_t)K * ng);
        float lo[4], di[4], up[4];
        coefs4(F.L, nf, i0, lo, di, up);
        float o[4];
        if (K == 0) {
            float c[4], l, r;
            row4(F.g, v, 0, i0, c, l, r);
#pragma unroll
            for (int p = 0; p < 4; ++p) o[p] = sig * (c[p] - mu * c[p]);
        } else {
            float cp[4], c1[4], c2[4], lp_, rp_, l1_, r1_, l2_, r2_;
            row4(F.g, v, 2 * K - 2, i0, cp, lp_, rp_);
            row4(F.g, v, 2 * K - 1, i0, c1, l1_, r1_);
            row4(F.g, v, 2 * K, i0, c2, l2_, r2_);
            float Lp[4], L1[4], L2[4];
            lap4c(cp, lp_, rp_, lo, di, up, Lp);
            lap4c(c1, l1_, r1_, lo, di, up, L1);
            lap4c(c2, l2_, r2_, lo, di, up, L2);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float av1 = (c1[p] - a * L1[p]) - (cp[p] + b * Lp[p]);
                const float av2 = (c2[p] - a * L2[p]) - (c1[p] + b * L1[p]);
                const float t1 = av1 - mu * c1[p];
                const float t2 = av2 - mu * c2[p];
                o[p] = sig * (t1 + t2);
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (i0 + p >= nf) o[p] = 0.f;
            acc += o[p] * o[p];
        }
        st4f(out + gc.guard + (int64_t)K * gc.plane + i0, o);
    }
    return (double)acc;
}

// ---- 4.4-4.5 and step 5: x = sigma v - Z vt, w = A x --------------------------------------
// One item = one coarse step K and four points: fine step 0 for K = 0, fine steps 2K-1 and 2K
// (both interpolate coarse row K) otherwise, with x_{2K-2} (coarse row K-1) for w_{2K-1}.
__device__ __forceinline__ void zrow(const Geom &gc, const float *Xc, int mc, int64_t xcs, const float *ys,
                                     int K, int i0, float (&z)[4], float &zl, float &zr) {
#pragma unroll
    for (int p = 0; p < 4; ++p) z[p] = 0.f;
    zl = 0.f;
    zr = 0.f;
    for (int m = 0; m < mc; ++m) {
        const float ym = ys ? ys[m] : 1.f;
        float t[4], tl, tr;
        row4(gc, Xc + (int64_t)m * xcs, K, i0, t, tl, tr);
#pragma unroll
        for (int p = 0; p < 4; ++p) z[p] = (m == 0) ? mul_rn(ym, t[p]) : fma_rn(ym, t[p], z[p]);
        zl = (m == 0) ? mul_rn(ym, tl) : fma_rn(ym, tl, zl);
        zr = (m == 0) ? mul_rn(ym, tr) : fma_rn(ym, tr, zr);
    }
}

__device__ __forceinline__ void xfrom(const Geom &gf, const float *v, float sig, int k, int i0,
                                      const float (&z)[4], float zl, float zr, float (&x)[4],
                                      float &xl, float &xr) {
    const int nf = gf.nx;
    float c[4], l, r;
    row4(gf, v, k, i0, c, l, r);
#pragma unroll
    for (int p = 0; p < 4; ++p) x[p] = (i0 + p < nf) ? fma_rn(sig, c[p], -z[p]) : 0.f;
    xl = (i0 > 0) ? fma_rn(sig, l, -zl) : 0.f;
    xr = (i0 + 4 < nf) ? fma_rn(sig, r, -zr) : 0.f;
}

__device__ __noinline__ void interp_phase(const CoopLevel &F, const Geom &gc, const float *v, float sig,
                                          const float *Xc, int mc, int64_t xcs, const float *ys,
                                          float *xout, float *wout) {
    const int nf = F.g.nx, ng = (nf + 3) / 4;
    const int64_t items = (int64_t)(gc.nt + 1) * ng;
    const float a = F.a, b = F.b;
    for (int64_t t = (int64_t)blockIdx.x * CT + threadIdx.x; t < items; t += (int64_t)gridDim.x * CT) {
        const int K = (int)(t / ng);
        const int i0 = 4 * (int)(t - (int64_t)K * ng);
        float z1[4], z1l, z1r;
        zrow(gc, Xc, mc, xcs, ys, K, i0, z1, z1l, z1r);
        if (K == 0) {
            float x[4], xl, xr;
            xfrom(F.g, v, sig, 0, i0, z1, z1l, z1r, x, xl, xr);
            const int64_t idx = F.g.guard + i0;
            st4f(xout + idx, x);
            st4f(wout + idx, x);
            continue;
        }
        float z0[4], z0l, z0r;
        zrow(gc, Xc, mc, xcs, ys, K - 1, i0, z0, z0l, z0r);
        float lo[4], di[4], up[4];
        coefs4(F.L, nf, i0, lo, di, up);
        float xp[4], xpl, xpr, x1[4], x1l, x1r, x2[4], x2l, x2r;
        xfrom(F.g, v, sig, 2 * K - 2, i0, z0, z0l, z0r, xp, xpl, xpr);
        xfrom(F.g, v, sig, 2 * K - 1, i0, z1, z1l, z1r, x1, x1l, x1r);
        xfrom(F.g, v, sig, 2 * K, i0, z1, z1l, z1r, x2, x2l, x2r);
        float lxp[4], lx1[4], lx2[4], w1[4], w2[4];
        lap4c(xp, xpl, xpr, lo, di, up, lxp);
        lap4c(x1, x1l, x1r, lo, di, up, lx1);
        lap4c(x2, x2l, x2r, lo, di, up, lx2);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const bool in = i0 + p < nf;
            w1[p] = in ? (x1[p] - a * lx1[p]) - (xp[p] + b * lxp[p]) : 0.f;
            w2[p] = in ? (x2[p] - a * lx2[p]) - (x1[p] + b * lx1[p]) : 0.f;
        }
        const int64_t i1 = F.g.guard + (int64_t)(2 * K - 1) * F.g.plane + i0;
        const int64_t i2 = i1 + F.g.plane;
        st4f(xout + i1, x1);
        st4f(wout + i1, w1);
        st4f(xout + i2, x2);
        st4f(wout + i2, w2);
    }
}

// ---- Gram-Schmidt: d_i = <W, V_i> (i <= j) and ||W||^2, thread sums (FP32 products, FP64 sums
// across threads) --------------------------------------------------------------------------
__device__ __noinline__ void multidot_phase(const CoopLevel &F, int j, double (&d)[NSLOT]) {
    const int nv = j + 1;
    float s[NSLOT];
#pragma unroll
    for (int i = 0; i < NSLOT; ++i) s[i] = 0.f;
    const int64_t n4 = F.g.len / 4;
    for (int64_t e = (int64_t)blockIdx.x * CT + threadIdx.x; e < n4; e += (int64_t)gridDim.x * CT) {
        const float4 w = ldcg4(F.W + 4 * e);
#pragma unroll
        for (int i = 0; i < NSLOT - 1; ++i) {
            if (i < nv) {
                const float4 v = ldcg4(F.V + (int64_t)i * F.stride + 4 * e);
                s[i] += ((w.x * v.x + w.y * v.y) + w.z * v.z) + w.w * v.w;
            }
        }
        s[NSLOT - 1] += ((w.x * w.x + w.y * w.y) + w.z * w.z) + w.w * w.w;
    }
#pragma unroll
    for (int i = 0; i < NSLOT; ++i) d[i] = 0.0;
#pragma unroll
    for (int i = 0; i < NSLOT - 1; ++i)
        if (i < nv) d[i] = (double)s[i];
    d[nv] = (double)s[NSLOT - 1];
}

// V_{j+1} = W - sum_{i <= j} c_i V_i, c_i = h_ij sigma_i; returns the thread's sum of squares.
__device__ __noinline__ double update_phase(const CoopLevel &F, int j, const float *c) {
    const int nv = j + 1;
    float cc[NSLOT - 1];
#pragma unroll
    for (int i = 0; i < NSLOT - 1; ++i) cc[i] = (i < nv) ? c[i] : 0.f;
    float *out = F.V + (int64_t)(j + 1) * F.stride;
    float acc = 0.f;
    const int64_t n4 = F.g.len / 4;
    for (int64_t e = (int64_t)blockIdx.x * CT + threadIdx.x; e < n4; e += (int64_t)gridDim.x * CT) {
        const float4 w = ldcg4(F.W + 4 * e);
        float val[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < NSLOT - 1; ++i) {
            if (i < nv) {
                const float4 v = ldcg4(F.V + (int64_t)i * F.stride + 4 * e);
                val[0] -= cc[i] * v.x;
                val[1] -= cc[i] * v.y;
                val[2] -= cc[i] * v.z;
                val[3] -= cc[i] * v.w;
            }
        }
        st4f(out + 4 * e, val);
        acc += ((val[0] * val[0] + val[1] * val[1]) + val[2] * val[2]) + val[3] * val[3];
    }
    return (double)acc;
}

// ---- coarsest level: rh = DST(R) per row, per-mode recurrence over the slabs (or the coupled
// march), X = 2/(n+1) DST(xh) per row, X_0 = R_0 ---------------------------------------------
__device__ __noinline__ void dst_row_in(const CoopCoarse &C, const float *src, float2 *a) {
    const int n = C.g.nx, N = n + 1, N2 = C.N2;
    for (int m = threadIdx.x; m < N2; m += CT) {
        float v = 0.f;
        if (m > 0 && m < N) v = __ldcg(src + m - 1);
        else if (m > N) v = -__ldcg(src + N2 - m - 1);
        a[dstfft::pad(m)] = make_float2(v, 0.f);
    }
    __syncthreads();
    dstfft::fft_smem(a, N2, C.logN2, C.tw);
}

template <int RC>
__device__ __noinline__ void scan_units(const CoopCoarse &C, int coupled, int steps, int nslabs) {
    const int ng = (C.g.nx + 31) / 32;
    const ModeTable<float> coef{C.tab, C.tab + C.g.nx};
    for (int u = blockIdx.x; u < ng * nslabs; u += gridDim.x)
        mode_scan_unit<float, RC, CWARPS, true, ModeTable<float>>(C.g.nx, C.rh, C.ldd, coef, steps,
                                                                  coupled, u % ng, u / ng);
}

__device__ __noinline__ void coarse_solve(const CoopCoarse &C, float2 *a, cg::grid_group &grid) {
    const int n = C.g.nx, nt = C.g.nt;
    const int coupled = C.n_cgs <= 0 ? 1 : 0;
    const int nslabs = coupled ? 1 : C.n_cgs;
    const int steps = coupled ? nt : nt / C.n_cgs;
    const int k0 = coupled ? 0 : 1;
    for (int k = k0 + blockIdx.x; k <= nt; k += gridDim.x) {
        dst_row_in(C, C.R + C.g.guard + (int64_t)k * C.g.plane, a);
        float *out = C.rh + (int64_t)k * C.ldd;
        for (int j = threadIdx.x; j < n; j += CT) out[j] = -0.5f * a[dstfft::pad(j + 1)].y;
        __syncthreads();
    }
    grid.sync();
    if (!coupled && steps <= 32) {
        // short slabs: one thread per (mode, slab) walks the slab
        const int64_t items = (int64_t)n * nslabs;
        for (int64_t t = (int64_t)blockIdx.x * CT + threadIdx.x; t < items; t += (int64_t)gridDim.x * CT) {
            const int j = (int)(t % n), sl = (int)(t / n);
            const float al = C.tab[j], be = C.tab[n + j];
            float *p = C.rh + (int64_t)(1 + sl * steps) * C.ldd + j;
            float acc = 0.f;
            for (int i = 0; i < steps; ++i) {
                acc = al * acc + be * __ldcg(p + (int64_t)i * C.ldd);
                p[(int64_t)i * C.ldd] = acc;
            }
        }
    } else {
        const int len = coupled ? steps + 1 : steps;
        const int rc = mode_scan_rows(len, CWARPS);
        if (rc == 2) scan_units<2>(C, coupled, steps, nslabs);
        else if (rc == 4) scan_units<4>(C, coupled, steps, nslabs);
        else if (rc == 8) scan_units<8>(C, coupled, steps, nslabs);
        else if (rc == 16) scan_units<16>(C, coupled, steps, nslabs);
        else scan_units<32>(C, coupled, steps, nslabs);
    }
    grid.sync();
    const float sc = -1.f / (float)(n + 1);
    for (int k = blockIdx.x; k <= nt; k += gridDim.x) {
        float *xrow_ = C.X + C.g.guard + (int64_t)k * C.g.plane;
        if (k == 0) {
            const float *r0 = C.R + C.g.guard;
            for (int i = threadIdx.x; i < n; i += CT) xrow_[i] = __ldcg(r0 + i);
            continue;
        }
        dst_row_in(C, C.rh + (int64_t)k * C.ldd, a);
        for (int i = threadIdx.x; i < n; i += CT) xrow_[i] = sc * a[dstfft::pad(i + 1)].y;
        __syncthreads();
    }
    grid.sync();
}


// ---- epilogues, run by thread 0 of every block on its copy of the level state; block 0
// also writes the level's device state (read by the level-1 kernels after the launch) ----------
__device__ void beta_epilogue(const CoopLevel &F, LvState &st, double total) {
    const double beta = sqrt(total);
    st.beta = beta;
    st.sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    if (blockIdx.x == 0) {
        F.ks.misc()[5] = total;
        F.ks.misc()[0] = beta;
        F.ks.sigma()[0] = st.sigma[0];
        if (!isfinite(beta)) F.ks.flags[3] = 1;
    }
}

// h_ij = sigma_i d_i; on the last iteration the new column's subdiagonal by Pythagoras and the
// least squares min || beta e_1 - H y || by Givens rotations.
__device__ __noinline__ void multidot_epilogue(const CoopLevel &F, LvState &st, int j, const double *res, bool last) {
    const int m = F.m, ld = m + 1;
    double s2 = 0.0;
    for (int i = 0; i <= j; ++i) {
        const double h = st.sigma[i] * res[i];
        st.tmp[i] = h;
        st.H[i + j * ld] = h;
        s2 += h * h;
    }
    const bool b0 = blockIdx.x == 0;
    if (b0) {
        for (int i = 0; i <= j; ++i) {
            F.ks.tmp()[i] = st.tmp[i];
            F.ks.H()[i + (int64_t)j * ld] = st.tmp[i];
        }
        F.ks.misc()[2] = res[j + 1];
    }
    if (!last) return;
    const double nrm = sqrt(fmax(res[j + 1] - s2, 0.0));
    if (!isfinite(nrm)) {
        if (b0) {
            F.ks.flags[3] = 1;
            F.ks.flags[0] = 1;
            F.ks.flags[1] = 0;
        }
        return;
    }
    st.H[j + 1 + j * ld] = nrm;
    st.sigma[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    double R[(MK_MAX_INNER + 1) * MK_MAX_INNER], g[MK_MAX_INNER + 1];
    for (int i = 0; i < ld * m; ++i) R[i] = st.H[i];
    givens_solve(R, ld, m, st.beta, g, st.y, nullptr);
    if (b0) {
        F.ks.flags[2] = 0;
        F.ks.H()[j + 1 + (int64_t)j * ld] = nrm;
        F.ks.sigma()[j + 1] = st.sigma[j + 1];
        for (int i = 0; i < m; ++i) F.ks.y()[i] = st.y[i];
        for (int i = 0; i <= m; ++i) F.ks.g()[i] = g[i];
    }
}

__device__ void update_epilogue(const CoopLevel &F, LvState &st, int j, double total) {
    const int ld = F.m + 1;
    const double nrm = sqrt(total);
    const bool b0 = blockIdx.x == 0;
    if (!isfinite(nrm)) {
        if (b0) {
            F.ks.flags[3] = 1;
            F.ks.flags[0] = 1;
            F.ks.flags[1] = 0;
        }
        return;
    }
    st.H[j + 1 + j * ld] = nrm;
    st.sigma[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (b0) {
        F.ks.flags[2] = 0;
        F.ks.H()[j + 1 + (int64_t)j * ld] = nrm;
        F.ks.sigma()[j + 1] = st.sigma[j + 1];
    }
}

// The inner FGMRES recursion as a loop over (level, iteration) with an explicit stack.
__global__ void __launch_bounds__(CT, 3) k_inner_coop(const CoopParams *__restrict__ P,
                                                   const int *__restrict__ done) {
    if (done && *done) return;   // every block reads the same flag: all return together
    cg::grid_group grid = cg::this_grid();
    extern __shared__ float2 fftbuf[];
    __shared__ LvState st[MK_MAX_LEVELS];
    __shared__ double red[NSLOT * CWARPS];
    __shared__ double tot[NSLOT];
    __shared__ float cw[NSLOT];   // Gram-Schmidt coefficients, then the coarse weights y
    const int nl = P->nl;
    const int maxb = P->max_blocks;
    int buf = 0;                  // ping-pong partial buffers: a reduction's partials are not
                                  // overwritten before every block has read them
    auto partials = [&]() { return P->partials + (int64_t)buf * NSLOT * maxb; };
    if (threadIdx.x == 0) {
        st[0].beta = P->lv[0].ks.misc()[0];
        st[0].sigma[0] = P->lv[0].ks.sigma()[0];
    }
    __syncthreads();
    int js[MK_MAX_LEVELS];
    int l = 0;
    js[0] = 0;
    bool descend = true;
    for (;;) {
        const CoopLevel &F = P->lv[l];
        const int jl = js[l];
        const bool next_coarsest = (l == nl - 1);
        const Geom gc = next_coarsest ? P->c.g : P->lv[l + 1].g;
        const float sig = (float)st[l].sigma[jl];
        const float *vj = F.V + (int64_t)jl * F.stride;
        if (descend) {
            // 4.1-4.2: the shifted residual of V_l[j] restricted to level l+1
            float *dst = next_coarsest ? P->c.R : P->lv[l + 1].V;
            double d[NSLOT];
            d[0] = restrict_phase(F, gc, vj, sig, dst);
            if (!next_coarsest) put_partials(d, 1, partials(), maxb, red);
            grid.sync();
            if (next_coarsest) {
                coarse_solve(P->c, fftbuf, grid);     // 4.3 at the coarsest level
                descend = false;
            } else {
                grid_totals(partials(), maxb, 1, tot);
                buf ^= 1;
                if (threadIdx.x == 0) beta_epilogue(P->lv[l + 1], st[l + 1], tot[0]);
                __syncthreads();
                l += 1;                               // 4.3: the inner FGMRES of level l+1
                js[l] = 0;
            }
            continue;
        }
        // 4.4-4.5 and step 5: X_l[j] = sigma_j V_l[j] - Z vt, W = A_l X_l[j]
        {
            const float *Xc = next_coarsest ? P->c.X : P->lv[l + 1].X;
            const int mc = next_coarsest ? 1 : P->lv[l + 1].m;
            const int64_t xcs = next_coarsest ? 0 : P->lv[l + 1].stride;
            if (!next_coarsest && (int)threadIdx.x < mc) cw[threadIdx.x] = (float)st[l + 1].y[threadIdx.x];
            __syncthreads();
            interp_phase(F, gc, vj, sig, Xc, mc, xcs, next_coarsest ? nullptr : cw,
                         F.X + (int64_t)jl * F.stride, F.W);
            __syncthreads();   // cw is rewritten below
        }
        grid.sync();
        // classical Gram-Schmidt against V_0 .. V_j
        {
            double d[NSLOT];
            multidot_phase(F, jl, d);
            put_partials(d, jl + 2, partials(), maxb, red);
            grid.sync();
            grid_totals(partials(), maxb, jl + 2, tot);
            buf ^= 1;
        }
        const bool last = (jl == F.m - 1);
        if (threadIdx.x == 0) multidot_epilogue(F, st[l], jl, tot, last);
        __syncthreads();
        if (!last) {
            if ((int)threadIdx.x <= jl) cw[threadIdx.x] = (float)(st[l].tmp[threadIdx.x] * st[l].sigma[threadIdx.x]);
            __syncthreads();
            double d[NSLOT];
            d[0] = update_phase(F, jl, cw);
            put_partials(d, 1, partials(), maxb, red);
            grid.sync();
            grid_totals(partials(), maxb, 1, tot);
            buf ^= 1;
            if (threadIdx.x == 0) update_epilogue(F, st[l], jl, tot[0]);
            __syncthreads();
            js[l] = jl + 1;
            descend = true;
        } else {
            if (l == 0) break;      // level 2 done: X_2 and y_2 are in place
            l -= 1;
            descend = false;
        }
    }
}

}  // namespace

cudaError_t coop_set_attributes() {
    return cudaFuncSetAttribute(k_inner_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dst_smem_bytes(4096));
}

int coop_grid_size(int N2) {
    int dev = 0, coop = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inner_coop, CT, dst_smem_bytes(N2)) !=
        cudaSuccess)
        return 0;
    return nb * g_num_sms;
}

void launch_inner_coop(const CoopParams *Pdev, int N2, int grid, const int *done, cudaStream_t s) {
    void *args[] = {(void *)&Pdev, (void *)&done};
    prof_begin(s);
    cudaLaunchCooperativeKernel((const void *)k_inner_coop, grid, CT, args, dst_smem_bytes(N2), s);
    prof_end(s, PROF_INNER, 0.0);
    count_launch();
}

}  // namespace mk
