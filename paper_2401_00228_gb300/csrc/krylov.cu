// Krylov kernels of FGMRES (Algorithm 2): Arnoldi orthogonalisation by classical
// Gram-Schmidt (one pass, and a second pass when the norm drops by more than 1/sqrt(2)),
// the Hessenberg least-squares problem by Givens rotations, and the solution update
// u = u_0 + X_J y_J.
//
// The basis is stored unnormalised: v_i = sigma_i V_i with sigma_i = 1/||V_i|| kept on the
// device, so no separate scaling pass is needed.  Every scalar of the process (H, Givens
// rotations, y, flags) lives on the device and is updated by the last block of the
// reduction that produces it, so a whole restart cycle runs without a host round trip.
#include <type_traits>

#include "kernels.h"
#include "reduce.cuh"
#include "krylov_epilogue.cuh"

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
        const double *p = part + (int64_t)t * max_blocks;
        double acc = 0.0;
#pragma unroll 8
        for (int b = lane; b < nb; b += 32) acc += __ldcg(p + b);
        acc = warp_sum(acc);
        if (lane == 0) out_smem[t] = acc;
    }
    __syncthreads();
}

// h_i = sigma_i d_i (i < nv) into H's column j and tmp; ||w||^2 into misc[2] (first pass).
__device__ __forceinline__ void multidot_epilogue(const double *res, KState ks, int j, int nv,
                                                  int second) {
    double *H = ks.H() + (int64_t)j * (ks.m + 1);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        const double hc = ks.sigma()[i] * res[i];
        ks.tmp()[i] = hc;
        H[i] = second ? H[i] + hc : hc;
    }
    if (!second && threadIdx.x == 0) ks.misc()[2] = res[nv];
}

// Last inner iteration: h_{j+1,j}^2 = ||w||^2 - sum_i h_ij^2 (orthonormal basis), then the
// update epilogue of the given mode (least squares) without forming V_{j+1}.
__device__ __forceinline__ void close_iteration(const double *res, KState ks, int j, int nv,
                                                int mode) {
    __syncthreads();   // H's column j, written by several threads, is read by the epilogue
    double nrm2 = 0.0;
    if (threadIdx.x == 0) {
        double s2 = 0.0;
        for (int i = 0; i < nv; ++i) {
            const double h = ks.sigma()[i] * res[i];
            s2 += h * h;
        }
        nrm2 = fmax(res[nv] - s2, 0.0);
    }
    update_epilogue_block(nrm2, ks, j, mode, 0);
}

// ---------------------------------------------------------------------------------------
// multidot: d_i = <W, V_i>, i = 0..j ; first pass also ||W||^2.
// ---------------------------------------------------------------------------------------
template <typename TW, typename TV>
__global__ void __launch_bounds__(KR_THREADS) k_multidot(int64_t len, const TW *__restrict__ W,
                                                         const TV *__restrict__ V,
                                                         int64_t vstride, int j,
                                                         ReduceScratch rs, KState ks, int second,
                                                         const int *__restrict__ done,
                                                         int close_mode) {
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
    if (last_block_ticket(rs.counter, (int)threadIdx.x < nslots)) {
        double *res = smem;  // reuse
        finish_slots(rs.partials, rs.max_blocks, nslots, gridDim.x, res);
        multidot_epilogue(res, ks, j, nv, second);
        if (close_mode && !second) close_iteration(res, ks, j, nv, close_mode);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
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
    double bs = block_sum_t(acc);
    if (threadIdx.x == 0) rs.partials[blockIdx.x] = bs;
    if (last_block_ticket(rs.counter, threadIdx.x == 0)) {
        double tot = sum_partials(rs.partials, gridDim.x);
        update_epilogue_block(tot, ks, j, mode, second);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// FP32 vectors with more than MK_MAX_INNER basis vectors (level 1 with the FP32 basis).
// multidot: a tile is 8 consecutive elements per thread in two float4 loads (coalesced
// across the block), two basis vectors per sweep with the W tile re-read from L1; sums in
// FP32 per thread and warp, in FP64 across tiles and warps.  update: four consecutive
// elements per thread and step (float4), the basis loop unrolled so that its loads overlap.
// Vector lengths and strides are whole numbers of 2048-element tiles.  (Four float4 loads per
// thread and tile left a 33.6 MB vector with 2049 tiles on 608 blocks: 4 against 3.37 per
// block on average; two per thread raised the 1D level-1 multidot from 4.63 to 4.85 TB/s.)
// ---------------------------------------------------------------------------------------
constexpr int F4_Q = 2;                            // float4 loads per thread per tile
constexpr int F4_TILE = KR_THREADS * 4 * F4_Q;     // elements per block tile (2048)

__global__ void __launch_bounds__(KR_THREADS) k_multidot_f4(int64_t len, const float *__restrict__ W,
                                                            const float *__restrict__ V,
                                                            int64_t vstride, int j,
                                                            ReduceScratch rs, KState ks, int second,
                                                            const int *__restrict__ done,
                                                            int close_mode) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    extern __shared__ double smem[];
    const int nv = j + 1;
    const int nslots = second ? nv : nv + 1;
    double *acc = smem;                      // [nslots][KR_WARPS]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < nslots * KR_WARPS; t += KR_THREADS) acc[t] = 0.0;
    __syncthreads();
    const float4 *src = reinterpret_cast<const float4 *>(second ? V + (int64_t)(j + 1) * vstride : W);
    const float4 *V4 = reinterpret_cast<const float4 *>(V);
    const int64_t n4 = len / 4, vs4 = vstride / 4;
    constexpr int T4 = F4_TILE / 4;          // float4 per block tile
    for (int64_t base = (int64_t)blockIdx.x * T4 + threadIdx.x; base < n4;
         base += (int64_t)gridDim.x * T4) {
        if (!second) {
            float sw = 0.f;
#pragma unroll
            for (int q = 0; q < F4_Q; ++q) {
                const float4 w = src[base + q * KR_THREADS];
                sw = fmaf(w.x, w.x, sw);
                sw = fmaf(w.y, w.y, sw);
                sw = fmaf(w.z, w.z, sw);
                sw = fmaf(w.w, w.w, sw);
            }
            sw = warp_sum_t(sw);
            if (lane == 0) acc[nv * KR_WARPS + warp] += (double)sw;
        }
        for (int i = 0; i < nv; i += 2) {
            const bool pair = i + 1 < nv;
            const float4 *va = V4 + (int64_t)i * vs4;
            const float4 *vb = pair ? va + vs4 : va;
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int q = 0; q < F4_Q; ++q) {
                const int64_t e = base + q * KR_THREADS;
                const float4 w = src[e], x = va[e], y = vb[e];
                sa = fmaf(w.x, x.x, sa);
                sa = fmaf(w.y, x.y, sa);
                sa = fmaf(w.z, x.z, sa);
                sa = fmaf(w.w, x.w, sa);
                sb = fmaf(w.x, y.x, sb);
                sb = fmaf(w.y, y.y, sb);
                sb = fmaf(w.z, y.z, sb);
                sb = fmaf(w.w, y.w, sb);
            }
            sa = warp_sum_t(sa);
            sb = warp_sum_t(sb);
            if (lane == 0) {
                acc[i * KR_WARPS + warp] += (double)sa;
                if (pair) acc[(i + 1) * KR_WARPS + warp] += (double)sb;
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nslots; t += KR_THREADS) {
        double sum = 0.0;
        for (int w2 = 0; w2 < KR_WARPS; ++w2) sum += acc[t * KR_WARPS + w2];
        rs.partials[(int64_t)t * rs.max_blocks + blockIdx.x] = sum;
    }
    if (last_block_ticket(rs.counter, (int)threadIdx.x < nslots)) {
        double *res = smem;  // reuse
        finish_slots(rs.partials, rs.max_blocks, nslots, gridDim.x, res);
        multidot_epilogue(res, ks, j, nv, second);
        if (close_mode && !second) close_iteration(res, ks, j, nv, close_mode);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
    }
}

__global__ void __launch_bounds__(KR_THREADS) k_update_f4(int64_t len, const float *__restrict__ W,
                                                          float *__restrict__ V, int64_t vstride,
                                                          int j, int write_next, ReduceScratch rs,
                                                          KState ks, int mode, int second,
                                                          const int *__restrict__ done) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    __shared__ float c[MK_MAX_RESTART + 1];
    const int nv = j + 1;
    for (int i = threadIdx.x; i < nv; i += KR_THREADS) c[i] = (float)(ks.tmp()[i] * ks.sigma()[i]);
    __syncthreads();
    float4 *out = reinterpret_cast<float4 *>(V + (int64_t)(j + 1) * vstride);
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
    const float4 *V4 = reinterpret_cast<const float4 *>(V);
    const int64_t n4 = len / 4, vs4 = vstride / 4;
    float acc = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; e < n4;
         e += (int64_t)gridDim.x * KR_THREADS) {
        float4 val = second ? out[e] : W4[e];
#pragma unroll 4
        for (int i = 0; i < nv; ++i) {
            const float4 v = V4[(int64_t)i * vs4 + e];
            const float ci = c[i];
            val.x = fmaf(-ci, v.x, val.x);
            val.y = fmaf(-ci, v.y, val.y);
            val.z = fmaf(-ci, v.z, val.z);
            val.w = fmaf(-ci, v.w, val.w);
        }
        if (write_next) out[e] = val;
        acc = fmaf(val.x, val.x, acc);
        acc = fmaf(val.y, val.y, acc);
        acc = fmaf(val.z, val.z, acc);
        acc = fmaf(val.w, val.w, acc);
    }
    double bs = block_sum_t(acc);
    if (threadIdx.x == 0) rs.partials[blockIdx.x] = bs;
    if (last_block_ticket(rs.counter, threadIdx.x == 0)) {
        double tot = sum_partials(rs.partials, gridDim.x);
        update_epilogue_block(tot, ks, j, mode, second);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// Short-basis variants (j + 1 = NV <= MK_MAX_INNER vectors: every inner level, and the
// first iterations of level 1 in FP64).  Each thread takes 8 consecutive elements per step
// with 16-byte loads, and the vector count is a compile-time constant, so all NV + 1 loads
// of a step are in flight together.  A vector's padded length is a multiple of 4096, so an
// 8-element group never straddles its end.
// ---------------------------------------------------------------------------------------
constexpr int SB_EPT = 8;

template <typename T>
__device__ __forceinline__ void ld8(const T *p, T (&o)[SB_EPT]);
template <>
__device__ __forceinline__ void ld8<float>(const float *p, float (&o)[SB_EPT]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
template <>
__device__ __forceinline__ void ld8<double>(const double *p, double (&o)[SB_EPT]) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + h);
        o[2 * h] = a.x;
        o[2 * h + 1] = a.y;
    }
}
// Plain (coherent) load: the source of a second Gram-Schmidt pass is written by this kernel.
template <typename T>
__device__ __forceinline__ void ld8_rw(const T *p, T (&o)[SB_EPT]) {
#pragma unroll
    for (int q = 0; q < SB_EPT; ++q) o[q] = p[q];
}
template <typename T>
__device__ __forceinline__ void st8(T *p, const T (&o)[SB_EPT]) {
#pragma unroll
    for (int q = 0; q < SB_EPT; ++q) p[q] = o[q];
}

template <int NV, typename T>
__global__ void __launch_bounds__(KR_THREADS) k_multidot_sb(int64_t len, const T *__restrict__ W,
                                                            const T *__restrict__ V,
                                                            int64_t vstride, ReduceScratch rs,
                                                            KState ks, int second,
                                                            const int *__restrict__ done,
                                                            int close_mode) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    constexpr int j = NV - 1;
    __shared__ double acc[(NV + 1) * KR_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T *src = second ? (const T *)(V + (int64_t)(j + 1) * vstride) : W;
    T d[NV + 1];
#pragma unroll
    for (int i = 0; i <= NV; ++i) d[i] = (T)0;
    for (int64_t base = ((int64_t)blockIdx.x * KR_THREADS + threadIdx.x) * SB_EPT; base < len;
         base += (int64_t)gridDim.x * KR_THREADS * SB_EPT) {
        T w[SB_EPT], v[NV][SB_EPT];
        if (second) ld8_rw(src + base, w); else ld8(src + base, w);
#pragma unroll
        for (int i = 0; i < NV; ++i) ld8(V + (int64_t)i * vstride + base, v[i]);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            T s = (T)0;
#pragma unroll
            for (int q = 0; q < SB_EPT; ++q) s += w[q] * v[i][q];
            d[i] += s;
        }
        T s = (T)0;
#pragma unroll
        for (int q = 0; q < SB_EPT; ++q) s += w[q] * w[q];
        d[NV] += s;
    }
    const int nslots = second ? NV : NV + 1;
#pragma unroll
    for (int i = 0; i <= NV; ++i) {
        const double t = (double)warp_sum_t(d[i]);   // warp stage in the arithmetic type
        if (lane == 0) acc[i * KR_WARPS + warp] = t;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nslots; t += KR_THREADS) {
        double sum = 0.0;
        for (int w2 = 0; w2 < KR_WARPS; ++w2) sum += acc[t * KR_WARPS + w2];
        rs.partials[(int64_t)t * rs.max_blocks + blockIdx.x] = sum;
    }
    if (last_block_ticket(rs.counter, (int)threadIdx.x < nslots)) {
        double *res = acc;  // reuse
        finish_slots(rs.partials, rs.max_blocks, nslots, gridDim.x, res);
        multidot_epilogue(res, ks, j, NV, second);
        if (close_mode && !second) close_iteration(res, ks, j, NV, close_mode);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
    }
}

template <int NV, typename T>
__global__ void __launch_bounds__(KR_THREADS) k_update_sb(int64_t len, const T *__restrict__ W,
                                                          T *__restrict__ V, int64_t vstride,
                                                          int write_next, ReduceScratch rs,
                                                          KState ks, int mode, int second,
                                                          const int *__restrict__ done) {
    if (done && *done) return;
    if (second && !ks.flags[2]) return;
    constexpr int j = NV - 1;
    // the coefficients c_i = tmp_i sigma_i, formed once per block (FP64 products and
    // conversions issue at GB300's FP64 rate)
    __shared__ T c_s[NV];
    if (threadIdx.x < NV) c_s[threadIdx.x] = (T)(ks.tmp()[threadIdx.x] * ks.sigma()[threadIdx.x]);
    __syncthreads();
    T c[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) c[i] = c_s[i];
    T *out = V + (int64_t)(j + 1) * vstride;
    T acc = (T)0;
    for (int64_t base = ((int64_t)blockIdx.x * KR_THREADS + threadIdx.x) * SB_EPT; base < len;
         base += (int64_t)gridDim.x * KR_THREADS * SB_EPT) {
        T val[SB_EPT], v[NV][SB_EPT];
        if (second) ld8_rw(out + base, val); else ld8(W + base, val);
#pragma unroll
        for (int i = 0; i < NV; ++i) ld8(V + (int64_t)i * vstride + base, v[i]);
#pragma unroll
        for (int i = 0; i < NV; ++i)
#pragma unroll
            for (int q = 0; q < SB_EPT; ++q) val[q] -= c[i] * v[i][q];
        if (write_next) st8(out + base, val);
#pragma unroll
        for (int q = 0; q < SB_EPT; ++q) acc += val[q] * val[q];
    }
    double bs = block_sum_t(acc);
    if (threadIdx.x == 0) rs.partials[blockIdx.x] = bs;
    if (last_block_ticket(rs.counter, threadIdx.x == 0)) {
        double tot = sum_partials(rs.partials, gridDim.x);
        update_epilogue_block(tot, ks, j, mode, second);
        if (threadIdx.x == 0) rs.counter[0] = 0u;
    }
}

// blocks per SM of the small-basis kernels for the launches that follow on this host thread
// (0: 4, one resident wave; the autotuner may pick fewer, fatter blocks for L2-resident
// vectors, where each block's reduction tail and ticket cost more than the sweep)
thread_local int t_sb_bpsm = 0;

void set_krylov_hint(int blocks_per_sm) { t_sb_bpsm = blocks_per_sm; }

static int sb_grid(int64_t len) {
    int64_t g = (len + KR_THREADS * SB_EPT - 1) / (KR_THREADS * SB_EPT);
    const int64_t cap = (int64_t)g_num_sms * (t_sb_bpsm > 0 ? t_sb_bpsm : 4);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ---------------------------------------------------------------------------------------
// combine: u += sum_{i < jf} y_i X_i
// ---------------------------------------------------------------------------------------
// aug (recycled corrections, may be null): the cycle's correction sum y_i X_i is also stored in
// ring slot flags[5] mod augk.
template <typename TX>
__global__ void __launch_bounds__(KR_THREADS) k_combine(int64_t len, double *__restrict__ u,
                                                        const TX *__restrict__ X,
                                                        int64_t xstride, KState ks,
                                                        TX *__restrict__ aug, int augk) {
    __shared__ double y[MK_MAX_RESTART];
    const int jf = ks.flags[1];
    if (jf <= 0 || ks.flags[3]) return;
    for (int i = threadIdx.x; i < jf; i += KR_THREADS) y[i] = ks.y()[i];
    __syncthreads();
    TX *d = aug ? aug + (int64_t)(ks.flags[5] % augk) * xstride : nullptr;
    for (int64_t e = (int64_t)blockIdx.x * KR_THREADS + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * KR_THREADS) {
        if (d) {
            double c = 0.0;
            for (int i = 0; i < jf; ++i) c += y[i] * (double)X[(int64_t)i * xstride + e];
            u[e] += c;
            d[e] = (TX)c;
        } else {
            double acc = u[e];
            for (int i = 0; i < jf; ++i) acc += y[i] * (double)X[(int64_t)i * xstride + e];
            u[e] = acc;
        }
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
                     cudaStream_t s, int close_mode) {
    int grid = krylov_grid(len, MD_TILE);
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    size_t shm = sizeof(double) * (size_t)(j + 2) * KR_WARPS;
    if (shm < sizeof(double) * (size_t)(j + 2)) shm = sizeof(double) * (size_t)(j + 2);
    prof_begin(s);
    if constexpr (std::is_same<TW, TV>::value) {
        if (j + 1 <= MK_MAX_INNER && len % (KR_THREADS * SB_EPT) == 0) {
            const int g = sb_grid(len);
            const int sec = second_pass ? 1 : 0;
            switch (j + 1) {
#define MK_MD(N) \
    case N:                                                                                   \
        k_multidot_sb<N, TV><<<g, KR_THREADS, 0, s>>>(len, W, V, vstride, rs, ks, sec, done,  \
                                                      close_mode);                            \
        break;
                MK_MD(1) MK_MD(2) MK_MD(3) MK_MD(4) MK_MD(5) MK_MD(6) MK_MD(7) MK_MD(8)
#undef MK_MD
            }
            prof_end(s, PROF_MULTIDOT, (double)(j + 2) * alg_n * sizeof(TV));
            count_launch();
            return;
        }
    }
    if constexpr (std::is_same<TW, float>::value && std::is_same<TV, float>::value) {
        if (len % F4_TILE == 0 && vstride % F4_TILE == 0) {
            k_multidot_f4<<<grid, KR_THREADS, shm, s>>>(len, W, V, vstride, j, rs, ks,
                                                       second_pass ? 1 : 0, done, close_mode);
            prof_end(s, PROF_MULTIDOT, (double)(j + 2) * alg_n * sizeof(TV));
            count_launch();
            return;
        }
    }
    k_multidot<TW, TV><<<grid, KR_THREADS, shm, s>>>(len, W, V, vstride, j, rs, ks,
                                                      second_pass ? 1 : 0, done, close_mode);
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
    if constexpr (std::is_same<TW, TV>::value) {
        if (j + 1 <= MK_MAX_INNER && len % (KR_THREADS * SB_EPT) == 0) {
            const int g = sb_grid(len);
            const int wn = write_next ? 1 : 0, sec = second_pass ? 1 : 0;
            switch (j + 1) {
#define MK_UP(N)                                                                              \
    case N:                                                                                   \
        k_update_sb<N, TV><<<g, KR_THREADS, 0, s>>>(len, W, V, vstride, wn, rs, ks, mode, sec, \
                                                    done);                                    \
        break;
                MK_UP(1) MK_UP(2) MK_UP(3) MK_UP(4) MK_UP(5) MK_UP(6) MK_UP(7) MK_UP(8)
#undef MK_UP
            }
            prof_end(s, PROF_UPDATE, (double)(j + 2 + (write_next ? 1 : 0)) * alg_n * sizeof(TV));
            count_launch();
            return;
        }
    }
    if constexpr (std::is_same<TW, float>::value && std::is_same<TV, float>::value) {
        if (len % F4_TILE == 0 && vstride % F4_TILE == 0) {
            k_update_f4<<<grid, KR_THREADS, 0, s>>>(len, W, V, vstride, j, write_next ? 1 : 0, rs,
                                                    ks, mode, second_pass ? 1 : 0, done);
            prof_end(s, PROF_UPDATE, (double)(j + 2 + (write_next ? 1 : 0)) * alg_n * sizeof(TV));
            count_launch();
            return;
        }
    }
    k_update<TW, TV><<<grid, KR_THREADS, 0, s>>>(len, W, V, vstride, j, write_next ? 1 : 0, rs,
                                                  ks, mode, second_pass ? 1 : 0, done);
    prof_end(s, PROF_UPDATE, (double)(j + 2 + (write_next ? 1 : 0)) * alg_n * sizeof(TV));
    count_launch();
}

template <typename TX>
void launch_combine(int64_t len, double *u, const TX *X, int64_t xstride, KState ks,
                    cudaStream_t s, TX *aug, int augk) {
    const double alg_n = prof_alg_n() > 0 ? prof_alg_n() : (double)len;
    int grid = krylov_grid(len, (int64_t)KR_THREADS * 8);
    prof_begin(s);
    k_combine<TX><<<grid, KR_THREADS, 0, s>>>(len, u, X, xstride, ks, aug, augk);
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
                                              const int *, cudaStream_t, int);
template void launch_multidot<float, float>(int64_t, const float *, const float *, int64_t, int,
                                            const ReduceScratch &, KState, bool, const int *,
                                            cudaStream_t, int);
template void launch_update<double, double>(int64_t, const double *, double *, int64_t, int, bool,
                                            const ReduceScratch &, KState, int, bool,
                                            const int *, cudaStream_t);
template void launch_update<float, float>(int64_t, const float *, float *, int64_t, int, bool,
                                          const ReduceScratch &, KState, int, bool, const int *,
                                          cudaStream_t);
template void launch_combine<double>(int64_t, double *, const double *, int64_t, KState,
                                     cudaStream_t, double *, int);
template void launch_combine<float>(int64_t, double *, const float *, int64_t, KState,
                                    cudaStream_t, float *, int);

}  // namespace mk
