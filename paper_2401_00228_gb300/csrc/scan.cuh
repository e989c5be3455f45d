// Per-mode first-order recurrences over time, the core of the coarsest-level solves in an
// eigenbasis of the spatial operator (Sec. 3.3.2, Eq. (Qhtilde) for the decoupled slabs;
// Sec. 3.3.1 for the coupled coarse march, n_cgs = 0).
//
// In the eigenbasis every step (I - a L) x_k = r_k + (I + b L) x_{k-1} of a slab is the scalar
// recurrence xh_k = alpha_m xh_{k-1} + beta_m rh_k per mode m, with beta_m = 1 / (1 - a lam_m)
// and alpha_m = (1 + b lam_m) beta_m.  Rows are stored rh[k * ld + m]; slab i of n_cgs covers
// rows 1 + i s .. (i + 1) s (s = nt / n_cgs) and starts from xh = 0 (the dropped coupling);
// the coupled march covers rows 0..nt with xh_0 = rh_0 (x_0 = r_0).
//
// k_mode_scan runs the recurrence as a blocked scan over time.  A block covers 32 consecutive
// modes (one per lane, so that every row access is one coalesced segment) and SCAN_CHUNKS
// warps; warp q owns C consecutive rows of the current tile of SCAN_CHUNKS * C rows.  Each warp
// keeps its rows in registers, runs the recurrence from zero over them and publishes its last
// value e_q; the value entering chunk q is c_q = alpha^C c_{q-1} + e_{q-1} (c_0 = the value
// carried out of the previous tile), and row i of the chunk gains alpha^{i+1} c_q.  Every row
// is read once and written once, and the dependent chain per thread is C + SCAN_CHUNKS steps
// instead of the slab's length.
#pragma once

#include <cstdint>

namespace mk {

// alpha, beta per mode from tables (1D sine basis: [alpha (n) | beta (n)])
template <typename T>
struct ModeTable {
    const T *alpha, *beta;
    __device__ __forceinline__ void get(int m, T &al, T &be) const {
        al = alpha[m];
        be = beta[m];
    }
};

// alpha, beta of mode m = j nx + i of L = Lx (+) Ly from the eigenvalues of both directions
template <typename T>
struct ModeEig2D {
    const T *lamx, *lamy;
    int nx;
    T a, b;
    __device__ __forceinline__ void get(int m, T &al, T &be) const {
        const int j = m / nx, i = m - j * nx;
        const T lam = lamy[j] + lamx[i];
        be = (T)1 / ((T)1 - a * lam);
        al = ((T)1 + b * lam) * be;
    }
};

constexpr int SCAN_CHUNKS = 16;

// One (group of 32 modes, slab) unit of the blocked scan by a block of 32 * CHUNKS threads.
// CG: the rows were written earlier in the same kernel by other blocks (read through L2).
template <typename T, int C, int CHUNKS, bool CG, typename Coef>
__device__ __forceinline__ void mode_scan_unit(int nm, T *__restrict__ rh, int64_t ld, const Coef &coef,
                                               int steps, int coupled, int group, int slab) {
    __shared__ T ends[CHUNKS][32];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int m = group * 32 + lane;
    const bool act = m < nm;
    T al = (T)0, be = (T)0;
    if (act) coef.get(m, al, be);
    T alc = al;   // alpha^C (C a power of two)
#pragma unroll
    for (int c = 1; c < C; c *= 2) alc *= alc;
    const int first = coupled ? 0 : 1 + slab * steps;
    const int len = coupled ? steps + 1 : steps;
    T carry = (T)0;
    for (int t0 = 0; t0 < len; t0 += CHUNKS * C) {
        const int c0 = t0 + q * C;
        const int cl = min(C, max(0, len - c0));
        T *p = rh + (int64_t)(first + c0) * ld + m;
        T v[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
            if (act && i < cl) v[i] = CG ? __ldcg(p + (int64_t)i * ld) : p[(int64_t)i * ld];
            else v[i] = (T)0;
        }
        T acc = (T)0;
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const T b = (coupled && c0 + i == 0) ? v[i] : be * v[i];
            acc = al * acc + b;
            v[i] = acc;
        }
        ends[q][lane] = acc;
        __syncthreads();
        T cin = carry;
        for (int p2 = 0; p2 < q; ++p2) cin = alc * cin + ends[p2][lane];
        T cout = cin;
        for (int p2 = q; p2 < CHUNKS; ++p2) cout = alc * cout + ends[p2][lane];
        __syncthreads();
        T pw = al;
#pragma unroll
        for (int i = 0; i < C; ++i) {
            if (act && i < cl) p[(int64_t)i * ld] = v[i] + pw * cin;
            pw *= al;
        }
        carry = cout;   // used only when another tile follows, i.e. this one was full
    }
}

template <typename T, int C, typename Coef>
__global__ void __launch_bounds__(32 * SCAN_CHUNKS) k_mode_scan(int nm, T *__restrict__ rh, int64_t ld,
                                                                Coef coef, int steps, int coupled,
                                                                const int *__restrict__ done) {
    if (done && *done) return;
    mode_scan_unit<T, C, SCAN_CHUNKS, false, Coef>(nm, rh, ld, coef, steps, coupled, blockIdx.x, blockIdx.y);
}

// Rows per warp for a slab of len rows and CHUNKS warps: the smallest power of two that
// covers the slab in one tile, at most 32 (longer slabs take several tiles).
__host__ __device__ inline int mode_scan_rows(int len, int chunks) {
    int C = 2;
    while (C < 32 && chunks * C < len) C *= 2;
    return C;
}

// One launch over nm modes and n_cgs slabs (n_cgs = 0: the coupled march over rows 0..nt).
template <typename T, typename Coef>
inline void launch_mode_scan(int nm, T *rh, int64_t ld, Coef coef, int n_cgs, int nt, const int *done,
                             cudaStream_t s) {
    const int coupled = n_cgs <= 0 ? 1 : 0;
    const int nslabs = coupled ? 1 : n_cgs;
    const int steps = coupled ? nt : nt / n_cgs;
    const int len = coupled ? steps + 1 : steps;
    const int C = mode_scan_rows(len, SCAN_CHUNKS);
    const dim3 grid((nm + 31) / 32, nslabs);
#define MK_SCAN(CC)                                                                            \
    if (C == CC)                                                                               \
    k_mode_scan<T, CC, Coef><<<grid, 32 * SCAN_CHUNKS, 0, s>>>(nm, rh, ld, coef, steps, coupled, done)
    MK_SCAN(2);
    MK_SCAN(4);
    MK_SCAN(8);
    MK_SCAN(16);
    MK_SCAN(32);
#undef MK_SCAN
}

}  // namespace mk
