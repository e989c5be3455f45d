// Shared-memory FFT of the sine-transform solvers (slab_dst.cu, inner_coop.cu): a complex
// FFT of length N = 2^logN <= 4096 by 256 threads in the Stockham auto-sort form (natural
// order in and out), radix-8 passes and one final radix-4 or radix-2 pass.  Each thread keeps
// its butterfly groups in registers between two barriers, the twiddles of each pass come from
// a table computed once on the host (a thread's R-1 factors are contiguous), and the shared
// array has one pad slot per 32 elements so that the strided stores of the early passes
// spread over the banks.  Every thread of the block must call these functions.
#pragma once

#include <cuda_runtime.h>

namespace mk {
namespace dstfft {

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


}  // namespace dstfft
}  // namespace mk
