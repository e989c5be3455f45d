// Deterministic two-stage reductions.
//
// Stage 1: each block reduces its values (warp shuffles, then one warp over the warp sums)
// and writes one partial per block.  Stage 2: the last block to arrive (atomic ticket after
// a memory fence) adds the partials in block order and runs a small epilogue on the
// result.  The order of every addition is fixed by the launch shape, so results are
// bitwise reproducible run to run.
#pragma once

#include "kernels.h"

namespace mk {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; result valid in thread 0.  Works for any blockDim <= 1024.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red_smem[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    v = warp_sum(v);
    __syncthreads();  // red_smem may still be read by a previous call
    if (lane == 0) red_smem[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        int nw = (nthreads + 31) >> 5;
        r = (lane < nw) ? red_smem[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// The same for a per-thread value in its arithmetic type T: the warp stage runs in T (an FP32
// value is summed by FP32 shuffles and adds, not at GB300's FP64 rate, 1/58 of FP32), the
// warp sums are then added in FP64.  Result valid in thread 0.
template <typename T>
__device__ __forceinline__ double block_sum_t(T v) {
    __shared__ double red_smem_t[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    const double wv = (double)warp_sum_t(v);
    __syncthreads();  // red_smem_t may still be read by a previous call
    if (lane == 0) red_smem_t[warp] = wv;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        int nw = (nthreads + 31) >> 5;
        r = (lane < nw) ? red_smem_t[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

__device__ __forceinline__ int linear_block() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ int num_blocks() { return gridDim.x * gridDim.y * gridDim.z; }

// Ticket: returns true in every thread of the last block to finish.  `wrote`: this thread
// stored one of the block's partials; only those threads fence (making the partial visible
// GPU-wide before the block's ticket is taken), the others' stores need no ordering here.
__device__ __forceinline__ bool last_block_ticket(unsigned *counter, bool wrote) {
    __shared__ bool am_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (wrote) __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned t = atomicAdd(counter, 1u);
        am_last = (t == (unsigned)num_blocks() - 1u);
    }
    __syncthreads();
    return am_last;
}

// Sum of nb partials in order, by the whole block; result in thread 0.
__device__ __forceinline__ double sum_partials(const double *p, int nb) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    // each thread sums a contiguous run so that the order is fixed by (nb, nthreads)
    int per = (nb + nthreads - 1) / nthreads;
    int s0 = tid * per, s1 = min(s0 + per, nb);
    double acc = 0.0;
    // L2 loads (the partials were written by other blocks before their fence), unrolled so
    // that they are in flight together
#pragma unroll 8
    for (int s = s0; s < s1; ++s) acc += __ldcg(p + s);
    return block_sum(acc);
}

// Epilogues on a completed sum of squares.
__device__ __forceinline__ void run_epilogue(double total, KState ks, int epi) {
    double *misc = ks.misc();
    misc[5] = total;
    if (epi == EPI_BETA) {
        double beta = sqrt(total);
        misc[0] = beta;
        ks.sigma()[0] = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(beta)) ks.flags[3] = 1;
    } else if (epi == EPI_OUTER_START || epi == EPI_OUTER_INIT) {
        double beta = sqrt(total);
        if (epi == EPI_OUTER_INIT) {
            misc[3] = beta;
            misc[1] = misc[7] * beta;
            ks.flags[4] = 0;
        }
        misc[0] = beta;
        misc[4] = beta;
        ks.sigma()[0] = beta > 0.0 ? 1.0 / beta : 0.0;
        ks.g()[0] = beta;
        ks.flags[1] = 0;
        ks.flags[2] = 0;
        ks.flags[0] = (beta <= misc[1]) ? 1 : 0;   // misc[1] = tol * ||f||
        if (!isfinite(beta)) {
            ks.flags[3] = 1;
            ks.flags[0] = 1;
        }
    }
}

// Block partial of a per-thread value in its arithmetic type (block_sum_t) -> partial slot;
// last block sums and runs the epilogue.
template <typename T>
__device__ __forceinline__ void block_partial_and_finish_t(T v, const ReduceScratch &rs, int slot,
                                                           KState ks, int epi) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    double bs = block_sum_t(v);
    double *part = rs.partials + (int64_t)slot * rs.max_blocks;
    if (tid == 0) part[linear_block()] = bs;
    if (last_block_ticket(rs.counter + slot, tid == 0)) {
        double tot = sum_partials(part, num_blocks());
        if (tid == 0) {
            run_epilogue(tot, ks, epi);
            rs.counter[slot] = 0u;
        }
    }
}

// Block partial of `v` -> partial slot; last block sums and runs the epilogue.
__device__ __forceinline__ void block_partial_and_finish(double v, const ReduceScratch &rs,
                                                         int slot, KState ks, int epi) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    double bs = block_sum(v);
    double *part = rs.partials + (int64_t)slot * rs.max_blocks;
    if (tid == 0) part[linear_block()] = bs;
    if (last_block_ticket(rs.counter + slot, tid == 0)) {
        double tot = sum_partials(part, num_blocks());
        if (tid == 0) {
            run_epilogue(tot, ks, epi);
            rs.counter[slot] = 0u;
        }
    }
}

}  // namespace mk
