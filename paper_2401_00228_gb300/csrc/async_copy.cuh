// Asynchronous global -> shared copies (cp.async, sm_80 and later) for kernels that stage the
// loads of later time steps in shared memory instead of registers.  A thread that reads back
// only the words it copied itself needs no block barrier: cp.async.wait_group makes its own
// completed copies visible to it.
#pragma once

#include <cuda_runtime.h>

namespace mk {

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// both addresses 8-byte aligned
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// close the copies issued since the last commit into one group (an empty group is allowed)
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// wait until at most N of this thread's groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace mk
