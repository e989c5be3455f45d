// Products and multiply-adds with fixed rounding (see the kernels that form the
// interpolated correction x = sigma v - Z vt).
#pragma once

#include <cuda_runtime.h>

namespace mk {

// A product and a multiply-add with fixed rounding: mul_rn is never contracted into an FMA and
// fma_rn always fuses.  A value formed at several sites of one kernel (a point's own x and the
// same x formed again as a neighbour's stencil operand) then rounds the same way at each.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return fma(a, b, c); }

}  // namespace mk
