// Reciprocal square root for the far-field and matrix-free hot loops: the
// hardware approximation (PTX rsqrt.approx.ftz.f32, about 2^-22.9 relative)
// without the special-case handling of subnormal inputs; every caller passes
// a positive normal argument (a squared distance between distinct points)
// or masks the result.
#pragma once
#include <cuda_runtime.h>

namespace pcm {

#ifndef PCM_RSQRT_PTX
#define PCM_RSQRT_PTX 1
#endif

__device__ __forceinline__ float rsqrt_fast(float x)
{
#if PCM_RSQRT_PTX
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return rsqrtf(x);
#endif
}

}  // namespace pcm
