// Packed FP32 pairs for sm_100-class GPUs: one FADD2 / FMUL2 / FFMA2
// instruction evaluates two independent lanes, each rounded exactly as the
// scalar FADD / FMUL / FFMA would (round to nearest even, no contraction
// between separate calls).  The integral kernels are bound by instruction
// issue rather than by the FP32 pipe, so evaluating two primitive pairs per
// instruction halves the issue cost of their floating-point work.
#pragma once
#include <cuda_runtime.h>

namespace pcm {

struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ explicit f2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
};

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    f2 r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    f2 r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
// a - b with one rounding: b * (-1) is exact
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return fma2(b, f2(-1.f), a); }
__device__ __forceinline__ f2 &operator+=(f2 &a, f2 b)
{
    a = a + b;
    return a;
}
__device__ __forceinline__ f2 hmadd(f2 a, f2 b, f2 c) { return fma2(a, b, c); }

}  // namespace pcm
