// Double-float helpers (a value carried as FP32 hi + lo) for 1/R from split
// coordinates, shared by the stored-A build and the matrix-free operator.
#pragma once
#include <cuda_runtime.h>

namespace pcm {

__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void df_fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ void df_rsqrt(float dxh, float dxl, float dyh, float dyl, float dzh, float dzl, float &ih,
                                         float &il, float &r2)
{
    // R^2 = sum_d (dh + dl)^2 = dh^2 + (2 dh dl + dl^2)
    const float px = dxh * dxh, py = dyh * dyh, pz = dzh * dzh;
    const float ex = fmaf(dxh, dxh, -px) + dxl * fmaf(2.f, dxh, dxl);
    const float ey = fmaf(dyh, dyh, -py) + dyl * fmaf(2.f, dyh, dyl);
    const float ez = fmaf(dzh, dzh, -pz) + dzl * fmaf(2.f, dzh, dzl);
    float s1, t1, s2, t2;
    df_two_sum(px, py, s1, t1);
    df_two_sum(s1, pz, s2, t2);
    float Sh, Sl;
    df_fast_two_sum(s2, (t1 + t2) + ((ex + ey) + ez), Sh, Sl);
    // FP32 Newton step on the hardware estimate, then one double-float step:
    // r1 = r0 + r0 e / 2 with e = 1 - S r0^2 formed from the exact products
    float r0 = rsqrtf(Sh);
    r0 = fmaf(0.5f * r0, fmaf(-Sh * r0, r0, 1.f), r0);
    const float th = Sh * r0;
    const float tl = fmaf(Sh, r0, -th) + Sl * r0;
    const float uh = th * r0;
    const float ul = fmaf(th, r0, -uh) + tl * r0;
    const float e = (1.f - uh) - ul;
    df_fast_two_sum(r0, 0.5f * r0 * e, ih, il);
    r2 = Sh;
}

}  // namespace pcm
