// Boys function F_m(T) = \int_0^1 u^{2m} exp(-T u^2) du on the device.
//
// T < BOYS_TMAX: tabulated values at T_i = i * BOYS_DT and a Taylor expansion
// in d = T - T_i, using dF_m/dT = -F_{m+1}:
//     F_m(T) = sum_k F_{m+k}(T_i) (-d)^k / k!
// (7 terms in FP64, 5 in FP32 with F_m(T_i) split as hi + lo; |d| <= BOYS_DT / 2).
// T >= BOYS_TMAX: F_0 = sqrt(pi / T) / 2 and F_m = F_{m-1} (2m - 1) / (2T);
// the neglected exp(-T) terms are below 1e-14 relative for m <= 6 there.
#pragma once
#include "common.cuh"
#include "f2.cuh"

namespace pcm {

constexpr double BOYS_TMAX = 48.0;
constexpr double BOYS_DT = 1.0 / 32.0;
constexpr double BOYS_INV_DT = 32.0;
constexpr int BOYS_NROW = 1540;            // rows 0 .. 48*32 (+ margin)
constexpr int BOYS_STRIDE64 = 16;          // doubles per row: m = 0 .. 15
constexpr int BOYS_STRIDE32 = 16;          // floats per row: F_0..F_9 (hi) then the lo parts of F_0..F_5
constexpr int BOYS_LO32 = 10;              // offset of the lo parts
constexpr int BOYS_MCOL = 16;              // columns generated
// The FP32 table holds a second block of BOYS_NROW rows after the first, for
// m <= 1: the Taylor coefficients pre-scaled for Horner evaluation in d,
//   h_{m,k} = (-1)^k F_{m+k}(T_i) / k!,  k = 0..4,
// laid out per row as h00 h01 h02 h03 | h04 lo0 h10 h11 | h12 h13 h14 lo1 | pad,
// with lo_m the FP32 residual of F_m(T_i) - h_{m,0}.
constexpr int BOYS_H32 = BOYS_NROW * BOYS_STRIDE32;
constexpr int BOYS_ALLOC32 = 2 * BOYS_NROW * BOYS_STRIDE32;

template <int MM>
__device__ __forceinline__ void boys_eval(double T, const double *__restrict__ tab, double (&F)[MM + 1])
{
    static_assert(MM + 6 < BOYS_STRIDE64, "Boys table too narrow");
    if (T < BOYS_TMAX) {
        const int i = min(max(__double2int_rn(T * BOYS_INV_DT), 0), BOYS_NROW - 1);
        const double d = T - (double)i * BOYS_DT;      // exact: BOYS_DT is a power of two
        const double *row = tab + (size_t)i * BOYS_STRIDE64;
        double r[MM + 7];
#pragma unroll
        for (int k = 0; k < MM + 7; ++k) r[k] = __ldg(row + k);
        const double e1 = -d, e2 = -d * 0.5, e3 = -d * (1.0 / 3.0), e4 = -d * 0.25, e5 = -d * 0.2,
                     e6 = -d * (1.0 / 6.0);
#pragma unroll
        for (int m = 0; m <= MM; ++m) {
            double s = fma(r[m + 6], e6, r[m + 5]);
            s = fma(s, e5, r[m + 4]);
            s = fma(s, e4, r[m + 3]);
            s = fma(s, e3, r[m + 2]);
            s = fma(s, e2, r[m + 1]);
            F[m] = fma(s, e1, r[m]);
        }
    } else {
        const double rs = rsqrt(T);
        const double half_inv_T = 0.5 * rs * rs;
        F[0] = 0.88622692545275801365 * rs;           // sqrt(pi) / 2
#pragma unroll
        for (int m = 1; m <= MM; ++m) F[m] = F[m - 1] * (double)(2 * m - 1) * half_inv_T;
    }
}

// FP32 near branch: row i of the table (T_i = i * BOYS_DT) and d = T - T_i
template <int MM>
__device__ __forceinline__ void boys_near32(int i, float d, const float *__restrict__ tab, float (&F)[MM + 1])
{
    if constexpr (MM <= 1) {
        // pre-scaled coefficients: Horner in d, the small terms first and
        // one rounding of the sum with the leading term
        const float4 *row = reinterpret_cast<const float4 *>(tab + BOYS_H32 + i * BOYS_STRIDE32);
        const float4 a = __ldg(row), b = __ldg(row + 1);
        F[0] = fmaf(fmaf(fmaf(fmaf(b.x, d, a.w), d, a.z), d, a.y), d, b.y) + a.x;
        if constexpr (MM == 1) {
            const float4 c = __ldg(row + 2);
            F[1] = fmaf(fmaf(fmaf(fmaf(c.z, d, c.y), d, c.x), d, b.w), d, c.w) + b.z;
        }
    } else {
        const float4 *row = reinterpret_cast<const float4 *>(tab + i * BOYS_STRIDE32);
        float r[BOYS_STRIDE32];
#pragma unroll
        for (int v = 0; v < BOYS_STRIDE32 / 4; ++v) {
            const float4 x = __ldg(row + v);
            r[4 * v] = x.x;
            r[4 * v + 1] = x.y;
            r[4 * v + 2] = x.z;
            r[4 * v + 3] = x.w;
        }
        const float e1 = -d, e2 = -d * 0.5f, e3 = -d * (1.0f / 3.0f), e4 = -d * 0.25f;
#pragma unroll
        for (int m = 0; m <= MM; ++m) {
            float s = fmaf(r[m + 4], e4, r[m + 3]);
            s = fmaf(s, e3, r[m + 2]);
            s = fmaf(s, e2, r[m + 1]);
            F[m] = fmaf(s, e1, r[BOYS_LO32 + m]) + r[m];  // the small terms first, one rounding of the sum
        }
    }
}

// sqrt(pi)/2 carried as hi + lo so that its FP32 rounding does not bias
// every far-field interaction the same way
constexpr float BOYS_C_HI = 0.88622692545275801365f;
constexpr float BOYS_C_LO = (float)(0.88622692545275801365 - (double)BOYS_C_HI);

template <int MM>
__device__ __forceinline__ void boys_eval(float T, const float *__restrict__ tab, float (&F)[MM + 1])
{
    // 5-term Taylor from F_m(T_i) stored as hi + lo: the table's FP32 rounding
    // and the truncation (whose d^4 remainder has one sign) would otherwise
    // both bias the result in the same direction for every interaction
    static_assert(MM + 4 < BOYS_LO32 && MM <= 5, "Boys table too narrow");
    if (T < (float)BOYS_TMAX) {
        // nearest row without float<->int conversions: adding 1.5 * 2^23 leaves
        // round(T * 32) in the low mantissa bits (0 <= T * 32 < 2^22)
        const float t = fmaf(T, (float)BOYS_INV_DT, 12582912.0f);
        const int i = __float_as_int(t) - 0x4B400000;
        const float d = fmaf(t - 12582912.0f, -(float)BOYS_DT, T);
        boys_near32<MM>(i, d, tab, F);
    } else {
        // hardware reciprocal square root, then one Newton step: the rounding
        // error left is that of the last FMA, without the approximation's
        // structured (input-correlated) error
        const float r0 = rsqrtf(T);
        const float e = fmaf(-T * r0, r0, 1.0f);
        const float rs = fmaf(0.5f * r0, e, r0);
        const float half_inv_T = 0.5f * rs * rs;
        F[0] = fmaf(BOYS_C_HI, rs, BOYS_C_LO * rs);
#pragma unroll
        for (int m = 1; m <= MM; ++m) F[m] = F[m - 1] * (float)(2 * m - 1) * half_inv_T;
    }
}

// The same evaluation for two lanes (two independent arguments).  Both lanes
// near: the row and offset are formed packed, the table Horner runs per lane
// (each lane reads its own row).  Both far: the far branch packed.  Mixed:
// each lane on its own.  Every lane's result equals the scalar boys_eval's.
template <int MM>
__device__ __forceinline__ void boys_eval2(f2 T, const float *__restrict__ tab, f2 (&F)[MM + 1])
{
    const bool n0 = T.v.x < (float)BOYS_TMAX, n1 = T.v.y < (float)BOYS_TMAX;
    if (n0 && n1) {
        const f2 t = fma2(T, f2((float)BOYS_INV_DT), f2(12582912.0f));
        const int i0 = __float_as_int(t.v.x) - 0x4B400000, i1 = __float_as_int(t.v.y) - 0x4B400000;
        const f2 d = fma2(t + f2(-12582912.0f), f2(-(float)BOYS_DT), T);
        float a[MM + 1], b[MM + 1];
        boys_near32<MM>(i0, d.v.x, tab, a);
        boys_near32<MM>(i1, d.v.y, tab, b);
#pragma unroll
        for (int m = 0; m <= MM; ++m) F[m] = f2(a[m], b[m]);
    } else if (!n0 && !n1) {
        const f2 r0(rsqrtf(T.v.x), rsqrtf(T.v.y));
        const f2 e = fma2((T * f2(-1.f)) * r0, r0, f2(1.0f));
        const f2 rs = fma2(f2(0.5f) * r0, e, r0);
        const f2 half_inv_T = (f2(0.5f) * rs) * rs;
        F[0] = fma2(f2(BOYS_C_HI), rs, f2(BOYS_C_LO) * rs);
#pragma unroll
        for (int m = 1; m <= MM; ++m) F[m] = (F[m - 1] * f2((float)(2 * m - 1))) * half_inv_T;
    } else {
        float a[MM + 1], b[MM + 1];
        boys_eval<MM>(T.v.x, tab, a);
        boys_eval<MM>(T.v.y, tab, b);
#pragma unroll
        for (int m = 0; m <= MM; ++m) F[m] = f2(a[m], b[m]);
    }
}

}  // namespace pcm
