// Elements of A (Eq. 2, Eq. 3 read as zeta_k sqrt(2/pi) / S_k, Eq. 8) for
// the kernels that need single elements: the RBJ set-up (Section 4b-ii) and
// the near-pair list of the matrix-free operator.
//
//   AStored  reads a stored FP64 A;
//   AStoredDF reads the stored double-float A of PCM_MIXED as hi + lo (that
//            mode keeps no FP64 copy);
//   AFree    evaluates the element from the surface: exact() in FP64 exactly
//            as the stored A is built, bin() the coarse ordering key of
//            |A_kj| from an FP32 estimate (erf only where zeta' R < 6.5),
//            falling back to the FP64 value when the estimate lies within
//            1.2e-4 (relative) of a bin edge, so that the coarse bins agree
//            with those of the FP64 values.
#pragma once
#include "common.cuh"

namespace pcm {

// coarse bin of |A|: top 11 bits of the FP32 value (monotone in |A|)
__device__ __forceinline__ int rbj_bin(double a) { return (int)(__float_as_uint((float)fabs(a)) >> 20); }
// exact ordering key: FP64 bits (|A| >= 0, so bit order = value order)
__device__ __forceinline__ unsigned long long rbj_key64(double a)
{
    return (unsigned long long)__double_as_longlong(fabs(a));
}

// the FP32 distance test shared by every kernel that splits A into near
// pairs (stored exactly) and far pairs (1/R): one fixed sequence of roundings
__device__ __forceinline__ float r2_test32(float4 a, float4 b)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(dz, dz)));
}

struct AStored {
    const double *A;
    int lda;
    __device__ __forceinline__ double exact(int k, int j) const { return A[(size_t)k * lda + j]; }
    __device__ __forceinline__ int bin(int k, int j) const { return rbj_bin(A[(size_t)k * lda + j]); }
};

struct AStoredDF {
    const float *hi, *lo;
    int lda;
    __device__ __forceinline__ double exact(int k, int j) const
    {
        const size_t i = (size_t)k * lda + j;
        return (double)hi[i] + (double)lo[i];
    }
    __device__ __forceinline__ int bin(int k, int j) const { return rbj_bin(exact(k, j)); }
};

struct AFree {
    const double *px, *py, *pz, *pzeta, *pS;
    const int *pcls;
    int ncls;
    const double *zp;      // ncls x ncls: zeta' of Eq. 8 per pair of classes
    const float4 *pts;     // FP32 coordinates (x, y, z, -)

    __device__ __forceinline__ double exact(int k, int j) const
    {
        if (k == j) return pzeta[k] * 0.79788456080286535588 / pS[k];  // sqrt(2/pi)
        const double dx = px[k] - px[j], dy = py[k] - py[j], dz = pz[k] - pz[j];
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double inv = rsqrt(d2);
        const double a = zp[pcls[k] * ncls + pcls[j]] * (d2 * inv);
        // erf(a) rounds to 1 in FP64 for a > 6
        return (a > 6.0) ? inv : erf(a) * inv;
    }

    __device__ __forceinline__ int bin(int k, int j) const
    {
        const float4 a = pts[k], b = pts[j];
        const float r2 = r2_test32(a, b);
        const float rs = rsqrtf(r2);
        const float x = (float)zp[pcls[k] * ncls + pcls[j]] * (r2 * rs);
        const float v = (x < 6.5f) ? erff(x) * rs : rs;
        const unsigned u = __float_as_uint(v);
        const unsigned m = u & 0xFFFFFu;
        if (k == j || m < 1024u || m > 0xFFFFFu - 1024u) return rbj_bin(exact(k, j));
        return (int)(u >> 20);
    }
};

}  // namespace pcm
