// Row-pair GEMV shared by the single-molecule and the batched solvers.
#pragma once
#include "common.cuh"

namespace pcm {

// Row-pair GEMV: a block of 8 warps computes two rows, four warps per row,
// each warp a quarter of the columns (whole vector loads), so the grid has
// M/2 blocks and no wave tail.  Returns, in thread 0, the block's x.y partial
// (x64 the FP64 copy of the input vector).  rp: the row pair (rows 2 rp, 2 rp + 1).
template <typename TA>
__device__ __forceinline__ double gemv_rowpair(int rp, int M, int lda, const TA *__restrict__ A,
                                               const TA *__restrict__ x, const double *__restrict__ x64,
                                               double *__restrict__ y)
{
    __shared__ double sh[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = rp * 2 + (w >> 2), seg = w & 3;
    constexpr int V = 16 / sizeof(TA);                    // elements per 16-byte load
    const int seglen = ((M + 3) / 4 + 32 * V - 1) / (32 * V) * (32 * V);
    const int c0 = seg * seglen, c1 = min(M, c0 + seglen);
    double part = 0.0;
    if (row < M && c0 < c1) {
        const TA *a = A + (size_t)row * lda;
        TA s0 = TA(0), s1 = TA(0);
        int col = c0 + V * lane;
        for (; col + 32 * V + V - 1 < c1; col += 64 * V) {
            if constexpr (sizeof(TA) == 4) {
                const float4 a0 = *reinterpret_cast<const float4 *>(a + col);
                const float4 a1 = *reinterpret_cast<const float4 *>(a + col + 32 * V);
                const float4 x0 = *reinterpret_cast<const float4 *>(x + col);
                const float4 x1 = *reinterpret_cast<const float4 *>(x + col + 32 * V);
                s0 = fmaf(a0.x, x0.x, fmaf(a0.y, x0.y, fmaf(a0.z, x0.z, fmaf(a0.w, x0.w, s0))));
                s1 = fmaf(a1.x, x1.x, fmaf(a1.y, x1.y, fmaf(a1.z, x1.z, fmaf(a1.w, x1.w, s1))));
            } else {
                const double2 a0 = *reinterpret_cast<const double2 *>(a + col);
                const double2 a1 = *reinterpret_cast<const double2 *>(a + col + 32 * V);
                const double2 x0 = *reinterpret_cast<const double2 *>(x + col);
                const double2 x1 = *reinterpret_cast<const double2 *>(x + col + 32 * V);
                s0 = fma(a0.x, x0.x, fma(a0.y, x0.y, s0));
                s1 = fma(a1.x, x1.x, fma(a1.y, x1.y, s1));
            }
        }
        for (; col < c1; col += 32 * V)
#pragma unroll
            for (int t = 0; t < V; ++t)
                if (col + t < c1) s0 += a[col + t] * x[col + t];
        part = (double)warp_sum(s0 + s1);
    }
    if (lane == 0) sh[w] = part;
    __syncthreads();
    double blk = 0.0;
    if (threadIdx.x == 0) {
        for (int r2 = 0; r2 < 2; ++r2) {
            const int rr = rp * 2 + r2;
            if (rr < M) {
                const double v = sh[4 * r2] + sh[4 * r2 + 1] + sh[4 * r2 + 2] + sh[4 * r2 + 3];
                y[rr] = v;
                blk = fma(x64[rr], v, blk);
            }
        }
    }
    __syncthreads();
    return blk;
}

// The same GEMV in double-float arithmetic on the FP32 pipes: A = Ahi + Alo
// (two FP32 matrices), x = xhi + xlo.  Per element the product Ahi xhi is
// formed exactly (p + e, e = fma(Ahi, xhi, -p)), the cross terms Ahi xlo +
// Alo xhi are added to e, and (p, e) enter a float-float running sum (TwoSum
// on the high part, the errors collected in the low part); Alo xlo is dropped.
// Each element's product carries about 2^-47 of its size in error, so y is
// accurate to ~1e-14 of sum_l |A_kl x_l|: the FP64 result without the FP64
// pipe, which on this GPU runs 64 times slower than FP32 and would bound an
// FP64 GEMV below the HBM rate.
__device__ __forceinline__ void df_acc(float &S, float &C, float a, float al, float x, float xl)
{
    const float p = a * x;
    const float e = fmaf(a, xl, fmaf(al, x, fmaf(a, x, -p)));
    const float s = S + p;
    const float bp = s - S;
    const float err = (S - (s - bp)) + (p - bp);
    C += err + e;
    S = s;
}

__device__ __forceinline__ double gemv_rowpair_df(int rp, int M, int lda, const float *__restrict__ Ahi,
                                                  const float *__restrict__ Alo, const float *__restrict__ xhi,
                                                  const float *__restrict__ xlo, const double *__restrict__ x64,
                                                  double *__restrict__ y)
{
    __shared__ double sh[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = rp * 2 + (w >> 2), seg = w & 3;
    constexpr int V = 4;
    const int seglen = ((M + 3) / 4 + 32 * V - 1) / (32 * V) * (32 * V);
    const int c0 = seg * seglen, c1 = min(M, c0 + seglen);
    double part = 0.0;
    if (row < M && c0 < c1) {
        const float *a = Ahi + (size_t)row * lda, *al = Alo + (size_t)row * lda;
        float S = 0.f, C = 0.f;
        int col = c0 + V * lane;
        for (; col + V - 1 < c1; col += 32 * V) {
            const float4 h = *reinterpret_cast<const float4 *>(a + col);
            const float4 l = *reinterpret_cast<const float4 *>(al + col);
            const float4 u = *reinterpret_cast<const float4 *>(xhi + col);
            const float4 v = *reinterpret_cast<const float4 *>(xlo + col);
            df_acc(S, C, h.x, l.x, u.x, v.x);
            df_acc(S, C, h.y, l.y, u.y, v.y);
            df_acc(S, C, h.z, l.z, u.z, v.z);
            df_acc(S, C, h.w, l.w, u.w, v.w);
        }
        for (int t = 0; t < V; ++t)
            if (col + t < c1) df_acc(S, C, a[col + t], al[col + t], xhi[col + t], xlo[col + t]);
        part = warp_sum((double)S + (double)C);
    }
    if (lane == 0) sh[w] = part;
    __syncthreads();
    double blk = 0.0;
    if (threadIdx.x == 0) {
        for (int r2 = 0; r2 < 2; ++r2) {
            const int rr = rp * 2 + r2;
            if (rr < M) {
                const double v = sh[4 * r2] + sh[4 * r2 + 1] + sh[4 * r2 + 2] + sh[4 * r2 + 3];
                y[rr] = v;
                blk = fma(x64[rr], v, blk);
            }
        }
    }
    __syncthreads();
    return blk;
}

}  // namespace pcm
