// Randomized block-Jacobi apply (Section 4b-ii) of one RBJ block for a
// thread block: shared by the PCG update kernel and the persistent solver.
#pragma once
#include "common.cuh"

namespace pcm {

constexpr int RBJ_SPLIT = 4;   // threads per row in the block-Jacobi apply

// Randomized block-Jacobi apply for RBJ block b: its indices are
// perm[b*l .. b*l + nb) and its inverse is inv[b] (l x l, symmetric).  Unless
// init, first x += alpha p and r -= alpha Ap on the block's indices; then
// z = Minv r there.  Returns the block's r.r and r.z in thread 0.
__device__ __forceinline__ void rbj_apply_block(int M, int l, int b, const int *__restrict__ perm,
                                                const int *__restrict__ bstart, const double *__restrict__ inv,
                                                double *__restrict__ x, double *__restrict__ r,
                                                double *__restrict__ z, const double *__restrict__ p,
                                                const double *__restrict__ Ap, double alpha, int init, double *srb,
                                                double *rr_out, double *rz_out)
{
    const int base = bstart ? bstart[b] : b * l;
    const int nb = bstart ? bstart[b + 1] - base : min(l, M - base);
    double rr = 0.0, rz = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int k = perm[base + i];
        double rk = r[k];
        if (!init) {
            x[k] = fma(alpha, p[k], x[k]);
            rk = fma(-alpha, Ap[k], rk);
            r[k] = rk;
        }
        srb[i] = rk;
    }
    __syncthreads();
    const double *Mi = inv + (size_t)b * l * l;
    // z_i = sum_j Minv_ji r_j (Minv symmetric): RBJ_SPLIT threads share a row,
    // each summing every RBJ_SPLIT-th column, combined by shuffles
    const int sub = threadIdx.x % RBJ_SPLIT;
    for (int i0 = threadIdx.x / RBJ_SPLIT; i0 < ((nb + 31) / 32) * 32; i0 += blockDim.x / RBJ_SPLIT) {
        const int i = i0;
        double s = 0.0;
        if (i < nb)
            for (int j = sub; j < nb; j += RBJ_SPLIT) s = fma(Mi[(size_t)j * l + i], srb[j], s);
#pragma unroll
        for (int o = RBJ_SPLIT / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sub == 0 && i < nb) {
            z[perm[base + i]] = s;
            rr = fma(srb[i], srb[i], rr);
            rz = fma(srb[i], s, rz);
        }
    }
    __shared__ double sh[2][32];
    rr = warp_sum(rr);
    rz = warp_sum(rz);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = rr;
        sh[1][threadIdx.x >> 5] = rz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += sh[0][i];
            c += sh[1][i];
        }
        *rr_out = a;
        *rz_out = c;
    }
}

}  // namespace pcm
