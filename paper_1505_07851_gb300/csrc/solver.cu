// Solve A q = rhs (Eq. 1) by preconditioned conjugate gradients with the
// residual test of Eq. 20 (Section 4b), Jacobi or randomized block-Jacobi
// preconditioning (Section 4b-ii), and the energy of Eq. 13.
//
// A is stored in FP64 (row-major, leading dimension lda).  Each PCG
// iteration is three kernels:
//   pcg_gemv     Ap = A p, p.Ap                       -> alpha
//   pcg_update   x += alpha p, r -= alpha Ap, z = C r, r.r, r.z -> beta, stop test
//   pcg_dir      p = z + beta p
// Scalars stay on the device; reductions use per-block partial sums added in
// block order by the last block to finish (deterministic).  Every kernel
// returns at once when the stop flag is set, so the host may enqueue a batch
// of iterations and look at the flag once per batch.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "context.h"

namespace pcm {

enum { S_RZ = 0, S_PAP, S_ALPHA, S_BETA, S_RNORM, S_DELTA, S_RR, S_NSCAL };
enum { I_DONE = 0, I_ITER, I_MAXIT, I_CONV, I_NINT };
constexpr int GV_NT = 256;          // 8 warps, one row per warp at a time
constexpr int UP_NT = 256;
constexpr int MAX_PART = 8192;      // partial-sum slots

// last-block pattern: returns true in the block that finished last; that
// block's thread 0 may then read every partial written before the fence.
__device__ __forceinline__ bool last_block(unsigned int *counter)
{
    __shared__ bool amlast;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(counter, 1u);
        amlast = (prev == gridDim.x - 1);
    }
    __syncthreads();
    return amlast;
}

// y = A x for rows handled by this block; partial[b] = sum_rows x_row y_row
__device__ __forceinline__ double gemv_rows(int M, int lda, const double *__restrict__ A,
                                            const double *__restrict__ x, double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * GV_NT + threadIdx.x) >> 5;
    const int nw = (gridDim.x * GV_NT) >> 5;
    double dotp = 0.0;
    for (int row = wg; row < M; row += nw) {
        const double *a = A + (size_t)row * lda;
        double s0 = 0.0, s1 = 0.0;
        int col = 2 * lane;
        // lda is a multiple of 32: double2 loads are aligned
        for (; col + 193 < M; col += 256) {
            const double2 a0 = *reinterpret_cast<const double2 *>(a + col);
            const double2 a1 = *reinterpret_cast<const double2 *>(a + col + 64);
            const double2 a2 = *reinterpret_cast<const double2 *>(a + col + 128);
            const double2 a3 = *reinterpret_cast<const double2 *>(a + col + 192);
            s0 = fma(a0.x, __ldg(x + col), s0);
            s1 = fma(a0.y, __ldg(x + col + 1), s1);
            s0 = fma(a1.x, __ldg(x + col + 64), s0);
            s1 = fma(a1.y, __ldg(x + col + 65), s1);
            s0 = fma(a2.x, __ldg(x + col + 128), s0);
            s1 = fma(a2.y, __ldg(x + col + 129), s1);
            s0 = fma(a3.x, __ldg(x + col + 192), s0);
            s1 = fma(a3.y, __ldg(x + col + 193), s1);
        }
        for (; col < M; col += 64) {
            s0 = fma(a[col], __ldg(x + col), s0);
            if (col + 1 < M) s1 = fma(a[col + 1], __ldg(x + col + 1), s1);
        }
        const double s = warp_sum(s0 + s1);
        if (lane == 0) {
            y[row] = s;
            dotp = fma(x[row], s, dotp);
        }
    }
    return dotp;  // valid in lane 0 of each warp
}

__device__ __forceinline__ double block_sum_warps(double v /* lane-0 values */)
{
    __shared__ double sh[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(GV_NT) pcg_gemv_kernel(int M, int lda, const double *__restrict__ A,
                                                         const double *__restrict__ p, double *__restrict__ Ap,
                                                         double *__restrict__ part, double *__restrict__ scal,
                                                         int *__restrict__ iscal, unsigned int *__restrict__ counter)
{
    if (iscal[I_DONE]) return;
    const double d = gemv_rows(M, lda, A, p, Ap);
    const double bsum = block_sum_warps(d);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum;
    if (last_block(counter)) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (unsigned int b = 0; b < gridDim.x; ++b) s += ((volatile double *)part)[b];
            scal[S_PAP] = s;
            scal[S_ALPHA] = scal[S_RZ] / s;
            *counter = 0;
        }
    }
}

// After the reductions of r.r and r.z: stop test (Eq. 20) and beta.
__device__ __forceinline__ void finish_update(double rr, double rz, double *scal, int *iscal)
{
    const double rn = sqrt(rr);
    scal[S_RNORM] = rn;
    scal[S_RR] = rr;
    const int it = iscal[I_ITER] + 1;
    iscal[I_ITER] = it;
    if (rn < scal[S_DELTA]) {
        iscal[I_DONE] = 1;
        iscal[I_CONV] = 1;
    } else if (it >= iscal[I_MAXIT]) {
        iscal[I_DONE] = 1;
    }
    scal[S_BETA] = rz / scal[S_RZ];
    scal[S_RZ] = rz;
}

// Jacobi (dinv != null) or no preconditioner
__global__ void __launch_bounds__(UP_NT) pcg_update_diag_kernel(int M, const double *__restrict__ dinv,
                                                                double *__restrict__ x, double *__restrict__ r,
                                                                double *__restrict__ z, const double *__restrict__ p,
                                                                const double *__restrict__ Ap, double *__restrict__ part,
                                                                double *__restrict__ scal, int *__restrict__ iscal,
                                                                unsigned int *__restrict__ counter)
{
    if (iscal[I_DONE]) return;
    const double alpha = scal[S_ALPHA];
    double rr = 0.0, rz = 0.0;
    for (int k = blockIdx.x * UP_NT + threadIdx.x; k < M; k += gridDim.x * UP_NT) {
        x[k] = fma(alpha, p[k], x[k]);
        const double rk = fma(-alpha, Ap[k], r[k]);
        r[k] = rk;
        const double zk = dinv ? rk * dinv[k] : rk;
        z[k] = zk;
        rr = fma(rk, rk, rr);
        rz = fma(rk, zk, rz);
    }
    __shared__ double sh[2][UP_NT / 32];
    rr = warp_sum(rr);
    rz = warp_sum(rz);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = rr;
        sh[1][threadIdx.x >> 5] = rz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < UP_NT / 32; ++i) {
            a += sh[0][i];
            b += sh[1][i];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (last_block(counter)) {
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (unsigned int i = 0; i < gridDim.x; ++i) {
                a += ((volatile double *)part)[2 * i];
                b += ((volatile double *)part)[2 * i + 1];
            }
            finish_update(a, b, scal, iscal);
            *counter = 0;
        }
    }
}

// Randomized block-Jacobi: one block per RBJ block; the block's indices are
// perm[b*l .. b*l + nb) and its inverse is inv[b] (l x l, symmetric).
// With alpha_from_scal = false (initialisation) x and r are left unchanged.
__global__ void pcg_update_rbj_kernel(int M, int l, const int *__restrict__ perm, const double *__restrict__ inv,
                                      double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                                      const double *__restrict__ p, const double *__restrict__ Ap,
                                      double *__restrict__ part, double *__restrict__ scal, int *__restrict__ iscal,
                                      unsigned int *__restrict__ counter, int init)
{
    extern __shared__ double srb[];  // l entries
    if (iscal[I_DONE]) return;
    const int b = blockIdx.x;
    const int base = b * l;
    const int nb = min(l, M - base);
    const double alpha = init ? 0.0 : scal[S_ALPHA];
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
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s = fma(Mi[(size_t)j * l + i], srb[j], s);
        z[perm[base + i]] = s;
        rr = fma(srb[i], srb[i], rr);
        rz = fma(srb[i], s, rz);
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
        part[2 * b] = a;
        part[2 * b + 1] = c;
    }
    if (last_block(counter)) {
        if (threadIdx.x == 0) {
            double a = 0.0, c = 0.0;
            for (unsigned int i = 0; i < gridDim.x; ++i) {
                a += ((volatile double *)part)[2 * i];
                c += ((volatile double *)part)[2 * i + 1];
            }
            if (init) {
                scal[S_RZ] = c;
                scal[S_RR] = a;
                scal[S_RNORM] = sqrt(a);
                if (sqrt(a) < scal[S_DELTA]) {
                    iscal[I_DONE] = 1;
                    iscal[I_CONV] = 1;
                }
            } else {
                finish_update(a, c, scal, iscal);
            }
            *counter = 0;
        }
    }
}

__global__ void pcg_dir_kernel(int M, const double *__restrict__ z, double *__restrict__ p,
                               const double *__restrict__ scal, const int *__restrict__ iscal)
{
    if (iscal[I_DONE]) return;
    const double beta = scal[S_BETA];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x)
        p[k] = fma(beta, p[k], z[k]);
}

// initialisation: r = b - (A x0) or r = b; x = x0 or 0
__global__ void pcg_init_kernel(int M, const double *__restrict__ b, const double *__restrict__ Ax0, int warm,
                                double *__restrict__ x, double *__restrict__ r)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        if (warm) {
            r[k] = b[k] - Ax0[k];
        } else {
            x[k] = 0.0;
            r[k] = b[k];
        }
    }
}

// z = D r for the diagonal preconditioners at initialisation, with r.r, r.z
__global__ void __launch_bounds__(UP_NT) pcg_init_diag_kernel(int M, const double *__restrict__ dinv,
                                                              const double *__restrict__ r, double *__restrict__ z,
                                                              double *__restrict__ part, double *__restrict__ scal,
                                                              int *__restrict__ iscal, unsigned int *__restrict__ counter)
{
    double rr = 0.0, rz = 0.0;
    for (int k = blockIdx.x * UP_NT + threadIdx.x; k < M; k += gridDim.x * UP_NT) {
        const double rk = r[k];
        const double zk = dinv ? rk * dinv[k] : rk;
        z[k] = zk;
        rr = fma(rk, rk, rr);
        rz = fma(rk, zk, rz);
    }
    __shared__ double sh[2][UP_NT / 32];
    rr = warp_sum(rr);
    rz = warp_sum(rz);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = rr;
        sh[1][threadIdx.x >> 5] = rz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < UP_NT / 32; ++i) {
            a += sh[0][i];
            b += sh[1][i];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (last_block(counter)) {
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (unsigned int i = 0; i < gridDim.x; ++i) {
                a += ((volatile double *)part)[2 * i];
                b += ((volatile double *)part)[2 * i + 1];
            }
            scal[S_RZ] = b;
            scal[S_RR] = a;
            scal[S_RNORM] = sqrt(a);
            if (sqrt(a) < scal[S_DELTA]) {
                iscal[I_DONE] = 1;
                iscal[I_CONV] = 1;
            }
            *counter = 0;
        }
    }
}

__global__ void copy_kernel(int M, const double *__restrict__ a, double *__restrict__ b)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) b[k] = a[k];
}

__global__ void gemv_plain_kernel(int M, int lda, const double *__restrict__ A, const double *__restrict__ x,
                                  double *__restrict__ y, double *__restrict__ part)
{
    const double d = gemv_rows(M, lda, A, x, y);
    const double bsum = block_sum_warps(d);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum;
}

// ---------------------------------------------------------------------------
// RBJ permutation (Section 4b-ii), one block of 1024 threads walking the
// pivots in sequence.  Pivot j is position floor((r_j >> 32) * nU / 2^32) of
// the ascending list of unassigned indices, r_j = splitmix64 output j; its
// block is the pivot followed by the l - 1 unassigned indices of largest
// |A_kj| (ties: lower index first).
// ---------------------------------------------------------------------------
constexpr int RBJ_NT = 1024;

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t j)
{
    // published splitmix64: state advances by the golden gamma, then mix
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(RBJ_NT) rbj_perm_kernel(int M, int lda, const double *__restrict__ A, int l,
                                                          unsigned long long seed, int *__restrict__ U,
                                                          int *__restrict__ U2, int *__restrict__ perm,
                                                          int *__restrict__ status)
{
    __shared__ unsigned int hist[256];
    __shared__ int sh_int[RBJ_NT / 32 + 1];
    __shared__ int s_nU, s_k, s_cnt_gt, s_need_eq;
    __shared__ unsigned long long s_prefix;
    for (int i = threadIdx.x; i < M; i += RBJ_NT) U[i] = i;
    if (threadIdx.x == 0) s_nU = M;
    __syncthreads();
    int out = 0;
    uint64_t draw = 0;
    int guard = 0;
    while (s_nU > 0) {
        if (++guard > M + 1) {  // cannot happen: every pass removes at least the pivot
            if (threadIdx.x == 0) *status = 1;
            return;
        }
        const int nU = s_nU;
        if (threadIdx.x == 0) {
            const uint64_t r = splitmix64_at(seed, draw);
            const int pos = (int)(((r >> 32) * (uint64_t)nU) >> 32);
            s_k = U[pos];
        }
        ++draw;
        __syncthreads();
        const int k = s_k;
        const int nsel = min(l - 1, nU - 1);
        const double *row = A + (size_t)k * lda;
        // radix select of the nsel-th largest key (bits of |A_kj|, j != k)
        unsigned long long prefix = 0, mask = 0;
        int need = nsel;  // how many still to take at or below the current prefix
        if (nsel > 0) {
            for (int shift = 56; shift >= 0; shift -= 8) {
                for (int i = threadIdx.x; i < 256; i += RBJ_NT) hist[i] = 0;
                __syncthreads();
                for (int i = threadIdx.x; i < nU; i += RBJ_NT) {
                    const int j = U[i];
                    if (j == k) continue;
                    const unsigned long long key = (unsigned long long)__double_as_longlong(fabs(row[j]));
                    if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255], 1u);
                }
                __syncthreads();
                // the bin holding the need-th largest key: warp 0 scans the 256
                // bins from the top, 8 per lane
                if (threadIdx.x < 32) {
                    const int lane = threadIdx.x;
                    int loc = 0;
                    for (int b = 0; b < 8; ++b) loc += (int)hist[255 - 8 * lane - b];
                    int inc = loc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    const unsigned ball = __ballot_sync(0xffffffffu, inc >= need);
                    if (lane == __ffs(ball) - 1) {
                        int acc = inc - loc, bin = 255 - 8 * lane;
                        for (int b = 0; b < 7; ++b, --bin) {
                            if (acc + (int)hist[bin] >= need) break;
                            acc += (int)hist[bin];
                        }
                        s_prefix = prefix | ((unsigned long long)bin << shift);
                        s_need_eq = need - acc;
                    }
                }
                __syncthreads();
                prefix = s_prefix;
                need = s_need_eq;
                mask |= 255ull << shift;
                __syncthreads();
            }
            // keys > prefix are all taken; `need` of the keys == prefix (lowest index first)
        }
        const unsigned long long thr = prefix;
        const int need_eq = need;
        // scan in list order: flag = taken (pivot, key > thr, or among the first need_eq keys == thr)
        if (threadIdx.x == 0) {
            perm[out] = k;
            s_cnt_gt = 0;
        }
        __syncthreads();
        int taken_base = out + 1;
        int eq_seen = 0, kept_base = 0;
        for (int c0 = 0; c0 < nU; c0 += RBJ_NT) {
            const int i = c0 + threadIdx.x;
            int j = -1, sel = 0, iseq = 0;
            if (i < nU) {
                j = U[i];
                if (j != k && nsel > 0) {
                    const unsigned long long key = (unsigned long long)__double_as_longlong(fabs(row[j]));
                    if (key > thr) sel = 1;
                    else if (key == thr) iseq = 1;
                }
            }
            // rank among equal keys in this chunk
            int eqx;
            {
                int tot;
                const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
                int xs = iseq;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, xs, o);
                    if (lane >= o) xs += y;
                }
                if (lane == 31) sh_int[wid] = xs;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int run = 0;
                    for (int w = 0; w < RBJ_NT / 32; ++w) {
                        int t = sh_int[w];
                        sh_int[w] = run;
                        run += t;
                    }
                    sh_int[RBJ_NT / 32] = run;
                }
                __syncthreads();
                eqx = sh_int[wid] + xs - iseq;
                tot = sh_int[RBJ_NT / 32];
                __syncthreads();
                if (iseq && eq_seen + eqx < need_eq) sel = 1;
                eq_seen += tot;
            }
            // compact: selected -> perm, unselected (and not pivot) -> U2
            const int keep = (i < nU && j != k && !sel) ? 1 : 0;
            int ex_sel, ex_keep, tot_sel, tot_keep;
            {
                const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
                int packed = (sel << 16) | keep;  // counts < 65536 per chunk
                int xs = packed;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, xs, o);
                    if (lane >= o) xs += y;
                }
                if (lane == 31) sh_int[wid] = xs;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int run = 0;
                    for (int w = 0; w < RBJ_NT / 32; ++w) {
                        int t = sh_int[w];
                        sh_int[w] = run;
                        run += t;
                    }
                    sh_int[RBJ_NT / 32] = run;
                }
                __syncthreads();
                const int ex = sh_int[wid] + xs - packed;
                const int tt = sh_int[RBJ_NT / 32];
                __syncthreads();
                ex_sel = ex >> 16;
                ex_keep = ex & 0xffff;
                tot_sel = tt >> 16;
                tot_keep = tt & 0xffff;
            }
            if (sel) perm[taken_base + ex_sel] = j;
            if (keep) U2[kept_base + ex_keep] = j;
            taken_base += tot_sel;
            kept_base += tot_keep;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kept_base; i += RBJ_NT) U[i] = U2[i];
        out = taken_base;
        if (threadIdx.x == 0) s_nU = kept_base;
        __syncthreads();
    }
    if (threadIdx.x == 0 && out != M) *status = 2;
}

// In-place Cholesky of one l x l block (lower), then the inverse by solving
// L L^T X = I column by column.  One thread block per RBJ block.
__global__ void rbj_invert_kernel(int M, int lda, const double *__restrict__ A, int l, const int *__restrict__ perm,
                                  double *__restrict__ work, double *__restrict__ inv, int *__restrict__ status)
{
    const int b = blockIdx.x;
    const int base = b * l;
    const int nb = min(l, M - base);
    double *W = work + (size_t)b * l * l;
    double *X = inv + (size_t)b * l * l;
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        W[(size_t)i * l + j] = A[(size_t)perm[base + i] * lda + perm[base + j]];
    }
    __syncthreads();
    __shared__ double dkk;
    for (int k = 0; k < nb; ++k) {
        if (threadIdx.x == 0) {
            const double a = W[(size_t)k * l + k];
            if (!(a > 0.0)) *status = 3;
            dkk = sqrt(fmax(a, 1e-300));
            W[(size_t)k * l + k] = dkk;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) W[(size_t)i * l + k] /= dkk;
        __syncthreads();
        for (int t = threadIdx.x; t < (nb - k - 1) * (nb - k - 1); t += blockDim.x) {
            const int i = k + 1 + t / (nb - k - 1), j = k + 1 + t % (nb - k - 1);
            if (j <= i) W[(size_t)i * l + j] -= W[(size_t)i * l + k] * W[(size_t)j * l + k];
        }
        __syncthreads();
    }
    // columns of the inverse: L y = e_c, L^T x = y (x overwrites column c of X)
    for (int col = threadIdx.x; col < nb; col += blockDim.x) {
        for (int i = 0; i < nb; ++i) {
            double s = (i == col) ? 1.0 : 0.0;
            for (int j = col; j < i; ++j) s -= W[(size_t)i * l + j] * X[(size_t)j * l + col];
            X[(size_t)i * l + col] = (i < col) ? 0.0 : s / W[(size_t)i * l + i];
        }
        for (int i = nb - 1; i >= 0; --i) {
            double s = X[(size_t)i * l + col];
            for (int j = i + 1; j < nb; ++j) s -= W[(size_t)j * l + i] * X[(size_t)j * l + col];
            X[(size_t)i * l + col] = s / W[(size_t)i * l + i];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int gemv_grid(pcm_ctx *c) { return std::min(MAX_PART, std::max(1, (c->M + 7) / 8)); }

int solver_prepare(pcm_ctx *c)
{
    if (c->pc_ready) return PCM_OK;
    const int M = c->M;
    int kind = c->opt.precond;
    if (kind == PCM_PRECOND_AUTO) kind = (M < c->opt.jacobi_below) ? PCM_PRECOND_JACOBI : PCM_PRECOND_RBJ;
    c->pc_kind = kind;
    PCM_TRY(c->iscal.alloc(64));
    if (kind == PCM_PRECOND_RBJ) {
        const int l = std::max(1, std::min(c->opt.rbj_block, M));
        c->rbj_l = l;
        c->rbj_nblk = (M + l - 1) / l;
        PCM_TRY(c->rbj_perm.alloc(M));
        DBuf<int> &U = c->si[0], &U2 = c->si[1];
        PCM_TRY(U.alloc(M));
        PCM_TRY(U2.alloc(M));
        PCM_CUDA(cudaMemsetAsync(c->iscal.p, 0, 64 * sizeof(int), c->stream));
        rbj_perm_kernel<<<1, RBJ_NT, 0, c->stream>>>(M, c->lda, c->A.p, l, c->opt.seed, U.p, U2.p, c->rbj_perm.p,
                                                     c->iscal.p + 16);
        PCM_LAUNCHED(c);
        PCM_TRY(c->rbj_inv.alloc((size_t)c->rbj_nblk * l * l));
        DBuf<double> &work = c->sd[0];
        PCM_TRY(work.alloc((size_t)c->rbj_nblk * l * l));
        const int nt = std::min(1024, std::max(32, (l + 31) / 32 * 32));
        rbj_invert_kernel<<<c->rbj_nblk, nt, 0, c->stream>>>(M, c->lda, c->A.p, l, c->rbj_perm.p, work.p,
                                                             c->rbj_inv.p, c->iscal.p + 16);
        PCM_LAUNCHED(c);
        int st = 0;
        PCM_CUDA(cudaMemcpyAsync(&st, c->iscal.p + 16, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        if (st != 0) {
            set_last_error("RBJ set-up failed (status %d: %s)", st,
                           st == 3 ? "a diagonal block is not positive definite" : "bad permutation");
            return PCM_ERR_CUDA;
        }
    }
    c->pc_ready = true;
    return PCM_OK;
}

int solver_run(pcm_ctx *c, const double *drhs, double delta, double *dq, bool warm, pcm_stats *st)
{
    PCM_TRY(solver_prepare(c));
    const int M = c->M;
    PCM_TRY(c->vr.alloc(M));
    PCM_TRY(c->vz.alloc(M));
    PCM_TRY(c->vp.alloc(M));
    PCM_TRY(c->vAp.alloc(M));
    PCM_TRY(c->red.alloc(2 * (size_t)std::max(MAX_PART, c->rbj_nblk)));
    PCM_TRY(c->scal.alloc(S_NSCAL));
    PCM_TRY(c->counter.alloc(4));
    PCM_CUDA(cudaMemsetAsync(c->counter.p, 0, 4 * sizeof(unsigned int), c->stream));
    PCM_CUDA(cudaMemsetAsync(c->iscal.p, 0, I_NINT * sizeof(int), c->stream));
    {
        double hs[S_NSCAL] = {0, 0, 0, 0, 0, delta, 0};
        int hi[I_NINT] = {0, 0, c->opt.max_iter, 0};
        PCM_CUDA(cudaMemcpyAsync(c->scal.p, hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream));
        PCM_CUDA(cudaMemcpyAsync(c->iscal.p, hi, sizeof(hi), cudaMemcpyHostToDevice, c->stream));
        // hs, hi are read before the synchronisation below
        PCM_CUDA(cudaStreamSynchronize(c->stream));
    }
    double *x = dq, *r = c->vr.p, *z = c->vz.p, *p = c->vp.p, *Ap = c->vAp.p;
    const int gv = gemv_grid(c);
    const int ub = std::min(MAX_PART, (M + UP_NT - 1) / UP_NT);
    if (warm) {
        gemv_plain_kernel<<<gv, GV_NT, 0, c->stream>>>(M, c->lda, c->A.p, x, Ap, c->red.p);
        PCM_LAUNCHED(c);
    }
    pcg_init_kernel<<<std::min(1024, (M + 255) / 256), 256, 0, c->stream>>>(M, drhs, Ap, warm ? 1 : 0, x, r);
    PCM_LAUNCHED(c);
    const double *dinv = (c->pc_kind == PCM_PRECOND_JACOBI) ? c->dinv.p : nullptr;
    const bool rbj = c->pc_kind == PCM_PRECOND_RBJ;
    const int rbj_nt = std::min(1024, std::max(32, (c->rbj_l + 31) / 32 * 32));
    const size_t rbj_smem = (size_t)c->rbj_l * sizeof(double);
    if (rbj) {
        if (rbj_smem > 48 * 1024)
            PCM_CUDA(cudaFuncSetAttribute(pcg_update_rbj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)rbj_smem));
        pcg_update_rbj_kernel<<<c->rbj_nblk, rbj_nt, rbj_smem, c->stream>>>(
            M, c->rbj_l, c->rbj_perm.p, c->rbj_inv.p, x, r, z, p, Ap, c->red.p, c->scal.p, c->iscal.p, c->counter.p, 1);
    } else {
        pcg_init_diag_kernel<<<ub, UP_NT, 0, c->stream>>>(M, dinv, r, z, c->red.p, c->scal.p, c->iscal.p,
                                                          c->counter.p);
    }
    PCM_LAUNCHED(c);
    copy_kernel<<<std::min(1024, (M + 255) / 256), 256, 0, c->stream>>>(M, z, p);
    PCM_LAUNCHED(c);

    const int batch = 8;
    int h_i[I_NINT] = {0, 0, 0, 0};
    for (int done_it = 0;;) {
        for (int b = 0; b < batch; ++b) {
            pcg_gemv_kernel<<<gv, GV_NT, 0, c->stream>>>(M, c->lda, c->A.p, p, Ap, c->red.p, c->scal.p, c->iscal.p,
                                                         c->counter.p);
            if (rbj)
                pcg_update_rbj_kernel<<<c->rbj_nblk, rbj_nt, rbj_smem, c->stream>>>(
                    M, c->rbj_l, c->rbj_perm.p, c->rbj_inv.p, x, r, z, p, Ap, c->red.p, c->scal.p, c->iscal.p,
                    c->counter.p, 0);
            else
                pcg_update_diag_kernel<<<ub, UP_NT, 0, c->stream>>>(M, dinv, x, r, z, p, Ap, c->red.p, c->scal.p,
                                                                    c->iscal.p, c->counter.p);
            pcg_dir_kernel<<<std::min(1024, (M + 255) / 256), 256, 0, c->stream>>>(M, z, p, c->scal.p, c->iscal.p);
            c->stats.launches += 3;
        }
        PCM_CUDA(cudaGetLastError());
        PCM_CUDA(cudaMemcpyAsync(h_i, c->iscal.p, sizeof(h_i), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        done_it += batch;
        if (h_i[I_DONE]) break;
        if (done_it > c->opt.max_iter + 2 * batch) {  // the device cap ends the loop first
            set_last_error("solver loop did not stop at its iteration cap");
            return PCM_ERR_TIMEOUT;
        }
    }
    double h_s[S_NSCAL];
    PCM_CUDA(cudaMemcpyAsync(h_s, c->scal.p, sizeof(h_s), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    c->stats.iterations = h_i[I_ITER];
    c->stats.converged = h_i[I_CONV];
    c->stats.rnorm = h_s[S_RNORM];
    c->stats.delta = delta;
    c->stats.refinements = 0;
    if (st) *st = c->stats;
    return h_i[I_CONV] ? PCM_OK : PCM_ERR_NOT_CONVERGED;
}

// E = (Bz)^T q + c^T q + q^T A q / (2 f)  (Eq. 13)
__global__ void dot2_kernel(int M, const double *__restrict__ a, const double *__restrict__ b,
                            const double *__restrict__ q, double *__restrict__ part)
{
    double s1 = 0.0, s2 = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        s1 = fma(a[k], q[k], s1);
        s2 = fma(b[k], q[k], s2);
    }
    __shared__ double sh[2][32];
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s1;
        sh[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            x += sh[0][i];
            y += sh[1][i];
        }
        part[2 * blockIdx.x] = x;
        part[2 * blockIdx.x + 1] = y;
    }
}

int energy_compute(pcm_ctx *c, const double *dq, const double *dcv, double *E)
{
    const int M = c->M;
    PCM_TRY(c->vtmp.alloc(M));
    const int gv = gemv_grid(c);
    PCM_TRY(c->red.alloc(2 * MAX_PART));
    DBuf<double> &part2 = c->sd[1];
    const int nb = std::min(1024, (M + 255) / 256);
    PCM_TRY(part2.alloc(2 * nb));
    gemv_plain_kernel<<<gv, GV_NT, 0, c->stream>>>(M, c->lda, c->A.p, dq, c->vtmp.p, c->red.p);
    PCM_LAUNCHED(c);
    dot2_kernel<<<nb, 256, 0, c->stream>>>(M, c->Bz.p, dcv, dq, part2.p);
    PCM_LAUNCHED(c);
    std::vector<double> h1(gv), h2(2 * nb);
    PCM_CUDA(cudaMemcpyAsync(h1.data(), c->red.p, gv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaMemcpyAsync(h2.data(), part2.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    double qAq = 0.0, bzq = 0.0, cq = 0.0;
    for (int i = 0; i < gv; ++i) qAq += h1[i];
    for (int i = 0; i < nb; ++i) {
        bzq += h2[2 * i];
        cq += h2[2 * i + 1];
    }
    const double f = (c->opt.eps - 1.0) / (c->opt.eps + c->opt.k);
    *E = bzq + cq + qAq / (2.0 * f);
    return PCM_OK;
}

}  // namespace pcm
