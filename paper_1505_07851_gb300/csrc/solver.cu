// Solve A q = rhs (Eq. 1) by preconditioned conjugate gradients with the
// residual test of Eq. 20 (Section 4b), Jacobi or randomized block-Jacobi
// preconditioning (Section 4b-ii), and the energy of Eq. 13.
//
// A is stored in FP64 (row-major, leading dimension lda) for PCM_FP64, and
// for PCM_MIXED as FP32 hi and lo parts only (A32, A32lo; no FP64 copy), or
// not at all (the matrix-free operator).  Each PCG iteration is three
// kernels:
//   pcg_gemv_rp  Ap = A p, p.Ap                       -> alpha
//   pcg_update   x += alpha p, r -= alpha Ap, z = C r, r.r, r.z -> beta, stop test
//   pcg_dir      p = z + beta p
// Scalars stay on the device; reductions use per-block partial sums added in
// a fixed order by the last block to finish (deterministic).  Every kernel
// returns at once when the stop flag is set; the iterations run as a CUDA
// graph whose WHILE node the direction kernel ends once the flag is set.
// PCM_MIXED refines FP32-GEMV inner solves with true residuals formed in
// double-float from A32 + A32lo.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "context.h"
#include "aelem.cuh"
#include "rbj_apply.cuh"
#include "gemv.cuh"

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

// fixed-order sum of n partials by the whole (last) block; valid in thread 0
__device__ __forceinline__ double sum_partials(const double *part, int n)
{
    __shared__ double sh[32];
    // four loads in flight per thread before their additions (each load is
    // an L2 round trip; a single running sum would wait for each in turn)
    const volatile double *v = part;
    const int st = blockDim.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int j = threadIdx.x;
    for (; j + 3 * st < n; j += 4 * st) {
        const double a = v[j], b = v[j + st], c = v[j + 2 * st], d = v[j + 3 * st];
        s0 += a;
        s1 += b;
        s2 += c;
        s3 += d;
    }
    for (; j < n; j += st) s0 += v[j];
    double s = (s0 + s1) + (s2 + s3);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;
}

// the same for n interleaved pairs (part[2 i], part[2 i + 1]): both sums
// valid in thread 0.  Every thread of the block takes a share of the loads, so
// the partials are read in parallel rather than one after another.
__device__ __forceinline__ void sum_partials2(const double *part, int n, double *a_out, double *b_out)
{
    __shared__ double sh[2][32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += ((volatile const double *)part)[2 * i];
        b += ((volatile const double *)part)[2 * i + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a;
        sh[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            x += sh[0][i];
            y += sh[1][i];
        }
        *a_out = x;
        *b_out = y;
    }
}

// Ap = A p (FP64 A), p.Ap -> alpha
template <typename TA>
__global__ void __launch_bounds__(GV_NT) pcg_gemv_rp_kernel(int M, int lda, const TA *__restrict__ A,
                                                            const TA *__restrict__ px, const double *__restrict__ p,
                                                            double *__restrict__ Ap, double *__restrict__ part,
                                                            double *__restrict__ scal, int *__restrict__ iscal,
                                                            unsigned int *__restrict__ counter)
{
    if (iscal[I_DONE]) return;
    const double bsum = gemv_rowpair<TA>(blockIdx.x, M, lda, A, px, p, Ap);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum;
    if (last_block(counter)) {
        const double t = sum_partials(part, gridDim.x);
        if (threadIdx.x == 0) {
            scal[S_PAP] = t;
            scal[S_ALPHA] = scal[S_RZ] / t;
            *counter = 0;
        }
    }
}

// y = A x (FP64), block partials of x.y
__global__ void __launch_bounds__(GV_NT) gemv_rp_plain_kernel(int M, int lda, const double *__restrict__ A,
                                                              const double *__restrict__ x, double *__restrict__ y,
                                                              double *__restrict__ part)
{
    const double bsum = gemv_rowpair<double>(blockIdx.x, M, lda, A, x, x, y);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum;
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
        double a, b;
        sum_partials2(part, gridDim.x, &a, &b);
        if (threadIdx.x == 0) {
            finish_update(a, b, scal, iscal);
            *counter = 0;
        }
    }
}

// Randomized block-Jacobi update, one block per RBJ block; the last block
// to finish sums the partials.  With init (initialisation) x and r are left
// unchanged.
__global__ void pcg_update_rbj_kernel(int M, int l, const int *__restrict__ perm, const int *__restrict__ bstart,
                                      const double *__restrict__ inv, double *__restrict__ x, double *__restrict__ r,
                                      double *__restrict__ z, const double *__restrict__ p,
                                      const double *__restrict__ Ap, double *__restrict__ part,
                                      double *__restrict__ scal, int *__restrict__ iscal,
                                      unsigned int *__restrict__ counter, int init)
{
    extern __shared__ double srb[];  // l entries
    if (iscal[I_DONE]) return;
    const int b = blockIdx.x;
    const double alpha = init ? 0.0 : scal[S_ALPHA];
    double a = 0.0, c = 0.0;
    rbj_apply_block(M, l, b, perm, bstart, inv, x, r, z, p, Ap, alpha, init, srb, &a, &c);
    if (threadIdx.x == 0) {
        part[2 * b] = a;
        part[2 * b + 1] = c;
    }
    if (last_block(counter)) {
        double a, c;
        sum_partials2(part, gridDim.x, &a, &c);
        if (threadIdx.x == 0) {
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

// Inside the solver's CUDA graph the direction kernel also sets the loop
// condition of the graph's WHILE node: continue while the stop flag is clear.
__device__ __forceinline__ void pcg_set_condition(cudaGraphConditionalHandle h, int set_cond, const int *iscal)
{
    if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, iscal[I_DONE] ? 0u : 1u);
}

__global__ void pcg_dir_kernel(int M, const double *__restrict__ z, double *__restrict__ p,
                               const double *__restrict__ scal, const int *__restrict__ iscal,
                               cudaGraphConditionalHandle h, int set_cond)
{
    pcg_set_condition(h, set_cond, iscal);
    if (iscal[I_DONE]) return;
    const double beta = scal[S_BETA];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x)
        p[k] = fma(beta, p[k], z[k]);
}

// x -> FP32 hi + lo parts for the double-float GEMV
__global__ void split_x_kernel(int M, const double *__restrict__ x, float *__restrict__ xh, float *__restrict__ xl)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const float h = (float)x[k];
        xh[k] = h;
        xl[k] = (float)(x[k] - (double)h);
    }
}

// y = A x in double-float (PCM_MIXED), block partials of x.y
__global__ void __launch_bounds__(GV_NT) gemv_df_kernel(int M, int lda, const float *__restrict__ Ahi,
                                                        const float *__restrict__ Alo, const float *__restrict__ xh,
                                                        const float *__restrict__ xl, const double *__restrict__ x,
                                                        double *__restrict__ y, double *__restrict__ part)
{
    const double bsum = gemv_rowpair_df(blockIdx.x, M, lda, Ahi, Alo, xh, xl, x, y);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum;
}

// y = A x with the stored A: FP64, or double-float from A32 + A32lo when the
// context is PCM_MIXED; block partials of x.y in part
static int gemv_a(pcm_ctx *c, const double *x, double *y, double *part, int *np)
{
    const int M = c->M;
    const int gv = std::max(1, (M + 1) / 2);
    if (np) *np = gv;
    if (matrix_free(c)) return matfree_dfmv(c, x, y, part, np);
    if (c->opt.precision == PCM_MIXED) {
        // hi part at 0, lo part at lda (a multiple of 32 floats): both start on
        // the 16-byte boundary the GEMV's float4 loads need
        PCM_TRY(c->vxs32.alloc(2 * (size_t)c->lda));
        float *xh = c->vxs32.p, *xl = c->vxs32.p + c->lda;
        const int eb = std::min(1024, (M + 255) / 256);
        split_x_kernel<<<eb, 256, 0, c->stream>>>(M, x, xh, xl);
        PCM_LAUNCHED(c);
        gemv_df_kernel<<<gv, GV_NT, 0, c->stream>>>(M, c->lda, c->A32.p, c->A32lo.p, xh, xl, x, y, part);
    } else {
        gemv_rp_plain_kernel<<<gv, GV_NT, 0, c->stream>>>(M, c->lda, c->A.p, x, y, part);
    }
    PCM_LAUNCHED(c);
    return PCM_OK;
}

// y = A x for pcm_apply_a: the solver's accurate product (FP64 stored A, or
// double-float from A32 + A32lo or matrix-free), or with fp32 the inner
// solver's FP32 matrix-free product
int apply_a(pcm_ctx *c, const double *x, double *y, bool fp32)
{
    PCM_TRY(join_side(c));
    if (fp32) return matfree_mv32(c, x, y);
    PCM_TRY(c->red.alloc(2 * (size_t)std::max(MAX_PART, std::max(1, (c->M + 1) / 2))));
    return gemv_a(c, x, y, c->red.p, nullptr);
}

// r = b - y and per-block partial sums of r.r
__global__ void residual_kernel(int M, const double *__restrict__ b, const double *__restrict__ y,
                                double *__restrict__ r, double *__restrict__ part)
{
    double s = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const double v = y ? b[k] - y[k] : b[k];
        r[k] = v;
        s = fma(v, v, s);
    }
    __shared__ double sh[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        part[blockIdx.x] = t;
    }
}

__global__ void axpy_kernel(int M, const double *__restrict__ d, double *__restrict__ x)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) x[k] += d[k];
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
        double a, b;
        sum_partials2(part, gridDim.x, &a, &b);
        if (threadIdx.x == 0) {
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

// block-wide exclusive scan of one int per thread (RBJ_NT threads); returns
// the exclusive prefix and writes the block total to *total
__device__ __forceinline__ int rbj_block_scan(int v, int *sh /* RBJ_NT/32 + 1 */, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int t = sh[lane];
        int xs = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xs, o);
            if (lane >= o) xs += y;
        }
        sh[lane] = xs - t;
        if (lane == 31) sh[32] = xs;
    }
    __syncthreads();
    const int r = sh[wid] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

constexpr int RBJ_NBIN = 2048;   // histogram of the top 11 bits of the FP32 key
constexpr int RBJ_LMAX = 3072;   // boundary-bin elements resolved exactly in shared memory


// The points are walked in their canonical order (the surface candidate index
// I n + i: atom-major, the order of the points before they are grouped by
// exponent class), so that the pivots and the ties of the selection, and with
// them the blocks, do not depend on how the library stores the points.  pidx:
// candidate index of each stored point; T: scratch of ncand ints.
template <typename AE>
__global__ void __launch_bounds__(RBJ_NT) rbj_perm_kernel(int M, AE acc, int l,
                                                          unsigned long long seed, const int *__restrict__ pidx,
                                                          long long ncand, int *__restrict__ T,
                                                          int *__restrict__ U, int *__restrict__ U2,
                                                          int *__restrict__ perm, int *__restrict__ status)
{
    __shared__ unsigned int hist[RBJ_NBIN];
    __shared__ unsigned long long lkey[RBJ_LMAX];
    __shared__ int lidx[RBJ_LMAX];   // candidate index of each boundary-bin element
    __shared__ unsigned char lsel[RBJ_LMAX];
    __shared__ int sh_int[RBJ_NT / 32 + 1];
    __shared__ int s_nU, s_k, s_bin, s_need, s_nlist;
    // U = the stored points in ascending candidate index: scatter into the
    // candidate table, then compact it in order
    for (long long t = threadIdx.x; t < ncand; t += RBJ_NT) T[t] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += RBJ_NT) T[pidx[i]] = i;
    __syncthreads();
    {
        int base = 0;
        for (long long c0 = 0; c0 < ncand; c0 += RBJ_NT) {
            const long long t = c0 + threadIdx.x;
            const int v = t < ncand ? T[t] : -1;
            int tot;
            const int ex = rbj_block_scan(v >= 0 ? 1 : 0, sh_int, &tot);
            if (v >= 0) U[base + ex] = v;
            base += tot;
        }
        if (threadIdx.x == 0) {
            s_nU = M;
            if (base != M) *status = 2;
        }
    }
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
            s_bin = RBJ_NBIN;          // above every bin: nothing selected
            s_need = 0;
            s_nlist = 0;
        }
        ++draw;
        for (int i = threadIdx.x; i < RBJ_NBIN; i += RBJ_NT) hist[i] = 0;
        __syncthreads();
        const int k = s_k;
        const int nsel = min(l - 1, nU - 1);
        if (nsel > 0) {
            // 1. coarse histogram
            for (int i = threadIdx.x; i < nU; i += RBJ_NT) {
                const int j = U[i];
                if (j != k) atomicAdd(&hist[acc.bin(k, j)], 1u);
            }
            __syncthreads();
            // 2. bin holding the nsel-th largest key: warp 0 scans from the top, 64 bins per lane
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                const int top = RBJ_NBIN - 1 - 64 * lane;
                int loc = 0;
                for (int b = 0; b < 64; ++b) loc += (int)hist[top - b];
                int inc = loc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const unsigned ball = __ballot_sync(0xffffffffu, inc >= nsel);
                if (lane == __ffs(ball) - 1) {
                    int acc = inc - loc, bin = top;
                    for (int b = 0; b < 63; ++b, --bin) {
                        if (acc + (int)hist[bin] >= nsel) break;
                        acc += (int)hist[bin];
                    }
                    s_bin = bin;
                    s_need = nsel - acc;   // taken from the boundary bin
                }
            }
            __syncthreads();
            // 3. boundary-bin elements with their exact keys
            const int bstar = s_bin;
            for (int i = threadIdx.x; i < nU; i += RBJ_NT) {
                const int j = U[i];
                if (j != k && acc.bin(k, j) == bstar) {
                    const int p = atomicAdd(&s_nlist, 1);
                    if (p < RBJ_LMAX) {
                        lkey[p] = rbj_key64(acc.exact(k, j));
                        lidx[p] = pidx[j];
                    }
                }
            }
            __syncthreads();
            const int nl = s_nlist;
            if (nl > RBJ_LMAX) {  // more equal-bin keys than shared memory holds
                if (threadIdx.x == 0) *status = 4;
                return;
            }
            // 4. exact rank in the boundary bin: larger key first, then lower
            // candidate index
            const int need = s_need;
            for (int a = threadIdx.x; a < nl; a += RBJ_NT) {
                const unsigned long long ka = lkey[a];
                const int ja = lidx[a];
                int rank = 0;
                for (int b = 0; b < nl; ++b) {
                    const unsigned long long kb = lkey[b];
                    rank += (kb > ka || (kb == ka && lidx[b] < ja)) ? 1 : 0;
                }
                lsel[a] = rank < need ? 1 : 0;
            }
            __syncthreads();
        }
        // 5. one compaction pass in list order: taken -> perm (after the pivot), kept -> U2
        if (threadIdx.x == 0) perm[out] = k;
        const int bstar = s_bin, nl = min(s_nlist, RBJ_LMAX);
        int taken_base = out + 1, kept_base = 0;
        for (int c0 = 0; c0 < nU; c0 += RBJ_NT) {
            const int i = c0 + threadIdx.x;
            int j = -1, sel = 0, keep = 0;
            if (i < nU) {
                j = U[i];
                if (j != k) {
                    if (nsel > 0) {
                        const int bn = acc.bin(k, j);
                        if (bn > bstar) {
                            sel = 1;
                        } else if (bn == bstar) {
                            const int cj = pidx[j];
                            for (int b = 0; b < nl; ++b)
                                if (lidx[b] == cj) {
                                    sel = lsel[b];
                                    break;
                                }
                        }
                    }
                    keep = !sel;
                }
            }
            // one scan of both counts: chunk totals stay below 2^16
            int tot;
            const int ex = rbj_block_scan((sel << 16) | keep, sh_int, &tot);
            const int ex_sel = ex >> 16, ex_keep = ex & 0xffff, tot_sel = tot >> 16, tot_keep = tot & 0xffff;
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
template <typename AE>
__global__ void rbj_invert_kernel(int M, AE acc, int l, const int *__restrict__ perm,
                                  const int *__restrict__ bstart, double *__restrict__ work, double *__restrict__ inv,
                                  int *__restrict__ status)
{
    const int b = blockIdx.x;
    // fixed-size blocks (RBJ) or the blocks listed in bstart (octree), stored with stride l
    const int base = bstart ? bstart[b] : b * l;
    const int nb = bstart ? bstart[b + 1] - base : min(l, M - base);
    double *W = work + (size_t)b * l * l;
    double *X = inv + (size_t)b * l * l;
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int i = t / nb, j = t % nb;
        W[(size_t)i * l + j] = acc.exact(perm[base + i], perm[base + j]);
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
static int gemv_grid(pcm_ctx *c) { return std::max(1, (c->M + 1) / 2); }

// Octree partition of the points for the block-Jacobi comparison of Section
// 4b-ii: the bounding cube (centred on the bounding box, side = its largest
// extent) is split at its centre into octants (index 4 [x >= cx] + 2 [y >= cy]
// + [z >= cz]) until a box holds at most `leaf` points; non-empty leaves in
// depth-first octant order, points of a leaf in ascending index.  perm lists
// the points leaf after leaf; start[b] is where leaf b begins (size nleaf + 1).
static void octree_split(const std::vector<double> &x, const std::vector<double> &y, const std::vector<double> &z,
                         const std::vector<int> &idx, double cx, double cy, double cz, double h, int leaf,
                         int depth, std::vector<int> &perm, std::vector<int> &start)
{
    if ((int)idx.size() <= leaf || depth >= 40) {
        if (idx.empty()) return;
        start.push_back((int)perm.size());
        perm.insert(perm.end(), idx.begin(), idx.end());
        return;
    }
    std::vector<int> part[8];
    for (int k : idx) part[4 * (x[k] >= cx) + 2 * (y[k] >= cy) + (z[k] >= cz)].push_back(k);
    const double q = 0.5 * h;
    for (int o = 0; o < 8; ++o)
        octree_split(x, y, z, part[o], cx + ((o & 4) ? q : -q), cy + ((o & 2) ? q : -q), cz + ((o & 1) ? q : -q), q,
                     leaf, depth + 1, perm, start);
}

void octree_partition(const std::vector<double> &x, const std::vector<double> &y, const std::vector<double> &z,
                      int leaf, std::vector<int> &perm, std::vector<int> &start)
{
    const int M = (int)x.size();
    perm.clear();
    start.clear();
    double lo[3] = {x[0], y[0], z[0]}, hi[3] = {x[0], y[0], z[0]};
    for (int k = 0; k < M; ++k) {
        lo[0] = std::min(lo[0], x[k]);
        hi[0] = std::max(hi[0], x[k]);
        lo[1] = std::min(lo[1], y[k]);
        hi[1] = std::max(hi[1], y[k]);
        lo[2] = std::min(lo[2], z[k]);
        hi[2] = std::max(hi[2], z[k]);
    }
    const double h = 0.5 * std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    std::vector<int> all(M);
    for (int k = 0; k < M; ++k) all[k] = k;
    octree_split(x, y, z, all, 0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2]), h, leaf, 0,
                 perm, start);
    start.push_back(M);
}

static int precond_kind(pcm_ctx *c)
{
    int kind = c->opt.precond;
    if (kind == PCM_PRECOND_AUTO) kind = (c->M < c->opt.jacobi_below) ? PCM_PRECOND_JACOBI : PCM_PRECOND_RBJ;
    return kind;
}

static int rbj_status_error(int st)
{
    set_last_error("RBJ set-up failed (status %d: %s)", st,
                   st == 3 ? "a diagonal block is not positive definite"
                           : (st == 4 ? "too many equal keys for the selection buffer" : "bad permutation"));
    return PCM_ERR_CUDA;
}

static AStoredDF astored_df(pcm_ctx *c) { return AStoredDF{c->A32.p, c->A32lo.p, c->lda}; }

// RBJ permutation and block inverses (Section 4b-ii) on stream s, with the
// context's own RBJ scratch; the status lands in rbj_status[0]
static int rbj_build(pcm_ctx *c, cudaStream_t s)
{
    const int M = c->M;
    const int l = std::max(1, std::min(c->opt.rbj_block, M));
    c->rbj_l = l;
    c->rbj_nblk = (M + l - 1) / l;
    PCM_TRY(c->rbj_perm.alloc(M));
    PCM_TRY(c->rbj_U.alloc(M));
    PCM_TRY(c->rbj_U2.alloc(M));
    PCM_TRY(c->rbj_status.alloc(16));
    PCM_CUDA(cudaMemsetAsync(c->rbj_status.p, 0, 16 * sizeof(int), s));
    const long long ncand = (long long)c->natom * c->npts_sphere;
    PCM_TRY(c->rbj_T.alloc(ncand));
    if (matrix_free(c))
        rbj_perm_kernel<AFree><<<1, RBJ_NT, 0, s>>>(M, afree(c), l, c->opt.seed, c->pindex.p, ncand, c->rbj_T.p,
                                                    c->rbj_U.p, c->rbj_U2.p, c->rbj_perm.p, c->rbj_status.p);
    else if (c->opt.precision == PCM_MIXED)
        rbj_perm_kernel<AStoredDF><<<1, RBJ_NT, 0, s>>>(M, astored_df(c), l, c->opt.seed, c->pindex.p, ncand,
                                                        c->rbj_T.p, c->rbj_U.p, c->rbj_U2.p, c->rbj_perm.p,
                                                        c->rbj_status.p);
    else
        rbj_perm_kernel<AStored><<<1, RBJ_NT, 0, s>>>(M, AStored{c->A.p, c->lda}, l, c->opt.seed, c->pindex.p, ncand,
                                                      c->rbj_T.p, c->rbj_U.p, c->rbj_U2.p, c->rbj_perm.p,
                                                      c->rbj_status.p);
    PCM_LAUNCHED(c);
    PCM_TRY(c->rbj_inv.alloc((size_t)c->rbj_nblk * l * l));
    PCM_TRY(c->rbj_work.alloc((size_t)c->rbj_nblk * l * l));
    const int nt = std::min(1024, std::max(32, (l + 31) / 32 * 32));
    if (matrix_free(c))
        rbj_invert_kernel<AFree><<<c->rbj_nblk, nt, 0, s>>>(M, afree(c), l, c->rbj_perm.p, nullptr, c->rbj_work.p,
                                                            c->rbj_inv.p, c->rbj_status.p);
    else if (c->opt.precision == PCM_MIXED)
        rbj_invert_kernel<AStoredDF><<<c->rbj_nblk, nt, 0, s>>>(M, astored_df(c), l, c->rbj_perm.p, nullptr,
                                                                c->rbj_work.p, c->rbj_inv.p, c->rbj_status.p);
    else
        rbj_invert_kernel<AStored><<<c->rbj_nblk, nt, 0, s>>>(M, AStored{c->A.p, c->lda}, l, c->rbj_perm.p, nullptr,
                                                              c->rbj_work.p, c->rbj_inv.p, c->rbj_status.p);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

int ensure_operator(pcm_ctx *c)
{
    if (!c->op_stale) return PCM_OK;
    c->op_stale = false;
    return operator_build_async(c);
}

int operator_build_async(pcm_ctx *c)
{
    PCM_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    PCM_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[13], c->side));
    if (matrix_free(c))
        PCM_TRY(matfree_build(c, c->side));
    else
        PCM_TRY(a_build(c, c->side));
    const int kind = precond_kind(c);
    c->side_rbj = false;
    if (kind != PCM_PRECOND_OCTREE) {   // the octree partition needs the points on the host: built at the solve
        c->pc_kind = kind;
        if (kind == PCM_PRECOND_RBJ) {
            PCM_TRY(rbj_build(c, c->side));
            c->side_rbj = true;
        }
        c->pc_ready = true;
    }
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_b[13], c->side));
    PCM_CUDA(cudaEventRecord(c->ev_side, c->side));
    c->side_pending = true;
    return PCM_OK;
}

int join_side(pcm_ctx *c)
{
    PCM_TRY(ensure_operator(c));
    if (!c->side_pending) return PCM_OK;
    c->side_pending = false;
    PCM_CUDA(cudaEventSynchronize(c->ev_side));
    PCM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_side, 0));
    if (c->have_events) {
        float ms = 0.f;
        PCM_CUDA(cudaEventElapsedTime(&ms, c->ev_a[13], c->ev_b[13]));
        c->stats.ms_precond = ms;
    }
    if (c->side_rbj) {
        int st = 0;
        PCM_CUDA(cudaMemcpy(&st, c->rbj_status.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (st != 0) {
            c->pc_ready = false;
            return rbj_status_error(st);
        }
    }
    return PCM_OK;
}

int solver_prepare(pcm_ctx *c)
{
    PCM_TRY(join_side(c));
    if (c->pc_ready) return PCM_OK;
    const int M = c->M;
    const int kind = precond_kind(c);
    c->pc_kind = kind;
    PCM_TRY(c->iscal.alloc(64));
    if (kind == PCM_PRECOND_OCTREE) {
        // blocks: the leaves of an octree over the points (sizes up to the leaf
        // capacity), inverted like RBJ blocks; stride = the largest leaf
        std::vector<double> hx(M), hy(M), hz(M);
        PCM_CUDA(cudaMemcpyAsync(hx.data(), c->px.p, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaMemcpyAsync(hy.data(), c->py.p, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaMemcpyAsync(hz.data(), c->pz.p, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        std::vector<int> perm, start;
        octree_partition(hx, hy, hz, std::max(1, c->opt.octree_leaf), perm, start);
        int lmax = 1;
        for (size_t b = 0; b + 1 < start.size(); ++b) lmax = std::max(lmax, start[b + 1] - start[b]);
        c->rbj_l = lmax;
        c->rbj_nblk = (int)start.size() - 1;
        PCM_TRY(c->rbj_perm.alloc(M));
        PCM_TRY(c->rbj_bstart.alloc(start.size()));
        PCM_CUDA(cudaMemcpyAsync(c->rbj_perm.p, perm.data(), M * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        PCM_CUDA(cudaMemcpyAsync(c->rbj_bstart.p, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 c->stream));
        PCM_TRY(c->rbj_inv.alloc((size_t)c->rbj_nblk * lmax * lmax));
        PCM_TRY(c->rbj_work.alloc((size_t)c->rbj_nblk * lmax * lmax));
        PCM_TRY(c->rbj_status.alloc(16));
        PCM_CUDA(cudaMemsetAsync(c->rbj_status.p, 0, sizeof(int), c->stream));
        const int nt = std::min(1024, std::max(32, (lmax + 31) / 32 * 32));
        if (matrix_free(c))
            rbj_invert_kernel<AFree><<<c->rbj_nblk, nt, 0, c->stream>>>(M, afree(c), lmax, c->rbj_perm.p,
                                                                        c->rbj_bstart.p, c->rbj_work.p, c->rbj_inv.p,
                                                                        c->rbj_status.p);
        else if (c->opt.precision == PCM_MIXED)
            rbj_invert_kernel<AStoredDF><<<c->rbj_nblk, nt, 0, c->stream>>>(M, astored_df(c), lmax, c->rbj_perm.p,
                                                                            c->rbj_bstart.p, c->rbj_work.p,
                                                                            c->rbj_inv.p, c->rbj_status.p);
        else
            rbj_invert_kernel<AStored><<<c->rbj_nblk, nt, 0, c->stream>>>(M, AStored{c->A.p, c->lda}, lmax,
                                                                          c->rbj_perm.p, c->rbj_bstart.p,
                                                                          c->rbj_work.p, c->rbj_inv.p,
                                                                          c->rbj_status.p);
        PCM_LAUNCHED(c);
        int st = 0;
        PCM_CUDA(cudaMemcpyAsync(&st, c->rbj_status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));  // perm, start are read by the copies above
        if (st != 0) {
            set_last_error("octree block-Jacobi set-up failed: a diagonal block is not positive definite");
            return PCM_ERR_CUDA;
        }
    }
    if (kind == PCM_PRECOND_RBJ) {
        PCM_TRY(rbj_build(c, c->stream));
        int st = 0;
        PCM_CUDA(cudaMemcpyAsync(&st, c->rbj_status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        if (st != 0) return rbj_status_error(st);
    }
    c->pc_ready = true;
    return PCM_OK;
}

// Everything a solve needs before its first iteration: the preconditioner
// (the stored parts of A come with the operator build).
int solver_prepare_full(pcm_ctx *c)
{
    PCM_TRY(solver_prepare(c));
    return PCM_OK;
}

// One PCG iteration of the FP64 solver (gemv, update, dir) on stream st;
// set_cond: the direction kernel sets the graph's loop condition h
static void pcg_iteration(pcm_ctx *c, cudaStream_t st, double *x, cudaGraphConditionalHandle h, int set_cond)
{
    const int M = c->M;
    double *r = c->vr.p, *z = c->vz.p, *p = c->vp.p, *Ap = c->vAp.p;
    const int gv = gemv_grid(c);
    const int ub = std::min(MAX_PART, (M + UP_NT - 1) / UP_NT);
    const int eb = std::min(1024, (M + 255) / 256);
    const double *dinv = (c->pc_kind == PCM_PRECOND_JACOBI) ? c->dinv.p : nullptr;
    const bool rbj = c->pc_kind == PCM_PRECOND_RBJ || c->pc_kind == PCM_PRECOND_OCTREE;
    const int *bstart = c->pc_kind == PCM_PRECOND_OCTREE ? c->rbj_bstart.p : nullptr;
    const int rbj_nt = std::min(1024, RBJ_SPLIT * std::max(32, (c->rbj_l + 31) / 32 * 32));
    const size_t rbj_smem = (size_t)c->rbj_l * sizeof(double);
    pcg_gemv_rp_kernel<double><<<gv, GV_NT, 0, st>>>(M, c->lda, c->A.p, p, p, Ap, c->red.p, c->scal.p, c->iscal.p,
                                                      c->counter.p);
    if (rbj)
        pcg_update_rbj_kernel<<<c->rbj_nblk, rbj_nt, rbj_smem, st>>>(M, c->rbj_l, c->rbj_perm.p, bstart,
                                                                     c->rbj_inv.p, x, r, z, p, Ap, c->red.p,
                                                                     c->scal.p, c->iscal.p, c->counter.p, 0);
    else
        pcg_update_diag_kernel<<<ub, UP_NT, 0, st>>>(M, dinv, x, r, z, p, Ap, c->red.p, c->scal.p, c->iscal.p,
                                                     c->counter.p);
    pcg_dir_kernel<<<eb, 256, 0, st>>>(M, z, p, c->scal.p, c->iscal.p, h, set_cond);
}

// The iteration loop as a CUDA graph: a conditional WHILE node whose body is
// one iteration; the direction kernel clears the condition once the stop flag
// is set (the test of Eq. 20, or the iteration cap in finish_update), so every
// graph launch ends after at most max_iter + 1 bodies.  Rebuilt when anything
// the captured launches read changes.
static int pcg_graph(pcm_ctx *c, double *x)
{
    const uintptr_t key[] = {(uintptr_t)x, (uintptr_t)c->M, (uintptr_t)c->lda, (uintptr_t)c->A.p,
                             (uintptr_t)c->vr.p, (uintptr_t)c->vz.p, (uintptr_t)c->vp.p, (uintptr_t)c->vAp.p,
                             (uintptr_t)c->red.p, (uintptr_t)c->scal.p, (uintptr_t)c->iscal.p,
                             (uintptr_t)c->counter.p, (uintptr_t)c->pc_kind, (uintptr_t)c->dinv.p,
                             (uintptr_t)c->rbj_perm.p, (uintptr_t)c->rbj_bstart.p, (uintptr_t)c->rbj_inv.p,
                             (uintptr_t)c->rbj_l, (uintptr_t)c->rbj_nblk};
    static_assert(sizeof(key) <= sizeof(c->pcg_key), "graph key too long");
    if (c->pcg_exec && memcmp(key, c->pcg_key, sizeof(key)) == 0) return PCM_OK;
    if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
    if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
    c->pcg_exec = nullptr;
    c->pcg_graph = nullptr;
    memset(c->pcg_key, 0, sizeof(c->pcg_key));
    if (!c->cap_stream) PCM_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    PCM_CUDA(cudaGraphCreate(&c->pcg_graph, 0));
    cudaGraphConditionalHandle handle;
    PCM_CUDA(cudaGraphConditionalHandleCreate(&handle, c->pcg_graph, 1, cudaGraphCondAssignDefault));
    // the parameter struct has no default constructor: zeroed raw storage
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams *cp = reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = handle;
    cp->conditional.type = cudaGraphCondTypeWhile;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    PCM_CUDA(cudaGraphAddNode(&node, c->pcg_graph, nullptr, nullptr, 0, cp));
    cudaGraph_t body = cp->conditional.phGraph_out[0];
    PCM_CUDA(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    pcg_iteration(c, c->cap_stream, x, handle, 1);
    const cudaError_t e = cudaGetLastError();
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &captured);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        set_last_error("solver graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        return PCM_ERR_CUDA;
    }
    PCM_CUDA(cudaGraphInstantiate(&c->pcg_exec, c->pcg_graph, 0));
    memcpy(c->pcg_key, key, sizeof(key));
    return PCM_OK;
}

// Preconditioned CG on A x = b with the FP64 stored A from x (warm) or 0
// until the recursively updated residual is below delta or max_iter steps.
// Returns iterations, the stop flag and the final residual norm.
static int pcg_core(pcm_ctx *c, const double *drhs, double *x, bool warm, double delta, int max_iter, int *iters,
                    int *conv, double *rnorm)
{
    const int M = c->M;
    if (!c->h_pinned) PCM_CUDA(cudaMallocHost((void **)&c->h_pinned, 32 * sizeof(double)));
    double *hs = c->h_pinned;
    int *hi = reinterpret_cast<int *>(c->h_pinned + 16);
    // the pinned scalars of the previous call were read after its final synchronisation
    for (int i = 0; i < S_NSCAL; ++i) hs[i] = 0.0;
    hs[S_DELTA] = delta;
    hi[I_DONE] = 0;
    hi[I_ITER] = 0;
    hi[I_MAXIT] = max_iter;
    hi[I_CONV] = 0;
    PCM_CUDA(cudaMemsetAsync(c->counter.p, 0, 4 * sizeof(unsigned int), c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->scal.p, hs, S_NSCAL * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->iscal.p, hi, I_NINT * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    double *r = c->vr.p, *z = c->vz.p, *p = c->vp.p, *Ap = c->vAp.p;
    const int gv = gemv_grid(c);
    const int ub = std::min(MAX_PART, (M + UP_NT - 1) / UP_NT);
    const int eb = std::min(1024, (M + 255) / 256);
    if (warm) {
        gemv_rp_plain_kernel<<<gv, GV_NT, 0, c->stream>>>(M, c->lda, c->A.p, x, Ap, c->red.p);
        PCM_LAUNCHED(c);
    }
    pcg_init_kernel<<<eb, 256, 0, c->stream>>>(M, drhs, Ap, warm ? 1 : 0, x, r);
    PCM_LAUNCHED(c);
    const double *dinv = (c->pc_kind == PCM_PRECOND_JACOBI) ? c->dinv.p : nullptr;
    const bool rbj = c->pc_kind == PCM_PRECOND_RBJ || c->pc_kind == PCM_PRECOND_OCTREE;
    const int *bstart = c->pc_kind == PCM_PRECOND_OCTREE ? c->rbj_bstart.p : nullptr;
    const int rbj_nt = std::min(1024, RBJ_SPLIT * std::max(32, (c->rbj_l + 31) / 32 * 32));
    const size_t rbj_smem = (size_t)c->rbj_l * sizeof(double);
    if (rbj) {
        if (rbj_smem > 48 * 1024)
            PCM_CUDA(cudaFuncSetAttribute(pcg_update_rbj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)rbj_smem));
        pcg_update_rbj_kernel<<<c->rbj_nblk, rbj_nt, rbj_smem, c->stream>>>(
            M, c->rbj_l, c->rbj_perm.p, bstart, c->rbj_inv.p, x, r, z, p, Ap, c->red.p, c->scal.p, c->iscal.p,
            c->counter.p, 1);
    } else {
        pcg_init_diag_kernel<<<ub, UP_NT, 0, c->stream>>>(M, dinv, r, z, c->red.p, c->scal.p, c->iscal.p,
                                                          c->counter.p);
    }
    PCM_LAUNCHED(c);
    copy_kernel<<<eb, 256, 0, c->stream>>>(M, z, p);
    PCM_LAUNCHED(c);

    PCM_TRY(pcg_graph(c, x));
    PCM_CUDA(cudaGraphLaunch(c->pcg_exec, c->stream));
    PCM_CUDA(cudaMemcpyAsync(hi, c->iscal.p, I_NINT * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaMemcpyAsync(hs, c->scal.p, S_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    if (!hi[I_DONE]) {  // the graph's loop ends only with the flag set
        set_last_error("solver loop ended without its stop flag");
        return PCM_ERR_TIMEOUT;
    }
    *iters = hi[I_ITER];
    *conv = hi[I_CONV];
    *rnorm = hs[S_RNORM];
    c->stats.launches += 3 * (long long)std::max(1, hi[I_ITER]);  // graph bodies run
    return PCM_OK;
}

// ||b - A x||_2 with the FP64 stored A; r receives the residual
// r = b - A x (FP64) and |r|; x == nullptr stands for x = 0 (r = b, no GEMV)
static int true_residual(pcm_ctx *c, const double *b, const double *x, double *r, double *norm)
{
    const int M = c->M;
    if (x) PCM_TRY(gemv_a(c, x, c->vtmp.p, c->red.p, nullptr));
    const int nb = std::min(256, (M + 255) / 256);
    residual_kernel<<<nb, 256, 0, c->stream>>>(M, b, x ? c->vtmp.p : nullptr, r, c->red.p);
    PCM_LAUNCHED(c);
    double h[256];
    PCM_CUDA(cudaMemcpyAsync(h, c->red.p, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += h[i];
    *norm = sqrt(s);
    return PCM_OK;
}

// the last solve's charges and A q = b - r (r: the final true residual b - A q)
__global__ void aq_store_kernel(int M, const double *__restrict__ b, const double *__restrict__ r,
                                const double *__restrict__ q, double *__restrict__ q_keep, double *__restrict__ y)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) {
        q_keep[k] = q[k];
        y[k] = b[k] - r[k];
    }
}

int solver_run(pcm_ctx *c, const double *drhs, double delta, double *dq, bool warm, pcm_stats *st)
{
    c->aq_valid = false;
    PCM_TRY(join_side(c));
    const bool fresh = !c->pc_ready;
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[13], c->stream));
    PCM_TRY(solver_prepare(c));
    if (fresh) c->stats.ms_precond = 0.0;
    if (c->have_events && fresh) {
        PCM_CUDA(cudaEventRecord(c->ev_b[13], c->stream));
        PCM_CUDA(cudaEventSynchronize(c->ev_b[13]));
        float ms = 0.f;
        PCM_CUDA(cudaEventElapsedTime(&ms, c->ev_a[13], c->ev_b[13]));
        c->stats.ms_precond = ms;
    }
    const int M = c->M;
    PCM_TRY(c->vr.alloc(M));
    PCM_TRY(c->vz.alloc(M));
    PCM_TRY(c->vp.alloc(M));
    PCM_TRY(c->vAp.alloc(M));
    PCM_TRY(c->vtmp.alloc(M));
    PCM_TRY(c->red.alloc(2 * (size_t)std::max(std::max(MAX_PART, c->rbj_nblk), gemv_grid(c))));
    PCM_TRY(c->scal.alloc(S_NSCAL));
    PCM_TRY(c->counter.alloc(4));
    PCM_CUDA(cudaMemsetAsync(c->iscal.p, 0, I_NINT * sizeof(int), c->stream));
    int iters = 0, conv = 0, refinements = 0;
    double rnorm = 0.0;
    if (c->opt.precision != PCM_MIXED) {
        // the iterate lives in a context buffer, so that the solver graph
        // (which holds its address) is reused whatever output the caller passes
        PCM_TRY(c->vd.alloc(M));
        if (warm) PCM_CUDA(cudaMemcpyAsync(c->vd.p, dq, M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        PCM_TRY(pcg_core(c, drhs, c->vd.p, warm, delta, c->opt.max_iter, &iters, &conv, &rnorm));
        PCM_CUDA(cudaMemcpyAsync(dq, c->vd.p, M * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else {
        // FP64 iterative refinement around FP32 inner solves: the true
        // residual b - A x is formed in double-float, each inner solve reduces
        // it by ETA (or to delta / 2), and x accumulates the corrections.  The
        // matrix-free inner solve goes further per refinement (its FP32
        // operator is accurate to ~1e-7, and every refinement restarts CG and
        // costs a double-float product)
        const double ETA = matrix_free(c) ? 1e-6 : 1e-3;
        constexpr int MAX_REFINE = 12;
        PCM_TRY(c->vro.alloc(M));
        PCM_TRY(c->vd.alloc(M));
        if (!warm) PCM_CUDA(cudaMemsetAsync(dq, 0, M * sizeof(double), c->stream));
        for (bool zero = !warm;; zero = false) {
            PCM_TRY(true_residual(c, drhs, zero ? nullptr : dq, c->vro.p, &rnorm));
            if (rnorm < delta) {
                conv = 1;
                break;
            }
            if (iters >= c->opt.max_iter || refinements >= MAX_REFINE || !std::isfinite(rnorm)) break;
            int it_in = 0, conv_in = 0;
            double rn_in = 0.0;
            const double tol = std::max(ETA * rnorm, 0.5 * delta);
            PCM_TRY(persistent_pcg(c, c->vro.p, c->vd.p, tol, std::max(1, c->opt.max_iter - iters), &it_in, &conv_in,
                                   &rn_in));
            iters += it_in;
            ++refinements;
            const int eb = std::min(1024, (M + 255) / 256);
            axpy_kernel<<<eb, 256, 0, c->stream>>>(M, c->vd.p, dq);
            PCM_LAUNCHED(c);
        }
        // every exit of the loop follows a true residual of the final x
        if (std::isfinite(rnorm)) {
            PCM_TRY(c->aq_q.alloc(M));
            PCM_TRY(c->aq_y.alloc(M));
            aq_store_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, drhs, c->vro.p, dq, c->aq_q.p, c->aq_y.p);
            PCM_LAUNCHED(c);
            c->aq_valid = true;
        }
    }
    c->stats.iterations = iters;
    c->stats.converged = conv;
    c->stats.rnorm = rnorm;
    c->stats.delta = delta;
    c->stats.refinements = refinements;
    if (st) *st = c->stats;
    return conv ? PCM_OK : PCM_ERR_NOT_CONVERGED;
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

// The energy's three dot products with A q taken from the last solve (qk, y)
// when q is that solve's result: per block q.y, Bz.q, c.q and the number of
// elements where q differs from qk (then the caller forms A q itself)
__global__ void energy_kept_kernel(int M, const double *__restrict__ q, const double *__restrict__ qk,
                                   const double *__restrict__ y, const double *__restrict__ Bz,
                                   const double *__restrict__ cv, double *__restrict__ part)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, nd = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const double v = q[k];
        nd += v != qk[k] ? 1.0 : 0.0;
        s0 = fma(v, y[k], s0);
        s1 = fma(Bz[k], v, s1);
        s2 = fma(cv[k], v, s2);
    }
    __shared__ double sh[4][32];
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    nd = warp_sum(nd);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
        sh[2][threadIdx.x >> 5] = s2;
        sh[3][threadIdx.x >> 5] = nd;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[threadIdx.x][i];
        part[4 * blockIdx.x + threadIdx.x] = t;
    }
}

int energy_compute(pcm_ctx *c, const double *dq, const double *dcv, double *E)
{
    PCM_TRY(join_side(c));
    const int M = c->M;
    const double f = (c->opt.eps - 1.0) / (c->opt.eps + c->opt.k);
    if (c->aq_valid) {
        // q^T A q = q^T (b - r) with the last solve's final true residual, when
        // q is that solve's result (checked element by element)
        const int nb = std::min(1024, (M + 255) / 256);
        DBuf<double> &part4 = c->sd[1];
        PCM_TRY(part4.alloc(4 * (size_t)nb));
        energy_kept_kernel<<<nb, 256, 0, c->stream>>>(M, dq, c->aq_q.p, c->aq_y.p, c->Bz.p, dcv, part4.p);
        PCM_LAUNCHED(c);
        std::vector<double> h(4 * (size_t)nb);
        PCM_CUDA(cudaMemcpyAsync(h.data(), part4.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        double qAq = 0.0, bzq = 0.0, cq = 0.0, nd = 0.0;
        for (int i = 0; i < nb; ++i) {
            qAq += h[4 * i];
            bzq += h[4 * i + 1];
            cq += h[4 * i + 2];
            nd += h[4 * i + 3];
        }
        if (nd == 0.0) {
            *E = bzq + cq + qAq / (2.0 * f);
            return PCM_OK;
        }
    }
    PCM_TRY(c->vtmp.alloc(M));
    const int gv = gemv_grid(c);
    PCM_TRY(c->red.alloc(2 * (size_t)std::max(MAX_PART, gv)));
    DBuf<double> &part2 = c->sd[1];
    const int nb = std::min(1024, (M + 255) / 256);
    PCM_TRY(part2.alloc(2 * nb));
    int np = gv;
    PCM_TRY(gemv_a(c, dq, c->vtmp.p, c->red.p, &np));
    dot2_kernel<<<nb, 256, 0, c->stream>>>(M, c->Bz.p, dcv, dq, part2.p);
    PCM_LAUNCHED(c);
    std::vector<double> h1(np), h2(2 * nb);
    PCM_CUDA(cudaMemcpyAsync(h1.data(), c->red.p, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaMemcpyAsync(h2.data(), part2.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    double qAq = 0.0, bzq = 0.0, cq = 0.0;
    for (int i = 0; i < np; ++i) qAq += h1[i];
    for (int i = 0; i < nb; ++i) {
        bzq += h2[2 * i];
        cq += h2[2 * i + 1];
    }
    *E = bzq + cq + qAq / (2.0 * f);
    return PCM_OK;
}

}  // namespace pcm
