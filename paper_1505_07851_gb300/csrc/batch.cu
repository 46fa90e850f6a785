// Batched C-PCM: ESP, solve, Fock correction and energy for many molecules
// of uneven size in one call.
//
// Each molecule keeps its own context (surface, stored A and its FP32 parts,
// pair lists, RBJ preconditioner).  The integral stages prepare each
// molecule's tiles on the batch's stream; in PCM_MIXED the packed ESP and Fock
// blocks of all molecules then run in one launch per angular class (job
// tables), the one-centre and epilogue kernels per molecule.  The linear
// solves of all molecules run in lockstep: every vector of the batch lives in
// one concatenated array (each molecule's slice starts on a 32-element
// boundary), and one launch per step serves all molecules:
//   bgemv      A p for every molecule (row pairs of all matrices, one table);
//              PCM_MIXED: bsym over the 128 x 128 tiles of the upper triangle
//              of every A32 (A is symmetric: each tile serves A_IJ p_J and
//              A_IJ^T p_I, half the bytes of the row GEMV), partial sums per
//              tile column block, then bsym_reduce adds them per row
//   balpha     alpha_m = r.z / p.Ap per molecule (fixed-order partial sums)
//   bupdate    x, r update and z = C r per RBJ block of every molecule
//   bscalar    per-molecule stop test (Eq. 20) and beta; sets the loop condition
//   bdir       p = z + beta p
// The iteration loop is a CUDA graph with a conditional WHILE node whose
// condition the bscalar kernel sets on the device: no host round trip per
// iteration.  Every molecule stops on its own test; converged molecules skip
// their work.  The loop is bounded: bscalar clears the condition once the
// iteration count reaches the cap.  PCM_MIXED wraps the FP32-GEMV loop in the
// iterative refinement of the single-molecule solver (true residuals in
// double-float from A32 + A32lo, inner tolerance max(eta |r|, delta / 2)).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "context.h"
#include "gemv.cuh"

namespace pcm {

constexpr int BG_NT = 256;       // row-pair GEMV block (8 warps)
constexpr int BR_SPLIT = 4;      // threads per row in the block-Jacobi apply
constexpr int BS_NT = 256;       // per-molecule scalar kernel
constexpr int BR_NT_MAX = 1024;

struct BatchDev {
    // per molecule
    const double **A64;
    const float **A32;
    const float **A32lo;   // PCM_MIXED: A - A32, for the double-float true residual
    const int **perm;
    const double **inv;
    const double **dinv;   // Jacobi (l == 1) when perm is null
    const int *lda, *M, *off, *l, *nblk;
    // block tables
    const int *gb_mol, *gb_rp, *gb_start;   // GEMV row-pair blocks; per-molecule ranges (nmol + 1)
    const int *rb_mol, *rb_blk, *rb_start;  // preconditioner blocks
    const int *elem_mol;                    // molecule of each (padded) element, -1 for padding
    // PCM_MIXED symmetric products: tile blocks (molecule, I << 16 | J), the start of each
    // molecule's partial slots (ceil(M / 128) slices of its padded length), reduction blocks
    // (molecule, first row) with per-molecule ranges (nmol + 1)
    const int *gt_mol, *gt_ij;
    const long long *slot_off;
    const int *rd_mol, *rd_row, *rd_start;
};

}  // namespace pcm

struct pcm_batch {
    pcm_options opt;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int nmol = 0;
    std::vector<pcm_ctx *> mol;
    std::vector<char> ready;
    bool layout_ok = false;
    int Mtot = 0, ngb = 0, nrb = 0, rbj_l_max = 1;
    std::vector<int> h_off;
    pcm::BatchDev dev{};
    // device tables
    pcm::DBuf<const double *> dA64, dinvp, ddinv;
    pcm::DBuf<const float *> dA32, dA32lo;
    pcm::DBuf<const int *> dperm;
    pcm::DBuf<int> dlda, dM, doff, dl, dnblk, gb_mol, gb_rp, gb_start, rb_mol, rb_blk, rb_start, elem_mol;
    pcm::DBuf<int> gt_mol, gt_ij, rd_mol, rd_row, rd_start;
    pcm::DBuf<long long> slot_off;
    pcm::DBuf<double> ypart;           // partial sums of the symmetric products
    int ngt = 0, nrd = 0;
    // vectors (Mtot) and per-molecule scalars
    pcm::DBuf<double> x, b, r, z, p, Ap, d, ro, y;
    pcm::DBuf<float> p32, xh32, xl32;  // FP32 copy of p; hi and lo parts of x for the residual
    pcm::DBuf<double> rz, pAp, alpha, beta, rr, tol, rnorm, gpart, rpart;
    pcm::DBuf<int> idone, iters, conv, maxit, gcount;
    // the inner loop as a graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_mixed = false;
    // the packed integral blocks of all molecules, one launch per class
    pcm::JobSink sink;
    pcm::DBuf<pcm::EspJob> dej;
    pcm::DBuf<pcm::FockJob> dfj;
    pcm::DBuf<int> derr;
    // results
    std::vector<pcm_stats> st;
    long long launches = 0;            // batch-level kernels (the molecules count their own)
    pcm::DBuf<double> dF;
};

namespace pcm {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// y = A x for every row pair of every molecule still iterating; per-block
// x.y partials (zero for skipped blocks)
template <typename TA>
__global__ void __launch_bounds__(BG_NT) bgemv_kernel(BatchDev B, const TA *__restrict__ x, const double *__restrict__ x64,
                                                      double *__restrict__ y, const int *__restrict__ idone,
                                                      double *__restrict__ part)
{
    const int m = B.gb_mol[blockIdx.x];
    if (idone[m]) {
        if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
        return;
    }
    const int o = B.off[m];
    const TA *A;
    if constexpr (sizeof(TA) == 4) A = B.A32[m];
    else A = B.A64[m];
    const double s = gemv_rowpair<TA>(B.gb_rp[blockIdx.x], B.M[m], B.lda[m], A, x + o, x64 + o, y + o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// y = A x over the tiles of the upper triangle of every molecule's A32 (DF:
// double-float from A32 + A32lo and x = xh + xl, as gemv_rowpair_df; else FP32
// from A32 and xh).  Block = tile (I, J) of molecule m: warp w takes rows
// I0 + w + 8 i (i < 16), lane l columns J0 + 4 l .. + 3.  Row sums (reduced
// across the lanes by halving) go to slot J of the rows, column sums of an
// off-diagonal tile (reduced across the warps in shared memory) to slot I of
// the columns; each (slot, row) is written by exactly one tile.
constexpr int BT_TB = 128;
template <bool DF>
__global__ void __launch_bounds__(BG_NT) bsym_kernel(BatchDev B, const float *__restrict__ xh,
                                                     const float *__restrict__ xl, const int *__restrict__ idone,
                                                     double *__restrict__ ypart)
{
    __shared__ double cs[BG_NT / 32][BT_TB];
    const int m = B.gt_mol[blockIdx.x];
    if (idone[m]) return;
    const int ij = B.gt_ij[blockIdx.x], I = ij >> 16, J = ij & 0xffff;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int M = B.M[m], lda = B.lda[m], o = B.off[m], Mp = B.off[m + 1] - o;
    const float *__restrict__ A = B.A32[m];
    const float *__restrict__ Al = B.A32lo[m];
    double *__restrict__ yp = ypart + B.slot_off[m];
    const int I0 = I * BT_TB, J0 = J * BT_TB, c0 = J0 + 4 * lane;
    const bool cok = c0 < M;   // then c0 + 3 < Mp <= lda: whole 16-byte loads stay in the slices
    float xj[4] = {0.f, 0.f, 0.f, 0.f}, xjl[4] = {0.f, 0.f, 0.f, 0.f};
    if (cok) {
        const float4 v = *reinterpret_cast<const float4 *>(xh + o + c0);
        xj[0] = v.x, xj[1] = v.y, xj[2] = v.z, xj[3] = v.w;
        if (DF) {
            const float4 u = *reinterpret_cast<const float4 *>(xl + o + c0);
            xjl[0] = u.x, xjl[1] = u.y, xjl[2] = u.z, xjl[3] = u.w;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (c0 + t >= M) xj[t] = xjl[t] = 0.f;
    }
    double rp[16];
    double cc[4] = {0.0, 0.0, 0.0, 0.0};
    float cS[4] = {0.f, 0.f, 0.f, 0.f}, cC[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        float4 a4[8], l4[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = I0 + w + 8 * (8 * hh + i);
            const bool ok = cok && row < M;
            a4[i] = ok ? *reinterpret_cast<const float4 *>(A + (size_t)row * lda + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (DF)
                l4[i] = ok ? *reinterpret_cast<const float4 *>(Al + (size_t)row * lda + c0)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = I0 + w + 8 * (8 * hh + i);
            float a[4] = {a4[i].x, a4[i].y, a4[i].z, a4[i].w};
            float al[4] = {0.f, 0.f, 0.f, 0.f};
            if (DF) al[0] = l4[i].x, al[1] = l4[i].y, al[2] = l4[i].z, al[3] = l4[i].w;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (c0 + t >= M) a[t] = al[t] = 0.f;   // columns beyond M: unwritten entries
            float xi = 0.f, xil = 0.f;
            if (row < M) {
                xi = xh[o + row];
                if (DF) xil = xl[o + row];
            }
            if (DF) {
                float S = 0.f, C = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    df_acc(S, C, a[t], al[t], xj[t], xjl[t]);
                    df_acc(cS[t], cC[t], a[t], al[t], xi, xil);
                }
                rp[8 * hh + i] = (double)S + (double)C;
            } else {
                rp[8 * hh + i] = (double)fmaf(a[0], xj[0], fmaf(a[1], xj[1], fmaf(a[2], xj[2], a[3] * xj[3])));
#pragma unroll
                for (int t = 0; t < 4; ++t) cS[t] = fmaf(a[t], xi, cS[t]);
            }
        }
    }
    // rows: halve the sixteen partials across the lanes (row 8 b4 + 4 b3 + 2 b2 + b1 ends in lanes 2i, 2i + 1)
#pragma unroll
    for (int h = 8, off = 16; h >= 1; h >>= 1, off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? rp[i] : rp[i + h];
            const double keep = up ? rp[i + h] : rp[i];
            rp[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    const double rsum = rp[0] + __shfl_xor_sync(0xffffffffu, rp[0], 1);
    {
        const int mm = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        const int row = I0 + w + 8 * mm;
        if ((lane & 1) == 0 && row < M) yp[(size_t)J * Mp + row] = rsum;
    }
    if (I != J) {
#pragma unroll
        for (int t = 0; t < 4; ++t) cc[t] = DF ? (double)cS[t] + (double)cC[t] : (double)cS[t];
#pragma unroll
        for (int t = 0; t < 4; ++t) cs[w][4 * lane + t] = cc[t];
        __syncthreads();
        if (threadIdx.x < BT_TB) {
            double v = cs[0][threadIdx.x];
#pragma unroll
            for (int q = 1; q < BG_NT / 32; ++q) v += cs[q][threadIdx.x];
            const int col = J0 + threadIdx.x;
            if (col < M) yp[(size_t)I * Mp + col] = v;
        }
    }
}

// y = the sum of a molecule's partial slots per row (fixed order), per-block
// partials of x.y
__global__ void __launch_bounds__(256) bsym_reduce_kernel(BatchDev B, const double *__restrict__ ypart,
                                                          const double *__restrict__ x64, const int *__restrict__ idone,
                                                          double *__restrict__ y, double *__restrict__ part)
{
    __shared__ double red[8];
    const int m = B.rd_mol[blockIdx.x];
    if (idone[m]) {
        if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
        return;
    }
    const int M = B.M[m], o = B.off[m], Mp = B.off[m + 1] - o;
    const int ntb = (M + BT_TB - 1) / BT_TB;
    const double *__restrict__ yp = ypart + B.slot_off[m];
    const int k = B.rd_row[blockIdx.x] + threadIdx.x;
    double d = 0.0;
    if (k < M) {
        double v = 0.0;
        for (int s = 0; s < ntb; ++s) v += yp[(size_t)s * Mp + k];
        y[o + k] = v;
        d = x64[o + k] * v;
    }
    d = block_sum<double, 256>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = d;
}

__global__ void bsplit_kernel(int n, const double *__restrict__ x, float *__restrict__ xh, float *__restrict__ xl)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float h = (float)x[k];
        xh[k] = h;
        xl[k] = (float)(x[k] - (double)h);
    }
}

// alpha_m = rz_m / (p.Ap)_m from the GEMV partials of molecule m (one warp per molecule)
__global__ void balpha_kernel(int nmol, const int *__restrict__ start, const double *__restrict__ part,
                              const int *__restrict__ idone, const double *__restrict__ rz, double *__restrict__ pAp,
                              double *__restrict__ alpha)
{
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= nmol || idone[m]) return;
    double s = 0.0;
    for (int i = start[m] + lane; i < start[m + 1]; i += 32) s += part[i];
    s = warp_sum(s);
    if (lane == 0) {
        pAp[m] = s;
        alpha[m] = rz[m] / s;
    }
}

// Preconditioner block of a molecule: RBJ (perm != null) or Jacobi.  Unless
// init, x += alpha p and r -= alpha Ap on the block's indices first.
__global__ void bupdate_kernel(BatchDev B, double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                               const double *__restrict__ p, const double *__restrict__ Ap,
                               const double *__restrict__ alpha, const int *__restrict__ idone,
                               double *__restrict__ part, int init)
{
    extern __shared__ double srb[];
    const int m = B.rb_mol[blockIdx.x];
    if (idone[m]) {
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = 0.0;
            part[2 * blockIdx.x + 1] = 0.0;
        }
        return;
    }
    const int o = B.off[m], M = B.M[m], l = B.l[m], blk = B.rb_blk[blockIdx.x];
    const double a = init ? 0.0 : alpha[m];
    double *xm = x + o, *rm = r + o, *zm = z + o;
    const double *pm = p + o, *Apm = Ap + o;
    const int *perm = B.perm[m];
    const int base = blk * l;
    const int nb = min(l, M - base);
    double rr = 0.0, rz = 0.0;
    if (!perm) {
        // Jacobi: l consecutive indices, z = r / A_kk
        const double *dinv = B.dinv[m];
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const int k = base + i;
            double rk = rm[k];
            if (!init) {
                xm[k] = fma(a, pm[k], xm[k]);
                rk = fma(-a, Apm[k], rk);
                rm[k] = rk;
            }
            const double zk = rk * dinv[k];
            zm[k] = zk;
            rr = fma(rk, rk, rr);
            rz = fma(rk, zk, rz);
        }
    } else {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const int k = perm[base + i];
            double rk = rm[k];
            if (!init) {
                xm[k] = fma(a, pm[k], xm[k]);
                rk = fma(-a, Apm[k], rk);
                rm[k] = rk;
            }
            srb[i] = rk;
        }
        __syncthreads();
        const double *Mi = B.inv[m] + (size_t)blk * l * l;
        const int sub = threadIdx.x % BR_SPLIT;
        for (int i = threadIdx.x / BR_SPLIT; i < ((nb + 31) / 32) * 32; i += blockDim.x / BR_SPLIT) {
            double s = 0.0;
            if (i < nb)
                for (int j = sub; j < nb; j += BR_SPLIT) s = fma(Mi[(size_t)j * l + i], srb[j], s);
#pragma unroll
            for (int off = BR_SPLIT / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (sub == 0 && i < nb) {
                zm[perm[base + i]] = s;
                rr = fma(srb[i], srb[i], rr);
                rz = fma(srb[i], s, rz);
            }
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
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            s0 += sh[0][i];
            s1 += sh[1][i];
        }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

// Per molecule: r.r and r.z from the preconditioner partials in block order,
// the stop test of Eq. 20 against tol_m and the iteration cap, beta.  With
// init only r.z and the test.  Then the loop condition: some molecule still
// iterating and the global count below its cap.
__global__ void __launch_bounds__(BS_NT) bscalar_kernel(int nmol, BatchDev B, const double *__restrict__ part,
                                                        int *__restrict__ idone, int *__restrict__ iters,
                                                        int *__restrict__ conv, const int *__restrict__ maxit,
                                                        const double *__restrict__ tol, double *__restrict__ rz,
                                                        double *__restrict__ rr, double *__restrict__ beta,
                                                        int *__restrict__ gcount, int cap, int init,
                                                        cudaGraphConditionalHandle handle, int set_cond)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < nmol; m += BS_NT) {
        if (idone[m]) continue;
        double a = 0.0, c = 0.0;
        for (int i = B.rb_start[m]; i < B.rb_start[m + 1]; ++i) {
            a += part[2 * i];
            c += part[2 * i + 1];
        }
        const double rn = sqrt(a);
        rr[m] = a;
        int done = 0;
        if (!init) {
            const int it = iters[m] + 1;
            iters[m] = it;
            beta[m] = c / rz[m];
            if (it >= maxit[m]) done = 1;
        }
        rz[m] = c;
        if (rn < tol[m]) {
            done = 1;
            conv[m] = 1;
        }
        if (!(rn == rn)) done = 1;  // NaN: stop this molecule (not converged)
        if (done) idone[m] = 1;
        else atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int g = *gcount + 1;
        *gcount = g;
        if (set_cond) cudaGraphSetConditional(handle, (any && g < cap) ? 1u : 0u);
    }
}

// p = z + beta p (p = z at init) and its FP32 copy, molecules still iterating
__global__ void bdir_kernel(int Mtot, BatchDev B, const double *__restrict__ z, double *__restrict__ p,
                            float *__restrict__ p32, const double *__restrict__ beta, const int *__restrict__ idone,
                            int init)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Mtot; k += gridDim.x * blockDim.x) {
        const int m = B.elem_mol[k];
        if (m < 0 || idone[m]) continue;
        const double v = init ? z[k] : fma(beta[m], p[k], z[k]);
        p[k] = v;
        p32[k] = (float)v;
    }
}

// ro = b - y, |ro| per molecule (one block per molecule, fixed order)
__global__ void bresid_kernel(BatchDev B, const double *__restrict__ b, const double *__restrict__ y,
                              double *__restrict__ ro, double *__restrict__ rnorm)
{
    const int m = blockIdx.x;
    const int o = B.off[m], M = B.M[m];
    double s = 0.0;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const double v = b[o + k] - y[o + k];
        ro[o + k] = v;
        s = fma(v, v, s);
    }
    __shared__ double sh[32];
    const double t = block_sum<double, 1024>(s, sh);
    if (threadIdx.x == 0) rnorm[m] = sqrt(t);
}

// start of an inner solve: r = ro, correction d = 0 for active molecules
__global__ void binit_kernel(int Mtot, BatchDev B, const double *__restrict__ ro, double *__restrict__ r,
                             double *__restrict__ d, const int *__restrict__ idone)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Mtot; k += gridDim.x * blockDim.x) {
        const int m = B.elem_mol[k];
        d[k] = 0.0;
        if (m < 0 || idone[m]) continue;
        r[k] = ro[k];
    }
}

// x += d
__global__ void baxpy_kernel(int Mtot, const double *__restrict__ d, double *__restrict__ x)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Mtot; k += gridDim.x * blockDim.x) x[k] += d[k];
}

__global__ void brhs_kernel(int M, double f, const double *__restrict__ Bz, const double *__restrict__ c,
                            double *__restrict__ rhs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) rhs[k] = -f * (Bz[k] + c[k]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int batch_layout(pcm_batch *bt)
{
    if (bt->layout_ok) return PCM_OK;
    const int n = bt->nmol;
    std::vector<const double *> A64(n), inv(n), dinv(n);
    std::vector<const float *> A32(n), A32lo(n);
    std::vector<const int *> perm(n);
    std::vector<int> lda(n), M(n), off(n + 1), l(n), nblk(n), gbm, gbr, gbs(n + 1), rbm, rbb, rbs(n + 1);
    int o = 0;
    bt->rbj_l_max = 1;
    for (int m = 0; m < n; ++m) {
        pcm_ctx *c = bt->mol[m];
        A64[m] = c->A.p;
        A32[m] = c->A32.p;
        A32lo[m] = c->A32lo.p;
        lda[m] = c->lda;
        M[m] = c->M;
        off[m] = o;
        o += (c->M + 31) / 32 * 32;   // 32-element aligned slices (vector loads in the GEMV)
        if (c->pc_kind == PCM_PRECOND_RBJ) {
            perm[m] = c->rbj_perm.p;
            inv[m] = c->rbj_inv.p;
            l[m] = c->rbj_l;
            nblk[m] = c->rbj_nblk;
        } else {
            perm[m] = nullptr;
            inv[m] = nullptr;
            l[m] = 256;                  // Jacobi: chunks of consecutive indices
            nblk[m] = (c->M + 255) / 256;
        }
        dinv[m] = c->dinv.p;
        bt->rbj_l_max = std::max(bt->rbj_l_max, perm[m] ? l[m] : 1);
        gbs[m] = (int)gbm.size();
        for (int rp = 0; rp < (c->M + 1) / 2; ++rp) {
            gbm.push_back(m);
            gbr.push_back(rp);
        }
        rbs[m] = (int)rbm.size();
        for (int k = 0; k < nblk[m]; ++k) {
            rbm.push_back(m);
            rbb.push_back(k);
        }
    }
    off[n] = o;
    gbs[n] = (int)gbm.size();
    rbs[n] = (int)rbm.size();
    // PCM_MIXED: tiles of the upper triangles, partial slots, reduction blocks
    std::vector<int> gtm, gtij, rdm, rdr, rds(n + 1);
    std::vector<long long> soff(n + 1, 0);
    const bool sym = bt->opt.precision == PCM_MIXED;
    for (int m = 0; m < n && sym; ++m) {
        const int ntb = (M[m] + BT_TB - 1) / BT_TB;
        if (bt->mol[m]->A32.p)
            for (int I = 0; I < ntb; ++I)
                for (int J = I; J < ntb; ++J) {
                    gtm.push_back(m);
                    gtij.push_back((I << 16) | J);
                }
        soff[m + 1] = soff[m] + (long long)ntb * (off[m + 1] - off[m]);
        rds[m] = (int)rdm.size();
        for (int k = 0; k < M[m]; k += 256) {
            rdm.push_back(m);
            rdr.push_back(k);
        }
    }
    rds[n] = (int)rdm.size();
    bt->ngt = (int)gtm.size();
    bt->nrd = (int)rdm.size();
    if (sym && bt->ngt > 0) PCM_TRY(bt->ypart.alloc((size_t)std::max(1LL, soff[n])));
    if (gtm.empty()) gtm.push_back(0), gtij.push_back(0);
    if (rdm.empty()) rdm.push_back(0), rdr.push_back(0);
    bt->h_off = off;
    bt->Mtot = o;
    bt->ngb = (int)gbm.size();
    bt->nrb = (int)rbm.size();
    std::vector<int> em(o, -1);
    for (int m = 0; m < n; ++m)
        for (int k = 0; k < M[m]; ++k) em[off[m] + k] = m;
    auto up = [&](auto &buf, const auto &v) -> int {
        PCM_TRY(buf.alloc(v.size()));
        PCM_CUDA(cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, bt->stream));
        return PCM_OK;
    };
    PCM_TRY(up(bt->dA64, A64));
    PCM_TRY(up(bt->dA32, A32));
    PCM_TRY(up(bt->dA32lo, A32lo));
    PCM_TRY(up(bt->dperm, perm));
    PCM_TRY(up(bt->dinvp, inv));
    PCM_TRY(up(bt->ddinv, dinv));
    PCM_TRY(up(bt->dlda, lda));
    PCM_TRY(up(bt->dM, M));
    PCM_TRY(up(bt->doff, off));
    PCM_TRY(up(bt->dl, l));
    PCM_TRY(up(bt->dnblk, nblk));
    PCM_TRY(up(bt->gb_mol, gbm));
    PCM_TRY(up(bt->gb_rp, gbr));
    PCM_TRY(up(bt->gb_start, gbs));
    PCM_TRY(up(bt->rb_mol, rbm));
    PCM_TRY(up(bt->rb_blk, rbb));
    PCM_TRY(up(bt->rb_start, rbs));
    PCM_TRY(up(bt->elem_mol, em));
    PCM_TRY(up(bt->gt_mol, gtm));
    PCM_TRY(up(bt->gt_ij, gtij));
    PCM_TRY(up(bt->slot_off, soff));
    PCM_TRY(up(bt->rd_mol, rdm));
    PCM_TRY(up(bt->rd_row, rdr));
    PCM_TRY(up(bt->rd_start, rds));
    PCM_CUDA(cudaStreamSynchronize(bt->stream));  // the host vectors go out of scope
    BatchDev &D = bt->dev;
    D.A64 = bt->dA64.p;
    D.A32 = bt->dA32.p;
    D.A32lo = bt->dA32lo.p;
    D.perm = bt->dperm.p;
    D.inv = bt->dinvp.p;
    D.dinv = bt->ddinv.p;
    D.lda = bt->dlda.p;
    D.M = bt->dM.p;
    D.off = bt->doff.p;
    D.l = bt->dl.p;
    D.nblk = bt->dnblk.p;
    D.gb_mol = bt->gb_mol.p;
    D.gb_rp = bt->gb_rp.p;
    D.gb_start = bt->gb_start.p;
    D.rb_mol = bt->rb_mol.p;
    D.rb_blk = bt->rb_blk.p;
    D.rb_start = bt->rb_start.p;
    D.elem_mol = bt->elem_mol.p;
    D.gt_mol = bt->gt_mol.p;
    D.gt_ij = bt->gt_ij.p;
    D.slot_off = bt->slot_off.p;
    D.rd_mol = bt->rd_mol.p;
    D.rd_row = bt->rd_row.p;
    D.rd_start = bt->rd_start.p;
    const size_t Mt = std::max(1, o);
    for (DBuf<double> *v : {&bt->x, &bt->b, &bt->r, &bt->z, &bt->p, &bt->Ap, &bt->d, &bt->ro, &bt->y}) {
        PCM_TRY(v->alloc(Mt));
        PCM_CUDA(cudaMemsetAsync(v->p, 0, Mt * sizeof(double), bt->stream));
    }
    for (DBuf<float> *v : {&bt->p32, &bt->xh32, &bt->xl32}) {
        PCM_TRY(v->alloc(Mt));
        PCM_CUDA(cudaMemsetAsync(v->p, 0, Mt * sizeof(float), bt->stream));
    }
    for (DBuf<double> *v : {&bt->rz, &bt->pAp, &bt->alpha, &bt->beta, &bt->rr, &bt->tol, &bt->rnorm})
        PCM_TRY(v->alloc(n));
    for (DBuf<int> *v : {&bt->idone, &bt->iters, &bt->conv, &bt->maxit}) PCM_TRY(v->alloc(n));
    PCM_TRY(bt->gcount.alloc(1));
    PCM_TRY(bt->gpart.alloc(std::max(1, std::max(bt->ngb, bt->nrd))));
    PCM_TRY(bt->rpart.alloc(2 * (size_t)std::max(1, bt->nrb)));
    if (bt->exec) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    if (bt->graph) {
        cudaGraphDestroy(bt->graph);
        bt->graph = nullptr;
    }
    bt->layout_ok = true;
    return PCM_OK;
}

static int rbj_threads(int l) { return std::min(BR_NT_MAX, BR_SPLIT * std::max(32, (l + 31) / 32 * 32)); }

// one inner iteration (GEMV, alpha, update, scalars, direction) on the stream
static void batch_iteration(pcm_batch *bt, bool use32, int cap, cudaGraphConditionalHandle handle, int set_cond)
{
    const int n = bt->nmol;
    const BatchDev &D = bt->dev;
    if (use32) {
        if (bt->ngt > 0)
            bsym_kernel<false><<<bt->ngt, BG_NT, 0, bt->stream>>>(D, bt->p32.p, nullptr, bt->idone.p, bt->ypart.p);
        if (bt->nrd > 0)
            bsym_reduce_kernel<<<bt->nrd, 256, 0, bt->stream>>>(D, bt->ypart.p, bt->p.p, bt->idone.p, bt->Ap.p,
                                                               bt->gpart.p);
    } else {
        bgemv_kernel<double><<<bt->ngb, BG_NT, 0, bt->stream>>>(D, bt->p.p, bt->p.p, bt->Ap.p, bt->idone.p,
                                                                bt->gpart.p);
    }
    balpha_kernel<<<(n + 7) / 8, 256, 0, bt->stream>>>(n, use32 ? bt->rd_start.p : bt->gb_start.p, bt->gpart.p,
                                                       bt->idone.p, bt->rz.p, bt->pAp.p, bt->alpha.p);
    bupdate_kernel<<<bt->nrb, rbj_threads(bt->rbj_l_max), bt->rbj_l_max * sizeof(double), bt->stream>>>(
        D, bt->d.p, bt->r.p, bt->z.p, bt->p.p, bt->Ap.p, bt->alpha.p, bt->idone.p, bt->rpart.p, 0);
    bscalar_kernel<<<1, BS_NT, 0, bt->stream>>>(n, D, bt->rpart.p, bt->idone.p, bt->iters.p, bt->conv.p,
                                                bt->maxit.p, bt->tol.p, bt->rz.p, bt->rr.p, bt->beta.p, bt->gcount.p,
                                                cap, 0, handle, set_cond);
    const int eb = std::min(4096, (bt->Mtot + 255) / 256);
    bdir_kernel<<<eb, 256, 0, bt->stream>>>(bt->Mtot, D, bt->z.p, bt->p.p, bt->p32.p, bt->beta.p, bt->idone.p, 0);
}

static int build_graph(pcm_batch *bt, bool use32, int cap)
{
    if (bt->exec && bt->graph_mixed == use32) return PCM_OK;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    bt->exec = nullptr;
    bt->graph = nullptr;
    PCM_CUDA(cudaGraphCreate(&bt->graph, 0));
    cudaGraphConditionalHandle handle;
    PCM_CUDA(cudaGraphConditionalHandleCreate(&handle, bt->graph, 1, cudaGraphCondAssignDefault));
    // the parameter struct has no default constructor: zeroed raw storage
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams *cp = reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = handle;
    cp->conditional.type = cudaGraphCondTypeWhile;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    PCM_CUDA(cudaGraphAddNode(&node, bt->graph, nullptr, nullptr, 0, cp));
    cudaGraph_t body = cp->conditional.phGraph_out[0];
    PCM_CUDA(cudaStreamBeginCaptureToGraph(bt->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    batch_iteration(bt, use32, cap, handle, 1);
    cudaError_t e = cudaGetLastError();
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(bt->stream, &captured);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        set_last_error("graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        return PCM_ERR_CUDA;
    }
    PCM_CUDA(cudaGraphInstantiate(&bt->exec, bt->graph, 0));
    bt->graph_mixed = use32;
    return PCM_OK;
}

// Lockstep PCG over every molecule on A d = ro from d = 0 to tol_m (device
// arrays already set): initialisation, then the graph.  Returns with the
// iteration counts on the device.
static int batch_inner(pcm_batch *bt, bool use32, int cap)
{
    const int n = bt->nmol;
    const BatchDev &D = bt->dev;
    const int eb = std::min(4096, (bt->Mtot + 255) / 256);
    binit_kernel<<<eb, 256, 0, bt->stream>>>(bt->Mtot, D, bt->ro.p, bt->r.p, bt->d.p, bt->idone.p);
    bupdate_kernel<<<bt->nrb, rbj_threads(bt->rbj_l_max), bt->rbj_l_max * sizeof(double), bt->stream>>>(
        D, bt->d.p, bt->r.p, bt->z.p, bt->p.p, bt->Ap.p, bt->alpha.p, bt->idone.p, bt->rpart.p, 1);
    PCM_CUDA(cudaMemsetAsync(bt->gcount.p, 0, sizeof(int), bt->stream));
    bscalar_kernel<<<1, BS_NT, 0, bt->stream>>>(n, D, bt->rpart.p, bt->idone.p, bt->iters.p, bt->conv.p, bt->maxit.p,
                                                bt->tol.p, bt->rz.p, bt->rr.p, bt->beta.p, bt->gcount.p, cap, 1,
                                                cudaGraphConditionalHandle(), 0);
    bdir_kernel<<<eb, 256, 0, bt->stream>>>(bt->Mtot, D, bt->z.p, bt->p.p, bt->p32.p, bt->beta.p, bt->idone.p, 1);
    PCM_CUDA(cudaGetLastError());
    PCM_CUDA(cudaMemsetAsync(bt->gcount.p, 0, sizeof(int), bt->stream));
    PCM_TRY(build_graph(bt, use32, cap));
    PCM_CUDA(cudaGraphLaunch(bt->exec, bt->stream));
    return PCM_OK;
}

// Solve A_m q_m = b_m for every molecule to ||r||_2 < delta (Eq. 20).
static int batch_solve(pcm_batch *bt, double delta)
{
    const int n = bt->nmol;
    const bool mixed = bt->opt.precision == PCM_MIXED;
    const BatchDev &D = bt->dev;
    const int maxit = bt->opt.max_iter;
    const int cap = maxit + 1;     // bound of the graph loop (each molecule has its own cap)
    std::vector<int> done(n, 0), conv(n, 0), total(n, 0), refine(n, 0), hi(n), hc(n);
    std::vector<double> tol(n), rn(n, 0.0), final_rn(n, 0.0);
    PCM_CUDA(cudaMemsetAsync(bt->x.p, 0, (size_t)bt->Mtot * sizeof(double), bt->stream));
    constexpr double ETA = 1e-3;
    const int max_round = mixed ? 12 : 1;
    for (int round = 0; round <= max_round; ++round) {
        // true residual of every molecule not yet done
        PCM_CUDA(cudaMemcpyAsync(bt->idone.p, done.data(), n * sizeof(int), cudaMemcpyHostToDevice, bt->stream));
        if (mixed) {
            // double-float A x: the FP64 pipe would bound an FP64 GEMV below the HBM rate
            const int sb = std::min(4096, (bt->Mtot + 255) / 256);
            bsplit_kernel<<<sb, 256, 0, bt->stream>>>(bt->Mtot, bt->x.p, bt->xh32.p, bt->xl32.p);
            if (bt->ngt > 0)
                bsym_kernel<true><<<bt->ngt, BG_NT, 0, bt->stream>>>(D, bt->xh32.p, bt->xl32.p, bt->idone.p,
                                                                    bt->ypart.p);
            if (bt->nrd > 0)
                bsym_reduce_kernel<<<bt->nrd, 256, 0, bt->stream>>>(D, bt->ypart.p, bt->x.p, bt->idone.p, bt->y.p,
                                                                   bt->gpart.p);
        } else {
            bgemv_kernel<double><<<bt->ngb, BG_NT, 0, bt->stream>>>(D, bt->x.p, bt->x.p, bt->y.p, bt->idone.p,
                                                                    bt->gpart.p);
        }
        bresid_kernel<<<n, 1024, 0, bt->stream>>>(D, bt->b.p, bt->y.p, bt->ro.p, bt->rnorm.p);
        PCM_CUDA(cudaGetLastError());
        PCM_CUDA(cudaMemcpyAsync(rn.data(), bt->rnorm.p, n * sizeof(double), cudaMemcpyDeviceToHost, bt->stream));
        PCM_CUDA(cudaStreamSynchronize(bt->stream));
        bt->launches += 2;
        int active = 0;
        for (int m = 0; m < n; ++m) {
            if (done[m]) continue;
            final_rn[m] = rn[m];
            if (rn[m] < delta) {
                done[m] = 1;
                conv[m] = 1;
            } else if (total[m] >= maxit || round == max_round || !std::isfinite(rn[m])) {
                done[m] = 1;
            } else {
                tol[m] = mixed ? std::max(ETA * rn[m], 0.5 * delta) : delta;
                ++active;
            }
        }
        if (!active) break;
        std::vector<int> mi(n), zero(n, 0);
        for (int m = 0; m < n; ++m) mi[m] = std::max(1, maxit - total[m]);
        PCM_CUDA(cudaMemcpyAsync(bt->idone.p, done.data(), n * sizeof(int), cudaMemcpyHostToDevice, bt->stream));
        PCM_CUDA(cudaMemcpyAsync(bt->tol.p, tol.data(), n * sizeof(double), cudaMemcpyHostToDevice, bt->stream));
        PCM_CUDA(cudaMemcpyAsync(bt->maxit.p, mi.data(), n * sizeof(int), cudaMemcpyHostToDevice, bt->stream));
        PCM_CUDA(cudaMemcpyAsync(bt->iters.p, zero.data(), n * sizeof(int), cudaMemcpyHostToDevice, bt->stream));
        PCM_CUDA(cudaMemcpyAsync(bt->conv.p, zero.data(), n * sizeof(int), cudaMemcpyHostToDevice, bt->stream));
        PCM_TRY(batch_inner(bt, mixed, cap));
        const int eb = std::min(4096, (bt->Mtot + 255) / 256);
        baxpy_kernel<<<eb, 256, 0, bt->stream>>>(bt->Mtot, bt->d.p, bt->x.p);
        PCM_CUDA(cudaGetLastError());
        PCM_CUDA(cudaMemcpyAsync(hi.data(), bt->iters.p, n * sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
        PCM_CUDA(cudaMemcpyAsync(hc.data(), bt->conv.p, n * sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
        PCM_CUDA(cudaStreamSynchronize(bt->stream));  // mi, zero, done, tol are read by the copies above
        int most = 0;
        for (int m = 0; m < n; ++m)
            if (!done[m]) {
                total[m] += hi[m];
                most = std::max(most, hi[m]);
                ++refine[m];
                if (!mixed) {
                    // FP64: the inner loop is the whole solve, with the recursively
                    // updated residual's test (as the single-molecule solver)
                    done[m] = 1;
                    conv[m] = hc[m];
                }
            }
        bt->launches += 5 + 5 * (long long)(most + 1) + 1;
        if (!mixed) break;
    }
    for (int m = 0; m < n; ++m) {
        pcm_stats &s = bt->st[m];
        s.iterations = total[m];
        s.converged = conv[m];
        s.delta = delta;
        s.rnorm = final_rn[m];
        s.refinements = mixed ? refine[m] : 0;
    }
    return PCM_OK;
}

}  // namespace pcm

using namespace pcm;

extern "C" {

int pcm_batch_create(pcm_batch **out, const pcm_options *opt, int nmol)
{
    if (!out || nmol <= 0) {
        set_last_error("pcm_batch_create: bad arguments");
        return PCM_ERR_ARG;
    }
    *out = nullptr;
    pcm_options o;
    if (opt) o = *opt;
    else pcm_default_options(&o);
    pcm_batch *bt = new (std::nothrow) pcm_batch();
    if (!bt) return PCM_ERR_OOM;
    bt->opt = o;
    bt->nmol = nmol;
    bt->device = o.device;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(o.device) != cudaSuccess) {
        delete bt;
        set_last_error("pcm_batch_create: device %d is not available", o.device);
        return PCM_ERR_ARG;
    }
    if (o.stream) {
        bt->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete bt;
            cudaSetDevice(prev);
            set_last_error("cudaStreamCreate failed");
            return PCM_ERR_CUDA;
        }
        bt->own_stream = true;
    }
    pcm_options mo = o;
    mo.stream = bt->stream;
    bt->mol.assign(nmol, nullptr);
    bt->ready.assign(nmol, 0);
    bt->st.assign(nmol, pcm_stats{});
    for (int m = 0; m < nmol; ++m) {
        int s = pcm_create(&bt->mol[m], &mo);
        if (s != PCM_OK) {
            pcm_batch_destroy(bt);
            cudaSetDevice(prev);
            return s;
        }
        // the lockstep solver reads each molecule's stored A; with
        // PCM_OPERATOR_FREE the molecules keep none and are solved one after
        // another by the matrix-free solver
        bt->mol[m]->store_a = o.operator_mode != PCM_OPERATOR_FREE;
    }
    cudaSetDevice(prev);
    *out = bt;
    return PCM_OK;
}

int pcm_batch_destroy(pcm_batch *bt)
{
    if (!bt) return PCM_OK;
    cudaSetDevice(bt->device);
    cudaStreamSynchronize(bt->stream);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    for (pcm_ctx *c : bt->mol)
        if (c) pcm_destroy(c);
    bt->mol.clear();
    const bool own = bt->own_stream;
    cudaStream_t s = bt->stream;
    delete bt;  // device buffers free themselves
    if (own) cudaStreamDestroy(s);
    return PCM_OK;
}

int pcm_batch_set_molecule(pcm_batch *bt, int i, int natom, const double *xyz, const double *Z, const double *radius,
                           int pts_per_sphere, int nshell, const int *shell_atom, const int *shell_l,
                           const int *shell_nprim, const double *exps, const double *coefs)
{
    if (!bt || i < 0 || i >= bt->nmol) {
        set_last_error("pcm_batch_set_molecule: bad molecule index");
        return PCM_ERR_ARG;
    }
    if (bt->opt.precond == PCM_PRECOND_OCTREE) {
        set_last_error("pcm_batch_set_molecule: batches use RBJ or Jacobi preconditioners");
        return PCM_ERR_UNSUPPORTED;
    }
    pcm_ctx *c = bt->mol[i];
    bt->ready[i] = 0;
    bt->layout_ok = false;
    PCM_TRY(pcm_build_surface(c, natom, xyz, Z, radius, pts_per_sphere, nullptr));
    PCM_TRY(pcm_set_basis(c, nshell, shell_atom, shell_l, shell_nprim, exps, coefs, nullptr));
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(bt->device);
    int s = solver_prepare_full(c);
    cudaSetDevice(prev);
    if (s != PCM_OK) return s;
    bt->ready[i] = 1;
    bt->st[i].M = c->M;
    bt->st[i].nbf = c->nbf;
    return PCM_OK;
}

int pcm_batch_sizes(pcm_batch *bt, int i, int *M, int *nbf)
{
    if (!bt || i < 0 || i >= bt->nmol || !bt->ready[i]) {
        set_last_error("pcm_batch_sizes: molecule %d is not set", i);
        return PCM_ERR_ARG;
    }
    if (M) *M = bt->mol[i]->M;
    if (nbf) *nbf = bt->mol[i]->nbf;
    return PCM_OK;
}

int pcm_batch_run(pcm_batch *bt, const double *const *P, double delta, double *E, double *const *q,
                  double *const *dF, int flags)
{
    if (!bt || !P || !E || !(delta > 0.0)) {
        set_last_error("pcm_batch_run: bad arguments (delta must be positive)");
        return PCM_ERR_ARG;
    }
    for (int m = 0; m < bt->nmol; ++m)
        if (!bt->ready[m] || !P[m]) {
            set_last_error("pcm_batch_run: molecule %d is not set or has no density", m);
            return PCM_ERR_ARG;
        }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(bt->device);
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};
    PCM_TRY(batch_layout(bt));
    const double f = (bt->opt.eps - 1.0) / (bt->opt.eps + bt->opt.k);
    const bool dev = (flags & PCM_PTR_DEVICE) != 0;
    // PCM_MIXED with the packed kernels: every molecule's packed ESP and Fock
    // blocks are collected and run in one launch per angular class
    const bool batched = bt->opt.precision == PCM_MIXED && bt->opt.fp32x2;
    struct Undefer {
        pcm_batch *bt;
        ~Undefer()
        {
            for (pcm_ctx *c : bt->mol) c->jobs = nullptr;
        }
    } undefer{bt};
    if (batched) {
        bt->sink.clear();
        if (!bt->derr.p) {
            PCM_TRY(bt->derr.alloc(1));
            PCM_CUDA(cudaMemsetAsync(bt->derr.p, 0, sizeof(int), bt->stream));
        }
    }
    // ESP of every molecule, and the right-hand sides
    for (int m = 0; m < bt->nmol; ++m) {
        pcm_ctx *c = bt->mol[m];
        const size_t n2 = (size_t)c->nbf * c->nbf;
        const double *dP = P[m];
        if (!dev) {
            PCM_TRY(c->dP.alloc(n2));
            PCM_CUDA(cudaMemcpyAsync(c->dP.p, P[m], n2 * sizeof(double), cudaMemcpyHostToDevice, bt->stream));
            dP = c->dP.p;
        }
        PCM_TRY(c->c_last.alloc(c->M));
        c->jobs = batched ? &bt->sink : nullptr;
        PCM_TRY(esp_compute(c, dP, c->c_last.p));
        c->jobs = nullptr;
        c->have_c = true;
        bt->st[m].integrals_esp = c->stats.integrals_esp;
        bt->st[m].pairs_esp = c->stats.pairs_esp;
    }
    if (batched) {
        PCM_TRY(launch_jobs(bt->sink, bt->dej, bt->dfj, bt->mol[0]->boys32.p, bt->derr.p, bt->stream));
        bt->launches += 10;
        for (int m = 0; m < bt->nmol; ++m) PCM_TRY(esp_mixed_finish(bt->mol[m]));
    }
    for (int m = 0; m < bt->nmol; ++m) {
        pcm_ctx *c = bt->mol[m];
        brhs_kernel<<<(c->M + 255) / 256, 256, 0, bt->stream>>>(c->M, f, c->Bz.p, c->c_last.p,
                                                                 bt->b.p + bt->h_off[m]);
        PCM_LAUNCHED(c);
    }
    if (bt->opt.precision == PCM_MIXED && bt->opt.operator_mode == PCM_OPERATOR_FREE) {
        // matrix-free molecules: each solve is one persistent inner solver per
        // refinement, molecule after molecule
        for (int m = 0; m < bt->nmol; ++m) {
            pcm_ctx *c = bt->mol[m];
            pcm_stats sm{};
            const int st = solver_run(c, bt->b.p + bt->h_off[m], delta, bt->x.p + bt->h_off[m], false, &sm);
            if (st != PCM_OK && st != PCM_ERR_NOT_CONVERGED) return st;
            bt->st[m].iterations = sm.iterations;
            bt->st[m].converged = sm.converged;
            bt->st[m].rnorm = sm.rnorm;
            bt->st[m].refinements = sm.refinements;
            bt->st[m].delta = delta;
        }
    } else {
        // every solve in lockstep
        PCM_TRY(batch_solve(bt, delta));
        if (bt->opt.precision == PCM_MIXED) {
            // the refinement ends on a true residual of every molecule's final
            // charges: y = A x is the energy's A q (as a single solve keeps it)
            for (int m = 0; m < bt->nmol; ++m) {
                pcm_ctx *c = bt->mol[m];
                PCM_TRY(c->aq_q.alloc(c->M));
                PCM_TRY(c->aq_y.alloc(c->M));
                PCM_CUDA(cudaMemcpyAsync(c->aq_q.p, bt->x.p + bt->h_off[m], c->M * sizeof(double),
                                         cudaMemcpyDeviceToDevice, bt->stream));
                PCM_CUDA(cudaMemcpyAsync(c->aq_y.p, bt->y.p + bt->h_off[m], c->M * sizeof(double),
                                         cudaMemcpyDeviceToDevice, bt->stream));
                c->aq_valid = true;
            }
        }
    }
    // Fock correction and energy of every molecule
    std::vector<double *> ddFs(bt->nmol, nullptr);
    if (batched) bt->sink.clear();
    for (int m = 0; m < bt->nmol; ++m) {
        pcm_ctx *c = bt->mol[m];
        const double *dq = bt->x.p + bt->h_off[m];
        if (dF && dF[m]) {
            const size_t n2 = (size_t)c->nbf * c->nbf;
            double *ddF = dF[m];
            if (!dev) {
                PCM_TRY(c->dF.alloc(n2));
                ddF = c->dF.p;
            }
            ddFs[m] = ddF;
            c->jobs = batched ? &bt->sink : nullptr;
            PCM_TRY(fock_compute(c, dq, ddF));
            c->jobs = nullptr;
            bt->st[m].integrals_fock = c->stats.integrals_fock;
        }
    }
    if (batched) {
        PCM_TRY(launch_jobs(bt->sink, bt->dej, bt->dfj, bt->mol[0]->boys32.p, bt->derr.p, bt->stream));
        bt->launches += 10;
        for (int m = 0; m < bt->nmol; ++m)
            if (ddFs[m]) PCM_TRY(fock_mixed_finish(bt->mol[m], ddFs[m]));
    }
    for (int m = 0; m < bt->nmol; ++m) {
        pcm_ctx *c = bt->mol[m];
        const double *dq = bt->x.p + bt->h_off[m];
        if (ddFs[m] && !dev) {
            const size_t n2 = (size_t)c->nbf * c->nbf;
            PCM_CUDA(cudaMemcpyAsync(dF[m], ddFs[m], n2 * sizeof(double), cudaMemcpyDeviceToHost, bt->stream));
        }
        PCM_TRY(energy_compute(c, dq, c->c_last.p, &E[m]));
        if (q && q[m])
            PCM_CUDA(cudaMemcpyAsync(q[m], dq, c->M * sizeof(double),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, bt->stream));
    }
    PCM_CUDA(cudaStreamSynchronize(bt->stream));
    if (batched) {
        int h = 0;
        PCM_CUDA(cudaMemcpy(&h, bt->derr.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (h) {
            PCM_CUDA(cudaMemset(bt->derr.p, 0, sizeof(int)));
            set_last_error("pcm_batch_run: a bounded device wait gave up in a batched integral kernel");
            return PCM_ERR_TIMEOUT;
        }
    }
    return PCM_OK;
}

int pcm_batch_get_stats(pcm_batch *bt, int i, pcm_stats *st)
{
    if (!bt || !st || i < -1 || i >= bt->nmol) return PCM_ERR_ARG;
    if (i == -1) {
        // batch totals: the lockstep solver's kernels and every molecule's
        memset(st, 0, sizeof(*st));
        st->launches = bt->launches;
        for (int m = 0; m < bt->nmol; ++m) {
            st->launches += bt->mol[m]->stats.launches;
            st->integrals_esp += bt->st[m].integrals_esp;
            st->integrals_fock += bt->st[m].integrals_fock;
            st->iterations = std::max(st->iterations, bt->st[m].iterations);
            st->M += bt->st[m].M;
            st->nbf += bt->st[m].nbf;
        }
        return PCM_OK;
    }
    *st = bt->st[i];
    st->launches = bt->mol[i]->stats.launches;
    return PCM_OK;
}

}  // extern "C"
