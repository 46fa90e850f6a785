// Matrix-free A (Eq. 2, Eq. 3, Eq. 8) for the PCM_MIXED solver.
//
// A_kl = erf(zeta'_kl R_kl) / R_kl equals 1/R_kl to FP64 precision once
// zeta' R > 6.  Pairs closer than rc = 6.1 / min(zeta') (the diagonal
// included) are kept in a near-pair list with their exact FP64 values (CSR,
// about twenty per row); every other element is recomputed as 1/R whenever a
// product with A is needed, in tiles of rows x columns:
//   - the inner PCG's A p in FP32 (the hardware reciprocal square root; the
//     FP32 pipes evaluate 1/R faster than HBM streams a stored FP32 A),
//   - true residuals and the energy's A q in double-float (1/R from split
//     coordinates to ~3e-14 relative, float-float sums), near pairs in FP64.
// One FP32 distance test (r2_test32 on the FP32 coordinates) decides near or
// far everywhere, so each element is counted exactly once.
//
// The inner PCG runs as one persistent cooperative kernel per inner solve:
// per iteration the product (matrix-free: work items of 512 rows x up to 1024
// columns over all blocks, partial products per column chunk; stored FP32 A:
// the tiles of its upper triangle only, each streamed from HBM once and used
// for both A_IJ p_J and A_IJ^T p_I, since A is symmetric), the update and
// preconditioner (Jacobi, or one randomized block-Jacobi block per thread
// block), and the direction update, separated by grid-wide barriers whose
// waits are bounded.  The stored-operator variant serves PCM_MIXED surfaces
// small enough to keep A32 + A32lo.
#include <math.h>

#include <algorithm>
#include <vector>

#include "aelem.cuh"
#include "common.cuh"
#include "context.h"
#include "dfloat.cuh"
#include "f2.cuh"
#include "fastmath.cuh"
#include "gemv.cuh"
#include "rbj_apply.cuh"

namespace pcm {

constexpr int MV_NT = 256;     // threads per block
constexpr int MV_ROWS = 512;   // rows per work item (two per thread)
constexpr int MV_CH = 1024;    // columns per work item
constexpr int MV_SUB = 256;    // columns staged in shared memory at a time
constexpr int NL_CH = 1024;    // columns staged per pass of the near-list build
constexpr int ST_TB = 128;     // tile side of the symmetric stored-operator product
constexpr int ST_RW = ST_TB / (MV_NT / 32);   // rows of a tile per warp (16)
constexpr int FS_TB = 256;     // tile side of the symmetric matrix-free product

__global__ void pts4_kernel(int M, const double *__restrict__ px, const double *__restrict__ py,
                            const double *__restrict__ pz, float4 *__restrict__ pts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) pts[k] = make_float4((float)px[k], (float)py[k], (float)pz[k], 0.f);
}

// near pairs of row k (r2_test32 < rc2, the diagonal included): count, or
// write columns (ascending), exact values, and for the FP32 product the values
// less the constant rsqrt(rc2) that product adds for each near pair
template <bool FILL>
__global__ void __launch_bounds__(MV_NT) near_rows_kernel(int M, const float4 *__restrict__ pts, float rc2,
                                                          int *__restrict__ cnt, const int *__restrict__ off,
                                                          AFree acc, int *__restrict__ col,
                                                          double *__restrict__ val, float *__restrict__ val32)
{
    __shared__ float4 sc[NL_CH];
    const int k = blockIdx.x * MV_NT + threadIdx.x;
    const float4 a = pts[min(k, M - 1)];
    int n = 0, o = FILL && k < M ? off[k] : 0;
    for (int c0 = 0; c0 < M; c0 += NL_CH) {
        const int nc = min(NL_CH, M - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < nc; t += MV_NT) sc[t] = pts[c0 + t];
        __syncthreads();
        if (k < M)
            for (int j = 0; j < nc; ++j)
                if (r2_test32(a, sc[j]) < rc2) {
                    if (FILL) {
                        const double v = acc.exact(k, c0 + j);
                        col[o] = c0 + j;
                        val[o] = v;
                        // the FP32 product adds rsqrt(rc2) for every near pair
                        val32[o] = (float)(v - (double)rsqrt_fast(rc2));
                        ++o;
                    } else {
                        ++n;
                    }
                }
    }
    if (!FILL && k < M) cnt[k] = n;
}

// exclusive scan of n ints by one block: off[0..n] (off[n] = total)
__global__ void scan_one_block_kernel(int n, const int *__restrict__ cnt, int *__restrict__ off)
{
    __shared__ int sh[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = sh[t];
            sh[t] = acc;
            acc += v;
        }
        off[n] = acc;
    }
    __syncthreads();
    int acc = sh[threadIdx.x];
    for (int i = b; i < e; ++i) {
        off[i] = acc;
        acc += cnt[i];
    }
}

// 1 / A_kk for the Jacobi preconditioner: S_k / (zeta_k sqrt(2/pi))
__global__ void dinv_free_kernel(int M, const double *__restrict__ pzeta, const double *__restrict__ pS,
                                 double *__restrict__ dinv)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) dinv[k] = 1.0 / (pzeta[k] * 0.79788456080286535588 / pS[k]);
}

AFree afree(pcm_ctx *c)
{
    AFree a;
    a.px = c->px.p;
    a.py = c->py.p;
    a.pz = c->pz.p;
    a.pzeta = c->pzeta.p;
    a.pS = c->pS.p;
    a.pcls = c->pcls.p;
    a.ncls = c->ncls;
    a.zp = c->zp_cls.p;
    a.pts = c->mf_pts.p;
    return a;
}

// zeta'_kl = zeta_k zeta_l / sqrt(zeta_k^2 + zeta_l^2) (Eq. 8) for every pair
// of exponent classes, on the host (IEEE division and square root, as on the
// device), uploaded on stream s
int zeta_pairs(pcm_ctx *c, cudaStream_t s)
{
    const int nc = c->ncls;
    std::vector<double> &zp = c->h_zp_cls;  // kept in the context: the copy reads it later
    zp.assign((size_t)nc * nc, 0.0);
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) {
            const double za = c->h_cls_zeta[a], zb = c->h_cls_zeta[b];
            zp[(size_t)a * nc + b] = za * zb / sqrt(za * za + zb * zb);
        }
    PCM_TRY(c->zp_cls.alloc(std::max<size_t>(1, zp.size())));
    PCM_CUDA(cudaMemcpyAsync(c->zp_cls.p, zp.data(), zp.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    return PCM_OK;
}

// The matrix-free operator of a surface on stream s: FP32 coordinates, the
// near-pair list and 1 / A_kk
int matfree_build(pcm_ctx *c, cudaStream_t s)
{
    const int M = c->M;
    c->st_arow_ok = false;
    PCM_TRY(zeta_pairs(c, s));
    double zmin = 1e300;
    for (double z : c->h_zp_cls) zmin = std::min(zmin, z);
    const double rc = 6.1 / zmin;
    c->mf_rc2 = (float)(rc * rc);
    PCM_TRY(c->mf_pts.alloc(M));
    pts4_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, c->px.p, c->py.p, c->pz.p, c->mf_pts.p);
    PCM_LAUNCHED(c);
    PCM_TRY(c->mf_off.alloc(M + 1));
    PCM_TRY(c->mf_cnt.alloc(M));
    const AFree acc = afree(c);
    const int nb = (M + MV_NT - 1) / MV_NT;
    near_rows_kernel<false><<<nb, MV_NT, 0, s>>>(M, c->mf_pts.p, c->mf_rc2, c->mf_cnt.p, nullptr, acc, nullptr,
                                                 nullptr, nullptr);
    PCM_LAUNCHED(c);
    scan_one_block_kernel<<<1, 1024, 0, s>>>(M, c->mf_cnt.p, c->mf_off.p);
    PCM_LAUNCHED(c);
    int nnz = 0;
    PCM_CUDA(cudaMemcpyAsync(&nnz, c->mf_off.p + M, sizeof(int), cudaMemcpyDeviceToHost, s));
    PCM_CUDA(cudaStreamSynchronize(s));
    c->mf_nnz = nnz;
    PCM_TRY(c->mf_col.alloc(std::max(1, nnz)));
    PCM_TRY(c->mf_val.alloc(std::max(1, nnz)));
    PCM_TRY(c->mf_val32.alloc(std::max(1, nnz)));
    near_rows_kernel<true><<<nb, MV_NT, 0, s>>>(M, c->mf_pts.p, c->mf_rc2, nullptr, c->mf_off.p, acc, c->mf_col.p,
                                                c->mf_val.p, c->mf_val32.p);
    PCM_LAUNCHED(c);
    PCM_TRY(c->dinv.alloc(M));
    dinv_free_kernel<<<(M + 127) / 128, 128, 0, s>>>(M, c->pzeta.p, c->pS.p, c->dinv.p);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

// ---------------------------------------------------------------------------
// y = A x in double-float: far pairs 1/R from the split coordinates (FP32 hi
// on a 2^-10 grid + lo), float-float sums over tiles of the upper triangle
// (dfmv_sym_kernel); then per row the tile partials and the near pairs (FP64)
// added in a fixed order, with block partials of x.y
// ---------------------------------------------------------------------------
__global__ void split_vec_kernel(int M, const double *__restrict__ x, float2 *__restrict__ xs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) {
        const float h = (float)x[k];
        xs[k] = make_float2(h, (float)(x[k] - (double)h));
    }
}

__global__ void __launch_bounds__(MV_NT) dfmv_reduce_kernel(int M, int S, const double *__restrict__ ypart,
                                                            const int *__restrict__ off, const int *__restrict__ col,
                                                            const double *__restrict__ val,
                                                            const double *__restrict__ x, double *__restrict__ y,
                                                            double *__restrict__ part)
{
    __shared__ double red[MV_NT / 32];
    const int k = blockIdx.x * MV_NT + threadIdx.x;
    double d = 0.0;
    if (k < M) {
        double v = 0.0;
        for (int e = off[k]; e < off[k + 1]; ++e) v = fma(val[e], x[col[e]], v);
        for (int s = 0; s < S; ++s) v += ypart[(size_t)s * M + k];
        y[k] = v;
        d = x[k] * v;
    }
    d = block_sum<double, MV_NT>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = d;
}

// The same product over the tiles of the upper triangle only (A symmetric:
// each double-float 1/R serves A_ij x_j and A_ji x_i).  Tile t (I <= J,
// DS_TB x DS_TB, row-major order) goes to block t mod grid; warp w takes rows
// I0 + 32 w + lane, one per lane, against the tile's columns, which it visits
// in groups of 32: at step s of a group, lane l takes column (l + s) mod 32,
// so the 32 lanes touch 32 different columns and each column's float-float
// sum (this warp's part, in shared memory) has one writer per step, in a
// fixed order.  Near pairs and the diagonal (r2_test32 < rc2) contribute
// nothing here.  Row sums go to ypart[J][row], column sums (the warps' parts
// added in warp order) to ypart[I][column]: each row of y receives exactly
// one partial per tile column block, summed by dfmv_reduce_kernel.
constexpr int DS_TB = 256;

__global__ void __launch_bounds__(MV_NT) dfmv_sym_kernel(int M, int ntb, const float4 *__restrict__ pts,
                                                         const float *__restrict__ ph, const float *__restrict__ pl,
                                                         const float2 *__restrict__ xs, float rc2,
                                                         double *__restrict__ ypart)
{
    __shared__ float4 sP[DS_TB], sH[DS_TB], sL[DS_TB];
    __shared__ float cS[MV_NT / 32][DS_TB], cC[MV_NT / 32][DS_TB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long ntiles = (long long)ntb * (ntb + 1) / 2;
    int I = 0;
    long long pos = blockIdx.x;
    while (I < ntb && pos >= ntb - I) {
        pos -= ntb - I;
        ++I;
    }
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int J = I + (int)pos;
        const int I0 = I * DS_TB, J0 = J * DS_TB;
        const bool diag = I == J;
        __syncthreads();
        {
            const int l = J0 + threadIdx.x;
            const int ll = min(l, M - 1);
            const float2 x = l < M ? xs[l] : make_float2(0.f, 0.f);
            sP[threadIdx.x] = pts[ll];
            sH[threadIdx.x] = make_float4(ph[ll], ph[(size_t)M + ll], ph[2 * (size_t)M + ll], x.x);
            sL[threadIdx.x] = make_float4(pl[ll], pl[(size_t)M + ll], pl[2 * (size_t)M + ll], x.y);
            if (!diag)
                for (int q = 0; q < MV_NT / 32; ++q) {
                    cS[q][threadIdx.x] = 0.f;
                    cC[q][threadIdx.x] = 0.f;
                }
        }
        const int k = I0 + 32 * w + lane;
        const int kk = min(k, M - 1);
        const float4 a = pts[kk];
        const float xh = ph[kk], yh = ph[(size_t)M + kk], zh = ph[2 * (size_t)M + kk];
        const float xl = pl[kk], yl = pl[(size_t)M + kk], zl = pl[2 * (size_t)M + kk];
        const float2 xk = k < M ? xs[kk] : make_float2(0.f, 0.f);
        __syncthreads();
        float S_ = 0.f, C_ = 0.f;
        for (int g = 0; g < DS_TB; g += 32) {
#pragma unroll 4
            for (int st = 0; st < 32; ++st) {
                const int j = g + ((lane + st) & 31);
                const float4 h = sH[j], lo = sL[j];
                float ih, il, r2;
                df_rsqrt(xh - h.x, xl - lo.x, yh - h.y, yl - lo.y, zh - h.z, zl - lo.z, ih, il, r2);
                const bool far = r2_test32(a, sP[j]) >= rc2;
                ih = far ? ih : 0.f;
                il = far ? il : 0.f;
                df_acc(S_, C_, ih, il, h.w, lo.w);
                if (!diag) {
                    float cs = cS[w][j], cc = cC[w][j];
                    df_acc(cs, cc, ih, il, xk.x, xk.y);
                    cS[w][j] = cs;
                    cC[w][j] = cc;
                }
                __syncwarp();   // the next step's lane for this column reads it
            }
        }
        if (k < M) ypart[(size_t)J * M + k] = (double)S_ + (double)C_;
        if (!diag) {
            __syncthreads();
            const int l = J0 + threadIdx.x;
            if (l < M) {
                double v = 0.0;
                for (int q = 0; q < MV_NT / 32; ++q) v += (double)cS[q][threadIdx.x] + (double)cC[q][threadIdx.x];
                ypart[(size_t)I * M + l] = v;
            }
        }
        pos += gridDim.x;
        while (I < ntb && pos >= ntb - I) {
            pos -= ntb - I;
            ++I;
        }
    }
}

// y = A x (double-float far part, FP64 near part); part receives per-block
// partials of x.y, *nparts their count
int matfree_dfmv(pcm_ctx *c, const double *x, double *y, double *part, int *nparts)
{
    const int M = c->M;
    const int ntb = (M + DS_TB - 1) / DS_TB;
    static int per = 0;
    if (per == 0) {
        PCM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dfmv_sym_kernel, MV_NT, 0));
        per = std::max(per, 1);
    }
    int nsm = 0;
    PCM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    PCM_TRY(c->mf_xs.alloc(M));
    PCM_TRY(c->mf_y64.alloc((size_t)ntb * M));
    split_vec_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, x, c->mf_xs.p);
    PCM_LAUNCHED(c);
    const long long ntiles = (long long)ntb * (ntb + 1) / 2;
    const int grid = (int)std::min<long long>(ntiles, (long long)per * nsm);
    dfmv_sym_kernel<<<grid, MV_NT, 0, c->stream>>>(M, ntb, c->mf_pts.p, c->p32.p, c->p32lo.p, c->mf_xs.p, c->mf_rc2,
                                                   c->mf_y64.p);
    PCM_LAUNCHED(c);
    const int nb = (M + MV_NT - 1) / MV_NT;
    dfmv_reduce_kernel<<<nb, MV_NT, 0, c->stream>>>(M, ntb, c->mf_y64.p, c->mf_off.p, c->mf_col.p, c->mf_val.p, x, y,
                                                    part);
    PCM_LAUNCHED(c);
    if (nparts) *nparts = nb;
    return PCM_OK;
}

// ---------------------------------------------------------------------------
// persistent inner PCG (cooperative launch: every block resident)
// ---------------------------------------------------------------------------
struct PcgArgs {
    int M, S, nitems, ch;        // points, column chunks, work items of the product (stored: blocks), chunk width
    const float *A32;            // stored FP32 A (row-major, leading dimension lda); null: matrix-free
    int lda;
    int ntb;                     // stored: tiles per side (ST_TB x ST_TB tiles)
    unsigned long long *acc;     // stored: A p in fixed point (M), read and cleared by the update
    unsigned *pmax;              // stored: [2] FP32 bits of max |p32| before each product (by its parity)
    const double *arow;          // max over rows of sum_l |A32_kl| (stored) or of the near-list |values| (matrix-free)
    double arow_add;             // matrix-free: M / rc, the bound of a row's far part
    const float4 *pts;           // FP32 coordinates
    float *p32;                  // FP32 copy of the direction (the product's input)
    float rc2;
    const int *off, *col;        // near pairs (CSR) and their FP32 values
    const float *val32;
    float *ypart;                // S x M partial products, row k at position iperm[k] (k without iperm)
    const int *iperm;            // position of each point in the preconditioner's block order
    double *idot;                // per work item partial of p.Ap
    const double *b;             // right-hand side; the solve starts from x = 0
    double *x, *r, *z, *p, *Ap;
    int rbj;                     // 0: Jacobi (dinv); 1: block Jacobi (perm, inv, bstart)
    const double *dinv;
    int l, nblk;
    const int *perm, *bstart;
    const double *inv;
    double *red;                 // partials of r.r and r.z (2 per slot)
    double delta;
    int max_iter;
    unsigned *bar;               // [0] arrivals, [1] generation
    int *out;                    // [0] iterations, [1] converged, [2] a barrier wait gave up
    double *rnorm;
};

// Grid-wide barrier with a bounded wait: true when every block arrived.
// Writes before it are visible to reads after it through L2 (the readers
// below load data written by other blocks with ld.global.cg).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned a = atomicAdd(bar, 1u);
        int good = 1;
        if (a == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            // poll with a growing pause (fewer loads on the line the last
            // arrival has to update)
            int it = 0;
            unsigned ns = 32;
            while (*gen == g && it < (1 << 22)) {
                __nanosleep(ns);
                ns = ns < 512 ? 2 * ns : ns;
                ++it;
            }
            good = *gen != g;
        }
        __threadfence();
        if (!good) atomicExch(err, 1);
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// fixed-order sum of n values written by other blocks; every block computes
// the same value; valid in all threads
__device__ __forceinline__ double grid_sum(const double *v, int n, int stride, int offset)
{
    __shared__ double sh[MV_NT / 32];
    __shared__ double res;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += MV_NT) s += __ldcg(v + (size_t)i * stride + offset);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < MV_NT / 32; ++w) t += sh[w];
        res = t;
    }
    __syncthreads();
    return res;
}

// The per-row FP32 matrix-free product (pcm_apply_a with PCM_APPLY_FP32):
// work items of rows rt*512 + t and + 256 (two lanes), columns [s*1024, ...);
// partial products to ypart[s], p.Ap partial to idot[item].  The inner solver
// evaluates the same elements over the upper triangle (pcg_product_free_sym).
__device__ __forceinline__ void pcg_product(const PcgArgs &a, float4 (*sc)[2])
{
    __shared__ double red[MV_NT / 32];
    const int M = a.M;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int rt = item / a.S, s = item % a.S;
        const int k0 = rt * MV_ROWS + threadIdx.x, k1 = k0 + MV_NT;
        const float4 q0 = a.pts[min(k0, M - 1)], q1 = a.pts[min(k1, M - 1)];
        const f2 rx(q0.x, q1.x), ry(q0.y, q1.y), rz(q0.z, q1.z);
        // four running sums (columns j mod 4), so that each FP32 sum adds a
        // quarter of the chunk.  A far pair contributes p_l / R; a near pair
        // (r2 < rc2, the diagonal included) the constant p_l rsqrt(rc2), which
        // the near list's FP32 values take back
        f2 acc[4] = {f2(0.f), f2(0.f), f2(0.f), f2(0.f)};
        const float rc2 = a.rc2;
        auto term = [&](const float4 u, const float4 v, f2 &acc_) {
            const f2 dx = rx - f2(u.x, u.y), dy = ry - f2(u.z, u.w), dz = rz - f2(v.x, v.y);
            const f2 r2 = fma2(dx, dx, fma2(dy, dy, dz * dz));
            const f2 rs(rsqrt_fast(fmaxf(r2.v.x, rc2)), rsqrt_fast(fmaxf(r2.v.y, rc2)));
            acc_ = fma2(rs, f2(v.z, v.w), acc_);
        };
        const int c0 = s * a.ch, c1 = min(M, c0 + a.ch);
        for (int b0 = c0; b0 < c1; b0 += MV_SUB) {
            const int nc = min(MV_SUB, c1 - b0);
            __syncthreads();
            for (int t = threadIdx.x; t < nc; t += MV_NT) {
                const float4 q = a.pts[b0 + t];
                const float pv = __ldcg(a.p32 + b0 + t);
                sc[t][0] = make_float4(q.x, q.x, q.y, q.y);
                sc[t][1] = make_float4(q.z, q.z, pv, pv);
            }
            __syncthreads();
            int j = 0;
#pragma unroll 2
            for (; j + 4 <= nc; j += 4) {
                term(sc[j][0], sc[j][1], acc[0]);
                term(sc[j + 1][0], sc[j + 1][1], acc[1]);
                term(sc[j + 2][0], sc[j + 2][1], acc[2]);
                term(sc[j + 3][0], sc[j + 3][1], acc[3]);
            }
            for (; j < nc; ++j) term(sc[j][0], sc[j][1], acc[0]);
        }
        const f2 accs = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        float y0 = accs.v.x, y1 = accs.v.y;
        if (s == 0) {
            // near pairs and the diagonal
            if (k0 < M)
                for (int e = a.off[k0]; e < a.off[k0 + 1]; ++e) y0 = fmaf(a.val32[e], __ldcg(a.p32 + a.col[e]), y0);
            if (k1 < M)
                for (int e = a.off[k1]; e < a.off[k1 + 1]; ++e) y1 = fmaf(a.val32[e], __ldcg(a.p32 + a.col[e]), y1);
        }
        double d = 0.0;
        if (k0 < M) {
            a.ypart[(size_t)s * M + (a.iperm ? a.iperm[k0] : k0)] = y0;
            d = __ldcg(a.p + k0) * (double)y0;
        }
        if (k1 < M) {
            a.ypart[(size_t)s * M + (a.iperm ? a.iperm[k1] : k1)] = y1;
            d = fma(__ldcg(a.p + k1), (double)y1, d);
        }
        d = block_sum<double, MV_NT>(d, red);
        if (threadIdx.x == 0) a.idot[item] = d;
    }
}


// Fixed-point scale of the symmetric products: every partial sum of a row of
// A p is bounded by arow max|p32| < 2^e (arow: a bound on the row sums of |A|
// as the product forms them), so sums of values v 2^(61 - e) rounded to
// integers stay below 2^61 in magnitude, and integer addition makes the
// result independent of the order in which the tiles add their parts.
__device__ __forceinline__ double st_scale(const PcgArgs &a, int n, double *inv)
{
    const float pm = __uint_as_float(__ldcg(a.pmax + (n & 1)));
    const double bound = (__ldcg(a.arow) + a.arow_add) * (double)pm;
    if (!(bound > 0.0) || !isfinite(bound)) {
        *inv = 1.0;
        return 1.0;
    }
    int e = 0;
    frexp(bound, &e);
    *inv = ldexp(1.0, e - 61);
    return ldexp(1.0, 61 - e);
}

__device__ __forceinline__ void st_add(unsigned long long *acc, float v, double scale)
{
    atomicAdd(acc, (unsigned long long)__double2ll_rn((double)v * scale));
}

// The matrix-free FP32 product over the tiles of the upper triangle (A
// symmetric: each 1/R evaluated once serves A_ij p_j and A_ji p_i).  Blocks
// take contiguous runs of the tiles (I <= J, FS_TB x FS_TB, row-major order),
// so a block stays on one tile row I for many tiles: the rows' coordinates
// and their running sums stay in registers across the run and are flushed
// once per row block.  In a tile, warp w takes columns J0 + 32 w + t (t < 32,
// staged in shared memory, read as broadcasts) against all FS_TB rows, eight
// per lane (rows I0 + 32 r + lane, two per packed FP32x2 word); the element is
// 1/R with R^2 clamped below at rc2 exactly as in the per-row product, near
// pairs and the diagonal thus adding the constant that the near list takes
// back.  The 32 column partials of a lane are reduced across the lanes by
// halving (31 shuffles); row sums are added across the warps in shared memory
// at the flush.  Diagonal tiles form row sums only (both triangles and the
// diagonal).  The near-pair corrections are one pass over the rows by the
// whole grid.  Sums enter the fixed-point accumulators; block partials of
// p.Ap to idot[block].
struct FsRows {
    f2 rx[4], ry[4], rz[4], rp[4], racc[4];
};

__device__ __forceinline__ void fs_rows_load(const PcgArgs &a, int I0, FsRows &R)
{
    const int lane = threadIdx.x & 31, M = a.M;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i0 = I0 + 64 * q + lane, i1 = i0 + 32;
        const float4 u0 = a.pts[min(i0, M - 1)], u1 = a.pts[min(i1, M - 1)];
        R.rx[q] = f2(u0.x, u1.x);
        R.ry[q] = f2(u0.y, u1.y);
        R.rz[q] = f2(u0.z, u1.z);
        R.rp[q] = f2(i0 < M ? __ldcg(a.p32 + i0) : 0.f, i1 < M ? __ldcg(a.p32 + i1) : 0.f);
        R.racc[q] = f2(0.f);
    }
}

// the warps' row sums of row block I0, added in warp order, into the accumulators
__device__ __forceinline__ void fs_rows_flush(const PcgArgs &a, int I0, const FsRows &R, float (*srow)[FS_TB],
                                              double scale, double &d)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        srow[w][64 * q + lane] = R.racc[q].v.x;
        srow[w][64 * q + 32 + lane] = R.racc[q].v.y;
    }
    __syncthreads();
    const int i = I0 + threadIdx.x;
    if (i < a.M) {
        float v = srow[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < MV_NT / 32; ++q) v += srow[q][threadIdx.x];
        st_add(a.acc + i, v, scale);
        d = fma(__ldcg(a.p + i), (double)v, d);
    }
}

template <bool DIAG>
__device__ __forceinline__ void fs_tile(const PcgArgs &a, int J0, double scale, const float4 *scol, FsRows &R,
                                        double &d)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float rc2 = a.rc2;
    float cp[32];
    const float4 *col = scol + 32 * w;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const float4 c = col[t];
        const f2 cx(c.x), cy(c.y), cz(c.z), cw(c.w);
        f2 ca(0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const f2 dx = R.rx[q] - cx, dy = R.ry[q] - cy, dz = R.rz[q] - cz;
            const f2 r2 = fma2(dx, dx, fma2(dy, dy, dz * dz));
            const f2 rs(rsqrt_fast(fmaxf(r2.v.x, rc2)), rsqrt_fast(fmaxf(r2.v.y, rc2)));
            R.racc[q] = fma2(rs, cw, R.racc[q]);
            if (!DIAG) ca = fma2(rs, R.rp[q], ca);
        }
        if (!DIAG) cp[t] = ca.v.x + ca.v.y;
    }
    if (!DIAG) {
        // column sums: halve the 32 partials across the lanes; lane l ends
        // with the sum for column 32 w + l
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
            const bool up = (lane & h) != 0;
#pragma unroll
            for (int m = 0; m < h; ++m) {
                const float send = up ? cp[m] : cp[m + h];
                const float keep = up ? cp[m + h] : cp[m];
                cp[m] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        const int jc = J0 + 32 * w + lane;
        if (jc < a.M) {
            st_add(a.acc + jc, cp[0], scale);
            d = fma(__ldcg(a.p + jc), (double)cp[0], d);
        }
    }
}

__device__ __forceinline__ void pcg_product_free_sym(const PcgArgs &a, int n)
{
    __shared__ double red[MV_NT / 32];
    __shared__ float4 scol[FS_TB];
    __shared__ float srow[MV_NT / 32][FS_TB];
    double inv;
    const double scale = st_scale(a, n, &inv);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.pmax[(n + 1) & 1] = 0u;
    const int M = a.M;
    double d = 0.0;
    const int ntb = a.ntb;
    const long long ntiles = (long long)ntb * (ntb + 1) / 2;
    const long long t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    int I = 0;
    long long pos = t0;
    while (I < ntb && pos >= ntb - I) {
        pos -= ntb - I;
        ++I;
    }
    FsRows R;
    int cur = -1;
    for (long long t = t0; t < t1; ++t) {
        const int J = I + (int)pos;
        if (I != cur) {
            if (cur >= 0) fs_rows_flush(a, cur * FS_TB, R, srow, scale, d);
            fs_rows_load(a, I * FS_TB, R);
            cur = I;
        }
        __syncthreads();   // the previous tile's readers of scol (and the flush's of srow) are done
        {
            const int j = J * FS_TB + threadIdx.x;
            const float4 q = a.pts[min(j, M - 1)];
            scol[threadIdx.x] = make_float4(q.x, q.y, q.z, j < M ? __ldcg(a.p32 + j) : 0.f);
        }
        __syncthreads();
        if (J == I)
            fs_tile<true>(a, J * FS_TB, scale, scol, R, d);
        else
            fs_tile<false>(a, J * FS_TB, scale, scol, R, d);
        if (++pos >= ntb - I) {
            pos = 0;
            ++I;
        }
    }
    if (cur >= 0) {
        __syncthreads();
        fs_rows_flush(a, cur * FS_TB, R, srow, scale, d);
    }
    // near pairs and the diagonal: A_kl - rsqrt(rc2) for the constant the tiles
    // add, one row per thread over the grid; the column indices and values of
    // eight entries are loaded before their directions, so that the dependent
    // loads overlap
    for (int i = blockIdx.x * MV_NT + threadIdx.x; i < M; i += gridDim.x * MV_NT) {
        float v = 0.f;
        const int e0 = a.off[i], e1 = a.off[i + 1];
        for (int e = e0; e < e1; e += 8) {
            int cl[8];
            float vl[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                cl[u] = e + u < e1 ? a.col[e + u] : 0;
                vl[u] = e + u < e1 ? a.val32[e + u] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) v = fmaf(vl[u], __ldcg(a.p32 + cl[u]), v);
        }
        st_add(a.acc + i, v, scale);
        d = fma(__ldcg(a.p + i), (double)v, d);
    }
    d = block_sum<double, MV_NT>(d, red);
    if (threadIdx.x == 0) a.idot[blockIdx.x] = d;
}

// The product with the stored FP32 A (A symmetric): tile t of the upper
// triangle (I <= J, ST_TB x ST_TB) goes to block t mod grid.  Warp w takes
// rows I0 + w + 8 m (m < 16), lane l columns J0 + 4 l .. + 3, all sixteen
// 16-byte loads of the warp in flight at once.  Row sums (A_IJ p_J) are
// reduced across the lanes; off-diagonal tiles also form column sums
// (A_IJ^T p_I), reduced across the warps in shared memory.  Both are added to
// the fixed-point accumulators; block partials of p.Ap to idot[block].
__device__ __forceinline__ void pcg_product_stored(const PcgArgs &a, int n)
{
    __shared__ double red[MV_NT / 32];
    __shared__ __align__(16) float cs[MV_NT / 32][ST_TB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int M = a.M, ntb = a.ntb;
    double inv;
    const double scale = st_scale(a, n, &inv);
    // the other parity's max |p| is cleared for the direction update before the next product
    if (blockIdx.x == 0 && threadIdx.x == 0) a.pmax[(n + 1) & 1] = 0u;
    const long long ntiles = (long long)ntb * (ntb + 1) / 2;
    // first tile of this block: row I of the triangle holds ntb - I tiles
    int I = 0;
    long long pos = blockIdx.x;
    while (I < ntb && pos >= ntb - I) {
        pos -= ntb - I;
        ++I;
    }
    double d = 0.0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int J = I + (int)pos;
        const int I0 = I * ST_TB, J0 = J * ST_TB;
        const int c0 = J0 + 4 * lane;
        const bool cok = c0 < M;
        float4 a4[ST_RW];
#pragma unroll
        for (int m = 0; m < ST_RW; ++m) {
            const int row = I0 + w + 8 * m;
            a4[m] = (cok && row < M) ? *reinterpret_cast<const float4 *>(a.A32 + (size_t)row * a.lda + c0)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float4 pj = __ldcg(reinterpret_cast<const float4 *>(a.p32 + c0));
        if (c0 + 3 >= M) {
            // columns beyond M: zero both the direction and the (unwritten) matrix entries
#pragma unroll
            for (int m = 0; m < ST_RW; ++m) {
                if (c0 + 1 >= M) a4[m].y = 0.f;
                if (c0 + 2 >= M) a4[m].z = 0.f;
                if (c0 + 3 >= M) a4[m].w = 0.f;
            }
            if (c0 >= M) pj.x = 0.f;
            if (c0 + 1 >= M) pj.y = 0.f;
            if (c0 + 2 >= M) pj.z = 0.f;
            if (c0 + 3 >= M) pj.w = 0.f;
        }
        float rp[ST_RW];
        float4 ca = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int m = 0; m < ST_RW; ++m) {
            rp[m] = fmaf(a4[m].x, pj.x, fmaf(a4[m].y, pj.y, fmaf(a4[m].z, pj.z, a4[m].w * pj.w)));
            const int row = I0 + w + 8 * m;
            const float pi = row < M ? __ldcg(a.p32 + row) : 0.f;
            ca.x = fmaf(a4[m].x, pi, ca.x);
            ca.y = fmaf(a4[m].y, pi, ca.y);
            ca.z = fmaf(a4[m].z, pi, ca.z);
            ca.w = fmaf(a4[m].w, pi, ca.w);
        }
        // reduce the sixteen row partials across the lanes by halving: after
        // the steps at 16, 8, 4, 2 and 1, lanes 2i and 2i + 1 hold the sum of
        // row m = 8 b4 + 4 b3 + 2 b2 + b1 (b: the bits of the lane)
#pragma unroll
        for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int m = 0; m < h; ++m) {
                const float send = up ? rp[m] : rp[m + h];
                const float keep = up ? rp[m + h] : rp[m];
                rp[m] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        const float rsum = rp[0] + __shfl_xor_sync(0xffffffffu, rp[0], 1);
        {
            const int m = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
            const int row = I0 + w + 8 * m;
            if ((lane & 1) == 0 && row < M) {
                st_add(a.acc + row, rsum, scale);
                d = fma(__ldcg(a.p + row), (double)rsum, d);
            }
        }
        if (I != J) {
            // column sums: the warps' parts in shared memory, added in warp order
            *reinterpret_cast<float4 *>(&cs[w][4 * lane]) = ca;
            __syncthreads();
            if (threadIdx.x < ST_TB) {
                float v = cs[0][threadIdx.x];
#pragma unroll
                for (int q = 1; q < MV_NT / 32; ++q) v += cs[q][threadIdx.x];
                const int col = J0 + threadIdx.x;
                if (col < M) {
                    st_add(a.acc + col, v, scale);
                    d = fma(__ldcg(a.p + col), (double)v, d);
                }
            }
            __syncthreads();
        }
        // next tile of this block
        pos += gridDim.x;
        while (I < ntb && pos >= ntb - I) {
            pos -= ntb - I;
            ++I;
        }
    }
    d = block_sum<double, MV_NT>(d, red);
    if (threadIdx.x == 0) a.idot[blockIdx.x] = d;
}

// A p at block position pos (the row at that place of the preconditioner's
// order): the column chunks' partial products, added in a fixed order
__device__ __forceinline__ double ap_pos(const PcgArgs &a, int pos)
{
    double v = 0.0;
    for (int s = 0; s < a.S; ++s) v += (double)__ldcg(a.ypart + (size_t)s * a.M + pos);
    return v;
}

// A p of point k from the stored product's accumulator, which is cleared for
// the next product
__device__ __forceinline__ double ap_acc(const PcgArgs &a, int k, double inv)
{
    const long long v = (long long)__ldcg(a.acc + k);
    a.acc[k] = 0ull;
    return (double)v * inv;
}

// update (init: only z = C r) on the rows this block owns; partials of r.r
// and r.z to red[2 slot], red[2 slot + 1]
__device__ __forceinline__ void pcg_update(const PcgArgs &a, double alpha, int init, double *srb, double inv)
{
    __shared__ double sh[2][MV_NT / 32];
    if (a.rbj) {
        for (int b = blockIdx.x; b < a.nblk; b += gridDim.x) {
            const int base = a.bstart ? a.bstart[b] : b * a.l;
            const int nb = a.bstart ? a.bstart[b + 1] - base : min(a.l, a.M - base);
            for (int i = threadIdx.x; i < nb; i += MV_NT) {
                const int k = a.perm[base + i];
                if (init) {
                    a.x[k] = 0.0;
                    a.r[k] = a.b[k];
                } else {
                    a.Ap[k] = a.acc ? ap_acc(a, k, inv) : ap_pos(a, base + i);
                }
            }
            __syncthreads();
            double rr, rz;
            rbj_apply_block(a.M, a.l, b, a.perm, a.bstart, a.inv, a.x, a.r, a.z, a.p, a.Ap, alpha, init, srb, &rr,
                            &rz);
            if (threadIdx.x == 0) {
                a.red[2 * b] = rr;
                a.red[2 * b + 1] = rz;
            }
            __syncthreads();
        }
    } else {
        double rr = 0.0, rz = 0.0;
        for (int k = blockIdx.x * MV_NT + threadIdx.x; k < a.M; k += gridDim.x * MV_NT) {
            double rk;
            if (init) {
                a.x[k] = 0.0;
                rk = a.b[k];
            } else {
                a.x[k] = fma(alpha, a.p[k], a.x[k]);
                rk = fma(-alpha, a.acc ? ap_acc(a, k, inv) : ap_pos(a, k), a.r[k]);
            }
            a.r[k] = rk;
            const double zk = a.dinv ? rk * a.dinv[k] : rk;
            a.z[k] = zk;
            rr = fma(rk, rk, rr);
            rz = fma(rk, zk, rz);
        }
        rr = warp_sum(rr);
        rz = warp_sum(rz);
        if ((threadIdx.x & 31) == 0) {
            sh[0][threadIdx.x >> 5] = rr;
            sh[1][threadIdx.x >> 5] = rz;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0, w = 0.0;
            for (int i = 0; i < MV_NT / 32; ++i) {
                u += sh[0][i];
                w += sh[1][i];
            }
            a.red[2 * blockIdx.x] = u;
            a.red[2 * blockIdx.x + 1] = w;
        }
        __syncthreads();
    }
}

// p = z + beta p on the owned rows (beta = 0: p = z), and its FP32 copy; for
// the stored product also max |p32| (slot n & 1 for product n)
__device__ __forceinline__ void pcg_direction(const PcgArgs &a, double beta, int n)
{
    float mx = 0.f;
    if (a.rbj) {
        for (int b = blockIdx.x; b < a.nblk; b += gridDim.x) {
            const int base = a.bstart ? a.bstart[b] : b * a.l;
            const int nb = a.bstart ? a.bstart[b + 1] - base : min(a.l, a.M - base);
            for (int i = threadIdx.x; i < nb; i += MV_NT) {
                const int k = a.perm[base + i];
                const double v = fma(beta, a.p[k], a.z[k]);
                a.p[k] = v;
                a.p32[k] = (float)v;
                mx = fmaxf(mx, fabsf((float)v));
            }
        }
    } else {
        for (int k = blockIdx.x * MV_NT + threadIdx.x; k < a.M; k += gridDim.x * MV_NT) {
            const double v = fma(beta, a.p[k], a.z[k]);
            a.p[k] = v;
            a.p32[k] = (float)v;
            mx = fmaxf(mx, fabsf((float)v));
        }
    }
    if (a.acc) {
        // non-negative floats order as their bit patterns
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(a.pmax + (n & 1), __float_as_uint(mx));
    }
}

template <bool STORED>
__global__ void __launch_bounds__(MV_NT) pcg_persistent_kernel(PcgArgs a)
{
    extern __shared__ double srb[];          // RBJ block: l entries
    int *err = a.out + 2;
    const int nslot = a.rbj ? a.nblk : (int)gridDim.x;
    // initialisation: x = 0, r = b, z = C r
    pcg_update(a, 0.0, 1, srb, 1.0);
    if (!grid_barrier(a.bar, err)) return;
    double rr = grid_sum(a.red, nslot, 2, 0);
    double rz = grid_sum(a.red, nslot, 2, 1);
    int it = 0, conv = sqrt(rr) < a.delta;
    if (!conv) {
        pcg_direction(a, 0.0, 0);
        if (!grid_barrier(a.bar, err)) return;
        while (true) {
            double inv = 1.0;
            st_scale(a, it, &inv);
            if constexpr (STORED)
                pcg_product_stored(a, it);
            else
                pcg_product_free_sym(a, it);
            if (!grid_barrier(a.bar, err)) return;
            const double pAp = grid_sum(a.idot, a.nitems, 1, 0);
            pcg_update(a, rz / pAp, 0, srb, inv);
            if (!grid_barrier(a.bar, err)) return;
            rr = grid_sum(a.red, nslot, 2, 0);
            const double rz_new = grid_sum(a.red, nslot, 2, 1);
            ++it;
            // Eq. 20 on the recursively updated residual, or the iteration cap
            if (sqrt(rr) < a.delta) {
                conv = 1;
                break;
            }
            if (it >= a.max_iter) break;
            pcg_direction(a, rz_new / rz, it);
            rz = rz_new;
            if (!grid_barrier(a.bar, err)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] = it;
        a.out[1] = conv;
        *a.rnorm = sqrt(rr);
    }
}

__global__ void iperm_kernel(int M, const int *__restrict__ perm, int *__restrict__ iperm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) iperm[perm[i]] = i;
}

// Column chunks of the FP32 product for a grid of `grid` blocks: chunks of at
// most MV_CH columns (a multiple of 4), and at least two work items per block
// where the rows allow it, so that small surfaces still fill the GPU.
static void mv_chunks(int M, int grid, int *S, int *ch)
{
    const int nrt = (M + MV_ROWS - 1) / MV_ROWS;
    const int s = std::max((M + MV_CH - 1) / MV_CH, (2 * grid + nrt - 1) / nrt);
    int w = (M + s - 1) / s;
    w = std::max(4, (w + 3) / 4 * 4);
    *ch = w;
    *S = (M + w - 1) / w;
}

// max over rows of sum_l |A32_kl| (FP64 row sums, one warp per row; the
// maximum of non-negative doubles taken on their bit patterns), the bound
// behind the fixed-point scale of the stored product
__global__ void __launch_bounds__(MV_NT) arow_kernel(int M, int lda, const float *__restrict__ A32,
                                                     unsigned long long *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int row = blockIdx.x * (MV_NT / 32) + (threadIdx.x >> 5); row < M; row += gridDim.x * (MV_NT / 32)) {
        const float *r = A32 + (size_t)row * lda;
        double s = 0.0;
        for (int col = lane; col < M; col += 32) s += fabs((double)r[col]);
        mx = fmax(mx, warp_sum(s));
    }
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// max over rows of sum_e |val32_e| over the row's near pairs (one warp per
// row), the near part of the matrix-free product's row-sum bound
__global__ void __launch_bounds__(MV_NT) near_abs_kernel(int M, const int *__restrict__ off,
                                                         const float *__restrict__ val32,
                                                         unsigned long long *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int row = blockIdx.x * (MV_NT / 32) + (threadIdx.x >> 5); row < M; row += gridDim.x * (MV_NT / 32)) {
        double s = 0.0;
        for (int e = off[row] + lane; e < off[row + 1]; e += 32) s += fabs((double)val32[e]);
        mx = fmax(mx, warp_sum(s));
    }
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// Inner PCG from x = 0 on A x = b with the FP32 product (matrix-free, or the
// stored A32 of PCM_MIXED) and the context's preconditioner, to ||r|| < delta
// (recursively updated residual) or max_iter steps, in one cooperative launch.
int persistent_pcg(pcm_ctx *c, const double *b, double *x, double delta, int max_iter, int *iters, int *conv,
                   double *rnorm)
{
    const int M = c->M;
    const bool stored = !matrix_free(c);
    const bool rbj = c->pc_kind == PCM_PRECOND_RBJ || c->pc_kind == PCM_PRECOND_OCTREE;
    const size_t smem = rbj ? (size_t)c->rbj_l * sizeof(double) : sizeof(double);
    const void *kern = stored ? (const void *)pcg_persistent_kernel<true> : (const void *)pcg_persistent_kernel<false>;
    const int v = stored ? 1 : 0;
    if (smem > 48 * 1024)
        PCM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (c->pg_grid[v] == 0 || c->pg_smem[v] != smem) {
        int per = 0, nsm = 0;
        PCM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, MV_NT, smem));
        PCM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
        if (per < 1) {
            set_last_error("inner solver: the persistent kernel cannot be resident");
            return PCM_ERR_CUDA;
        }
        c->pg_grid[v] = per * nsm;
        c->pg_smem[v] = smem;
    }
    const int grid = c->pg_grid[v];
    const int nslot = rbj ? c->rbj_nblk : grid;
    const int tb = stored ? ST_TB : FS_TB;
    const int ntb = (M + tb - 1) / tb;
    PCM_TRY(c->mf_idot.alloc((size_t)grid));
    PCM_TRY(c->st_acc.alloc(M));
    PCM_TRY(c->st_pmax.alloc(2));
    PCM_TRY(c->st_arow.alloc(1));
    if (!c->st_arow_ok) {
        // the row-sum bound of the fixed-point scale, once per operator
        PCM_CUDA(cudaMemsetAsync(c->st_arow.p, 0, sizeof(double), c->stream));
        unsigned long long *o = reinterpret_cast<unsigned long long *>(c->st_arow.p);
        if (stored)
            arow_kernel<<<std::min(4096, (M + 7) / 8), MV_NT, 0, c->stream>>>(M, c->lda, c->A32.p, o);
        else
            near_abs_kernel<<<std::min(4096, (M + 7) / 8), MV_NT, 0, c->stream>>>(M, c->mf_off.p, c->mf_val32.p, o);
        PCM_LAUNCHED(c);
        c->st_arow_ok = true;
    }
    PCM_CUDA(cudaMemsetAsync(c->st_acc.p, 0, (size_t)M * sizeof(unsigned long long), c->stream));
    PCM_CUDA(cudaMemsetAsync(c->st_pmax.p, 0, 2 * sizeof(unsigned), c->stream));
    // the stored product reads the direction in whole tiles: zero padding to ntb tiles
    const size_t np32 = (size_t)ntb * tb;
    PCM_TRY(c->mf_p32.alloc(np32));
    PCM_CUDA(cudaMemsetAsync(c->mf_p32.p, 0, np32 * sizeof(float), c->stream));
    PCM_TRY(c->vr.alloc(M));
    PCM_TRY(c->vz.alloc(M));
    PCM_TRY(c->vp.alloc(M));
    PCM_TRY(c->vAp.alloc(M));
    PCM_TRY(c->mf_red.alloc(2 * (size_t)std::max(nslot, 1)));
    if (rbj) {
        PCM_TRY(c->mf_iperm.alloc(M));
        iperm_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, c->rbj_perm.p, c->mf_iperm.p);
        PCM_LAUNCHED(c);
    }
    PCM_TRY(c->mf_bar.alloc(2));
    PCM_TRY(c->mf_out.alloc(4));
    PCM_TRY(c->mf_rn.alloc(1));
    PCM_CUDA(cudaMemsetAsync(c->mf_bar.p, 0, 2 * sizeof(unsigned), c->stream));
    PCM_CUDA(cudaMemsetAsync(c->mf_out.p, 0, 4 * sizeof(int), c->stream));
    PcgArgs a;
    a.M = M;
    a.S = 0;
    a.ch = 0;
    a.nitems = grid;
    a.A32 = stored ? c->A32.p : nullptr;
    a.lda = c->lda;
    a.ntb = ntb;
    a.acc = c->st_acc.p;
    a.pmax = c->st_pmax.p;
    a.arow = c->st_arow.p;
    a.arow_add = stored ? 0.0 : (double)M / sqrt((double)c->mf_rc2);
    a.pts = c->mf_pts.p;
    a.p32 = c->mf_p32.p;
    a.rc2 = c->mf_rc2;
    a.off = c->mf_off.p;
    a.col = c->mf_col.p;
    a.val32 = c->mf_val32.p;
    a.ypart = nullptr;
    a.iperm = rbj ? c->mf_iperm.p : nullptr;
    a.idot = c->mf_idot.p;
    a.b = b;
    a.x = x;
    a.r = c->vr.p;
    a.z = c->vz.p;
    a.p = c->vp.p;
    a.Ap = c->vAp.p;
    a.rbj = rbj ? 1 : 0;
    a.dinv = c->pc_kind == PCM_PRECOND_JACOBI ? c->dinv.p : nullptr;
    a.l = c->rbj_l;
    a.nblk = c->rbj_nblk;
    a.perm = c->rbj_perm.p;
    a.bstart = c->pc_kind == PCM_PRECOND_OCTREE ? c->rbj_bstart.p : nullptr;
    a.inv = c->rbj_inv.p;
    a.red = c->mf_red.p;
    a.delta = delta;
    a.max_iter = max_iter;
    a.bar = c->mf_bar.p;
    a.out = c->mf_out.p;
    a.rnorm = c->mf_rn.p;
    void *args[] = {&a};
    PCM_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(MV_NT), args, smem, c->stream));
    PCM_LAUNCHED(c);
    int h[4];
    double rn = 0.0;
    PCM_CUDA(cudaMemcpyAsync(h, c->mf_out.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaMemcpyAsync(&rn, c->mf_rn.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    if (h[2]) {
        set_last_error("inner solver: a grid barrier wait gave up");
        return PCM_ERR_TIMEOUT;
    }
    *iters = h[0];
    *conv = h[1];
    *rnorm = rn;
    return PCM_OK;
}

// y = A x with the FP32 matrix-free elements of the inner solver, summed per
// row over column chunks (pcg_product; pcm_apply_a with PCM_APPLY_FP32), y in
// FP64
__global__ void __launch_bounds__(MV_NT) mv32_reduce_kernel(int M, int S, const float *__restrict__ ypart,
                                                            double *__restrict__ y)
{
    const int k = blockIdx.x * MV_NT + threadIdx.x;
    if (k >= M) return;
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += (double)ypart[(size_t)s * M + k];
    y[k] = v;
}

__global__ void __launch_bounds__(MV_NT) mv32_items_kernel(PcgArgs a)
{
    __shared__ float4 sc[MV_SUB][2];
    pcg_product(a, sc);
}

__global__ void to_f32_kernel(int M, const double *__restrict__ x, float *__restrict__ x32, double *__restrict__ x64)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) {
        x32[k] = (float)x[k];
        x64[k] = x[k];
    }
}

int matfree_mv32(pcm_ctx *c, const double *x, double *y)
{
    const int M = c->M;
    const int nrt = (M + MV_ROWS - 1) / MV_ROWS;
    int S, ch;
    mv_chunks(M, 152 * 6, &S, &ch);
    PCM_TRY(c->mf_p32.alloc(M));
    PCM_TRY(c->vp.alloc(M));
    PCM_TRY(c->mf_ypart.alloc((size_t)S * M));
    PCM_TRY(c->mf_idot.alloc((size_t)nrt * S));
    to_f32_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, x, c->mf_p32.p, c->vp.p);
    PCM_LAUNCHED(c);
    PcgArgs a = {};
    a.M = M;
    a.S = S;
    a.ch = ch;
    a.nitems = nrt * S;
    a.pts = c->mf_pts.p;
    a.p32 = c->mf_p32.p;
    a.rc2 = c->mf_rc2;
    a.off = c->mf_off.p;
    a.col = c->mf_col.p;
    a.val32 = c->mf_val32.p;
    a.ypart = c->mf_ypart.p;
    a.idot = c->mf_idot.p;
    a.p = c->vp.p;
    mv32_items_kernel<<<std::min(a.nitems, 152 * 8), MV_NT, 0, c->stream>>>(a);
    PCM_LAUNCHED(c);
    mv32_reduce_kernel<<<(M + MV_NT - 1) / MV_NT, MV_NT, 0, c->stream>>>(M, S, c->mf_ypart.p, y);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

}  // namespace pcm
