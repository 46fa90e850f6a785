// Utility kernels: Boys-function tables and stable stream compaction.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "boys.cuh"
#include "common.cuh"
#include "context.h"

namespace pcm {

// ---------------------------------------------------------------------------
// Boys tables.  F_m(T_i) = \int_0^1 u^{2m} exp(-T_i u^2) du by composite
// Gauss-Legendre quadrature (BOYS_PANELS panels of BOYS_GL nodes); the
// integrand is smooth on [0, 1], so the rule converges to FP64 precision.
// ---------------------------------------------------------------------------
constexpr int BOYS_GL = 24;
constexpr int BOYS_PANELS = 16;

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(PCM_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
        }
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

__global__ void boys_table_kernel(const double *__restrict__ gx, const double *__restrict__ gw, double *tab64,
                                  float *tab32)
{
    const int row = blockIdx.x;
    const int m = threadIdx.x;  // 0 .. BOYS_MCOL-1 (launched with exactly BOYS_MCOL threads)
    const double T = row * BOYS_DT;
    double s = 0.0;
    const double h = 1.0 / BOYS_PANELS;
    for (int pnl = 0; pnl < BOYS_PANELS; ++pnl) {
        const double a = pnl * h;
        double ps = 0.0;
        for (int k = 0; k < BOYS_GL; ++k) {
            const double u = a + 0.5 * h * (gx[k] + 1.0);
            double u2m = 1.0;
            const double u2 = u * u;
            for (int j = 0; j < m; ++j) u2m *= u2;
            ps += gw[k] * u2m * exp(-T * u2);
        }
        s += 0.5 * h * ps;
    }
    tab64[(size_t)row * BOYS_STRIDE64 + m] = s;
    if (m < BOYS_LO32) tab32[(size_t)row * BOYS_STRIDE32 + m] = (float)s;
    if (m < BOYS_STRIDE32 - BOYS_LO32) tab32[(size_t)row * BOYS_STRIDE32 + BOYS_LO32 + m] = (float)(s - (double)(float)s);
    // Horner block for m <= 1 (layout in boys.cuh)
    __shared__ double F[BOYS_MCOL];
    F[m] = s;
    __syncthreads();
    if (m < BOYS_STRIDE32) {
        constexpr double inv_fact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};
        // slot -> (m, k) or the lo part of m
        static constexpr int SM[16] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1};
        static constexpr int SK[16] = {0, 1, 2, 3, 4, -1, 0, 1, 2, 3, 4, -1, 0, 0, 0, 0};
        const int mm = SM[m], k = SK[m];
        float v = 0.f;
        if (mm >= 0 && k >= 0) v = (float)(((k & 1) ? -1.0 : 1.0) * F[mm + k] * inv_fact[k]);
        else if (mm >= 0) v = (float)(F[mm] - (double)(float)F[mm]);
        tab32[BOYS_H32 + (size_t)row * BOYS_STRIDE32 + m] = v;
    }
}

int boys_build_tables(pcm_ctx *c)
{
    std::vector<double> x, w;
    gauss_legendre(BOYS_GL, x, w);
    DBuf<double> gx, gw;
    PCM_TRY(gx.alloc(BOYS_GL));
    PCM_TRY(gw.alloc(BOYS_GL));
    PCM_CUDA(cudaMemcpyAsync(gx.p, x.data(), BOYS_GL * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(gw.p, w.data(), BOYS_GL * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PCM_TRY(c->boys64.alloc((size_t)BOYS_NROW * BOYS_STRIDE64));
    PCM_TRY(c->boys32.alloc((size_t)BOYS_ALLOC32));
    PCM_CUDA(cudaMemsetAsync(c->boys64.p, 0, (size_t)BOYS_NROW * BOYS_STRIDE64 * sizeof(double), c->stream));
    boys_table_kernel<<<BOYS_NROW, BOYS_MCOL, 0, c->stream>>>(gx.p, gw.p, c->boys64.p, c->boys32.p);
    PCM_LAUNCHED(c);
    PCM_CUDA(cudaStreamSynchronize(c->stream));  // gx, gw are freed on return
    return PCM_OK;
}

// ---------------------------------------------------------------------------
// Stable compaction of byte flags (three passes: block counts, one-block
// scan of the counts, scatter).  Each thread owns CITEMS consecutive flags.
// ---------------------------------------------------------------------------
constexpr int CT = 256;
constexpr int CITEMS = 8;
constexpr int CCHUNK = CT * CITEMS;

__device__ __forceinline__ int block_exclusive_scan(int v, int *sh /* CT/32 + 1 */, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < CT / 32; ++i) {
            int t = sh[i];
            sh[i] = run;
            run += t;
        }
        sh[CT / 32] = run;
    }
    __syncthreads();
    int r = sh[wid] + x - v;
    *total = sh[CT / 32];
    __syncthreads();
    return r;
}

__global__ void compact_count(const unsigned char *__restrict__ f, long long n, int *__restrict__ bcount)
{
    __shared__ int sh[CT / 32 + 1];
    const long long base = (long long)blockIdx.x * CCHUNK + (long long)threadIdx.x * CITEMS;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < CITEMS; ++k)
        if (base + k < n && f[base + k]) ++cnt;
    int tot;
    block_exclusive_scan(cnt, sh, &tot);
    if (threadIdx.x == 0) bcount[blockIdx.x] = tot;
}

__global__ void compact_scan(int *bcount, int nb, int *count_dev)
{
    // one block: exclusive scan of nb block counts in place
    __shared__ int sh[CT / 32 + 1];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += CT) {
        int i = b0 + threadIdx.x;
        int v = i < nb ? bcount[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) bcount[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *count_dev = carry;
}

__global__ void compact_scatter(const unsigned char *__restrict__ f, long long n, const int *__restrict__ boff,
                                int *__restrict__ out, int *__restrict__ pos, const int *__restrict__ count_dev)
{
    __shared__ int sh[CT / 32 + 1];
    const long long base = (long long)blockIdx.x * CCHUNK + (long long)threadIdx.x * CITEMS;
    unsigned char loc[CITEMS];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < CITEMS; ++k) {
        loc[k] = (base + k < n) ? f[base + k] : 0;
        cnt += loc[k] ? 1 : 0;
    }
    int tot;
    int run = boff[blockIdx.x] + block_exclusive_scan(cnt, sh, &tot);
#pragma unroll
    for (int k = 0; k < CITEMS; ++k) {
        if (base + k < n) {
            if (pos) pos[base + k] = run;
            if (loc[k]) {
                if (out) out[run] = (int)(base + k);
                ++run;
            }
        }
    }
    if (pos && blockIdx.x == 0 && threadIdx.x == 0) pos[n] = *count_dev;
}

int compact_flags(pcm_ctx *c, const unsigned char *flags, long long n, int *out, int *pos, int *count_dev)
{
    long long nb = (n + CCHUNK - 1) / CCHUNK;
    if (nb < 1) nb = 1;
    PCM_TRY(c->scan32.alloc((size_t)nb + 1));
    compact_count<<<(unsigned)nb, CT, 0, c->stream>>>(flags, n, c->scan32.p);
    PCM_LAUNCHED(c);
    compact_scan<<<1, CT, 0, c->stream>>>(c->scan32.p, (int)nb, count_dev);
    PCM_LAUNCHED(c);
    compact_scatter<<<(unsigned)nb, CT, 0, c->stream>>>(flags, n, c->scan32.p, out, pos, count_dev);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

}  // namespace pcm

namespace pcm {

int device_error_flag(pcm_ctx *c)
{
    if (c->dev_err.p) return PCM_OK;
    PCM_TRY(c->dev_err.alloc(1));
    PCM_CUDA(cudaMemsetAsync(c->dev_err.p, 0, sizeof(int), c->stream));
    return PCM_OK;
}

// Read the device error flag after the stream has been synchronised: a kernel
// whose bounded wait gave up set it (and returned without its results).
int check_device_error(pcm_ctx *c, const char *where)
{
    if (!c->dev_err.p) return PCM_OK;
    int h = 0;
    PCM_CUDA(cudaMemcpy(&h, c->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        PCM_CUDA(cudaMemset(c->dev_err.p, 0, sizeof(int)));
        set_last_error("%s: a bounded device wait gave up (a bulk copy into shared memory did not complete)", where);
        return PCM_ERR_TIMEOUT;
    }
    return PCM_OK;
}

}  // namespace pcm
