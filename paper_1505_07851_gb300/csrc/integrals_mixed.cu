// PCM_MIXED integral kernels: the same McMurchie-Davidson contractions as
// integrals.cu, evaluated on the FP32 pipes (62x the FP64 rate on GB300) with
// FP64 accumulation across tiles.
//
// Error control.  FP32 rounding that is the same for every surface point
// (a per-pair constant) would bias c_k for all k alike and add up in the
// energy (dE = q^T dc); rounding that varies from point to point averages
// out, and so does a per-pair rounding whose sign varies from pair to pair.
// So the per-pair or per-(pair, class) constants that repeat over many pairs
// or dominate the sums are carried as FP32 hi + lo pairs computed in FP64:
// rho (T = rho_hi R^2 + rho_lo R^2, and (-2 rho)^n corrected to first order
// in rho_lo / rho_hi; rho depends only on p and the point class, so it
// repeats over every pair of the same exponents), the Hermite density
// U D_tuv (all components in the scalar and same-atom kernels, U D_000 in the
// packed cross-atom kernel), and sqrt(pi)/2 in the far-field Boys branch.
// Coordinates are split as hi (on a 2^-10 grid, so hi differences are exact)
// + lo, so every distance is the FP32 rounding of the exact one.  ESP sums
// are Kahan-compensated per interaction in FP32 over a pair segment and
// added in FP64; Fock sums run in FP32 within a tile of 128 points (64 per
// lane when packed) and in FP64 across tiles.
#include <math.h>

#include <algorithm>
#include <vector>

#include "boys.cuh"
#include "common.cuh"
#include "context.h"
#include "f2.cuh"
#include "tune.h"

namespace pcm {

__device__ __forceinline__ void split_val(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ void split_coord(double v, float &hi, float &lo)
{
    const double h = rint(v * 1024.0) * (1.0 / 1024.0);
    hi = (float)h;
    lo = (float)(v - h);
}

// point coordinates -> FP32 hi/lo [3][M] each
__global__ void point_split_kernel(int M, const double *__restrict__ px, const double *__restrict__ py,
                                   const double *__restrict__ pz, float *__restrict__ hi, float *__restrict__ lo)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    split_coord(px[k], hi[k], lo[k]);
    split_coord(py[k], hi[(size_t)M + k], lo[(size_t)M + k]);
    split_coord(pz[k], hi[2 * (size_t)M + k], lo[2 * (size_t)M + k]);
}

int points_split(pcm_ctx *c)
{
    PCM_TRY(c->p32.alloc(3 * (size_t)c->M));
    PCM_TRY(c->p32lo.alloc(3 * (size_t)c->M));
    point_split_kernel<<<(c->M + 127) / 128, 128, 0, c->stream>>>(c->M, c->px.p, c->py.p, c->pz.p, c->p32.p,
                                                                  c->p32lo.p);
    PCM_LAUNCHED(c);
    return fock_point_tiles_map(c);
}

// ---------------------------------------------------------------------------
// ESP: per-(class e, pair j) constants
//   eX[0..2][j] = hi(P), eX[3..5][j] = lo(P)
//   eC[e][0][j] = rho_hi, [1] = rho_lo, [2] = rho_lo / rho_hi,
//   eC[e][3 + h][j] = hi(U D_h), eC[e][3 + NH + h][j] = lo(U D_h)
// ---------------------------------------------------------------------------
template <int L>
__global__ void esp_mixed_prep_kernel(int nesp, int jend, int ncls, const double *__restrict__ cls_zeta,
                                      const double *__restrict__ eP, const double *__restrict__ eD,
                                      float *__restrict__ eX, float *__restrict__ eC)
{
    constexpr int NH = nherm(L);
    constexpr int F = 3 + 2 * NH;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= jend) return;
    for (int d = 0; d < 3; ++d) split_coord(eP[(size_t)d * nesp + j], eX[(size_t)d * nesp + j], eX[(size_t)(3 + d) * nesp + j]);
    const double p = eP[3 * (size_t)nesp + j];
    for (int e = 0; e < ncls; ++e) {
        float *C = eC + (size_t)e * F * nesp;
        const double z2 = cls_zeta[e] * cls_zeta[e];
        const double inv = 1.0 / (p + z2);
        const double rho = p * z2 * inv;
        const double U = sqrt(z2 * inv);
        float rh, rl;
        split_val(rho, rh, rl);
        C[0 * (size_t)nesp + j] = rh;
        C[1 * (size_t)nesp + j] = rl;
        C[2 * (size_t)nesp + j] = (float)((rho - (double)rh) / (double)rh);
        for (int h = 0; h < NH; ++h) {
            float dh, dl;
            split_val(U * eD[(size_t)h * nesp + j], dh, dl);
            C[(size_t)(3 + h) * nesp + j] = dh;
            C[(size_t)(3 + NH + h) * nesp + j] = dl;
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float helpers (a value carried as hi + lo FP32 parts) for the pairs
// whose two primitives sit on one atom: their contributions are the largest
// terms of every c_k, and their FP32 rounding sets the error of the energy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

// F_0 (hi, lo) and F_1..F_MM (FP32) at T = Th + Tl
template <int MM>
__device__ __forceinline__ void boys_df(float Th, float Tl, const float *__restrict__ tab, float &F0h, float &F0l,
                                        float (&F)[MM + 1])
{
    if (Th < (float)BOYS_TMAX) {
        const float t = fmaf(Th, (float)BOYS_INV_DT, 12582912.0f);
        const int i = __float_as_int(t) - 0x4B400000;
        const float d = fmaf(t - 12582912.0f, -(float)BOYS_DT, Th) + Tl;
        const float *row = tab + i * BOYS_STRIDE32;
        float r[MM + 5], lo[MM + 1];
#pragma unroll
        for (int k = 0; k < MM + 5; ++k) r[k] = __ldg(row + k);
#pragma unroll
        for (int k = 0; k <= MM; ++k) lo[k] = __ldg(row + BOYS_LO32 + k);
        const float e1 = -d, e2 = -d * 0.5f, e3 = -d * (1.0f / 3.0f), e4 = -d * 0.25f;
#pragma unroll
        for (int m = 0; m <= MM; ++m) {
            float s = fmaf(r[m + 4], e4, r[m + 3]);
            s = fmaf(s, e3, r[m + 2]);
            s = fmaf(s, e2, r[m + 1]);
            const float corr = fmaf(s, e1, lo[m]);
            if (m == 0) {
                F0h = r[0];
                F0l = corr;
            }
            F[m] = corr + r[m];
        }
    } else {
        constexpr float C_HI = 0.88622692545275801365f;
        constexpr float C_LO = (float)(0.88622692545275801365 - (double)C_HI);
        const float r0 = rsqrtf(Th);
        // 1/sqrt(T) = r0 (1 + e/2) with e = 1 - T r0^2 formed to ~2^-48
        const float hh = Th * r0;
        const float hl = fmaf(Th, r0, -hh);
        const float e = (fmaf(-hh, r0, 1.0f) - hl * r0) - Tl * r0 * r0;
        const float rsl = 0.5f * r0 * e;
        F0h = C_HI * r0;
        F0l = (fmaf(C_HI, r0, -F0h) + C_HI * rsl) + C_LO * r0;
        const float rs = r0 + rsl;
        const float half_inv_T = 0.5f * rs * rs;
        F[0] = F0h + F0l;
#pragma unroll
        for (int m = 1; m <= MM; ++m) F[m] = F[m - 1] * (float)(2 * m - 1) * half_inv_T;
    }
}

constexpr int MESP_NT = 128;
constexpr int MESP_TP = 32;
// points per thread: the autotuner picks 4 or 2 per class.  Default: 2 for
// the packed kernels (at 4 the register count cuts the resident warps by a
// third, measured slower for every class), else 4 for the light classes
// (more independent work per pair) and 2 for the others.
constexpr int esp_default_ppt(int L, bool packed) { return packed ? 2 : (L <= 1 ? 4 : 2); }

// Per tile of TP pairs, shared memory holds per pair float4 (xh, yh, zh, rho_hi),
// float4 (xl, yl, zl, rho_lo), rho_lo/rho_hi and NH float2 (hi, lo) of U D_h.
template <int L, bool SC, int PPT>
__global__ void __launch_bounds__(MESP_NT) esp_kernel_f32(int nesp, int jbeg, int jend, int seglen,
                                                          const float *__restrict__ eX, const float *__restrict__ eC,
                                                          const int *__restrict__ blk_off,
                                                          const int *__restrict__ blk_cls, const float *__restrict__ ph,
                                                          const float *__restrict__ pl, const float *__restrict__ boys,
                                                          int M, double *__restrict__ part)
{
    constexpr int NH = nherm(L);
    constexpr int F = 3 + 2 * NH;
    __shared__ float4 sA[MESP_TP], sB[MESP_TP];
    __shared__ float sR[MESP_TP];
    __shared__ float2 sD[NH][MESP_TP];
    const int k0 = blk_off[blockIdx.x], k1 = blk_off[blockIdx.x + 1];
    const float *C = eC + (size_t)blk_cls[blockIdx.x] * F * nesp;
    const int j0 = jbeg + blockIdx.y * seglen;
    const int j1 = min(jend, j0 + seglen);

    float xh[PPT], yh[PPT], zh[PPT], xl[PPT], yl[PPT], zl[PPT];
    // Kahan-compensated FP32 sums over the whole segment, one compensated
    // addition per interaction: adding a small term to a larger running sum in
    // plain FP32 drops its bits below half an ulp, always towards a smaller
    // magnitude for same-sign terms (a bias, not noise).  Plain FP32 sums over
    // tiles of pairs, compensated only across tiles, measured a ten times larger
    // energy error on the 300-atom spd cluster.
    float a32[PPT], k32[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = min(k0 + (int)threadIdx.x + q * MESP_NT, k1 - 1);
        xh[q] = ph[k];
        yh[q] = ph[(size_t)M + k];
        zh[q] = ph[2 * (size_t)M + k];
        xl[q] = pl[k];
        yl[q] = pl[(size_t)M + k];
        zl[q] = pl[2 * (size_t)M + k];
        a32[q] = k32[q] = 0.f;
    }
    for (int jt = j0; jt < j1; jt += MESP_TP) {
        const int nt = min(MESP_TP, j1 - jt);
        __syncthreads();
        for (int jj = threadIdx.x; jj < MESP_TP; jj += MESP_NT) {
            const bool v = jj < nt;
            const size_t j = jt + jj;
            sA[jj] = v ? make_float4(eX[j], eX[(size_t)nesp + j], eX[2 * (size_t)nesp + j], C[j])
                       : make_float4(0.f, 0.f, 0.f, 1.f);
            sB[jj] = v ? make_float4(eX[3 * (size_t)nesp + j], eX[4 * (size_t)nesp + j], eX[5 * (size_t)nesp + j],
                                     C[(size_t)nesp + j])
                       : make_float4(0.f, 0.f, 0.f, 0.f);
            sR[jj] = v ? C[2 * (size_t)nesp + j] : 0.f;
        }
        for (int t = threadIdx.x; t < NH * MESP_TP; t += MESP_NT) {
            const int h = t / MESP_TP, jj = t % MESP_TP;
            sD[h][jj] = jj < nt ? make_float2(C[(size_t)(3 + h) * nesp + jt + jj], C[(size_t)(3 + NH + h) * nesp + jt + jj])
                                : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int jj = 0; jj < nt; ++jj) {
            const float4 A = sA[jj], B = sB[jj];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if constexpr (SC) {
                    // double-float distance, T, F_0 and D_000 F_0; the Hermite
                    // terms beyond the charge stay FP32 (they are smaller)
                    float X, Xl, Y, Yl, Z, Zl;
                    two_sum(A.x - xh[q], B.x - xl[q], X, Xl);
                    two_sum(A.y - yh[q], B.y - yl[q], Y, Yl);
                    two_sum(A.z - zh[q], B.z - zl[q], Z, Zl);
                    const float p1 = X * X, p2 = Y * Y, p3 = Z * Z;
                    const float e1 = fmaf(X, X, -p1), e2 = fmaf(Y, Y, -p2), e3 = fmaf(Z, Z, -p3);
                    float s1, t1, s2, t2;
                    two_sum(p1, p2, s1, t1);
                    two_sum(s1, p3, s2, t2);
                    const float lo = ((e1 + e2) + e3) + (t1 + t2) + 2.f * (X * Xl + Y * Yl + Z * Zl);
                    float R2h, R2l;
                    fast_two_sum(s2, lo, R2h, R2l);
                    const float Th = A.w * R2h;
                    const float Tl = fmaf(A.w, R2h, -Th) + (A.w * R2l + B.w * R2h);
                    float F0h, F0l, Fb[L + 1];
                    boys_df<L>(Th, Tl, boys, F0h, F0l, Fb);
                    const float2 D0 = sD[0][jj];
                    const float ph0 = D0.x * F0h;
                    const float pl0 = (fmaf(D0.x, F0h, -ph0) + D0.x * F0l) + D0.y * F0h;
                    float rest = 0.f;
                    if constexpr (L > 0) {
                        const float dr = sR[jj];
                        const float m2r = -2.f * A.w;
                        float Rn[L + 1];
                        float f = 1.f;
#pragma unroll
                        for (int n = 0; n <= L; ++n) {
                            const float v = f * Fb[n];
                            Rn[n] = (n == 0) ? v : fmaf(v, (float)n * dr, v);
                            f *= m2r;
                        }
                        float R[NH];
                        hermite_R<L, float>(X, Y, Z, Rn, R);
#pragma unroll
                        for (int h = 1; h < NH; ++h) {
                            const float2 D = sD[h][jj];
                            rest = fmaf(D.x, R[h], fmaf(D.y, R[h], rest));
                        }
                    }
                    const float y = (ph0 - k32[q]) + (pl0 + rest);
                    const float t = a32[q] + y;
                    k32[q] = (t - a32[q]) - y;
                    a32[q] = t;
                    continue;
                }
                const float X = (A.x - xh[q]) + (B.x - xl[q]);
                const float Y = (A.y - yh[q]) + (B.y - yl[q]);
                const float Z = (A.z - zh[q]) + (B.z - zl[q]);
                const float R2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
                const float T = fmaf(A.w, R2, B.w * R2);
                float Fb[L + 1];
                boys_eval<L>(T, boys, Fb);
                float dot;
                if constexpr (L == 0) {
                    const float2 D = sD[0][jj];
                    dot = fmaf(D.x, Fb[0], D.y * Fb[0]);
                } else {
                    const float dr = sR[jj];
                    const float m2r = -2.f * A.w;
                    float Rn[L + 1];
                    float f = 1.f;
#pragma unroll
                    for (int n = 0; n <= L; ++n) {
                        const float v = f * Fb[n];
                        Rn[n] = (n == 0) ? v : fmaf(v, (float)n * dr, v);
                        f *= m2r;
                    }
                    float R[NH];
                    hermite_R<L, float>(X, Y, Z, Rn, R);
                    dot = 0.f;
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        const float2 D = sD[h][jj];
                        dot = fmaf(D.x, R[h], fmaf(D.y, R[h], dot));
                    }
                }
                const float y = dot - k32[q];
                const float t = a32[q] + y;
                k32[q] = (t - a32[q]) - y;
                a32[q] = t;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = k0 + threadIdx.x + q * MESP_NT;
        if (k < k1) part[(size_t)blockIdx.y * M + k] = (double)a32[q] - (double)k32[q];
    }
}

// ---------------------------------------------------------------------------
// Fock: NPT primitive pairs per thread (the point data staged in shared memory
// serve them all); per class rho and U in FP64 (hi/lo for rho), per point tile
// FP32 sums of q_k R_tuv, folded into FP64 with U.  The next tile's points are
// read into registers while the current one is computed.
// ---------------------------------------------------------------------------
constexpr int MF_NT = 128;
constexpr int MF_TQ = 128;
constexpr int fock_default_npt(int L) { return L <= 1 ? 2 : 1; }

// pairs per thread of the FP32 Fock kernel for class L: the autotuner's
// choice when it has one for this context's GPU, else the default
int fock_mixed_pairs_per_thread(pcm_ctx *c, int L, long long npair)
{
    const int t = c->opt.autotune ? tune_get(c->device, c->opt.fp32x2 ? TUNE_FOCK_NPT : TUNE_FOCK_NPT_SCALAR, L, tune_bucket(npair)) : -1;
    return t > 0 ? t : fock_default_npt(L);
}

template <int L, int NPT>
__global__ void __launch_bounds__(MF_NT) fock_kernel_f32(int npair, const double *__restrict__ gp,
                                                         const float *__restrict__ Phl, int ksplit,
                                                         const float *__restrict__ ph, const float *__restrict__ pl,
                                                         const double *__restrict__ q, int M, int ncls,
                                                         const int *__restrict__ cls_off,
                                                         const double *__restrict__ cls_zeta,
                                                         const float *__restrict__ boys, double *__restrict__ W)
{
    constexpr int NH = nherm(L);
    __shared__ float4 sH[MF_TQ], sL[MF_TQ];  // (xh, yh, zh, q) and (xl, yl, zl, 0) per point
    int r[NPT];
    bool active[NPT];
    float Pxh[NPT], Pyh[NPT], Pzh[NPT], Pxl[NPT], Pyl[NPT], Pzl[NPT];
    double p[NPT];
    double w64[NPT][NH];
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
        r[i] = (blockIdx.x * NPT + i) * MF_NT + threadIdx.x;
        active[i] = r[i] < npair;
        const int rr = active[i] ? r[i] : 0;
        Pxh[i] = Phl[rr];
        Pyh[i] = Phl[(size_t)npair + rr];
        Pzh[i] = Phl[2 * (size_t)npair + rr];
        Pxl[i] = Phl[3 * (size_t)npair + rr];
        Pyl[i] = Phl[4 * (size_t)npair + rr];
        Pzl[i] = Phl[5 * (size_t)npair + rr];
        p[i] = gp[rr];
#pragma unroll
        for (int h = 0; h < NH; ++h) w64[i][h] = 0.0;
    }
    const int ka = blockIdx.y * ksplit;
    const int kb = min(M, ka + ksplit);
    for (int ec = 0; ec < ncls; ++ec) {
        const int a = max(ka, cls_off[ec]), b = min(kb, cls_off[ec + 1]);
        if (a >= b) continue;
        const double z2 = cls_zeta[ec] * cls_zeta[ec];
        double U[NPT];
        float rh[NPT], rl[NPT], dr[NPT], m2r[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            const double inv = 1.0 / (p[i] + z2);
            const double rho = p[i] * z2 * inv;
            U[i] = sqrt(z2 * inv);
            rh[i] = (float)rho;
            rl[i] = (float)(rho - (double)rh[i]);
            dr[i] = (float)((rho - (double)rh[i]) / (double)rh[i]);
            m2r[i] = -2.f * rh[i];
        }
        // this thread's point of the first tile
        float4 nH = make_float4(0.f, 0.f, 0.f, 0.f), nL = nH;
        if (a + (int)threadIdx.x < b) {
            const int k = a + threadIdx.x;
            nH = make_float4(ph[k], ph[(size_t)M + k], ph[2 * (size_t)M + k], (float)q[k]);
            nL = make_float4(pl[k], pl[(size_t)M + k], pl[2 * (size_t)M + k], 0.f);
        }
        for (int t0 = a; t0 < b; t0 += MF_TQ) {
            const int nt = min(MF_TQ, b - t0);
            __syncthreads();
            sH[threadIdx.x] = nH;
            sL[threadIdx.x] = nL;
            __syncthreads();
            // prefetch the next tile while this one is computed
            if (t0 + MF_TQ + (int)threadIdx.x < b) {
                const int k = t0 + MF_TQ + threadIdx.x;
                nH = make_float4(ph[k], ph[(size_t)M + k], ph[2 * (size_t)M + k], (float)q[k]);
                nL = make_float4(pl[k], pl[(size_t)M + k], pl[2 * (size_t)M + k], 0.f);
            }
            float w32[NPT][NH];
#pragma unroll
            for (int i = 0; i < NPT; ++i)
#pragma unroll
                for (int h = 0; h < NH; ++h) w32[i][h] = 0.f;
            for (int kk = 0; kk < nt; ++kk) {
                const float4 H = sH[kk], Lo = sL[kk];
#pragma unroll
                for (int i = 0; i < NPT; ++i) {
                    const float X = (Pxh[i] - H.x) + (Pxl[i] - Lo.x);
                    const float Y = (Pyh[i] - H.y) + (Pyl[i] - Lo.y);
                    const float Z = (Pzh[i] - H.z) + (Pzl[i] - Lo.z);
                    const float R2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
                    const float T = fmaf(rh[i], R2, rl[i] * R2);
                    float Fb[L + 1];
                    boys_eval<L>(T, boys, Fb);
                    if constexpr (L == 0) {
                        w32[i][0] = fmaf(H.w, Fb[0], w32[i][0]);
                    } else {
                        float Rn[L + 1];
                        float f = H.w;
#pragma unroll
                        for (int n = 0; n <= L; ++n) {
                            const float v = f * Fb[n];
                            Rn[n] = (n == 0) ? v : fmaf(v, (float)n * dr[i], v);
                            f *= m2r[i];
                        }
                        float R[NH];
                        hermite_R<L, float>(X, Y, Z, Rn, R);
#pragma unroll
                        for (int h = 0; h < NH; ++h) w32[i][h] += R[h];
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NPT; ++i)
#pragma unroll
                for (int h = 0; h < NH; ++h) w64[i][h] = fma(U[i], (double)w32[i][h], w64[i][h]);
        }
    }
#pragma unroll
    for (int i = 0; i < NPT; ++i)
        if (active[i]) {
#pragma unroll
            for (int h = 0; h < NH; ++h) W[((size_t)blockIdx.y * NH + h) * npair + r[i]] = w64[i][h];
        }
}

// ---------------------------------------------------------------------------
// Point part of the integral gradient on the FP32 pipes (the FP64 statement
// is esp_grad_kernel in integrals.cu): per point the three sums
//   sum_pairs U sum_tuv eD_tuv R_{tuv + 1_d},  R up to L+1,
// from the ESP pairs' split constants (eX, eC as prepared for the ESP), with
// Kahan-compensated FP32 sums per segment.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(MESP_NT) esp_grad_kernel_f32(int nesp, int seglen, const float *__restrict__ eX,
                                                               const float *__restrict__ eC,
                                                               const int *__restrict__ blk_off,
                                                               const int *__restrict__ blk_cls,
                                                               const float *__restrict__ ph,
                                                               const float *__restrict__ pl,
                                                               const float *__restrict__ boys, int M,
                                                               double *__restrict__ part)
{
    constexpr int NH = nherm(L);
    constexpr int L1 = L + 1;
    constexpr int NH1 = nherm(L1);
    constexpr int F = 3 + 2 * NH;
    constexpr int PPT = esp_default_ppt(L, false);
    __shared__ float4 sA[MESP_TP], sB[MESP_TP];
    __shared__ float sR[MESP_TP];
    __shared__ float2 sD[NH][MESP_TP];
    const int k0 = blk_off[blockIdx.x], k1 = blk_off[blockIdx.x + 1];
    const float *C = eC + (size_t)blk_cls[blockIdx.x] * F * nesp;
    const int j0 = blockIdx.y * seglen;
    const int j1 = min(nesp, j0 + seglen);

    float xh[PPT], yh[PPT], zh[PPT], xl[PPT], yl[PPT], zl[PPT];
    float a32[3][PPT], k32[3][PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = min(k0 + (int)threadIdx.x + q * MESP_NT, k1 - 1);
        xh[q] = ph[k];
        yh[q] = ph[(size_t)M + k];
        zh[q] = ph[2 * (size_t)M + k];
        xl[q] = pl[k];
        yl[q] = pl[(size_t)M + k];
        zl[q] = pl[2 * (size_t)M + k];
#pragma unroll
        for (int d = 0; d < 3; ++d) a32[d][q] = k32[d][q] = 0.f;
    }
    for (int jt = j0; jt < j1; jt += MESP_TP) {
        const int nt = min(MESP_TP, j1 - jt);
        __syncthreads();
        for (int jj = threadIdx.x; jj < MESP_TP; jj += MESP_NT) {
            const bool v = jj < nt;
            const size_t j = jt + jj;
            sA[jj] = v ? make_float4(eX[j], eX[(size_t)nesp + j], eX[2 * (size_t)nesp + j], C[j])
                       : make_float4(0.f, 0.f, 0.f, 1.f);
            sB[jj] = v ? make_float4(eX[3 * (size_t)nesp + j], eX[4 * (size_t)nesp + j], eX[5 * (size_t)nesp + j],
                                     C[(size_t)nesp + j])
                       : make_float4(0.f, 0.f, 0.f, 0.f);
            sR[jj] = v ? C[2 * (size_t)nesp + j] : 0.f;
        }
        for (int t = threadIdx.x; t < NH * MESP_TP; t += MESP_NT) {
            const int h = t / MESP_TP, jj = t % MESP_TP;
            sD[h][jj] = jj < nt ? make_float2(C[(size_t)(3 + h) * nesp + jt + jj], C[(size_t)(3 + NH + h) * nesp + jt + jj])
                                : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int jj = 0; jj < nt; ++jj) {
            const float4 A = sA[jj], B = sB[jj];
            const float dr = sR[jj];
            const float m2r = -2.f * A.w;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const float X = (A.x - xh[q]) + (B.x - xl[q]);
                const float Y = (A.y - yh[q]) + (B.y - yl[q]);
                const float Z = (A.z - zh[q]) + (B.z - zl[q]);
                const float R2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
                const float T = fmaf(A.w, R2, B.w * R2);
                float Fb[L1 + 1];
                boys_eval<L1>(T, boys, Fb);
                float Rn[L1 + 1];
                float f = 1.f;
#pragma unroll
                for (int n = 0; n <= L1; ++n) {
                    const float v = f * Fb[n];
                    Rn[n] = (n == 0) ? v : fmaf(v, (float)n * dr, v);
                    f *= m2r;
                }
                float R[NH1];
                hermite_R<L1, float>(X, Y, Z, Rn, R);
                float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int v = 0; v <= L - t - u; ++v) {
                            const float2 D = sD[hidx(t, u, v)][jj];
                            const float Dt = D.x + D.y;
                            s[0] = fmaf(Dt, R[hidx(t + 1, u, v)], s[0]);
                            s[1] = fmaf(Dt, R[hidx(t, u + 1, v)], s[1]);
                            s[2] = fmaf(Dt, R[hidx(t, u, v + 1)], s[2]);
                        }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float y = s[d] - k32[d][q];
                    const float t = a32[d][q] + y;
                    k32[d][q] = (t - a32[d][q]) - y;
                    a32[d][q] = t;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = k0 + threadIdx.x + q * MESP_NT;
        if (k < k1)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                part[((size_t)blockIdx.y * 3 + d) * M + k] = (double)a32[d][q] - (double)k32[d][q];
    }
}


// The point part with two pairs per packed instruction (lanes as in
// esp_kernel_f32x2, 2 points per thread); each lane's arithmetic is that of
// esp_grad_kernel_f32: hi + lo distances, rho hi + lo, and U D_tuv as the
// FP32 sum of its hi and lo parts.  Shared memory per pair of pairs,
// lane-interleaved: float4 (xh, yh), (zh, rho_hi), (xl, yl); float2 zl, rho_lo,
// rho_lo / rho_hi and NH float2 U D_tuv.
template <int L>
__global__ void __launch_bounds__(MESP_NT) esp_grad_kernel_f32x2(int nesp, int seglen, const float *__restrict__ eX,
                                                                 const float *__restrict__ eC,
                                                                 const int *__restrict__ blk_off,
                                                                 const int *__restrict__ blk_cls,
                                                                 const float *__restrict__ ph,
                                                                 const float *__restrict__ pl,
                                                                 const float *__restrict__ boys, int M,
                                                                 double *__restrict__ part)
{
    constexpr int NH = nherm(L);
    constexpr int L1 = L + 1;
    constexpr int NH1 = nherm(L1);
    constexpr int F = 3 + 2 * NH;
    constexpr int PPT = 2;
    constexpr int TP2 = MESP_TP / 2;
    __shared__ float4 sXY[TP2], sZR[TP2], sXYl[TP2];
    __shared__ float2 sZl[TP2], sRl[TP2], sDr[TP2], sD[NH][TP2];
    const int k0 = blk_off[blockIdx.x], k1 = blk_off[blockIdx.x + 1];
    const float *C = eC + (size_t)blk_cls[blockIdx.x] * F * nesp;
    const int j0 = blockIdx.y * seglen;
    const int j1 = min(nesp, j0 + seglen);

    f2 nxh[PPT], nyh[PPT], nzh[PPT], nxl[PPT], nyl[PPT], nzl[PPT];
    f2 a32[3][PPT], k32[3][PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = min(k0 + (int)threadIdx.x + q * MESP_NT, k1 - 1);
        nxh[q] = f2(-ph[k]);
        nyh[q] = f2(-ph[(size_t)M + k]);
        nzh[q] = f2(-ph[2 * (size_t)M + k]);
        nxl[q] = f2(-pl[k]);
        nyl[q] = f2(-pl[(size_t)M + k]);
        nzl[q] = f2(-pl[2 * (size_t)M + k]);
#pragma unroll
        for (int d = 0; d < 3; ++d) a32[d][q] = k32[d][q] = f2(0.f);
    }
    for (int jt = j0; jt < j1; jt += MESP_TP) {
        const int nt = min(MESP_TP, j1 - jt);
        __syncthreads();
        for (int jj = threadIdx.x; jj < MESP_TP; jj += MESP_NT) {
            const bool v = jj < nt;
            const size_t j = jt + jj;
            const int s = jj >> 1, l = jj & 1;
            float *xy = reinterpret_cast<float *>(&sXY[s]), *zr = reinterpret_cast<float *>(&sZR[s]);
            float *xyl = reinterpret_cast<float *>(&sXYl[s]);
            xy[l] = v ? eX[j] : 0.f;
            xy[2 + l] = v ? eX[(size_t)nesp + j] : 0.f;
            zr[l] = v ? eX[2 * (size_t)nesp + j] : 0.f;
            zr[2 + l] = v ? C[j] : 1.f;
            xyl[l] = v ? eX[3 * (size_t)nesp + j] : 0.f;
            xyl[2 + l] = v ? eX[4 * (size_t)nesp + j] : 0.f;
            reinterpret_cast<float *>(&sZl[s])[l] = v ? eX[5 * (size_t)nesp + j] : 0.f;
            reinterpret_cast<float *>(&sRl[s])[l] = v ? C[(size_t)nesp + j] : 0.f;
            reinterpret_cast<float *>(&sDr[s])[l] = v ? C[2 * (size_t)nesp + j] : 0.f;
        }
        for (int t = threadIdx.x; t < NH * MESP_TP; t += MESP_NT) {
            const int h = t / MESP_TP, jj = t % MESP_TP;
            reinterpret_cast<float *>(&sD[h][jj >> 1])[jj & 1] =
                jj < nt ? C[(size_t)(3 + h) * nesp + jt + jj] + C[(size_t)(3 + NH + h) * nesp + jt + jj] : 0.f;
        }
        __syncthreads();
        const int np = (nt + 1) >> 1;
        for (int s = 0; s < np; ++s) {
            const float4 xy = sXY[s], zr = sZR[s], xyl = sXYl[s];
            const float2 zl = sZl[s], rlo = sRl[s], dr = sDr[s];
            const f2 Ax(xy.x, xy.y), Ay(xy.z, xy.w), Az(zr.x, zr.y), rh(zr.z, zr.w);
            const f2 Bx(xyl.x, xyl.y), By(xyl.z, xyl.w), Bz(zl.x, zl.y), rl(rlo.x, rlo.y);
            const f2 m2r = rh * f2(-2.f);
            f2 ndr[L1 + 1];
#pragma unroll
            for (int n = 1; n <= L1; ++n) ndr[n] = f2((float)n) * f2(dr.x, dr.y);
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const f2 X = (Ax + nxh[q]) + (Bx + nxl[q]);
                const f2 Y = (Ay + nyh[q]) + (By + nyl[q]);
                const f2 Z = (Az + nzh[q]) + (Bz + nzl[q]);
                const f2 R2 = fma2(X, X, fma2(Y, Y, Z * Z));
                const f2 T = fma2(rh, R2, rl * R2);
                f2 Fb[L1 + 1];
                boys_eval2<L1>(T, boys, Fb);
                f2 Rn[L1 + 1];
                Rn[0] = Fb[0];
                f2 f = m2r;
#pragma unroll
                for (int n = 1; n <= L1; ++n) {
                    const f2 v = f * Fb[n];
                    Rn[n] = fma2(v, ndr[n], v);
                    if (n < L1) f = f * m2r;
                }
                f2 R[NH1];
                hermite_R<L1, f2>(X, Y, Z, Rn, R);
                f2 sd[3] = {f2(0.f), f2(0.f), f2(0.f)};
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int v = 0; v <= L - t - u; ++v) {
                            const float2 Dv = sD[hidx(t, u, v)][s];
                            const f2 Dt(Dv.x, Dv.y);
                            sd[0] = fma2(Dt, R[hidx(t + 1, u, v)], sd[0]);
                            sd[1] = fma2(Dt, R[hidx(t, u + 1, v)], sd[1]);
                            sd[2] = fma2(Dt, R[hidx(t, u, v + 1)], sd[2]);
                        }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const f2 y = sd[d] - k32[d][q];
                    const f2 t = a32[d][q] + y;
                    k32[d][q] = (t - a32[d][q]) - y;
                    a32[d][q] = t;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = k0 + threadIdx.x + q * MESP_NT;
        if (k < k1)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                part[((size_t)blockIdx.y * 3 + d) * M + k] = ((double)a32[d][q].v.x - (double)k32[d][q].v.x) +
                                                             ((double)a32[d][q].v.y - (double)k32[d][q].v.y);
    }
}

// ---------------------------------------------------------------------------
// The "MS-driven" ESP of Section 4a (an autotuner candidate): one primitive
// pair per thread, looping over the surface points of its split in tiles
// staged in shared memory; for each point the block's pairs are summed (warp
// shuffles, then the four warps in fixed order, in FP64) into the block's
// partial c_k, part[blockIdx.x][k].  Same split constants as the pair-driven
// kernel; each interaction is a single FP32 term, so no running FP32 sum.
// ---------------------------------------------------------------------------
constexpr int MS_NT = 128;
constexpr int MS_TQ = 128;

template <int L>
__global__ void __launch_bounds__(MS_NT) esp_ms_kernel_f32(int nesp, int j0, int j1, int ksplit,
                                                           const float *__restrict__ eX, const float *__restrict__ eC,
                                                           int ncls, const int *__restrict__ cls_off,
                                                           const float *__restrict__ ph, const float *__restrict__ pl,
                                                           const float *__restrict__ boys, int M,
                                                           double *__restrict__ part)
{
    constexpr int NH = nherm(L);
    constexpr int F = 3 + 2 * NH;
    __shared__ float4 sH[MS_TQ], sL[MS_TQ];
    __shared__ float sw[MS_NT / 32][MS_TQ];
    const int j = j0 + blockIdx.x * MS_NT + threadIdx.x;
    const bool active = j < j1;
    const int jj = active ? j : j0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float xh = eX[jj], yh = eX[(size_t)nesp + jj], zh = eX[2 * (size_t)nesp + jj];
    const float xl = eX[3 * (size_t)nesp + jj], yl = eX[4 * (size_t)nesp + jj], zl = eX[5 * (size_t)nesp + jj];
    const int ka = blockIdx.y * ksplit;
    const int kb = min(M, ka + ksplit);
    double *out = part + (size_t)blockIdx.x * M;
    for (int e = 0; e < ncls; ++e) {
        const int a = max(ka, cls_off[e]), b = min(kb, cls_off[e + 1]);
        if (a >= b) continue;
        const float *C = eC + (size_t)e * F * nesp;
        const float rh = C[jj], rl = C[(size_t)nesp + jj], dr = C[2 * (size_t)nesp + jj];
        float2 D[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h)
            D[h] = active ? make_float2(C[(size_t)(3 + h) * nesp + jj], C[(size_t)(3 + NH + h) * nesp + jj])
                          : make_float2(0.f, 0.f);
        const float m2r = -2.f * rh;
        for (int t0 = a; t0 < b; t0 += MS_TQ) {
            const int nt = min(MS_TQ, b - t0);
            __syncthreads();
            if (threadIdx.x < nt) {
                const int k = t0 + threadIdx.x;
                sH[threadIdx.x] = make_float4(ph[k], ph[(size_t)M + k], ph[2 * (size_t)M + k], 0.f);
                sL[threadIdx.x] = make_float4(pl[k], pl[(size_t)M + k], pl[2 * (size_t)M + k], 0.f);
            }
            __syncthreads();
            for (int kk = 0; kk < nt; ++kk) {
                const float4 H = sH[kk], Lo = sL[kk];
                const float X = (xh - H.x) + (xl - Lo.x);
                const float Y = (yh - H.y) + (yl - Lo.y);
                const float Z = (zh - H.z) + (zl - Lo.z);
                const float R2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
                const float T = fmaf(rh, R2, rl * R2);
                float Fb[L + 1];
                boys_eval<L>(T, boys, Fb);
                float v;
                if constexpr (L == 0) {
                    v = fmaf(D[0].x, Fb[0], D[0].y * Fb[0]);
                } else {
                    float Rn[L + 1];
                    float f = 1.f;
#pragma unroll
                    for (int n = 0; n <= L; ++n) {
                        const float u = f * Fb[n];
                        Rn[n] = (n == 0) ? u : fmaf(u, (float)n * dr, u);
                        f *= m2r;
                    }
                    float R[NH];
                    hermite_R<L, float>(X, Y, Z, Rn, R);
                    v = 0.f;
#pragma unroll
                    for (int h = 0; h < NH; ++h) v = fmaf(D[h].x, R[h], fmaf(D[h].y, R[h], v));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) sw[wid][kk] = v;
            }
            __syncthreads();
            if (threadIdx.x < nt) {
                double s = 0.0;
#pragma unroll
                for (int w = 0; w < MS_NT / 32; ++w) s += (double)sw[w][threadIdx.x];
                out[t0 + threadIdx.x] = s;
            }
        }
    }
}

__global__ void esp_reduce_mixed_kernel(int M, int nseg, const double *__restrict__ part, double *__restrict__ c)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double s = 0.0;
    for (int g = 0; g < nseg; ++g) s += part[(size_t)g * M + k];
    c[k] = s;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static const int CLASS_L[6] = {0, 1, 2, 2, 3, 4};

// segments of [0, n) pairs for nblk point blocks: enough CTAs to fill the GPU
static void esp_plan(int n, int nblk, int *seglen, int *rows)
{
    if (n <= 0) {
        *seglen = 0;
        *rows = 0;
        return;
    }
    const int target = 152 * 8;
    const int maxseg = (n + MESP_TP - 1) / MESP_TP;
    const int ns = std::max(1, std::min(maxseg, (target + nblk - 1) / nblk));
    int sl = (n + ns - 1) / ns;
    sl = (sl + MESP_TP - 1) / MESP_TP * MESP_TP;
    *seglen = sl;
    *rows = (n + sl - 1) / sl;
}

template <int L, int PPT, bool PACKED>
static int esp_mixed_launch(pcm_ctx *c, PairClass &pc, int k, const int *blk, const int *bcls, int nblk, double *part)
{
    constexpr int NH = nherm(L);
    constexpr int F = 3 + 2 * NH;
    const int n = pc.nesp;
    // same-atom pairs [0, nesp_same) in double-float, the rest in FP32 (the
    // packed kernel prepares its own tiles for those)
    const int ns = pc.nesp_same, nx = n - ns;
    const int nprep = PACKED ? ns : n;
    PCM_TRY(pc.eX32.alloc(6 * (size_t)n));
    PCM_TRY(pc.eC32.alloc((size_t)c->ncls * F * n));
    if (nprep > 0) {
        esp_mixed_prep_kernel<L><<<(nprep + 127) / 128, 128, 0, c->stream>>>(n, nprep, c->ncls, c->cls_zeta.p,
                                                                             pc.eP.p, pc.eD.p, pc.eX32.p, pc.eC32.p);
        PCM_LAUNCHED(c);
    }
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[k], c->stream));
    int sl, rows;
    esp_plan(ns, nblk, &sl, &rows);
    if (rows > 0) {
        dim3 grid(nblk, rows);
        esp_kernel_f32<L, true, PPT><<<grid, MESP_NT, 0, c->stream>>>(n, 0, ns, sl, pc.eX32.p, pc.eC32.p, blk, bcls,
                                                                  c->p32.p, c->p32lo.p, c->boys32.p, c->M, part);
        PCM_LAUNCHED(c);
        part += (size_t)rows * c->M;
    }
    esp_plan(nx, nblk, &sl, &rows);
    if (rows > 0) {
        dim3 grid(nblk, rows);
        if constexpr (PACKED) {
            PCM_TRY(esp_packed(c, pc, L, PPT, ns, n, blk, bcls, nblk, part));
        } else {
            esp_kernel_f32<L, false, PPT><<<grid, MESP_NT, 0, c->stream>>>(n, ns, n, sl, pc.eX32.p, pc.eC32.p, blk,
                                                                            bcls, c->p32.p, c->p32lo.p, c->boys32.p,
                                                                            c->M, part);
            PCM_LAUNCHED(c);
        }
    }
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_b[k], c->stream));
    return PCM_OK;
}

// single-class point blocks of at most MESP_NT * PPT points (two layouts:
// PPT 4 and 2) in c->si[4..5] (offsets) and c->si[6..7] (classes); returns
// the number of blocks of each layout
static int mixed_point_blocks(pcm_ctx *c, int nblk[2])
{
    std::vector<int> off[2], bc[2];
    for (int v = 0; v < 2; ++v) {
        const int cap = MESP_NT * (v == 0 ? 4 : 2);
        off[v].push_back(0);
        for (int e = 0; e < c->ncls; ++e)
            for (int k = c->h_cls_off[e]; k < c->h_cls_off[e + 1]; k += cap) {
                off[v].push_back(std::min(c->h_cls_off[e + 1], k + cap));
                bc[v].push_back(e);
            }
    }
    DBuf<int> *blk = &c->si[4], *bcls = &c->si[6];
    for (int v = 0; v < 2; ++v) {
        // kept in the context: the copies below read them after this returns
        // (the next call that rewrites them comes after a synchronisation)
        c->h_pblk[v] = off[v];
        c->h_pbcls[v] = bc[v];
        PCM_TRY(blk[v].alloc(off[v].size()));
        PCM_TRY(bcls[v].alloc(bc[v].size()));
        PCM_CUDA(cudaMemcpyAsync(blk[v].p, c->h_pblk[v].data(), off[v].size() * sizeof(int), cudaMemcpyHostToDevice,
                                 c->stream));
        PCM_CUDA(cudaMemcpyAsync(bcls[v].p, c->h_pbcls[v].data(), bc[v].size() * sizeof(int),
                                 cudaMemcpyHostToDevice, c->stream));
        nblk[v] = (int)bc[v].size();
    }
    return PCM_OK;
}

// points of each split for the MS-driven kernel over n pairs: enough CTAs to
// fill the GPU, splits on whole point tiles
static void esp_ms_plan(pcm_ctx *c, int n, int *rows, int *nsplit, int *ksplit)
{
    *rows = (n + MS_NT - 1) / MS_NT;
    const int maxsplit = std::max(1, (c->M + MS_TQ - 1) / MS_TQ);
    int ns = *rows > 0 ? std::max(1, std::min(maxsplit, (152 * 8 + *rows - 1) / *rows)) : 1;
    int ks = (c->M + ns - 1) / ns;
    ks = (ks + MS_TQ - 1) / MS_TQ * MS_TQ;
    *ksplit = ks;
    *nsplit = (c->M + ks - 1) / ks;
}

// variant 2: the same-atom pairs as in the default layout, the others by the
// MS-driven kernel (L <= 2)
template <int L>
static int esp_ms_launch(pcm_ctx *c, PairClass &pc, int k, const int *blk, const int *bcls, int nblk, double *part)
{
    constexpr int NH = nherm(L);
    constexpr int F = 3 + 2 * NH;
    constexpr int PPT = esp_default_ppt(L, false);
    const int n = pc.nesp;
    PCM_TRY(pc.eX32.alloc(6 * (size_t)n));
    PCM_TRY(pc.eC32.alloc((size_t)c->ncls * F * n));
    esp_mixed_prep_kernel<L><<<(n + 127) / 128, 128, 0, c->stream>>>(n, n, c->ncls, c->cls_zeta.p, pc.eP.p, pc.eD.p,
                                                                     pc.eX32.p, pc.eC32.p);
    PCM_LAUNCHED(c);
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[k], c->stream));
    const int ns = pc.nesp_same;
    int sl, rows;
    esp_plan(ns, nblk, &sl, &rows);
    if (rows > 0) {
        dim3 grid(nblk, rows);
        esp_kernel_f32<L, true, PPT><<<grid, MESP_NT, 0, c->stream>>>(n, 0, ns, sl, pc.eX32.p, pc.eC32.p, blk,
                                                                       bcls, c->p32.p, c->p32lo.p, c->boys32.p, c->M,
                                                                       part);
        PCM_LAUNCHED(c);
        part += (size_t)rows * c->M;
    }
    int mrows, nsplit, ks;
    esp_ms_plan(c, n - ns, &mrows, &nsplit, &ks);
    if (mrows > 0) {
        dim3 grid(mrows, nsplit);
        esp_ms_kernel_f32<L><<<grid, MS_NT, 0, c->stream>>>(n, ns, n, ks, pc.eX32.p, pc.eC32.p, c->ncls,
                                                             c->cls_off.p, c->p32.p, c->p32lo.p, c->boys32.p, c->M,
                                                             part);
        PCM_LAUNCHED(c);
    }
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_b[k], c->stream));
    return PCM_OK;
}

// Variants of the FP32 ESP: pair-driven with 4 (v = 0) or 2 (v = 1) points per
// thread (two pairs per packed instruction unless the context asks for scalar
// FP32 instructions); MS-driven (v = 2).
static int esp_launch_variant(pcm_ctx *c, int k, int v, DBuf<int> *blk, DBuf<int> *bcls, const int nb[2], double *part)
{
    PairClass &pc = c->cls[k];
    if (v == 2) {
        const int d = esp_default_ppt(CLASS_L[k], false) == 4 ? 0 : 1;
        switch (CLASS_L[k]) {
        case 0: return esp_ms_launch<0>(c, pc, k, blk[d].p, bcls[d].p, nb[d], part);
        case 1: return esp_ms_launch<1>(c, pc, k, blk[d].p, bcls[d].p, nb[d], part);
        case 2: return esp_ms_launch<2>(c, pc, k, blk[d].p, bcls[d].p, nb[d], part);
        default: return PCM_ERR_ARG;
        }
    }
#define PCM_ESPV(LL)                                                                                         \
    case LL:                                                                                                 \
        if (c->opt.fp32x2)                                                                                   \
            return v == 0 ? esp_mixed_launch<LL, 4, true>(c, pc, k, blk[0].p, bcls[0].p, nb[0], part)        \
                          : esp_mixed_launch<LL, 2, true>(c, pc, k, blk[1].p, bcls[1].p, nb[1], part);       \
        return v == 0 ? esp_mixed_launch<LL, 4, false>(c, pc, k, blk[0].p, bcls[0].p, nb[0], part)           \
                      : esp_mixed_launch<LL, 2, false>(c, pc, k, blk[1].p, bcls[1].p, nb[1], part);
    switch (CLASS_L[k]) {
        PCM_ESPV(0)
        PCM_ESPV(1)
        PCM_ESPV(2)
        PCM_ESPV(3)
        PCM_ESPV(4)
    }
#undef PCM_ESPV
    return PCM_ERR_ARG;
}

static int esp_rows(pcm_ctx *c, int k, int nblk)
{
    int sl, r1, r2;
    esp_plan(c->cls[k].nesp_same, nblk, &sl, &r1);
    esp_plan(c->cls[k].nesp - c->cls[k].nesp_same, nblk, &sl, &r2);
    return r1 + r2;
}

// partial-sum rows of variant v of class k
static int esp_rows_v(pcm_ctx *c, int k, int v, const int nb[2])
{
    if (v < 2) return esp_rows(c, k, nb[v]);
    const int d = esp_default_ppt(CLASS_L[k], false) == 4 ? 0 : 1;
    int sl, r1, mrows, ns, ks;
    esp_plan(c->cls[k].nesp_same, nb[d], &sl, &r1);
    esp_ms_plan(c, c->cls[k].nesp - c->cls[k].nesp_same, &mrows, &ns, &ks);
    return r1 + mrows;
}

// The autotuner's trial for class k: every candidate run once untimed, then
// once timed with CUDA events on the context's stream; the fastest is
// remembered for this GPU, kernel family, angular momentum and size bucket.
static int esp_tune(pcm_ctx *c, int k, DBuf<int> *blk, DBuf<int> *bcls, const int nb[2], int *choice)
{
    // a batch member: its packed blocks join one launch with every other
    // molecule's, so only the packed layouts are candidates (their own record)
    const bool batching = c->jobs != nullptr && c->opt.fp32x2;
    struct NoDefer {
        pcm_ctx *c;
        JobSink *j;
        ~NoDefer() { c->jobs = j; }
    } nd{c, c->jobs};
    c->jobs = nullptr;   // the trials run now, whatever the caller collects
    const int L = CLASS_L[k];
    const int bucket = tune_bucket((long long)c->cls[k].nesp);
    const int kind = batching ? TUNE_ESP_PPT_BATCH : (c->opt.fp32x2 ? TUNE_ESP_PPT : TUNE_ESP_PPT_SCALAR);
    const int t = tune_get(c->device, kind, L, bucket);
    if (t >= 0) {
        *choice = t;
        return PCM_OK;
    }
    // candidates: pair-driven with 4 or 2 points per thread; MS-driven for L <= 2 (not in batches)
    const int nv = (L <= 2 && !batching) ? 3 : 2;
    int rmax = 1;
    for (int v = 0; v < nv; ++v) rmax = std::max(rmax, esp_rows_v(c, k, v, nb));
    PCM_TRY(c->esp_part.alloc((size_t)rmax * c->M));
    // one untimed pass first: the first launch of a variant also allocates
    // its tile buffers and loads its code, which is not what it costs per call
    for (int v = 0; v < nv; ++v) PCM_TRY(esp_launch_variant(c, k, v, blk, bcls, nb, c->esp_part.p));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    cudaEvent_t e[4];
    for (int i = 0; i <= nv; ++i) PCM_CUDA(cudaEventCreate(&e[i]));
    float ms[3] = {0.f, 0.f, 0.f};
    int st = PCM_OK;
    PCM_CUDA(cudaEventRecord(e[0], c->stream));
    for (int v = 0; v < nv && st == PCM_OK; ++v) {
        st = esp_launch_variant(c, k, v, blk, bcls, nb, c->esp_part.p);
        if (st == PCM_OK) PCM_CUDA(cudaEventRecord(e[v + 1], c->stream));
    }
    if (st == PCM_OK) {
        PCM_CUDA(cudaEventSynchronize(e[nv]));
        for (int v = 0; v < nv; ++v) PCM_CUDA(cudaEventElapsedTime(&ms[v], e[v], e[v + 1]));
    }
    for (int i = 0; i <= nv; ++i) cudaEventDestroy(e[i]);
    if (st != PCM_OK) return st;
    int best = 0;
    for (int v = 1; v < nv; ++v)
        if (ms[v] < ms[best]) best = v;
    *choice = best;
    tune_set(c->device, kind, L, bucket, best, ms[0], ms[1], ms[2]);
    return PCM_OK;
}

int esp_compute_mixed(pcm_ctx *c, double *dc)
{
    int nb[2];
    PCM_TRY(mixed_point_blocks(c, nb));
    DBuf<int> *blk = &c->si[4], *bcls = &c->si[6];  // blk[0..1], bcls[0..1]
    int var[6], rows[6], total = 0;
    for (int k = 0; k < 6; ++k) {
        var[k] = esp_default_ppt(CLASS_L[k], c->opt.fp32x2) == 4 ? 0 : 1;
        if (c->opt.esp_variant >= 0) {
            if (c->opt.esp_variant < 2 || CLASS_L[k] <= 2) var[k] = c->opt.esp_variant;
        } else if (c->opt.autotune && c->cls[k].nesp > 0) {
            PCM_TRY(esp_tune(c, k, blk, bcls, nb, &var[k]));
        }
        rows[k] = c->cls[k].nesp > 0 ? esp_rows_v(c, k, var[k], nb) : 0;
        total += rows[k];
    }
    if (total == 0) {
        c->esp_total_rows = 0;
        c->esp_out = dc;
        PCM_CUDA(cudaMemsetAsync(dc, 0, c->M * sizeof(double), c->stream));
        if (c->jobs) return PCM_OK;
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        return PCM_OK;
    }
    PCM_TRY(c->esp_part.alloc((size_t)total * c->M));
    int base = 0;
    for (int k = 0; k < 6; ++k) {
        if (c->cls[k].nesp == 0) continue;
        PCM_TRY(esp_launch_variant(c, k, var[k], blk, bcls, nb, c->esp_part.p + (size_t)base * c->M));
        base += rows[k];
    }
    c->esp_total_rows = total;
    c->esp_out = dc;
    if (c->jobs) return PCM_OK;   // the batch launches the packed blocks, then esp_mixed_finish
    PCM_TRY(esp_mixed_finish(c));
    PCM_CUDA(cudaStreamSynchronize(c->stream));  // the class timers are read next
    return check_device_error(c, "pcm_esp");
}

// c = the sum of the partial rows (after the packed blocks have run)
int esp_mixed_finish(pcm_ctx *c)
{
    if (c->esp_total_rows == 0) return PCM_OK;
    esp_reduce_mixed_kernel<<<(c->M + 255) / 256, 256, 0, c->stream>>>(c->M, c->esp_total_rows, c->esp_part.p,
                                                                       c->esp_out);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

int fock_mixed_class(pcm_ctx *c, int k, const double *dq, int nsplit, int ksplit, double *W, int npt)
{
    PairClass &pc = c->cls[k];
    // the packed kernel with two pairs per thread would spill for L >= 3
    if (c->opt.fp32x2 && CLASS_L[k] >= 3) npt = 1;
    const int per = MF_NT * npt;
    const int nb = (pc.npair + per - 1) / per;
    dim3 grid(nb, nsplit);
    if (c->opt.fp32x2) return fock_packed(c, CLASS_L[k], npt, pc.npair, pc.p.p, pc.Pxyz32.p, pc.fnear, dq, nsplit, W);
    switch (CLASS_L[k]) {
#define PCM_FOCK_F32(LL)                                                                                           \
    case LL:                                                                                                       \
        if (npt == 2)                                                                                              \
            fock_kernel_f32<LL, 2><<<grid, MF_NT, 0, c->stream>>>(pc.npair, pc.p.p, pc.Pxyz32.p, ksplit, c->p32.p, \
                                                                   c->p32lo.p, dq, c->M, c->ncls, c->cls_off.p,    \
                                                                   c->cls_zeta.p, c->boys32.p, W);                 \
        else                                                                                                       \
            fock_kernel_f32<LL, 1><<<grid, MF_NT, 0, c->stream>>>(pc.npair, pc.p.p, pc.Pxyz32.p, ksplit, c->p32.p, \
                                                                   c->p32lo.p, dq, c->M, c->ncls, c->cls_off.p,    \
                                                                   c->cls_zeta.p, c->boys32.p, W);                 \
        break;
        PCM_FOCK_F32(0)
        PCM_FOCK_F32(1)
        PCM_FOCK_F32(2)
        PCM_FOCK_F32(3)
        PCM_FOCK_F32(4)
#undef PCM_FOCK_F32
    }
    PCM_LAUNCHED(c);
    return PCM_OK;
}

// ---------------------------------------------------------------------------
// gradient (PCM_MIXED): point part and the W accumulation on the FP32 pipes
// ---------------------------------------------------------------------------
template <int L>
static int grad_point_mixed_class(pcm_ctx *c, PairClass &pc, const int *blk, const int *bcls, int nblk,
                                  double *part, int rows, int sl)
{
    constexpr int NH = nherm(L);
    constexpr int F = 3 + 2 * NH;
    const int n = pc.nesp;
    PCM_TRY(pc.eX32.alloc(6 * (size_t)n));
    PCM_TRY(pc.eC32.alloc((size_t)c->ncls * F * n));
    esp_mixed_prep_kernel<L><<<(n + 127) / 128, 128, 0, c->stream>>>(n, n, c->ncls, c->cls_zeta.p, pc.eP.p, pc.eD.p,
                                                                     pc.eX32.p, pc.eC32.p);
    PCM_LAUNCHED(c);
    dim3 grid(nblk, rows);
    if (c->opt.fp32x2)
        esp_grad_kernel_f32x2<L><<<grid, MESP_NT, 0, c->stream>>>(n, sl, pc.eX32.p, pc.eC32.p, blk, bcls, c->p32.p,
                                                                   c->p32lo.p, c->boys32.p, c->M, part);
    else
        esp_grad_kernel_f32<L><<<grid, MESP_NT, 0, c->stream>>>(n, sl, pc.eX32.p, pc.eC32.p, blk, bcls, c->p32.p,
                                                                 c->p32lo.p, c->boys32.p, c->M, part);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

// Point-part partial sums of every class into c->esp_part (rows x 3 x M);
// *total_rows receives the number of rows.  Needs the ESP preparation.
int grad_point_mixed(pcm_ctx *c, int *total_rows)
{
    int nb[2];
    PCM_TRY(mixed_point_blocks(c, nb));
    DBuf<int> *blk = &c->si[4], *bcls = &c->si[6];
    int rows[6], sls[6], total = 0;
    // point-block layout: 2 points per thread for the packed kernel, else the
    // scalar kernel's 4 (L <= 1) or 2
    int lay[6];
    for (int k = 0; k < 6; ++k) {
        lay[k] = (c->opt.fp32x2 || CLASS_L[k] > 1) ? 1 : 0;
        esp_plan(c->cls[k].nesp, nb[lay[k]], &sls[k], &rows[k]);
        total += rows[k];
    }
    *total_rows = total;
    if (total == 0) return PCM_OK;
    PCM_TRY(c->esp_part.alloc((size_t)total * 3 * c->M));
    int base = 0;
    for (int k = 0; k < 6; ++k) {
        PairClass &pc = c->cls[k];
        if (rows[k] == 0) continue;
        double *part = c->esp_part.p + (size_t)base * 3 * c->M;
        const int v = lay[k];
        switch (CLASS_L[k]) {
#define PCM_GPM(LL)                                                                                      \
    case LL:                                                                                             \
        PCM_TRY(grad_point_mixed_class<LL>(c, pc, blk[v].p, bcls[v].p, nb[v], part, rows[k], sls[k])); \
        break;
            PCM_GPM(0)
            PCM_GPM(1)
            PCM_GPM(2)
            PCM_GPM(3)
            PCM_GPM(4)
#undef PCM_GPM
        }
        base += rows[k];
    }
    return PCM_OK;
}

// W_tuv (t+u+v <= L+1) over the ESP pairs of class k on the FP32 pipes; the
// pairs' split centres come from the point-part preparation (eX32)
template <int LL>
static void grad_w_launch(pcm_ctx *c, PairClass &pc, const double *dq, dim3 grid, int ksplit, double *W, int npt)
{
    const int n = pc.nesp;
    const double *gp = pc.eP.p + 3 * (size_t)n;
    if (npt == 2)
        fock_kernel_f32<LL, 2><<<grid, MF_NT, 0, c->stream>>>(n, gp, pc.eX32.p, ksplit, c->p32.p, c->p32lo.p, dq, c->M,
                                                               c->ncls, c->cls_off.p, c->cls_zeta.p, c->boys32.p, W);
    else
        fock_kernel_f32<LL, 1><<<grid, MF_NT, 0, c->stream>>>(n, gp, pc.eX32.p, ksplit, c->p32.p, c->p32lo.p, dq, c->M,
                                                               c->ncls, c->cls_off.p, c->cls_zeta.p, c->boys32.p, W);
}

// W accumulation of the integral gradient: the Fock contraction with R up to
// L + 1 over the ESP pairs (the packed far-field kernel of fock_packed.cu by
// default; one pair per thread from L + 1 = 4 on)
int grad_w_mixed(pcm_ctx *c, int k, const double *dq, int nsplit, int ksplit, double *W, int npt)
{
    PairClass &pc = c->cls[k];
    const int L1 = CLASS_L[k] + 1;
    if (L1 >= 4) npt = 1;
    const int per = MF_NT * npt;
    const int nb = (pc.nesp + per - 1) / per;
    dim3 grid(nb, nsplit);
    if (c->opt.fp32x2)
        return fock_packed(c, L1, npt, pc.nesp, pc.eP.p + 3 * (size_t)pc.nesp, pc.eX32.p, pc.fnear, dq, nsplit, W);
    switch (L1) {
    case 1: grad_w_launch<1>(c, pc, dq, grid, ksplit, W, npt); break;
    case 2: grad_w_launch<2>(c, pc, dq, grid, ksplit, W, npt); break;
    case 3: grad_w_launch<3>(c, pc, dq, grid, ksplit, W, npt); break;
    case 4: grad_w_launch<4>(c, pc, dq, grid, ksplit, W, npt); break;
    case 5: grad_w_launch<5>(c, pc, dq, grid, ksplit, W, npt); break;
    }
    PCM_LAUNCHED(c);
    return PCM_OK;
}

}  // namespace pcm
