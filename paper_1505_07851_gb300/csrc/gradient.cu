// Nuclear gradient of the electrostatic solvation energy at fixed density P
// and fixed charges q (Eq. 14, with the integral term split as in Eq. 22):
//   g_I = z^T (dB^T/dR_I) q + (d*c^T/dR_I) q + q^T (dA/dR_I) q / (2 f).
// At the solution of Eq. 1 this is the derivative of Eq. 13 at fixed P,
// because Eq. 13 is stationary in q there.
//
// Every surface point r_k = R_I + R_I u_i moves with its atom I (zeta_k does
// not depend on the geometry), so the points of one atom form one rigid body;
// in library order they are contiguous.  The terms:
//   B:  q_k Z_J erf(zeta_k d)/d over point k and atom J != I(k)    (Eq. 4)
//   A:  off-diagonal erf(zeta'_kl r)/r over point pairs on different atoms,
//       diagonal zeta_k sqrt(2/pi)/S_k through the switching factors s_J of
//       the other atoms (Eq. 2, Eq. 3, Eq. 8, Eq. 9)
//   C:  the integrals' bra, ket and point centres (integrals.cu)
// Per-point contributions are summed per atom over its point range, per-atom
// ones by one block per atom; every sum has a fixed order.  PCM_MIXED runs
// the integral kernels and the off-diagonal A term on the FP32 pipes (FP64
// accumulation across tiles); the B and switching terms stay FP64.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "context.h"

namespace pcm {

constexpr double TWO_OVER_SQRT_PI = 1.1283791670955125739;
constexpr double INV_SQRT_PI = 0.56418958354775628695;
constexpr double SQRT_2_OVER_PI = 0.79788456080286535588;
constexpr int GPT_NT = 128;
constexpr int GATOM_TILE = 512;

// atom of each point; each atom's point range [a0, a1) (zeroed by the caller,
// so an atom without points keeps an empty range)
__global__ void point_atom_kernel(int M, int n, const int *__restrict__ pindex, int *__restrict__ patom)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) patom[k] = pindex[k] / n;
}

__global__ void atom_range_kernel(int M, int natom, const int *__restrict__ patom, int *__restrict__ range)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const int a = patom[k];
    if (k == 0 || patom[k - 1] != a) range[a] = k;
    if (k == M - 1 || patom[k + 1] != a) range[natom + a] = k + 1;
}

// d/dr_k of the (k, J) terms of z^T B q and of q_k^2 A_kk / (2 f), J != I(k),
// as a coefficient of (r_k - R_J):
//   B: q_k Z_J d/dd [erf(zeta_k d)/d] / d
//   A: -wdiag (ds_J/dd) / (s_J d),   wdiag = q_k^2 A_kk / (2 f)
// with s_J = (erfc(zeta (R_J - d)) + erfc(zeta (R_J + d))) / 2 (Eq. 9) and
// ds_J/dd = (zeta / sqrt(pi)) (exp(-zeta^2 (R_J - d)^2) - exp(-zeta^2 (R_J + d)^2)).
// An atom with zeta (d - R_J) > 6 has s_J = 1 in FP64 and does not enter S_k;
// erf(zeta d) rounds to 1 for zeta d > 6.
__device__ __forceinline__ double point_atom_coef(double zk, double qk, double wdiag, double ZJ, double RJ,
                                                  double d2, int terms)
{
    const double d = sqrt(d2);
    double coef = 0.0;
    if (terms & PCM_GRAD_B) {
        const double a = zk * d;
        const double gp = (a > 6.0) ? -1.0 / d2 : (TWO_OVER_SQRT_PI * zk * exp(-a * a) - erf(a) / d) / d;
        coef += qk * ZJ * gp;
    }
    if ((terms & PCM_GRAD_A) && zk * (d - RJ) <= 6.0) {
        const double u = zk * (RJ - d), v = zk * (RJ + d);
        const double s = 0.5 * (erfc(u) + erfc(v));
        const double ds = zk * INV_SQRT_PI * (exp(-u * u) - exp(-v * v));
        coef -= wdiag * ds / s;
    }
    return coef / d;
}

// point side: g[d][k] = sum_{J != I(k)} coef (r_k - R_J)_d  (initialises g)
__global__ void __launch_bounds__(GPT_NT) grad_point_side_kernel(
    int M, int natom, const double *__restrict__ px, const double *__restrict__ py, const double *__restrict__ pz,
    const double *__restrict__ pzeta, const double *__restrict__ pS, const int *__restrict__ patom,
    const double *__restrict__ q, const double *__restrict__ xyz, const double *__restrict__ Z,
    const double *__restrict__ radius, double inv2f, int terms, double *__restrict__ g)
{
    __shared__ double sx[GATOM_TILE], sy[GATOM_TILE], sz[GATOM_TILE], sZ[GATOM_TILE], sR[GATOM_TILE];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = k < M;
    const int kk = active ? k : 0;
    const double x = px[kk], y = py[kk], z = pz[kk], zk = pzeta[kk], qk = q[kk];
    const int I = patom[kk];
    const double wdiag = qk * qk * (zk * SQRT_2_OVER_PI / pS[kk]) * inv2f;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int J0 = 0; J0 < natom; J0 += GATOM_TILE) {
        const int nj = min(GATOM_TILE, natom - J0);
        __syncthreads();
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
            sx[j] = xyz[3 * (J0 + j) + 0];
            sy[j] = xyz[3 * (J0 + j) + 1];
            sz[j] = xyz[3 * (J0 + j) + 2];
            sZ[j] = Z[J0 + j];
            sR[j] = radius[J0 + j];
        }
        __syncthreads();
        if (active)
            for (int j = 0; j < nj; ++j) {
                if (J0 + j == I) continue;
                const double dx = x - sx[j], dy = y - sy[j], dz = z - sz[j];
                const double c = point_atom_coef(zk, qk, wdiag, sZ[j], sR[j], dx * dx + dy * dy + dz * dz, terms);
                gx = fma(c, dx, gx);
                gy = fma(c, dy, gy);
                gz = fma(c, dz, gz);
            }
    }
    if (active) {
        g[k] = gx;
        g[(size_t)M + k] = gy;
        g[2 * (size_t)M + k] = gz;
    }
}

// atom side: gJ[J] = -sum_{k: I(k) != J} coef (r_k - R_J), one block per atom
__global__ void __launch_bounds__(GPT_NT) grad_atom_side_kernel(
    int M, const double *__restrict__ px, const double *__restrict__ py, const double *__restrict__ pz,
    const double *__restrict__ pzeta, const double *__restrict__ pS, const int *__restrict__ patom,
    const double *__restrict__ q, const double *__restrict__ xyz, const double *__restrict__ Z,
    const double *__restrict__ radius, double inv2f, int terms, double *__restrict__ gJ)
{
    __shared__ double red[GPT_NT / 32];
    const int J = blockIdx.x;
    const double X = xyz[3 * J], Y = xyz[3 * J + 1], Zc = xyz[3 * J + 2], ZJ = Z[J], RJ = radius[J];
    double a[3] = {0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < M; k += GPT_NT) {
        if (patom[k] == J) continue;
        const double zk = pzeta[k], qk = q[k];
        const double wdiag = qk * qk * (zk * SQRT_2_OVER_PI / pS[k]) * inv2f;
        const double dx = px[k] - X, dy = py[k] - Y, dz = pz[k] - Zc;
        const double c = point_atom_coef(zk, qk, wdiag, ZJ, RJ, dx * dx + dy * dy + dz * dz, terms);
        a[0] = fma(c, dx, a[0]);
        a[1] = fma(c, dy, a[1]);
        a[2] = fma(c, dz, a[2]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = block_sum<double, GPT_NT>(a[d], red);
        if (threadIdx.x == 0) gJ[3 * J + d] = -v;
    }
}

// Off-diagonal A: g[d][k] += (q_k / f) sum_{l != k} q_l dA_kl/dr_k,
//   dA_kl/dr_k = h'(r) (r_k - r_l) / r,  h(r) = erf(zeta' r) / r,
//   h'(r) / r = (2 zeta' / sqrt(pi) exp(-zeta'^2 r^2) - A_kl) / r^2,
// with A_kl read from the stored matrix; where zeta' r > 6 the stored A_kl is
// 1/r and h'(r)/r = -A_kl^3.  (Both orders (k, l) and (l, k) of the sum over
// pairs give the same derivative: the factor 2 of (1/2f) x 2.)  Pairs on one
// atom cancel between k and l in the per-atom sum and need no exclusion.
constexpr int GAO_NT = 256;
__global__ void __launch_bounds__(GAO_NT) grad_aoff_kernel(int M, int lda, const double *__restrict__ A,
                                                           const double *__restrict__ px,
                                                           const double *__restrict__ py,
                                                           const double *__restrict__ pz,
                                                           const int *__restrict__ pcls, int ncls,
                                                           const double *__restrict__ cls_zeta,
                                                           const double *__restrict__ q, double inv_f,
                                                           double *__restrict__ g)
{
    __shared__ double zp_tab[16], zp2_tab[16];
    __shared__ double red[GAO_NT / 32];
    const int k = blockIdx.x;
    const int ck = pcls[k];
    for (int t = threadIdx.x; t < ncls && t < 16; t += GAO_NT) {
        const double a = cls_zeta[ck], b = cls_zeta[t];
        const double zp = a * b / sqrt(a * a + b * b);  // Eq. 8
        zp_tab[t] = zp;
        zp2_tab[t] = zp * zp;
    }
    __syncthreads();
    const double xk = px[k], yk = py[k], zk = pz[k];
    const double *row = A + (size_t)k * lda;
    double a[3] = {0.0, 0.0, 0.0};
    for (int l = threadIdx.x; l < M; l += GAO_NT) {
        if (l == k) continue;
        const double dx = xk - px[l], dy = yk - py[l], dz = zk - pz[l];
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double Akl = row[l];
        const int cl = pcls[l];
        double zp, zp2;
        if (ncls <= 16) {
            zp = zp_tab[cl];
            zp2 = zp2_tab[cl];
        } else {
            const double za = cls_zeta[ck], zb = cls_zeta[cl];
            zp = za * zb / sqrt(za * za + zb * zb);
            zp2 = zp * zp;
        }
        const double x2 = zp2 * d2;
        const double t = (x2 > 36.0) ? -Akl * Akl * Akl : (TWO_OVER_SQRT_PI * zp * exp(-x2) - Akl) / d2;
        const double w = q[l] * t;
        a[0] = fma(w, dx, a[0]);
        a[1] = fma(w, dy, a[1]);
        a[2] = fma(w, dz, a[2]);
    }
    const double s = q[k] * inv_f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = block_sum<double, GAO_NT>(a[d], red);
        if (threadIdx.x == 0) g[(size_t)d * M + k] += s * v;
    }
}

// The same on the FP32 pipes (PCM_MIXED) from the hi/lo split coordinates
// (hi on a 2^-10 grid, so hi differences are exact), with A_kl from the FP32
// copy of A when one is stored (A != null), else evaluated in FP32 (1/R, or
// erf(zeta' R) / R where zeta' R <= 6); per-thread FP32 sums, the block
// reduction in FP64.
__global__ void __launch_bounds__(GAO_NT) grad_aoff_kernel_f32(int M, int lda, const float *__restrict__ A,
                                                               const float *__restrict__ ph,
                                                               const float *__restrict__ pl,
                                                               const int *__restrict__ pcls, int ncls,
                                                               const double *__restrict__ cls_zeta,
                                                               const double *__restrict__ q, double inv_f,
                                                               double *__restrict__ g)
{
    __shared__ float zp_tab[16], zp2_tab[16];
    __shared__ double red[GAO_NT / 32];
    const int k = blockIdx.x;
    const int ck = pcls[k];
    for (int t = threadIdx.x; t < ncls && t < 16; t += GAO_NT) {
        const double a = cls_zeta[ck], b = cls_zeta[t];
        const double zp = a * b / sqrt(a * a + b * b);  // Eq. 8
        zp_tab[t] = (float)zp;
        zp2_tab[t] = (float)(zp * zp);
    }
    __syncthreads();
    const float xh = ph[k], yh = ph[(size_t)M + k], zh = ph[2 * (size_t)M + k];
    const float xl = pl[k], yl = pl[(size_t)M + k], zl = pl[2 * (size_t)M + k];
    const float *row = A ? A + (size_t)k * lda : nullptr;
    float a[3] = {0.f, 0.f, 0.f};
    for (int l = threadIdx.x; l < M; l += GAO_NT) {
        if (l == k) continue;
        const float dx = (xh - ph[l]) + (xl - pl[l]);
        const float dy = (yh - ph[(size_t)M + l]) + (yl - pl[(size_t)M + l]);
        const float dz = (zh - ph[2 * (size_t)M + l]) + (zl - pl[2 * (size_t)M + l]);
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const int cl = pcls[l];
        float zp, zp2;
        if (ncls <= 16) {
            zp = zp_tab[cl];
            zp2 = zp2_tab[cl];
        } else {
            const double za = cls_zeta[ck], zb = cls_zeta[cl];
            const double z = za * zb / sqrt(za * za + zb * zb);
            zp = (float)z;
            zp2 = (float)(z * z);
        }
        const float x2 = zp2 * d2;
        float Akl;
        if (row) {
            Akl = row[l];
        } else {
            const float rs = rsqrtf(d2);
            Akl = (x2 > 36.f) ? rs : erff(zp * (d2 * rs)) * rs;
        }
        const float t = (x2 > 36.f) ? -Akl * Akl * Akl
                                    : (1.1283791670955126f * zp * __expf(-x2) - Akl) / d2;
        const float w = (float)q[l] * t;
        a[0] = fmaf(w, dx, a[0]);
        a[1] = fmaf(w, dy, a[1]);
        a[2] = fmaf(w, dz, a[2]);
    }
    const double s = q[k] * inv_f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = block_sum<double, GAO_NT>((double)a[d], red);
        if (threadIdx.x == 0) g[(size_t)d * M + k] += s * v;
    }
}

// grad[I] = sum over the points of I of g_pt + gJ[I] + gpair[I], one block per atom
__global__ void __launch_bounds__(GPT_NT) grad_combine_kernel(int M, int natom, const int *__restrict__ range,
                                                              const double *__restrict__ gpt,
                                                              const double *__restrict__ gJ,
                                                              const double *__restrict__ gpair,
                                                              double *__restrict__ grad)
{
    __shared__ double red[GPT_NT / 32];
    const int I = blockIdx.x;
    const int k0 = range[I], k1 = range[natom + I];
    double a[3] = {0.0, 0.0, 0.0};
    for (int k = k0 + threadIdx.x; k < k1; k += GPT_NT)
#pragma unroll
        for (int d = 0; d < 3; ++d) a[d] += gpt[(size_t)d * M + k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = block_sum<double, GPT_NT>(a[d], red);
        if (threadIdx.x == 0) grad[3 * I + d] = v + gJ[3 * I + d] + gpair[3 * I + d];
    }
}

int gradient_compute(pcm_ctx *c, const double *dP, const double *dq, int terms, double *dgrad)
{
    PCM_TRY(join_side(c));
    const int M = c->M, natom = c->natom;
    const double f = (c->opt.eps - 1.0) / (c->opt.eps + c->opt.k);
    PCM_TRY(c->patom.alloc(M));
    PCM_TRY(c->arange.alloc(2 * (size_t)natom));
    PCM_TRY(c->g_pt.alloc(3 * (size_t)M));
    PCM_TRY(c->g_atom.alloc(3 * (size_t)natom));
    PCM_TRY(c->g_pair.alloc(3 * (size_t)natom));
    point_atom_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, c->npts_sphere, c->pindex.p, c->patom.p);
    PCM_LAUNCHED(c);
    PCM_CUDA(cudaMemsetAsync(c->arange.p, 0, 2 * (size_t)natom * sizeof(int), c->stream));
    atom_range_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, natom, c->patom.p, c->arange.p);
    PCM_LAUNCHED(c);

    // B and the diagonal of A: point side (initialises g_pt) and atom side
    const int pa_terms = terms & (PCM_GRAD_B | PCM_GRAD_A);
    grad_point_side_kernel<<<(M + GPT_NT - 1) / GPT_NT, GPT_NT, 0, c->stream>>>(
        M, natom, c->px.p, c->py.p, c->pz.p, c->pzeta.p, c->pS.p, c->patom.p, dq, c->xyz.p, c->Z.p, c->radius.p,
        0.5 / f, pa_terms, c->g_pt.p);
    PCM_LAUNCHED(c);
    grad_atom_side_kernel<<<natom, GPT_NT, 0, c->stream>>>(M, c->px.p, c->py.p, c->pz.p, c->pzeta.p, c->pS.p,
                                                           c->patom.p, dq, c->xyz.p, c->Z.p, c->radius.p, 0.5 / f,
                                                           pa_terms, c->g_atom.p);
    PCM_LAUNCHED(c);
    // off-diagonal A
    if (terms & PCM_GRAD_A) {
        if (c->opt.precision == PCM_MIXED) {
            const float *A32 = matrix_free(c) ? nullptr : c->A32.p;
            grad_aoff_kernel_f32<<<M, GAO_NT, 0, c->stream>>>(M, c->lda, A32, c->p32.p, c->p32lo.p, c->pcls.p,
                                                              c->ncls, c->cls_zeta.p, dq, 1.0 / f, c->g_pt.p);
        } else {
            grad_aoff_kernel<<<M, GAO_NT, 0, c->stream>>>(M, c->lda, c->A.p, c->px.p, c->py.p, c->pz.p, c->pcls.p,
                                                          c->ncls, c->cls_zeta.p, dq, 1.0 / f, c->g_pt.p);
        }
        PCM_LAUNCHED(c);
    }
    // integrals
    PCM_CUDA(cudaMemsetAsync(c->g_pair.p, 0, 3 * (size_t)natom * sizeof(double), c->stream));
    c->stats.integrals_grad = 0.0;
    if (terms & PCM_GRAD_C) PCM_TRY(grad_integrals(c, dP, dq, c->g_pt.p, c->g_pair.p));
    grad_combine_kernel<<<natom, GPT_NT, 0, c->stream>>>(M, natom, c->arange.p, c->g_pt.p, c->g_atom.p, c->g_pair.p,
                                                         dgrad);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

}  // namespace pcm
