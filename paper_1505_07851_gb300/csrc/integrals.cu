// The two contractions of the erf-screened one-electron integrals:
//   c_k        = -sum_{mu nu} P_{mu nu} (mu|J_k|nu)       (Eq. 5, Eq. 6, Eq. 19)
//   dF_{mu nu} = -sum_k q_k (mu|J_k|nu)                   (Eq. 10, Eq. 16, Eq. 17)
// with (mu|J_k|nu) contracted from primitives (Eq. 12).
//
// Integrals are evaluated in the McMurchie-Davidson (Hermite) form.  For a
// primitive pair with exponents a, b, p = a + b, centre P and
// K = exp(-ab/p |A-B|^2), and a point with exponent zeta:
//   rho = p zeta^2 / (p + zeta^2),  U = sqrt(zeta^2 / (p + zeta^2))
//   [a|J|b] = (2 pi / p) K U sum_tuv E^{ab}_tuv R_tuv(rho, P - C)
//   R^(n)_000 = (-2 rho)^n F_n(rho |P - C|^2)
// (the erf operator is the Coulomb operator between the pair's Gaussian
// charge and a Gaussian charge of exponent zeta^2).  The ESP kernel dots each
// pair's density-weighted Hermite coefficients D_tuv into R_tuv; the Fock
// kernel accumulates W_tuv = sum_k q_k U R_tuv per pair and contracts with
// E^{ab}_tuv at the end.  Both contractions are reduced on the device in a
// fixed order, so results are bit-reproducible.
#include <math.h>

#include <algorithm>
#include <vector>

#include "boys.cuh"
#include "common.cuh"
#include "context.h"
#include "tune.h"

namespace pcm {

__device__ inline double comp_factor_i(int l, int c)
{
    if (l < 2) return 1.0;
    return (c == 1 || c == 2 || c == 4) ? 1.7320508075688772935 : 1.0;
}

// ---------------------------------------------------------------------------
// ESP prologue: density test of Eq. 18 and Hermite density coefficients
//   D_tuv = -(2 pi / p) K sum_{a in A, b in B} W_ab c_a c_b E^{ab}_tuv
// with W_ab = P_ab + P_ba for off-diagonal primitive pairs (a pair stands for
// itself and its mirror image) and W_ab = P_ab for i = j in a diagonal shell pair.
// ---------------------------------------------------------------------------
// flag[r] (first npair bytes): pair kept and both primitives on one atom;
// flag[npair + r]: kept and on two atoms.  Same-atom pairs (centre P = the
// atom) come first in the ESP list; PCM_MIXED evaluates them more precisely.
template <int LA, int LB>
__global__ void esp_flag_kernel(int npair, const int *__restrict__ sp, const int *__restrict__ ia,
                                const int *__restrict__ ib, const int *__restrict__ spA, const int *__restrict__ spB,
                                const int *__restrict__ sh_bf, const int *__restrict__ sh_atom,
                                const double *__restrict__ Q, const double *__restrict__ Pm, int nbf, double thresh,
                                unsigned char *__restrict__ flag)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= npair) return;
    const int s = sp[r];
    const int A = spA[s], B = spB[s];
    const bool mirror = (A != B) || (ia[r] != ib[r]);
    const int fa = sh_bf[A], fb = sh_bf[B];
    double wmax = 0.0;
    for (int a = 0; a < ncart(LA); ++a)
        for (int b = 0; b < ncart(LB); ++b) {
            double w = Pm[(size_t)(fa + a) * nbf + fb + b];
            if (mirror) w += Pm[(size_t)(fb + b) * nbf + fa + a];
            wmax = fmax(wmax, fabs(w));
        }
    const bool kept = thresh <= 0.0 || wmax * Q[r] >= thresh;
    const bool same = sh_atom[A] == sh_atom[B];
    flag[r] = (kept && same) ? 1 : 0;
    flag[(size_t)npair + r] = (kept && !same) ? 1 : 0;
}

template <int LA, int LB>
__global__ void esp_coef_kernel(int nesp, const int *__restrict__ list, const int *__restrict__ sp,
                                const int *__restrict__ ia, const int *__restrict__ ib, const int *__restrict__ spA,
                                const int *__restrict__ spB, const int *__restrict__ sh_atom,
                                const int *__restrict__ sh_off, const int *__restrict__ sh_bf,
                                const double *__restrict__ cnorm, const double *__restrict__ xyz,
                                const double *__restrict__ Px, const double *__restrict__ Py,
                                const double *__restrict__ Pz, const double *__restrict__ pp,
                                const double *__restrict__ pref, const double *__restrict__ Pm, int nbf,
                                double *__restrict__ eP, double *__restrict__ eD)
{
    constexpr int L = LA + LB;
    constexpr int NH = nherm(L);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nesp) return;
    const int r = list[j];
    const int s = sp[r];
    const int A = spA[s], B = spB[s];
    const int i1 = ia[r], i2 = ib[r];
    const bool mirror = (A != B) || (i1 != i2);
    const double p = pp[r];
    const double P[3] = {Px[r], Py[r], Pz[r]};
    const double *RA = xyz + 3 * sh_atom[A], *RB = xyz + 3 * sh_atom[B];
    E1T<LA, LB> Ex, Ey, Ez;
    const double inv2p = 0.5 / p;
    hermite_E1T<LA, LB>(P[0] - RA[0], P[0] - RB[0], inv2p, Ex);
    hermite_E1T<LA, LB>(P[1] - RA[1], P[1] - RB[1], inv2p, Ey);
    hermite_E1T<LA, LB>(P[2] - RA[2], P[2] - RB[2], inv2p, Ez);
    const double cc = cnorm[sh_off[A] + i1] * cnorm[sh_off[B] + i2];
    const int fa = sh_bf[A], fb = sh_bf[B];
    double D[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) D[h] = 0.0;
#pragma unroll
    for (int a = 0; a < ncart(LA); ++a) {
        const int ax = cart_e(LA, a, 0), ay = cart_e(LA, a, 1), az = cart_e(LA, a, 2);
#pragma unroll
        for (int b = 0; b < ncart(LB); ++b) {
            const int bx = cart_e(LB, b, 0), by = cart_e(LB, b, 1), bz = cart_e(LB, b, 2);
            double w = Pm[(size_t)(fa + a) * nbf + fb + b];
            if (mirror) w += Pm[(size_t)(fb + b) * nbf + fa + a];
            w *= cc * comp_factor_i(LA, a) * comp_factor_i(LB, b);
            // E_t vanishes for t > i + j: the full loops add exact zeros there
#pragma unroll
            for (int t = 0; t <= L; ++t)
#pragma unroll
                for (int u = 0; u <= L - t; ++u)
#pragma unroll
                    for (int v = 0; v <= L - t - u; ++v)
                        D[hidx(t, u, v)] += w * Ex.e[ax][bx][t] * Ey.e[ay][by][u] * Ez.e[az][bz][v];
        }
    }
    const double scale = -pref[r];
    eP[0 * (size_t)nesp + j] = P[0];
    eP[1 * (size_t)nesp + j] = P[1];
    eP[2 * (size_t)nesp + j] = P[2];
    eP[3 * (size_t)nesp + j] = p;
#pragma unroll
    for (int h = 0; h < NH; ++h) eD[(size_t)h * nesp + j] = scale * D[h];
}

// ---------------------------------------------------------------------------
// ESP main kernel: one thread per surface point (PPT points per thread),
// looping over tiles of TP primitive pairs staged in shared memory.  The
// per-(pair, exponent class) factors rho and U are computed once per tile for
// the classes present in the block (at most MAXCB).
// grid.x: point blocks (ranges from blk_off), grid.y: pair segments.
// ---------------------------------------------------------------------------
constexpr int ESP_NT = 128;
constexpr int ESP_PPT = 2;
constexpr int ESP_TP = 32;
constexpr int ESP_MAXCB = 8;

template <int L>
__global__ void __launch_bounds__(ESP_NT) esp_kernel_f64(int nesp, int seglen, const double *__restrict__ eP,
                                                         const double *__restrict__ eD, const int *__restrict__ blk_off,
                                                         const double *__restrict__ px, const double *__restrict__ py,
                                                         const double *__restrict__ pz, const int *__restrict__ pcls,
                                                         const double *__restrict__ cls_zeta,
                                                         const double *__restrict__ boys, int M,
                                                         double *__restrict__ part)
{
    constexpr int NH = nherm(L);
    __shared__ double sP[4][ESP_TP];
    __shared__ double sD[NH][ESP_TP];
    __shared__ double sRho[ESP_MAXCB][ESP_TP];
    __shared__ double sU[ESP_MAXCB][ESP_TP];

    const int k0 = blk_off[blockIdx.x], k1 = blk_off[blockIdx.x + 1];
    const int cmin = pcls[k0];
    const int ncb = pcls[k1 - 1] - cmin + 1;  // <= ESP_MAXCB by construction of blk_off
    const int j0 = blockIdx.y * seglen;
    const int j1 = min(nesp, j0 + seglen);

    double x[ESP_PPT], y[ESP_PPT], z[ESP_PPT], acc[ESP_PPT];
    int e[ESP_PPT];
    bool on[ESP_PPT];
#pragma unroll
    for (int q = 0; q < ESP_PPT; ++q) {
        const int k = k0 + threadIdx.x + q * ESP_NT;
        on[q] = k < k1;
        const int kk = on[q] ? k : k0;
        x[q] = px[kk];
        y[q] = py[kk];
        z[q] = pz[kk];
        e[q] = pcls[kk] - cmin;
        acc[q] = 0.0;
    }

    for (int jt = j0; jt < j1; jt += ESP_TP) {
        const int nt = min(ESP_TP, j1 - jt);
        __syncthreads();
        for (int t = threadIdx.x; t < 4 * ESP_TP; t += ESP_NT) {
            const int f = t / ESP_TP, jj = t % ESP_TP;
            sP[f][jj] = jj < nt ? eP[(size_t)f * nesp + jt + jj] : 1.0;
        }
        for (int t = threadIdx.x; t < NH * ESP_TP; t += ESP_NT) {
            const int h = t / ESP_TP, jj = t % ESP_TP;
            sD[h][jj] = jj < nt ? eD[(size_t)h * nesp + jt + jj] : 0.0;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ncb * ESP_TP; t += ESP_NT) {
            const int ec = t / ESP_TP, jj = t % ESP_TP;
            const double zz = cls_zeta[cmin + ec];
            const double z2 = zz * zz;
            const double p = sP[3][jj];
            const double inv = 1.0 / (p + z2);
            sRho[ec][jj] = p * z2 * inv;
            sU[ec][jj] = sqrt(z2 * inv);
        }
        __syncthreads();
        for (int jj = 0; jj < nt; ++jj) {
            const double Px = sP[0][jj], Py = sP[1][jj], Pz = sP[2][jj];
#pragma unroll
            for (int q = 0; q < ESP_PPT; ++q) {
                const double rho = sRho[e[q]][jj];
                const double X = Px - x[q], Y = Py - y[q], Z = Pz - z[q];
                const double T = rho * (X * X + Y * Y + Z * Z);
                double F[L + 1];
                boys_eval<L>(T, boys, F);
                double dot;
                if constexpr (L == 0) {
                    dot = sD[0][jj] * F[0];
                } else {
                    double Rn[L + 1];
                    double m2r = -2.0 * rho, f = 1.0;
#pragma unroll
                    for (int n = 0; n <= L; ++n) {
                        Rn[n] = f * F[n];
                        f *= m2r;
                    }
                    double R[NH];
                    hermite_R<L, double>(X, Y, Z, Rn, R);
                    dot = 0.0;
#pragma unroll
                    for (int h = 0; h < NH; ++h) dot = fma(sD[h][jj], R[h], dot);
                }
                acc[q] = fma(sU[e[q]][jj], dot, acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < ESP_PPT; ++q) {
        const int k = k0 + threadIdx.x + q * ESP_NT;
        if (on[q]) part[(size_t)blockIdx.y * M + k] = acc[q];
    }
}

// c_k = sum over segments of the partial sums, in segment order.
__global__ void esp_reduce_kernel(int M, int nseg, const double *__restrict__ part, double *__restrict__ c)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double s = 0.0;
    for (int g = 0; g < nseg; ++g) s += part[(size_t)g * M + k];
    c[k] = s;
}

// ---------------------------------------------------------------------------
// Fock main kernel: one thread per primitive pair, looping over the points of
// its split in exponent-class order, staged in shared memory tiles of TQ.
// W[split][h][pair] = sum_k q_k U_k R_h(rho_k, P - C_k)
// ---------------------------------------------------------------------------
constexpr int FOCK_NT = 128;
constexpr int FOCK_TQ = 128;

template <int L>
__global__ void __launch_bounds__(FOCK_NT) fock_kernel_f64(int npair, const double *__restrict__ gPx,
                                                           const double *__restrict__ gPy,
                                                           const double *__restrict__ gPz,
                                                           const double *__restrict__ gp, int ksplit,
                                                           const double *__restrict__ px, const double *__restrict__ py,
                                                           const double *__restrict__ pz, const double *__restrict__ q,
                                                           int M, int ncls, const int *__restrict__ cls_off,
                                                           const double *__restrict__ cls_zeta,
                                                           const double *__restrict__ boys, double *__restrict__ W)
{
    constexpr int NH = nherm(L);
    __shared__ double sx[FOCK_TQ], sy[FOCK_TQ], sz[FOCK_TQ], sq[FOCK_TQ];
    const int r = blockIdx.x * FOCK_NT + threadIdx.x;
    const bool active = r < npair;
    const int rr = active ? r : 0;
    const double Px = gPx[rr], Py = gPy[rr], Pz = gPz[rr], p = gp[rr];
    const int ka = blockIdx.y * ksplit;
    const int kb = min(M, ka + ksplit);
    double w[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) w[h] = 0.0;
    for (int ec = 0; ec < ncls; ++ec) {
        const int a = max(ka, cls_off[ec]), b = min(kb, cls_off[ec + 1]);
        if (a >= b) continue;
        const double zz = cls_zeta[ec];
        const double z2 = zz * zz;
        const double inv = 1.0 / (p + z2);
        const double rho = p * z2 * inv;
        const double U = sqrt(z2 * inv);
        const double m2r = -2.0 * rho;
        for (int t0 = a; t0 < b; t0 += FOCK_TQ) {
            const int nt = min(FOCK_TQ, b - t0);
            __syncthreads();
            for (int t = threadIdx.x; t < nt; t += FOCK_NT) {
                sx[t] = px[t0 + t];
                sy[t] = py[t0 + t];
                sz[t] = pz[t0 + t];
                sq[t] = q[t0 + t];
            }
            __syncthreads();
            for (int kk = 0; kk < nt; ++kk) {
                const double X = Px - sx[kk], Y = Py - sy[kk], Z = Pz - sz[kk];
                const double T = rho * (X * X + Y * Y + Z * Z);
                double F[L + 1];
                boys_eval<L>(T, boys, F);
                const double sc = sq[kk] * U;
                if constexpr (L == 0) {
                    w[0] = fma(sc, F[0], w[0]);
                } else {
                    double Rn[L + 1];
                    double f = sc;
#pragma unroll
                    for (int n = 0; n <= L; ++n) {
                        Rn[n] = f * F[n];
                        f *= m2r;
                    }
                    double R[NH];
                    hermite_R<L, double>(X, Y, Z, Rn, R);
#pragma unroll
                    for (int h = 0; h < NH; ++h) w[h] += R[h];
                }
            }
        }
    }
    if (active) {
#pragma unroll
        for (int h = 0; h < NH; ++h) W[((size_t)blockIdx.y * NH + h) * npair + r] = w[h];
    }
}

// Fock epilogue: one thread per shell pair.  For each kept primitive pair of
// the shell pair, L_ab = -(2 pi/p) K sum_tuv E^{ab}_tuv W_tuv is contracted
// with c_a c_b (Eq. 16) and summed in pair order (Eq. 17).  A diagonal shell
// pair's off-diagonal primitive pair also adds its mirror image.  Both dF
// blocks (A,B) and (B,A) are written; every element of dF is written.
template <int LA, int LB>
__global__ void fock_epilogue_kernel(int nsp, int npair, int nsplit, const int *__restrict__ spA,
                                     const int *__restrict__ spB, const int *__restrict__ sp_start,
                                     const int *__restrict__ ia, const int *__restrict__ ib,
                                     const int *__restrict__ sh_atom, const int *__restrict__ sh_off,
                                     const int *__restrict__ sh_bf, const double *__restrict__ cnorm,
                                     const double *__restrict__ xyz, const double *__restrict__ Px,
                                     const double *__restrict__ Py, const double *__restrict__ Pz,
                                     const double *__restrict__ pp, const double *__restrict__ pref,
                                     const double *__restrict__ W, int nbf, double *__restrict__ dF)
{
    constexpr int L = LA + LB;
    constexpr int NH = nherm(L);
    constexpr int NA = ncart(LA), NB = ncart(LB);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsp) return;
    const int A = spA[s], B = spB[s];
    const double *RA = xyz + 3 * sh_atom[A], *RB = xyz + 3 * sh_atom[B];
    double G[NA * NB];
#pragma unroll
    for (int t = 0; t < NA * NB; ++t) G[t] = 0.0;
    for (int r = sp_start[s]; r < sp_start[s + 1]; ++r) {
        double w[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            double acc = 0.0;
            for (int g = 0; g < nsplit; ++g) acc += W[((size_t)g * NH + h) * npair + r];
            w[h] = acc;
        }
        const double p = pp[r];
        const double P[3] = {Px[r], Py[r], Pz[r]};
        E1T<LA, LB> Ex, Ey, Ez;
        const double inv2p = 0.5 / p;
        hermite_E1T<LA, LB>(P[0] - RA[0], P[0] - RB[0], inv2p, Ex);
        hermite_E1T<LA, LB>(P[1] - RA[1], P[1] - RB[1], inv2p, Ey);
        hermite_E1T<LA, LB>(P[2] - RA[2], P[2] - RB[2], inv2p, Ez);
        const int i1 = ia[r], i2 = ib[r];
        const double cc = -pref[r] * cnorm[sh_off[A] + i1] * cnorm[sh_off[B] + i2];
        const bool mirror = (A == B) && (i1 != i2);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int ax = cart_e(LA, a, 0), ay = cart_e(LA, a, 1), az = cart_e(LA, a, 2);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int bx = cart_e(LB, b, 0), by = cart_e(LB, b, 1), bz = cart_e(LB, b, 2);
                double v = 0.0;
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int vv = 0; vv <= L - t - u; ++vv)
                            v += Ex.e[ax][bx][t] * Ey.e[ay][by][u] * Ez.e[az][bz][vv] * w[hidx(t, u, vv)];
                v *= cc * comp_factor_i(LA, a) * comp_factor_i(LB, b);
                G[a * NB + b] += v;
                if (mirror) G[b * NB + a] += v;
            }
        }
    }
    const int fa = sh_bf[A], fb = sh_bf[B];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            dF[(size_t)(fa + a) * nbf + fb + b] = G[a * NB + b];
            dF[(size_t)(fb + b) * nbf + fa + a] = G[a * NB + b];
        }
}


// ---------------------------------------------------------------------------
// Integral part of the nuclear gradient (Eq. 14, second term; Eq. 22).
// Each integral [a|J_k|b] depends on the centre of a, the centre of b and the
// point r_k, which moves with its atom.
//
// Point part (gc of Eq. 22): d/dC R_tuv(P - C) = -R_{t+1,u,v} (and y, z), so
//   d c_k / dC_k = -sum_pairs U sum_tuv eD_tuv R_{tuv + 1_d}
// with the ESP pairs' density coefficients eD (t+u+v <= L) and R up to L+1.
// One thread per point as in the ESP kernel; three sums per point.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(ESP_NT) esp_grad_kernel(int nesp, int seglen, const double *__restrict__ eP,
                                                          const double *__restrict__ eD,
                                                          const int *__restrict__ blk_off,
                                                          const double *__restrict__ px, const double *__restrict__ py,
                                                          const double *__restrict__ pz, const int *__restrict__ pcls,
                                                          const double *__restrict__ cls_zeta,
                                                          const double *__restrict__ boys, int M,
                                                          double *__restrict__ part)
{
    constexpr int NH = nherm(L);
    constexpr int L1 = L + 1;
    constexpr int NH1 = nherm(L1);
    __shared__ double sP[4][ESP_TP];
    __shared__ double sD[NH][ESP_TP];
    __shared__ double sRho[ESP_MAXCB][ESP_TP];
    __shared__ double sU[ESP_MAXCB][ESP_TP];

    const int k0 = blk_off[blockIdx.x], k1 = blk_off[blockIdx.x + 1];
    const int cmin = pcls[k0];
    const int ncb = pcls[k1 - 1] - cmin + 1;
    const int j0 = blockIdx.y * seglen;
    const int j1 = min(nesp, j0 + seglen);

    double x[ESP_PPT], y[ESP_PPT], z[ESP_PPT], gx[ESP_PPT], gy[ESP_PPT], gz[ESP_PPT];
    int e[ESP_PPT];
    bool on[ESP_PPT];
#pragma unroll
    for (int q = 0; q < ESP_PPT; ++q) {
        const int k = k0 + threadIdx.x + q * ESP_NT;
        on[q] = k < k1;
        const int kk = on[q] ? k : k0;
        x[q] = px[kk];
        y[q] = py[kk];
        z[q] = pz[kk];
        e[q] = pcls[kk] - cmin;
        gx[q] = gy[q] = gz[q] = 0.0;
    }

    for (int jt = j0; jt < j1; jt += ESP_TP) {
        const int nt = min(ESP_TP, j1 - jt);
        __syncthreads();
        for (int t = threadIdx.x; t < 4 * ESP_TP; t += ESP_NT) {
            const int f = t / ESP_TP, jj = t % ESP_TP;
            sP[f][jj] = jj < nt ? eP[(size_t)f * nesp + jt + jj] : 1.0;
        }
        for (int t = threadIdx.x; t < NH * ESP_TP; t += ESP_NT) {
            const int h = t / ESP_TP, jj = t % ESP_TP;
            sD[h][jj] = jj < nt ? eD[(size_t)h * nesp + jt + jj] : 0.0;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ncb * ESP_TP; t += ESP_NT) {
            const int ec = t / ESP_TP, jj = t % ESP_TP;
            const double zz = cls_zeta[cmin + ec];
            const double z2 = zz * zz;
            const double p = sP[3][jj];
            const double inv = 1.0 / (p + z2);
            sRho[ec][jj] = p * z2 * inv;
            sU[ec][jj] = sqrt(z2 * inv);
        }
        __syncthreads();
        for (int jj = 0; jj < nt; ++jj) {
            const double Px = sP[0][jj], Py = sP[1][jj], Pz = sP[2][jj];
#pragma unroll
            for (int q = 0; q < ESP_PPT; ++q) {
                const double rho = sRho[e[q]][jj];
                const double X = Px - x[q], Y = Py - y[q], Z = Pz - z[q];
                const double T = rho * (X * X + Y * Y + Z * Z);
                double F[L1 + 1];
                boys_eval<L1>(T, boys, F);
                double Rn[L1 + 1];
                double m2r = -2.0 * rho, f = 1.0;
#pragma unroll
                for (int n = 0; n <= L1; ++n) {
                    Rn[n] = f * F[n];
                    f *= m2r;
                }
                double R[NH1];
                hermite_R<L1, double>(X, Y, Z, Rn, R);
                double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int v = 0; v <= L - t - u; ++v) {
                            const double d = sD[hidx(t, u, v)][jj];
                            sx = fma(d, R[hidx(t + 1, u, v)], sx);
                            sy = fma(d, R[hidx(t, u + 1, v)], sy);
                            sz = fma(d, R[hidx(t, u, v + 1)], sz);
                        }
                const double U = sU[e[q]][jj];
                gx[q] = fma(U, sx, gx[q]);
                gy[q] = fma(U, sy, gy[q]);
                gz[q] = fma(U, sz, gz[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < ESP_PPT; ++q) {
        const int k = k0 + threadIdx.x + q * ESP_NT;
        if (on[q]) {
            part[((size_t)blockIdx.y * 3 + 0) * M + k] = gx[q];
            part[((size_t)blockIdx.y * 3 + 1) * M + k] = gy[q];
            part[((size_t)blockIdx.y * 3 + 2) * M + k] = gz[q];
        }
    }
}

// g[d][k] += -q_k sum over segments of the point-part sums, in segment order
__global__ void grad_point_reduce_kernel(int M, int nseg, const double *__restrict__ part,
                                         const double *__restrict__ q, double *__restrict__ g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int seg = 0; seg < nseg; ++seg) s += part[((size_t)seg * 3 + d) * M + k];
        g[(size_t)d * M + k] -= q[k] * s;
    }
}

// Bra- and ket-centre parts (ga, gb of Eq. 22) for one ESP pair.  With
// W_tuv = sum_k q_k U_k R_tuv (t+u+v <= L+1, accumulated by the Fock kernel
// over the ESP pairs) and the derivative of a Cartesian Gaussian with respect
// to its centre, d/dA_x G_a = 2 alpha G_{a+1_x} - a_x G_{a-1_x},
//   d/dA_x sum_k q_k c_k (this pair) = -(2 pi/p) K sum_ab w_ab
//       sum_tuv (2 alpha E^{a+1_x,b}_t - a_x E^{a-1_x,b}_t) E^{ab}_u E^{ab}_v W_tuv
// (w_ab the density weights of the ESP prologue), and likewise for y, z and
// for the centre of b.  Written to gfull[d][r] (A) and gfull[3 + d][r] (B) at
// the kept-pair index r.
template <int LA, int LB>
__global__ void grad_pair_kernel(int nesp, int npair, int nsplit, const int *__restrict__ elist,
                                 const int *__restrict__ sp, const int *__restrict__ ia, const int *__restrict__ ib,
                                 const int *__restrict__ spA, const int *__restrict__ spB,
                                 const int *__restrict__ sh_atom, const int *__restrict__ sh_off,
                                 const int *__restrict__ sh_bf, const double *__restrict__ exps,
                                 const double *__restrict__ cnorm, const double *__restrict__ xyz,
                                 const double *__restrict__ Px, const double *__restrict__ Py,
                                 const double *__restrict__ Pz, const double *__restrict__ pp,
                                 const double *__restrict__ pref, const double *__restrict__ Pm, int nbf,
                                 const double *__restrict__ W, double *__restrict__ gfull)
{
    constexpr int L1 = LA + LB + 1;
    constexpr int NH1 = nherm(L1);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nesp) return;
    const int r = elist[j];
    const int s = sp[r];
    const int A = spA[s], B = spB[s];
    const int i1 = ia[r], i2 = ib[r];
    const bool mirror = (A != B) || (i1 != i2);
    double w[NH1];
#pragma unroll
    for (int h = 0; h < NH1; ++h) {
        double acc = 0.0;
        for (int g = 0; g < nsplit; ++g) acc += W[((size_t)g * NH1 + h) * nesp + j];
        w[h] = acc;
    }
    const double p = pp[r];
    const double P[3] = {Px[r], Py[r], Pz[r]};
    const double *RA = xyz + 3 * sh_atom[A], *RB = xyz + 3 * sh_atom[B];
    E1T<LA + 1, LB + 1> Ex, Ey, Ez;
    const double inv2p = 0.5 / p;
    hermite_E1T<LA + 1, LB + 1>(P[0] - RA[0], P[0] - RB[0], inv2p, Ex);
    hermite_E1T<LA + 1, LB + 1>(P[1] - RA[1], P[1] - RB[1], inv2p, Ey);
    hermite_E1T<LA + 1, LB + 1>(P[2] - RA[2], P[2] - RB[2], inv2p, Ez);
    const double al2 = 2.0 * exps[sh_off[A] + i1], be2 = 2.0 * exps[sh_off[B] + i2];
    const double cc = cnorm[sh_off[A] + i1] * cnorm[sh_off[B] + i2];
    const int fa = sh_bf[A], fb = sh_bf[B];
    double gA[3] = {0.0, 0.0, 0.0}, gB[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < ncart(LA); ++a) {
        const int ax = cart_e(LA, a, 0), ay = cart_e(LA, a, 1), az = cart_e(LA, a, 2);
#pragma unroll
        for (int b = 0; b < ncart(LB); ++b) {
            const int bx = cart_e(LB, b, 0), by = cart_e(LB, b, 1), bz = cart_e(LB, b, 2);
            double wab = Pm[(size_t)(fa + a) * nbf + fb + b];
            if (mirror) wab += Pm[(size_t)(fb + b) * nbf + fa + a];
            wab *= cc * comp_factor_i(LA, a) * comp_factor_i(LB, b);
            // one-dimensional factors: plain, centre-A derivative, centre-B derivative
            double X0[L1 + 1], XA[L1 + 1], XB[L1 + 1], Y0[L1 + 1], YA[L1 + 1], YB[L1 + 1];
            double Z0[L1 + 1], ZA[L1 + 1], ZB[L1 + 1];
#pragma unroll
            for (int t = 0; t <= L1; ++t) {
                X0[t] = Ex.e[ax][bx][t];
                Y0[t] = Ey.e[ay][by][t];
                Z0[t] = Ez.e[az][bz][t];
                XA[t] = al2 * Ex.e[ax + 1][bx][t] - (ax > 0 ? ax * Ex.e[ax > 0 ? ax - 1 : 0][bx][t] : 0.0);
                YA[t] = al2 * Ey.e[ay + 1][by][t] - (ay > 0 ? ay * Ey.e[ay > 0 ? ay - 1 : 0][by][t] : 0.0);
                ZA[t] = al2 * Ez.e[az + 1][bz][t] - (az > 0 ? az * Ez.e[az > 0 ? az - 1 : 0][bz][t] : 0.0);
                XB[t] = be2 * Ex.e[ax][bx + 1][t] - (bx > 0 ? bx * Ex.e[ax][bx > 0 ? bx - 1 : 0][t] : 0.0);
                YB[t] = be2 * Ey.e[ay][by + 1][t] - (by > 0 ? by * Ey.e[ay][by > 0 ? by - 1 : 0][t] : 0.0);
                ZB[t] = be2 * Ez.e[az][bz + 1][t] - (bz > 0 ? bz * Ez.e[az][bz > 0 ? bz - 1 : 0][t] : 0.0);
            }
            double sA[3] = {0.0, 0.0, 0.0}, sB[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int t = 0; t <= L1; ++t)
#pragma unroll
                for (int u = 0; u <= L1 - t; ++u)
#pragma unroll
                    for (int v = 0; v <= L1 - t - u; ++v) {
                        const double wh = w[hidx(t, u, v)];
                        sA[0] += XA[t] * Y0[u] * Z0[v] * wh;
                        sA[1] += X0[t] * YA[u] * Z0[v] * wh;
                        sA[2] += X0[t] * Y0[u] * ZA[v] * wh;
                        sB[0] += XB[t] * Y0[u] * Z0[v] * wh;
                        sB[1] += X0[t] * YB[u] * Z0[v] * wh;
                        sB[2] += X0[t] * Y0[u] * ZB[v] * wh;
                    }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                gA[d] = fma(wab, sA[d], gA[d]);
                gB[d] = fma(wab, sB[d], gB[d]);
            }
        }
    }
    const double scale = -pref[r];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        gfull[(size_t)d * npair + r] = scale * gA[d];
        gfull[(size_t)(3 + d) * npair + r] = scale * gB[d];
    }
}

// Per-atom sums of the pair parts: one block per atom walks its shell pairs
// (entry 2 s + side) and their kept primitive pairs; fixed-order reduction.
constexpr int GPA_NT = 128;
__global__ void __launch_bounds__(GPA_NT) pair_atom_reduce_kernel(int natom, const int *__restrict__ off,
                                                                  const int *__restrict__ ent,
                                                                  const int *__restrict__ sp_start, int npair,
                                                                  const double *__restrict__ gfull,
                                                                  double *__restrict__ g)
{
    __shared__ double red[GPA_NT / 32];
    const int I = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int e = off[I] + threadIdx.x; e < off[I + 1]; e += GPA_NT) {
        const int s = ent[e] >> 1, side = ent[e] & 1;
        for (int r = sp_start[s]; r < sp_start[s + 1]; ++r)
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[d] += gfull[(size_t)(3 * side + d) * npair + r];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = block_sum<double, GPA_NT>(acc[d], red);
        if (threadIdx.x == 0) g[3 * I + d] += v;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int target_ctas(pcm_ctx *) { return 152 * 8; }

// point blocks of at most ESP_NT*ESP_PPT points spanning at most ESP_MAXCB classes
static void esp_blocks(pcm_ctx *c, std::vector<int> &off)
{
    off.clear();
    const int cap = ESP_NT * ESP_PPT;
    int k = 0;
    // class of point k from the class offsets
    auto cls_of = [&](int kk) {
        return (int)(std::upper_bound(c->h_cls_off.begin(), c->h_cls_off.end(), kk) - c->h_cls_off.begin()) - 1;
    };
    off.push_back(0);
    while (k < c->M) {
        int end = std::min(c->M, k + cap);
        const int c0 = cls_of(k);
        if (cls_of(end - 1) - c0 + 1 > ESP_MAXCB) end = c->h_cls_off[c0 + ESP_MAXCB];
        off.push_back(end);
        k = end;
    }
}

template <int L>
static int launch_esp_class(pcm_ctx *c, PairClass &pc, const int *blk, int nblk, int seg_base, int nseg_cls,
                            int seglen)
{
    if (pc.nesp == 0) return PCM_OK;
    const int k = (int)(&pc - c->cls);
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[k], c->stream));
    dim3 grid(nblk, nseg_cls);
    esp_kernel_f64<L><<<grid, ESP_NT, 0, c->stream>>>(pc.nesp, seglen, pc.eP.p, pc.eD.p, blk, c->px.p, c->py.p,
                                                       c->pz.p, c->pcls.p, c->cls_zeta.p, c->boys64.p, c->M,
                                                       c->esp_part.p + (size_t)seg_base * c->M);
    PCM_LAUNCHED(c);
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_b[k], c->stream));
    return PCM_OK;
}

template <int LA, int LB>
static int esp_prepare_class(pcm_ctx *c, PairClass &pc, const double *dP)
{
    pc.nesp = 0;
    if (pc.npair == 0) return PCM_OK;
    PCM_TRY(c->flags8.alloc(2 * (size_t)pc.npair));
    PCM_TRY(pc.elist.alloc(pc.npair));
    esp_flag_kernel<LA, LB><<<(pc.npair + 127) / 128, 128, 0, c->stream>>>(
        pc.npair, pc.sp.p, pc.ia.p, pc.ib.p, pc.spA.p, pc.spB.p, c->sh_bf.p, c->sh_atom.p, pc.Q.p, dP, c->nbf,
        c->opt.schwarz, c->flags8.p);
    PCM_LAUNCHED(c);
    // same-atom pairs first, then the others, each in pair order
    PCM_TRY(compact_flags(c, c->flags8.p, pc.npair, pc.elist.p, nullptr, c->iscal.p));
    int cnt[2] = {0, 0};
    PCM_CUDA(cudaMemcpyAsync(&cnt[0], c->iscal.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    PCM_TRY(compact_flags(c, c->flags8.p + pc.npair, pc.npair, pc.elist.p + cnt[0], nullptr, c->iscal.p + 1));
    PCM_CUDA(cudaMemcpyAsync(&cnt[1], c->iscal.p + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    const int n = cnt[0] + cnt[1];
    pc.nesp = n;
    pc.nesp_same = cnt[0];
    if (n == 0) return PCM_OK;
    constexpr int NH = nherm(LA + LB);
    PCM_TRY(pc.eP.alloc(4 * (size_t)n));
    PCM_TRY(pc.eD.alloc((size_t)NH * n));
    esp_coef_kernel<LA, LB><<<(n + 127) / 128, 128, 0, c->stream>>>(
        n, pc.elist.p, pc.sp.p, pc.ia.p, pc.ib.p, pc.spA.p, pc.spB.p, c->sh_atom.p, c->sh_off.p, c->sh_bf.p,
        c->cnorm.p, c->xyz.p, pc.Px.p, pc.Py.p, pc.Pz.p, pc.p.p, pc.pref.p, dP, c->nbf, pc.eP.p, pc.eD.p);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

static int esp_class_stats(pcm_ctx *c)
{
    for (int k = 0; k < 6; ++k) {
        c->stats.esp_class_pairs[k] = c->cls[k].nesp;
        c->stats.ms_esp_class[k] = 0.0;
        if (c->have_events && c->cls[k].nesp > 0) {
            float ms = 0.f;
            PCM_CUDA(cudaEventElapsedTime(&ms, c->ev_a[k], c->ev_b[k]));
            c->stats.ms_esp_class[k] = ms;
        }
    }
    return PCM_OK;
}

// density test and Hermite density coefficients of every class
int esp_prepare_all(pcm_ctx *c, const double *dP)
{
    PCM_TRY((esp_prepare_class<0, 0>(c, c->cls[0], dP)));
    PCM_TRY((esp_prepare_class<1, 0>(c, c->cls[1], dP)));
    PCM_TRY((esp_prepare_class<1, 1>(c, c->cls[2], dP)));
    PCM_TRY((esp_prepare_class<2, 0>(c, c->cls[3], dP)));
    PCM_TRY((esp_prepare_class<2, 1>(c, c->cls[4], dP)));
    PCM_TRY((esp_prepare_class<2, 2>(c, c->cls[5], dP)));
    return PCM_OK;
}

int esp_compute(pcm_ctx *c, const double *dP, double *dc)
{
    // A and the preconditioner on the second stream, beside these integrals
    PCM_TRY(ensure_operator(c));
    PCM_TRY(esp_prepare_all(c, dP));

    if (c->opt.precision == PCM_MIXED) {
        long long pesp = 0;
        double ints = 0.0;
        for (int k = 0; k < 6; ++k) {
            pesp += c->cls[k].nesp;
            ints += (double)c->cls[k].nesp * ncart(c->cls[k].la) * ncart(c->cls[k].lb) * c->M;
        }
        c->stats.pairs_esp = pesp;
        c->stats.integrals_esp = ints;
        PCM_TRY(esp_compute_mixed(c, dc));
        return esp_class_stats(c);
    }
    std::vector<int> off;
    esp_blocks(c, off);
    const int nblk = (int)off.size() - 1;
    DBuf<int> &blk = c->si[5];
    PCM_TRY(blk.alloc(off.size()));
    PCM_CUDA(cudaMemcpyAsync(blk.p, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));

    // pair segments per class
    int nseg[6], seglen[6], total = 0;
    long long pesp = 0;
    double ints = 0.0;
    for (int k = 0; k < 6; ++k) {
        PairClass &pc = c->cls[k];
        pesp += pc.nesp;
        ints += (double)pc.nesp * ncart(pc.la) * ncart(pc.lb) * c->M;
        if (pc.nesp == 0) {
            nseg[k] = 0;
            seglen[k] = 0;
            continue;
        }
        const int maxseg = (pc.nesp + ESP_TP - 1) / ESP_TP;
        int ns = std::max(1, std::min(maxseg, (target_ctas(c) + nblk - 1) / nblk));
        int sl = (pc.nesp + ns - 1) / ns;
        sl = (sl + ESP_TP - 1) / ESP_TP * ESP_TP;
        ns = (pc.nesp + sl - 1) / sl;
        nseg[k] = ns;
        seglen[k] = sl;
        total += ns;
    }
    c->stats.pairs_esp = pesp;
    c->stats.integrals_esp = ints;
    if (total == 0) {
        PCM_CUDA(cudaMemsetAsync(dc, 0, c->M * sizeof(double), c->stream));
        return PCM_OK;
    }
    PCM_TRY(c->esp_part.alloc((size_t)total * c->M));
    int base = 0;
    PCM_TRY((launch_esp_class<0>(c, c->cls[0], blk.p, nblk, base, nseg[0], seglen[0])));
    base += nseg[0];
    PCM_TRY((launch_esp_class<1>(c, c->cls[1], blk.p, nblk, base, nseg[1], seglen[1])));
    base += nseg[1];
    PCM_TRY((launch_esp_class<2>(c, c->cls[2], blk.p, nblk, base, nseg[2], seglen[2])));
    base += nseg[2];
    PCM_TRY((launch_esp_class<2>(c, c->cls[3], blk.p, nblk, base, nseg[3], seglen[3])));
    base += nseg[3];
    PCM_TRY((launch_esp_class<3>(c, c->cls[4], blk.p, nblk, base, nseg[4], seglen[4])));
    base += nseg[4];
    PCM_TRY((launch_esp_class<4>(c, c->cls[5], blk.p, nblk, base, nseg[5], seglen[5])));
    base += nseg[5];
    esp_reduce_kernel<<<(c->M + 255) / 256, 256, 0, c->stream>>>(c->M, total, c->esp_part.p, dc);
    PCM_LAUNCHED(c);
    PCM_CUDA(cudaStreamSynchronize(c->stream));  // the class timers are read next
    return esp_class_stats(c);
}

// points of each split and the number of splits for a Fock launch of nb
// pair blocks: enough CTAs to fill the GPU, splits on whole point tiles
static void fock_split(pcm_ctx *c, int nb, int *nsplit, int *ks)
{
    const int maxsplit = std::max(1, (c->M + FOCK_TQ - 1) / FOCK_TQ);
    int ns = std::max(1, std::min(maxsplit, (target_ctas(c) + nb - 1) / nb));
    int k = (c->M + ns - 1) / ns;
    k = (k + FOCK_TQ - 1) / FOCK_TQ * FOCK_TQ;
    *ks = k;
    *nsplit = (c->M + k - 1) / k;
}

// The autotuner's trial for the FP32 Fock kernel of class k: one and two
// pairs per thread, each run once untimed and then timed once; the faster is
// remembered.
static int fock_tune(pcm_ctx *c, int k, int L, const double *dq)
{
    struct NoDefer {
        pcm_ctx *c;
        JobSink *j;
        ~NoDefer() { c->jobs = j; }
    } nd{c, c->jobs};
    c->jobs = nullptr;   // the trials run now, whatever the caller collects
    PairClass &pc = c->cls[k];
    const int bucket = tune_bucket(pc.npair);
    const int kind = c->opt.fp32x2 ? TUNE_FOCK_NPT : TUNE_FOCK_NPT_SCALAR;
    if (tune_get(c->device, kind, L, bucket) >= 0) return PCM_OK;
    float ms[2] = {0.f, 0.f};
    cudaEvent_t e0, e1;
    PCM_CUDA(cudaEventCreate(&e0));
    PCM_CUDA(cudaEventCreate(&e1));
    int st = PCM_OK;
    for (int npt = 1; npt <= 2 && st == PCM_OK; ++npt) {
        const int nb = (pc.npair + FOCK_NT * npt - 1) / (FOCK_NT * npt);
        int nsplit, ks;
        fock_split(c, nb, &nsplit, &ks);
        st = c->fock_W.alloc((size_t)nsplit * nherm(L) * pc.npair);
        if (st != PCM_OK) break;
        // an untimed run first (first-use allocations and code loading)
        st = fock_mixed_class(c, k, dq, nsplit, ks, c->fock_W.p, npt);
        if (st == PCM_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_last_error("autotuner: a Fock trial failed");
            st = PCM_ERR_CUDA;
        }
        if (st != PCM_OK) break;
        cudaEventRecord(e0, c->stream);
        st = fock_mixed_class(c, k, dq, nsplit, ks, c->fock_W.p, npt);
        cudaEventRecord(e1, c->stream);
        if (st == PCM_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms[npt - 1], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PCM_OK) return st;
    tune_set(c->device, kind, L, bucket, ms[1] < ms[0] ? 2 : 1, ms[0], ms[1]);
    return PCM_OK;
}

template <int LA, int LB>
static void fock_epilogue(pcm_ctx *c, PairClass &pc, int nsplit, const double *W, double *ddF)
{
    fock_epilogue_kernel<LA, LB><<<(pc.nsp + 127) / 128, 128, 0, c->stream>>>(
        pc.nsp, pc.npair, nsplit, pc.spA.p, pc.spB.p, pc.sp_start.p, pc.ia.p, pc.ib.p, c->sh_atom.p, c->sh_off.p,
        c->sh_bf.p, c->cnorm.p, c->xyz.p, pc.Px.p, pc.Py.p, pc.Pz.p, pc.p.p, pc.pref.p, W, c->nbf, ddF);
}

// the Fock epilogues a batch deferred until its packed blocks had run
int fock_mixed_finish(pcm_ctx *c, double *ddF)
{
    for (int k = 0; k < 6; ++k) {
        if (!c->fock_pending[k]) continue;
        c->fock_pending[k] = false;
        PairClass &pc = c->cls[k];
        const double *W = c->fock_Wk[k].p;
        const int ns = c->fock_nsplit_k[k];
        switch (k) {
        case 0: fock_epilogue<0, 0>(c, pc, ns, W, ddF); break;
        case 1: fock_epilogue<1, 0>(c, pc, ns, W, ddF); break;
        case 2: fock_epilogue<1, 1>(c, pc, ns, W, ddF); break;
        case 3: fock_epilogue<2, 0>(c, pc, ns, W, ddF); break;
        case 4: fock_epilogue<2, 1>(c, pc, ns, W, ddF); break;
        case 5: fock_epilogue<2, 2>(c, pc, ns, W, ddF); break;
        }
        PCM_LAUNCHED(c);
    }
    return PCM_OK;
}

template <int LA, int LB>
static int fock_class(pcm_ctx *c, PairClass &pc, const double *dq, double *ddF)
{
    constexpr int L = LA + LB;
    constexpr int NH = nherm(L);
    if (pc.nsp == 0) return PCM_OK;
    int nsplit = 1;
    const int kk = (int)(&pc - c->cls);
    // a batch collects the packed blocks of every molecule and runs the
    // epilogue afterwards (fock_mixed_finish), with one W per class
    const bool defer = c->jobs && c->opt.precision == PCM_MIXED && c->opt.fp32x2;
    if (pc.npair > 0) {
        const bool mixed = c->opt.precision == PCM_MIXED;
        const int k = kk;
        if (mixed && c->opt.autotune) PCM_TRY(fock_tune(c, k, L, dq));
        const int npt = mixed ? fock_mixed_pairs_per_thread(c, L, pc.npair) : 1;
        const int nb = (pc.npair + FOCK_NT * npt - 1) / (FOCK_NT * npt);
        int ks;
        fock_split(c, nb, &nsplit, &ks);
        if (defer) {
            PCM_TRY(c->fock_Wk[k].alloc((size_t)nsplit * NH * pc.npair));
            PCM_TRY(fock_mixed_class(c, k, dq, nsplit, ks, c->fock_Wk[k].p, npt));
            c->fock_nsplit_k[k] = nsplit;
            c->fock_pending[k] = true;
            c->stats.integrals_fock += (double)pc.npair * ncart(LA) * ncart(LB) * c->M;
            return PCM_OK;
        }
        PCM_TRY(c->fock_W.alloc((size_t)nsplit * NH * pc.npair));
        dim3 grid(nb, nsplit);
        if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[6 + k], c->stream));
        if (mixed) {
            PCM_TRY(fock_mixed_class(c, k, dq, nsplit, ks, c->fock_W.p, npt));
        } else {
            fock_kernel_f64<L><<<grid, FOCK_NT, 0, c->stream>>>(pc.npair, pc.Px.p, pc.Py.p, pc.Pz.p, pc.p.p, ks,
                                                                 c->px.p, c->py.p, c->pz.p, dq, c->M, c->ncls,
                                                                 c->cls_off.p, c->cls_zeta.p, c->boys64.p,
                                                                 c->fock_W.p);
            PCM_LAUNCHED(c);
        }
        if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_b[6 + k], c->stream));
    }
    if (defer) {
        // no kept pairs: the epilogue writes the class's zero blocks
        PCM_TRY(c->fock_Wk[kk].alloc(1));
        c->fock_nsplit_k[kk] = nsplit;
        c->fock_pending[kk] = true;
        return PCM_OK;
    }
    fock_epilogue<LA, LB>(c, pc, nsplit, c->fock_W.p, ddF);
    PCM_LAUNCHED(c);
    c->stats.integrals_fock += (double)pc.npair * ncart(LA) * ncart(LB) * c->M;
    return PCM_OK;
}

int fock_compute(pcm_ctx *c, const double *dq, double *ddF)
{
    c->stats.integrals_fock = 0.0;
    PCM_TRY((fock_class<0, 0>(c, c->cls[0], dq, ddF)));
    PCM_TRY((fock_class<1, 0>(c, c->cls[1], dq, ddF)));
    PCM_TRY((fock_class<1, 1>(c, c->cls[2], dq, ddF)));
    PCM_TRY((fock_class<2, 0>(c, c->cls[3], dq, ddF)));
    PCM_TRY((fock_class<2, 1>(c, c->cls[4], dq, ddF)));
    PCM_TRY((fock_class<2, 2>(c, c->cls[5], dq, ddF)));
    if (c->jobs) return PCM_OK;
    if (c->have_events) PCM_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 6; ++k) {
        c->stats.fock_class_pairs[k] = c->cls[k].npair;
        c->stats.ms_fock_class[k] = 0.0;
        if (c->have_events && c->cls[k].npair > 0) {
            float ms = 0.f;
            PCM_CUDA(cudaEventElapsedTime(&ms, c->ev_a[6 + k], c->ev_b[6 + k]));
            c->stats.ms_fock_class[k] = ms;
        }
    }
    return PCM_OK;
}

// ---------------------------------------------------------------------------
// integral part of the gradient (host side)
// ---------------------------------------------------------------------------
// shell pairs of a class listed by atom: for atom I, entries 2 s (atom of A is
// I) and 2 s + 1 (atom of B is I), in increasing s
static int pair_csr(pcm_ctx *c, PairClass &pc)
{
    if (pc.csr_ready) return PCM_OK;
    const int natom = c->natom;
    std::vector<int> off(natom + 1, 0), ent(2 * (size_t)pc.nsp);
    for (int s = 0; s < pc.nsp; ++s) {
        ++off[c->h_sh_atom[pc.h_spA[s]] + 1];
        ++off[c->h_sh_atom[pc.h_spB[s]] + 1];
    }
    for (int I = 0; I < natom; ++I) off[I + 1] += off[I];
    std::vector<int> pos(off.begin(), off.end() - 1);
    for (int s = 0; s < pc.nsp; ++s) {
        ent[pos[c->h_sh_atom[pc.h_spA[s]]]++] = 2 * s;
        ent[pos[c->h_sh_atom[pc.h_spB[s]]]++] = 2 * s + 1;
    }
    PCM_TRY(pc.csr_off.alloc(natom + 1));
    PCM_TRY(pc.csr_ent.alloc(ent.size()));
    PCM_CUDA(cudaMemcpyAsync(pc.csr_off.p, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (!ent.empty())
        PCM_CUDA(cudaMemcpyAsync(pc.csr_ent.p, ent.data(), ent.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    pc.csr_ready = true;
    return PCM_OK;
}

template <int L>
static void launch_esp_grad(pcm_ctx *c, PairClass &pc, const int *blk, int nblk, int seg_base, int nseg_cls,
                            int seglen)
{
    dim3 grid(nblk, nseg_cls);
    esp_grad_kernel<L><<<grid, ESP_NT, 0, c->stream>>>(pc.nesp, seglen, pc.eP.p, pc.eD.p, blk, c->px.p, c->py.p,
                                                        c->pz.p, c->pcls.p, c->cls_zeta.p, c->boys64.p, c->M,
                                                        c->esp_part.p + (size_t)seg_base * 3 * c->M);
}

template <int LA, int LB>
static int grad_pair_class(pcm_ctx *c, PairClass &pc, const double *dP, const double *dq, double *gpair)
{
    constexpr int L1 = LA + LB + 1;
    constexpr int NH1 = nherm(L1);
    if (pc.nesp == 0) return PCM_OK;
    const int n = pc.nesp;
    const int npt = c->opt.precision == PCM_MIXED ? fock_mixed_pairs_per_thread(c, L1, n) : 1;
    const int nb = (n + FOCK_NT * npt - 1) / (FOCK_NT * npt);
    int nsplit, ks;
    fock_split(c, nb, &nsplit, &ks);
    PCM_TRY(c->fock_W.alloc((size_t)nsplit * NH1 * n));
    if (c->opt.precision == PCM_MIXED) {
        PCM_TRY(grad_w_mixed(c, (int)(&pc - c->cls), dq, nsplit, ks, c->fock_W.p, npt));
    } else {
        dim3 grid(nb, nsplit);
        fock_kernel_f64<L1><<<grid, FOCK_NT, 0, c->stream>>>(n, pc.eP.p, pc.eP.p + n, pc.eP.p + 2 * (size_t)n,
                                                              pc.eP.p + 3 * (size_t)n, ks, c->px.p, c->py.p, c->pz.p,
                                                              dq, c->M, c->ncls, c->cls_off.p, c->cls_zeta.p,
                                                              c->boys64.p, c->fock_W.p);
        PCM_LAUNCHED(c);
    }
    PCM_TRY(c->g_full.alloc(6 * (size_t)pc.npair));
    PCM_CUDA(cudaMemsetAsync(c->g_full.p, 0, 6 * (size_t)pc.npair * sizeof(double), c->stream));
    grad_pair_kernel<LA, LB><<<(n + 127) / 128, 128, 0, c->stream>>>(
        n, pc.npair, nsplit, pc.elist.p, pc.sp.p, pc.ia.p, pc.ib.p, pc.spA.p, pc.spB.p, c->sh_atom.p, c->sh_off.p,
        c->sh_bf.p, c->exps.p, c->cnorm.p, c->xyz.p, pc.Px.p, pc.Py.p, pc.Pz.p, pc.p.p, pc.pref.p, dP, c->nbf,
        c->fock_W.p, c->g_full.p);
    PCM_LAUNCHED(c);
    PCM_TRY(pair_csr(c, pc));
    pair_atom_reduce_kernel<<<c->natom, GPA_NT, 0, c->stream>>>(c->natom, pc.csr_off.p, pc.csr_ent.p, pc.sp_start.p,
                                                                pc.npair, c->g_full.p, gpair);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

static int grad_pair_all(pcm_ctx *c, const double *dP, const double *dq, double *gpair)
{
    PCM_TRY((grad_pair_class<0, 0>(c, c->cls[0], dP, dq, gpair)));
    PCM_TRY((grad_pair_class<1, 0>(c, c->cls[1], dP, dq, gpair)));
    PCM_TRY((grad_pair_class<1, 1>(c, c->cls[2], dP, dq, gpair)));
    PCM_TRY((grad_pair_class<2, 0>(c, c->cls[3], dP, dq, gpair)));
    PCM_TRY((grad_pair_class<2, 1>(c, c->cls[4], dP, dq, gpair)));
    PCM_TRY((grad_pair_class<2, 2>(c, c->cls[5], dP, dq, gpair)));
    return PCM_OK;
}

// gk (3 x M): += the point part, -q_k d c_k / dC_k; gpair (natom x 3): += the
// bra/ket-centre parts.  PCM_FP64: FP64 throughout; PCM_MIXED: the point part
// and the W accumulation on the FP32 pipes (FP64 across tiles and segments),
// the per-pair contraction and every reduction in FP64.
int grad_integrals(pcm_ctx *c, const double *dP, const double *dq, double *gk, double *gpair)
{
    PCM_TRY(esp_prepare_all(c, dP));
    if (c->opt.precision == PCM_MIXED) {
        double ints = 0.0;
        for (int k = 0; k < 6; ++k)
            ints += (double)c->cls[k].nesp * ncart(c->cls[k].la) * ncart(c->cls[k].lb) * c->M;
        c->stats.integrals_grad = 2.0 * ints;
        int total = 0;
        PCM_TRY(grad_point_mixed(c, &total));
        if (total > 0) {
            grad_point_reduce_kernel<<<(c->M + 255) / 256, 256, 0, c->stream>>>(c->M, total, c->esp_part.p, dq,
                                                                                  gk);
            PCM_LAUNCHED(c);
        }
        return grad_pair_all(c, dP, dq, gpair);
    }
    std::vector<int> off;
    esp_blocks(c, off);
    const int nblk = (int)off.size() - 1;
    DBuf<int> &blk = c->si[5];
    PCM_TRY(blk.alloc(off.size()));
    PCM_CUDA(cudaMemcpyAsync(blk.p, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    int nseg[6], seglen[6], total = 0;
    double ints = 0.0;
    for (int k = 0; k < 6; ++k) {
        PairClass &pc = c->cls[k];
        nseg[k] = seglen[k] = 0;
        if (pc.nesp == 0) continue;
        ints += (double)pc.nesp * ncart(pc.la) * ncart(pc.lb) * c->M;
        const int maxseg = (pc.nesp + ESP_TP - 1) / ESP_TP;
        int ns = std::max(1, std::min(maxseg, (target_ctas(c) + nblk - 1) / nblk));
        int sl = (pc.nesp + ns - 1) / ns;
        sl = (sl + ESP_TP - 1) / ESP_TP * ESP_TP;
        nseg[k] = (pc.nesp + sl - 1) / sl;
        seglen[k] = sl;
        total += nseg[k];
    }
    c->stats.integrals_grad = 2.0 * ints;
    if (total > 0) {
        PCM_TRY(c->esp_part.alloc((size_t)total * 3 * c->M));
        int base = 0;
        static const int LSUM[6] = {0, 1, 2, 2, 3, 4};
        for (int k = 0; k < 6; ++k) {
            PairClass &pc = c->cls[k];
            if (nseg[k] == 0) continue;
            switch (LSUM[k]) {
            case 0: launch_esp_grad<0>(c, pc, blk.p, nblk, base, nseg[k], seglen[k]); break;
            case 1: launch_esp_grad<1>(c, pc, blk.p, nblk, base, nseg[k], seglen[k]); break;
            case 2: launch_esp_grad<2>(c, pc, blk.p, nblk, base, nseg[k], seglen[k]); break;
            case 3: launch_esp_grad<3>(c, pc, blk.p, nblk, base, nseg[k], seglen[k]); break;
            case 4: launch_esp_grad<4>(c, pc, blk.p, nblk, base, nseg[k], seglen[k]); break;
            }
            PCM_LAUNCHED(c);
            base += nseg[k];
        }
        grad_point_reduce_kernel<<<(c->M + 255) / 256, 256, 0, c->stream>>>(c->M, total, c->esp_part.p, dq, gk);
        PCM_LAUNCHED(c);
    }
    return grad_pair_all(c, dP, dq, gpair);
}

}  // namespace pcm
