// Shared device helpers for the C-PCM / ISWIG kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef PCM_PI
#define PCM_PI 3.141592653589793238462643383279502884
#endif

namespace pcm {

// ---------------------------------------------------------------------------
// Hermite index bookkeeping.  Hermite components (t, u, v) with t+u+v <= L are
// stored in one canonical order: by total degree n = t+u+v, then t descending,
// then u descending.  nherm(L) = (L+1)(L+2)(L+3)/6.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// position of (t,u,v) in the order above
__host__ __device__ constexpr int hidx(int t, int u, int v)
{
    // components of lower total degree come first
    return nherm(t + u + v - 1) +
           // within degree n: t descending, then u descending
           ((t + u + v) - t) * ((t + u + v) - t + 1) / 2 + ((t + u + v) - t - u);
}
// nherm(-1) must be 0
static_assert(nherm(-1) == 0, "nherm(-1)");
static_assert(hidx(0, 0, 0) == 0 && hidx(1, 0, 0) == 1 && hidx(0, 1, 0) == 2 && hidx(0, 0, 1) == 3, "hidx");
static_assert(hidx(2, 0, 0) == 4 && hidx(0, 0, 2) == 9 && hidx(0, 0, 4) == 34, "hidx");

// Cartesian component `c` of shell l in the order x^l, x^(l-1)y, x^(l-1)z, ..., z^l.
__host__ __device__ inline void cart_xyz(int l, int c, int &lx, int &ly, int &lz)
{
    int n = 0;
    for (int a = l; a >= 0; --a)
        for (int b = l - a; b >= 0; --b) {
            if (n == c) { lx = a; ly = b; lz = l - a - b; return; }
            ++n;
        }
    lx = ly = lz = 0;
}

// ---------------------------------------------------------------------------
// McMurchie-Davidson Hermite Coulomb integrals R_tuv (t+u+v <= L) from
// Rn[n] = (-2 rho)^n F_n(rho R^2) and the vector P - C = (X, Y, Z):
//   R^(n)_{t+1,u,v} = t R^(n+1)_{t-1,u,v} + X R^(n+1)_{t,u,v}   (and y, z).
// Fully unrolled for compile-time L so every array stays in registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float hmadd(float a, float b, float c) { return fmaf(a, b, c); }

template <int L, typename T>
__device__ __forceinline__ void hermite_R(T X, T Y, T Z, const T (&Rn)[L + 1], T (&R)[nherm(L)])
{
    // buf holds R^(n) for t+u+v <= L-n, rebuilt for n = L .. 0
    T buf[nherm(L)];
#pragma unroll
    for (int i = 0; i < nherm(L); ++i) buf[i] = T(0);
#pragma unroll
    for (int n = L; n >= 0; --n) {
        const int D = L - n;
        T nb[nherm(L)];
#pragma unroll
        for (int i = 0; i < nherm(L); ++i) nb[i] = T(0);
#pragma unroll
        for (int d = 0; d <= D; ++d)
#pragma unroll
            for (int t = d; t >= 0; --t)
#pragma unroll
                for (int u = d - t; u >= 0; --u) {
                    const int v = d - t - u;
                    T val;
                    if (d == 0) {
                        val = Rn[n];
                    } else if (t > 0) {
                        val = X * buf[hidx(t - 1, u, v)];
                        if (t > 1) val = hmadd(T(t - 1), buf[hidx(t - 2, u, v)], val);
                    } else if (u > 0) {
                        val = Y * buf[hidx(t, u - 1, v)];
                        if (u > 1) val = hmadd(T(u - 1), buf[hidx(t, u - 2, v)], val);
                    } else {
                        val = Z * buf[hidx(t, u, v - 1)];
                        if (v > 1) val = hmadd(T(v - 1), buf[hidx(t, u, v - 2)], val);
                    }
                    nb[hidx(t, u, v)] = val;
                }
#pragma unroll
        for (int i = 0; i < nherm(L); ++i) buf[i] = nb[i];
    }
#pragma unroll
    for (int i = 0; i < nherm(L); ++i) R[i] = buf[i];
}

// Hermite expansion coefficients E^{ij}_t of one Cartesian direction for
// i <= la, j <= lb (without the Gaussian-product prefactor K, which the
// callers carry separately):
//   E^{00}_0 = 1
//   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
//   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}
// E[i][j][t] laid out with fixed strides for lmax = 3.
struct E1D {
    double e[4][4][7];
};

__device__ inline void hermite_E1D(int la, int lb, double PA, double PB, double inv2p, E1D &E)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int t = 0; t < 7; ++t) E.e[i][j][t] = 0.0;
    E.e[0][0][0] = 1.0;
    for (int i = 0; i <= la; ++i) {
        if (i > 0) {
            for (int t = 0; t <= i; ++t) {
                double v = PA * E.e[i - 1][0][t];
                if (t > 0) v += inv2p * E.e[i - 1][0][t - 1];
                if (t + 1 <= i - 1) v += (t + 1) * E.e[i - 1][0][t + 1];
                E.e[i][0][t] = v;
            }
        }
        for (int j = 1; j <= lb; ++j)
            for (int t = 0; t <= i + j; ++t) {
                double v = PB * E.e[i][j - 1][t];
                if (t > 0) v += inv2p * E.e[i][j - 1][t - 1];
                if (t + 1 <= i + j - 1) v += (t + 1) * E.e[i][j - 1][t + 1];
                E.e[i][j][t] = v;
            }
    }
}

// Compile-time Cartesian exponents (l <= 3) in the order above, so that fully
// unrolled component loops index register arrays with constants.
__host__ __device__ constexpr int cart_e(int l, int c, int axis)
{
    // rows: x^l, x^(l-1) y, x^(l-1) z, ..., z^l
    int n = 0;
    for (int a = l; a >= 0; --a)
        for (int b = l - a; b >= 0; --b) {
            if (n == c) return axis == 0 ? a : (axis == 1 ? b : l - a - b);
            ++n;
        }
    return 0;
}
static_assert(cart_e(2, 1, 0) == 1 && cart_e(2, 1, 1) == 1 && cart_e(2, 4, 2) == 1 && cart_e(2, 5, 2) == 2, "cart_e");

// Hermite expansion coefficients of one direction, sized for (LA, LB) and
// fully unrolled (registers): same recurrences as hermite_E1D.
template <int LA, int LB, typename T = double>
struct E1T {
    T e[LA + 1][LB + 1][LA + LB + 1];
};

template <int LA, int LB, typename T = double>
__device__ __forceinline__ void hermite_E1T(T PA, T PB, T inv2p, E1T<LA, LB, T> &E)
{
#pragma unroll
    for (int i = 0; i <= LA; ++i)
#pragma unroll
        for (int j = 0; j <= LB; ++j)
#pragma unroll
            for (int t = 0; t <= LA + LB; ++t) E.e[i][j][t] = T(0);
    E.e[0][0][0] = T(1);
#pragma unroll
    for (int i = 0; i <= LA; ++i) {
        if (i > 0) {
#pragma unroll
            for (int t = 0; t <= i; ++t) {
                T v = PA * E.e[i - 1][0][t];
                if (t > 0) v += inv2p * E.e[i - 1][0][t - 1];
                if (t + 1 <= i - 1) v += T(t + 1) * E.e[i - 1][0][t + 1];
                E.e[i][0][t] = v;
            }
        }
#pragma unroll
        for (int j = 1; j <= LB; ++j)
#pragma unroll
            for (int t = 0; t <= i + j; ++t) {
                T v = PB * E.e[i][j - 1][t];
                if (t > 0) v += inv2p * E.e[i][j - 1][t - 1];
                if (t + 1 <= i + j - 1) v += T(t + 1) * E.e[i][j - 1][t + 1];
                E.e[i][j][t] = v;
            }
    }
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (deterministic); result valid in thread 0.
template <typename T, int NT>
__device__ __forceinline__ T block_sum(T v, T *smem /* NT/32 entries */)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[w] = v;
    __syncthreads();
    T r = T(0);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) r += smem[i];
    }
    __syncthreads();
    return r;
}

}  // namespace pcm
