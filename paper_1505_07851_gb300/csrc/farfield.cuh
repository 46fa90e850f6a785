// Far-field form of the McMurchie-Davidson Coulomb integrals.
//
// For T = rho R^2 beyond a threshold the Boys function equals its asymptotic
// form F_n(T) = (2n-1)!! / (2T)^n * sqrt(pi) / (2 sqrt(T)) up to a relative
// error below 1e-10 (the neglected part is the tail of the integral beyond
// u = 1, about e^-T 2^n T^(n-1/2) / ((2n-1)!! sqrt(pi)) of F_n).  There
//   U (-2 rho)^n F_n(rho R^2) = sqrt(pi) / (2 sqrt(p)) (-1)^n (2n-1)!! / R^(2n+1)
// because U / sqrt(rho) = 1 / sqrt(p): the point's exponent zeta_k cancels and
// every Hermite integral R_tuv becomes sqrt(pi)/(2 sqrt(p)) times the
// derivative d^t/dX d^u/dY d^v/dZ of 1/R, the field of a point charge.  The
// Hermite recurrence has the closed form
//   R_tuv = sum_ijk h(t,i) h(u,j) h(v,k) X^(t-2i) Y^(u-2j) Z^(v-2k) Rn[t+u+v-i-j-k],
//   h(t,i) = t! / (i! (t-2i)! 2^i),
// so a Hermite density D_tuv contracts to sum_n Rn[n] Q_n(X, Y, Z) with
// polynomials Q_n whose coefficients are fixed per primitive pair.  With
// Rn[n] = (-1)^n (2n-1)!! R^-(2n+1) the sign and the double factorial move
// into those coefficients too, and the far-field interaction is
//   sum_n R^-(2n+1) Q_n(X, Y, Z),
// evaluated per pair-point interaction from 1/R alone.
#pragma once
#include "common.cuh"

namespace pcm {

// smallest T at which the asymptotic form holds to 1e-10 relative for F_0..F_m
__host__ __device__ constexpr float far_T(int m)
{
    return m <= 1 ? 25.f : (m == 2 ? 30.f : (m == 3 ? 32.f : (m == 4 ? 34.f : 36.f)));
}

// terms (n; a, b, c) of the polynomials Q_n: the monomial X^a Y^b Z^c of
// degree d = a+b+c appears in Q_n when d <= n and 2n - d <= L
__host__ __device__ constexpr int far_nterms(int L)
{
    int cnt = 0;
    for (int n = 0; n <= L; ++n)
        for (int d = 0; d <= n; ++d)
            if (2 * n - d <= L) cnt += (d + 1) * (d + 2) / 2;
    return cnt;
}

struct FarTerms {
    int n[64], a[64], b[64], c[64];
    int count;
};

__host__ __device__ constexpr FarTerms far_terms(int L)
{
    FarTerms T{};
    int k = 0;
    for (int n = 0; n <= L; ++n)
        for (int d = 0; d <= n; ++d) {
            if (2 * n - d > L) continue;
            for (int a = d; a >= 0; --a)
                for (int b = d - a; b >= 0; --b) {
                    T.n[k] = n;
                    T.a[k] = a;
                    T.b[k] = b;
                    T.c[k] = d - a - b;
                    ++k;
                }
        }
    T.count = k;
    return T;
}

__host__ __device__ constexpr double herm_h(int t, int i)
{
    // t! / (i! (t-2i)! 2^i)
    double f = 1.0;
    for (int x = 2; x <= t; ++x) f *= x;
    double g = 1.0;
    for (int x = 2; x <= i; ++x) g *= x;
    double r = 1.0;
    for (int x = 2; x <= t - 2 * i; ++x) r *= x;
    double p2 = 1.0;
    for (int x = 0; x < i; ++x) p2 *= 2.0;
    return f / (g * r * p2);
}

__host__ __device__ constexpr double dfact_odd(int n)
{
    // (2n - 1)!!, 1 for n = 0
    double r = 1.0;
    for (int x = 2 * n - 1; x > 1; x -= 2) r *= x;
    return r;
}

// contributions of the Hermite density components to the terms:
// coef[term] += w * D[hidx(t, u, v)], with the sign (-1)^n and (2n-1)!! included
struct FarContrib {
    int term[320], h[320];
    double w[320];
    int count;
};

__host__ __device__ constexpr FarContrib far_contrib(int L)
{
    FarContrib C{};
    const FarTerms T = far_terms(L);
    int q = 0;
    for (int k = 0; k < T.count; ++k) {
        const int n = T.n[k], a = T.a[k], b = T.b[k], c = T.c[k];
        const int m = n - (a + b + c);
        const double sgn = (n % 2) ? -1.0 : 1.0;
        for (int i = 0; i <= m; ++i)
            for (int j = 0; j <= m - i; ++j) {
                const int l = m - i - j;
                const int t = a + 2 * i, u = b + 2 * j, v = c + 2 * l;
                C.term[q] = k;
                C.h[q] = hidx(t, u, v);
                C.w[q] = sgn * dfact_odd(n) * herm_h(t, i) * herm_h(u, j) * herm_h(v, l);
                ++q;
            }
    }
    C.count = q;
    return C;
}

// exponents (a, b, c) of the monomial at Hermite index i (degree order, then
// a descending, then b descending), for index i < nherm(L)
struct MonoTab {
    int a[84], b[84], c[84];
};

__host__ __device__ constexpr MonoTab mono_tab(int L)
{
    MonoTab M{};
    for (int d = 0; d <= L; ++d)
        for (int a = d; a >= 0; --a)
            for (int b = d - a; b >= 0; --b) {
                const int i = hidx(a, b, d - a - b);
                M.a[i] = a;
                M.b[i] = b;
                M.c[i] = d - a - b;
            }
    return M;
}

static_assert(far_nterms(0) == 1 && far_nterms(1) == 4 && far_nterms(2) == 11 && far_nterms(3) == 24 &&
                  far_nterms(4) == 46,
              "far_nterms");
static_assert(far_terms(4).count == 46, "far_terms");

}  // namespace pcm
