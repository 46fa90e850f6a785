/*
 * ORACLE -- test infrastructure only.  Plain, slow FP64 reference for the
 * erf-screened one-electron integrals of the C-PCM/ISWIG model.  Only the
 * tests, the package's smoke check and the benchmark's CPU-baseline leg use
 * it; the CUDA library shares no code with it and never calls it.
 *
 * What it computes (all in atomic units):
 *   [chi_a | J_k | chi_b] = \int chi_a(r) erf(zeta_k |r - r_k|) / |r - r_k| chi_b(r) dr
 * over raw Cartesian Gaussians chi = x_A^ax y_A^ay z_A^az exp(-alpha r_A^2)
 * (Eq. 6 and Eq. 12 of the paper), contracted over normalised primitives
 * (Eq. 11), and the two contractions of Section 2:
 *   c_k        = sum_{mu nu} P_{mu nu} L^k_{mu nu},  L^k = -(mu|J_k|nu)   (Eq. 5, Eq. 6)
 *   dF_{mu nu} = sum_k q_k L^k_{mu nu}                                  (Eq. 10)
 *
 * Method: Obara-Saika vertical (VRR) and horizontal (HRR) recurrences for
 * nuclear-attraction integrals, with every auxiliary Boys value F_m(T)
 * replaced by its erf-attenuated form.  With p = alpha + beta and
 * U^2 = zeta^2 / (p + zeta^2), the attenuated operator restricts the
 * Gaussian-transform variable u to [0, U] instead of [0, 1], so the
 * auxiliary integrals become
 *   Theta^(m)_00 = (2 pi / p) K_AB \int_0^U u^{2m} exp(-p R_PC^2 u^2) du
 *                = (2 pi / p) K_AB U^{2m+1} F_m(U^2 p R_PC^2)
 * and the recurrences keep their point-charge form.  zeta = +inf gives the
 * ordinary point-charge nuclear attraction integrals (U = 1).
 *
 * Gradient (Eq. 14, Eq. 22): the derivative of sum_k q_k c_k with respect
 * to the nuclear positions at fixed P.  Each integral depends on the centre
 * of chi_a (the atom of its shell), the centre of chi_b and the point r_k,
 * which moves with the atom of its sphere.  The centre derivatives follow
 * from differentiating the primitive itself,
 *   d/dA_x [x_A^ax ... exp(-alpha r_A^2)] = 2 alpha G_{a+1_x} - ax G_{a-1_x},
 * and the point derivative from translational invariance,
 *   d/dC = -(d/dA + d/dB).
 *
 * Boys function: the series e^-T sum_i (2T)^i / ((2m+1)(2m+3)...(2m+2i+1))
 * for T < 30, else F_0 = (1/2) sqrt(pi/T) erf(sqrt T) and upward recursion.
 * No screening of any kind is applied.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_LMAX 3                     /* per shell: s, p, d, f */
#define ORACLE_LPAIR (2 * ORACLE_LMAX)

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Boys function F_m(T) = \int_0^1 u^{2m} exp(-T u^2) du, m = 0..mmax. */
void oracle_boys(int mmax, double T, double *F)
{
    if (T < 30.0) {
        for (int m = 0; m <= mmax; m++) {
            double term = 1.0 / (2 * m + 1), sum = term;
            for (int i = 1; i < 2000; i++) {
                term *= 2.0 * T / (2 * m + 2 * i + 1);
                sum += term;
                if (term < 1e-18 * sum) break;
            }
            F[m] = exp(-T) * sum;
        }
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

int oracle_ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents of component `idx` of shell l, in the order
 * x^l, x^(l-1)y, x^(l-1)z, ..., z^l (d: xx, xy, xz, yy, yz, zz). */
static void cart_exponents(int l, int idx, int e[3])
{
    int n = 0;
    for (int lx = l; lx >= 0; lx--)
        for (int ly = l - lx; ly >= 0; ly--) {
            if (n == idx) { e[0] = lx; e[1] = ly; e[2] = l - lx - ly; return; }
            n++;
        }
}

static double dfact(int n) /* (n)!! with (-1)!! = 1 */
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

/* Normalisation of the Cartesian primitive x^lx y^ly z^lz exp(-a r^2):
 * each Cartesian component is normalised to unit self-overlap. */
double oracle_norm(double a, int lx, int ly, int lz)
{
    int L = lx + ly + lz;
    return pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * L) /
           sqrt(dfact(2 * lx - 1) * dfact(2 * ly - 1) * dfact(2 * lz - 1));
}

typedef struct {
    int L;                       /* la + lb */
    double PA[3], PC[3], AB[3], inv2p;
    double base[ORACLE_LPAIR + 1];
    double memo[(ORACLE_LPAIR + 1) * (ORACLE_LPAIR + 1) * (ORACLE_LPAIR + 1) * (ORACLE_LPAIR + 2)];
    unsigned char have[(ORACLE_LPAIR + 1) * (ORACLE_LPAIR + 1) * (ORACLE_LPAIR + 1) * (ORACLE_LPAIR + 2)];
} os_ctx;

static int os_idx(const os_ctx *c, int ax, int ay, int az, int m)
{
    int n = c->L + 1;
    return ((ax * n + ay) * n + az) * (n + 1) + m;
}

/* VRR: Theta^(m)_{a+1_i,0} = PA_i Theta^(m)_{a,0} - PC_i Theta^(m+1)_{a,0}
 *                           + a_i/(2p) (Theta^(m)_{a-1_i,0} - Theta^(m+1)_{a-1_i,0}) */
static double vrr(os_ctx *c, int ax, int ay, int az, int m)
{
    if (ax == 0 && ay == 0 && az == 0) return c->base[m];
    int id = os_idx(c, ax, ay, az, m);
    if (c->have[id]) return c->memo[id];
    int a[3] = {ax, ay, az};
    int i = ax > 0 ? 0 : (ay > 0 ? 1 : 2);
    a[i] -= 1;
    double v = c->PA[i] * vrr(c, a[0], a[1], a[2], m) - c->PC[i] * vrr(c, a[0], a[1], a[2], m + 1);
    if (a[i] > 0) {
        int b[3] = {a[0], a[1], a[2]};
        b[i] -= 1;
        v += a[i] * c->inv2p * (vrr(c, b[0], b[1], b[2], m) - vrr(c, b[0], b[1], b[2], m + 1));
    }
    c->have[id] = 1;
    c->memo[id] = v;
    return v;
}

/* HRR: Theta_{a,b+1_j} = Theta_{a+1_j,b} + AB_j Theta_{a,b}, AB = A - B. */
static double hrr(os_ctx *c, const int a[3], const int b[3])
{
    if (b[0] == 0 && b[1] == 0 && b[2] == 0) return vrr(c, a[0], a[1], a[2], 0);
    int j = b[0] > 0 ? 0 : (b[1] > 0 ? 1 : 2);
    int b1[3] = {b[0], b[1], b[2]};
    int a1[3] = {a[0], a[1], a[2]};
    b1[j] -= 1;
    a1[j] += 1;
    return hrr(c, a1, b1) + c->AB[j] * hrr(c, a, b1);
}

/* Raw primitive block [chi_a | J | chi_b] for all Cartesian components,
 * out[ia * ncart(lb) + ib].  zeta <= 0 or +inf selects the point charge. */
void oracle_prim(int la, double alpha, const double *A, int lb, double beta, const double *B,
                 const double *C, double zeta, double *out)
{
    os_ctx ctx, *c = &ctx;
    double p = alpha + beta;
    double P[3], ab2 = 0.0, pc2 = 0.0;
    for (int i = 0; i < 3; i++) {
        P[i] = (alpha * A[i] + beta * B[i]) / p;
        c->PA[i] = P[i] - A[i];
        c->PC[i] = P[i] - C[i];
        c->AB[i] = A[i] - B[i];
        ab2 += c->AB[i] * c->AB[i];
        pc2 += c->PC[i] * c->PC[i];
    }
    c->L = la + lb;
    c->inv2p = 0.5 / p;
    double U2 = (zeta > 0.0 && isfinite(zeta)) ? zeta * zeta / (p + zeta * zeta) : 1.0;
    double U = sqrt(U2);
    double K = exp(-alpha * beta / p * ab2);
    double F[ORACLE_LPAIR + 1];
    oracle_boys(c->L, U2 * p * pc2, F);
    double Um = U; /* U^{2m+1} */
    for (int m = 0; m <= c->L; m++) {
        c->base[m] = 2.0 * M_PI / p * K * Um * F[m];
        Um *= U2;
    }
    {
        int n = c->L + 1;
        memset(c->have, 0, (size_t)n * n * n * (n + 1));
    }
    int na = oracle_ncart(la), nb = oracle_ncart(lb);
    for (int ia = 0; ia < na; ia++)
        for (int ib = 0; ib < nb; ib++) {
            int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
            cart_exponents(la, ia, ea);
            cart_exponents(lb, ib, eb);
            out[ia * nb + ib] = hrr(c, ea, eb);
        }
}

/* Contracted block (mu | J | nu) over normalised primitives (Eq. 11, Eq. 12)
 * for shells sa, sb.  Shells are given expanded (l = 0, 1, 2, 3 only). */
static void shell_block(const int *sh_atom, const int *sh_l, const int *sh_nprim, const int *sh_off,
                        const double *exps, const double *coefs, const double *axyz, int sa, int sb,
                        const double *C, double zeta, double *out)
{
    int la = sh_l[sa], lb = sh_l[sb];
    int na = oracle_ncart(la), nb = oracle_ncart(lb);
    const double *A = axyz + 3 * sh_atom[sa], *B = axyz + 3 * sh_atom[sb];
    double prim[(ORACLE_LMAX + 1) * (ORACLE_LMAX + 2) / 2 * (ORACLE_LMAX + 1) * (ORACLE_LMAX + 2) / 2];
    for (int k = 0; k < na * nb; k++) out[k] = 0.0;
    for (int i = 0; i < sh_nprim[sa]; i++)
        for (int j = 0; j < sh_nprim[sb]; j++) {
            double a = exps[sh_off[sa] + i], b = exps[sh_off[sb] + j];
            double ca = coefs[sh_off[sa] + i], cb = coefs[sh_off[sb] + j];
            oracle_prim(la, a, A, lb, b, B, C, zeta, prim);
            double Na[16], Nb[16];
            for (int ia = 0; ia < na; ia++) {
                int e[3] = {0, 0, 0};
                cart_exponents(la, ia, e);
                Na[ia] = oracle_norm(a, e[0], e[1], e[2]);
            }
            for (int ib = 0; ib < nb; ib++) {
                int e[3] = {0, 0, 0};
                cart_exponents(lb, ib, e);
                Nb[ib] = oracle_norm(b, e[0], e[1], e[2]);
            }
            for (int ia = 0; ia < na; ia++)
                for (int ib = 0; ib < nb; ib++)
                    out[ia * nb + ib] += ca * cb * Na[ia] * Nb[ib] * prim[ia * nb + ib];
        }
}

void oracle_shell_block(const int *sh_atom, const int *sh_l, const int *sh_nprim, const int *sh_off,
                        const double *exps, const double *coefs, const double *axyz, int sa, int sb,
                        const double *C, double zeta, double *out)
{
    shell_block(sh_atom, sh_l, sh_nprim, sh_off, exps, coefs, axyz, sa, sb, C, zeta, out);
}

/* c_k = sum_{mu nu} P_{mu nu} L^k_{mu nu} = -sum_{mu nu} P_{mu nu} (mu|J_k|nu)  (Eq. 5, Eq. 6).
 * The double sum runs over shell pairs A <= B; a pair with A < B stands for
 * both (A,B) and (B,A), which contribute equally because P and L are
 * symmetric. */
void oracle_esp(int nshell, const int *sh_atom, const int *sh_l, const int *sh_nprim, const int *sh_off,
                const int *sh_bf, const double *exps, const double *coefs, const double *axyz, int nbf,
                const double *P, int npts, const double *pts, const double *zeta, double *c_out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < npts; k++) {
        double blk[100];
        double ck = 0.0;
        for (int sa = 0; sa < nshell; sa++)
            for (int sb = sa; sb < nshell; sb++) {
                int na = oracle_ncart(sh_l[sa]), nb = oracle_ncart(sh_l[sb]);
                shell_block(sh_atom, sh_l, sh_nprim, sh_off, exps, coefs, axyz, sa, sb, pts + 3 * k,
                            zeta[k], blk);
                double w = (sa == sb) ? 1.0 : 2.0, s = 0.0;
                for (int ia = 0; ia < na; ia++)
                    for (int ib = 0; ib < nb; ib++)
                        s += P[(size_t)(sh_bf[sa] + ia) * nbf + sh_bf[sb] + ib] * blk[ia * nb + ib];
                ck += w * s;
            }
        c_out[k] = -ck;
    }
}

/* dF_{mu nu} = sum_k q_k L^k_{mu nu} = -sum_k q_k (mu|J_k|nu) for the listed
 * shell pairs (Eq. 10); block p is written at out + off[p] as
 * ncart(A) x ncart(B), row-major. */
void oracle_fock_pairs(const int *sh_atom, const int *sh_l, const int *sh_nprim, const int *sh_off,
                       const double *exps, const double *coefs, const double *axyz, int npts,
                       const double *pts, const double *zeta, const double *q, int npairs,
                       const int *pa, const int *pb, const long *off, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npairs; p++) {
        double blk[100];
        int na = oracle_ncart(sh_l[pa[p]]), nb = oracle_ncart(sh_l[pb[p]]);
        double *o = out + off[p];
        for (int t = 0; t < na * nb; t++) o[t] = 0.0;
        for (int k = 0; k < npts; k++) {
            shell_block(sh_atom, sh_l, sh_nprim, sh_off, exps, coefs, axyz, pa[p], pb[p], pts + 3 * k,
                        zeta[k], blk);
            for (int t = 0; t < na * nb; t++) o[t] -= q[k] * blk[t];
        }
    }
}

/* Position of the Cartesian component with exponents e in shell l (the order
 * of cart_exponents). */
static int cart_index(int l, const int e[3])
{
    int m = l - e[0];
    return m * (m + 1) / 2 + (m - e[1]);
}

/* Gradient of sum_k q_k c_k = -sum_k q_k sum_{mu nu} P_{mu nu} (mu|J_k|nu)
 * with respect to the nuclear positions at fixed P (the second term of
 * Eq. 14, split as in Eq. 22 into the bra-centre, ket-centre and point parts).
 * point_atom[k]: the atom whose sphere holds point k.  grad: natom*3,
 * accumulated into (the caller zeroes it).  Points with q_k = 0 are skipped. */
void oracle_grad_c(int nshell, const int *sh_atom, const int *sh_l, const int *sh_nprim, const int *sh_off,
                   const int *sh_bf, const double *exps, const double *coefs, const double *axyz, int nbf,
                   const double *P, int npts, const double *pts, const double *zeta, const double *q,
                   const int *point_atom, int natom, double *grad)
{
#pragma omp parallel
    {
        double *g = (double *)calloc((size_t)natom * 3, sizeof(double));
        /* raw blocks of (la+1, lb), (la-1, lb), (la, lb+1), (la, lb-1): at most
         * ncart(3) x ncart(2) = 60 entries each */
        double up_a[60], dn_a[60], up_b[60], dn_b[60];
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < npts; k++) {
            if (q[k] == 0.0) continue;
            const double *C = pts + 3 * k;
            for (int sa = 0; sa < nshell; sa++)
                for (int sb = sa; sb < nshell; sb++) {
                    const int la = sh_l[sa], lb = sh_l[sb];
                    const int na = oracle_ncart(la), nb = oracle_ncart(lb);
                    const int IA = sh_atom[sa], IB = sh_atom[sb], IC = point_atom[k];
                    const double *A = axyz + 3 * IA, *B = axyz + 3 * IB;
                    const double w = (sa == sb) ? 1.0 : 2.0;
                    for (int i = 0; i < sh_nprim[sa]; i++)
                        for (int j = 0; j < sh_nprim[sb]; j++) {
                            const double al = exps[sh_off[sa] + i], be = exps[sh_off[sb] + j];
                            const double cc = coefs[sh_off[sa] + i] * coefs[sh_off[sb] + j];
                            oracle_prim(la + 1, al, A, lb, be, B, C, zeta[k], up_a);
                            if (la > 0) oracle_prim(la - 1, al, A, lb, be, B, C, zeta[k], dn_a);
                            oracle_prim(la, al, A, lb + 1, be, B, C, zeta[k], up_b);
                            if (lb > 0) oracle_prim(la, al, A, lb - 1, be, B, C, zeta[k], dn_b);
                            const int nbu = oracle_ncart(lb + 1), nbd = lb > 0 ? oracle_ncart(lb - 1) : 0;
                            for (int ia = 0; ia < na; ia++) {
                                int ea[3] = {0, 0, 0};
                                cart_exponents(la, ia, ea);
                                const double Na = oracle_norm(al, ea[0], ea[1], ea[2]);
                                for (int ib = 0; ib < nb; ib++) {
                                    int eb[3] = {0, 0, 0};
                                    cart_exponents(lb, ib, eb);
                                    const double Nb = oracle_norm(be, eb[0], eb[1], eb[2]);
                                    const double Pw = P[(size_t)(sh_bf[sa] + ia) * nbf + sh_bf[sb] + ib];
                                    /* this integral's weight in sum_k q_k c_k */
                                    const double s = -q[k] * w * Pw * cc * Na * Nb;
                                    for (int d = 0; d < 3; d++) {
                                        int e1[3] = {ea[0], ea[1], ea[2]};
                                        e1[d] += 1;
                                        double dA = 2.0 * al * up_a[cart_index(la + 1, e1) * nb + ib];
                                        if (ea[d] > 0) {
                                            int e2[3] = {ea[0], ea[1], ea[2]};
                                            e2[d] -= 1;
                                            dA -= ea[d] * dn_a[cart_index(la - 1, e2) * nb + ib];
                                        }
                                        int f1[3] = {eb[0], eb[1], eb[2]};
                                        f1[d] += 1;
                                        double dB = 2.0 * be * up_b[ia * nbu + cart_index(lb + 1, f1)];
                                        if (eb[d] > 0) {
                                            int f2[3] = {eb[0], eb[1], eb[2]};
                                            f2[d] -= 1;
                                            dB -= eb[d] * dn_b[ia * nbd + cart_index(lb - 1, f2)];
                                        }
                                        g[3 * IA + d] += s * dA;
                                        g[3 * IB + d] += s * dB;
                                        g[3 * IC + d] -= s * (dA + dB);
                                    }
                                }
                            }
                        }
                }
        }
#pragma omp critical
        for (int t = 0; t < natom * 3; t++) grad[t] += g[t];
        free(g);
    }
}
