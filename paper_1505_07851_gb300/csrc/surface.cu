// ISWIG cavity surface (Eq. 7, Eq. 9, Section 3), the stored A (Eq. 2, Eq. 3,
// Eq. 8) and B z (Eq. 4).
#include <math.h>

#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"
#include "context.h"

namespace pcm {

constexpr int SURF_T = 128;
constexpr int SURF_ATOM_TILE = 512;

// Per-atom exponent of Eq. 7 with equal weights w = 4 pi / n.
__global__ void atom_zeta_kernel(int natom, const double *__restrict__ radius, double zeta, int n,
                                 double *__restrict__ azeta)
{
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= natom) return;
    const double w = 4.0 * PCM_PI / n;
    azeta[I] = zeta / (radius[I] * sqrt(w));
}

// One thread per candidate point (atom I, Fibonacci index i):
//   u_i: z_i = 1 - (2i+1)/n, phi_i = i pi (3 - sqrt 5)
//   r_k = X_I + R_I u_i,  zeta_k = zeta_I
//   S_k = prod_{J != I} (erfc(zeta_k (R_J - d)) + erfc(zeta_k (R_J + d))) / 2
// (Eq. 9 with erf written as 1 - erfc).  An atom with zeta_k (d - R_J) > 6
// contributes a factor that rounds to exactly 1 in FP64 and is skipped.
__global__ void surface_candidates_kernel(int natom, int n, const double *__restrict__ xyz,
                                          const double *__restrict__ radius, const double *__restrict__ azeta,
                                          double drop, double *__restrict__ cx, double *__restrict__ cy,
                                          double *__restrict__ cz, double *__restrict__ cS,
                                          unsigned char *__restrict__ keep)
{
    __shared__ double sx[SURF_ATOM_TILE], sy[SURF_ATOM_TILE], sz[SURF_ATOM_TILE], sr[SURF_ATOM_TILE];
    const long long ncand = (long long)natom * n;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = k < ncand;
    int I = 0, i = 0;
    double rx = 0, ry = 0, rz = 0, zk = 1.0;
    if (active) {
        I = (int)(k / n);
        i = (int)(k - (long long)I * n);
        const double zc = 1.0 - (2.0 * i + 1.0) / n;
        const double phi = i * (PCM_PI * (3.0 - sqrt(5.0)));
        const double s = sqrt(1.0 - zc * zc);
        double sphi, cphi;
        sincos(phi, &sphi, &cphi);
        const double R = radius[I];
        rx = xyz[3 * I + 0] + R * (s * cphi);
        ry = xyz[3 * I + 1] + R * (s * sphi);
        rz = xyz[3 * I + 2] + R * zc;
        zk = azeta[I];
    }
    const double reach = 6.0 / zk;
    double S = 1.0;
    for (int J0 = 0; J0 < natom; J0 += SURF_ATOM_TILE) {
        const int nj = min(SURF_ATOM_TILE, natom - J0);
        __syncthreads();
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
            sx[j] = xyz[3 * (J0 + j) + 0];
            sy[j] = xyz[3 * (J0 + j) + 1];
            sz[j] = xyz[3 * (J0 + j) + 2];
            sr[j] = radius[J0 + j];
        }
        __syncthreads();
        if (active) {
            for (int j = 0; j < nj; ++j) {
                if (J0 + j == I) continue;
                const double dx = rx - sx[j], dy = ry - sy[j], dz = rz - sz[j];
                const double d2 = dx * dx + dy * dy + dz * dz;
                const double lim = sr[j] + reach;
                if (d2 > lim * lim) continue;
                const double d = sqrt(d2);
                S *= 0.5 * (erfc(zk * (sr[j] - d)) + erfc(zk * (sr[j] + d)));
            }
        }
    }
    if (active) {
        cx[k] = rx;
        cy[k] = ry;
        cz[k] = rz;
        cS[k] = S;
        keep[k] = S >= drop ? 1 : 0;
    }
}

// flags of the kept candidates of one exponent class
__global__ void class_flags_kernel(long long ncand, int n, const unsigned char *__restrict__ keep,
                                   const int *__restrict__ atom_cls, int e, unsigned char *__restrict__ f)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncand) return;
    f[k] = (keep[k] && atom_cls[k / n] == e) ? 1 : 0;
}

__global__ void gather_points_kernel(int M, int n, const int *__restrict__ idx, const double *__restrict__ cx,
                                     const double *__restrict__ cy, const double *__restrict__ cz,
                                     const double *__restrict__ cS, const double *__restrict__ azeta,
                                     const int *__restrict__ atom_cls, double *px, double *py, double *pz,
                                     double *pzeta, double *pS, int *pindex, int *pcls)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int k = idx[j];
    const int I = k / n;
    px[j] = cx[k];
    py[j] = cy[k];
    pz[j] = cz[k];
    pS[j] = cS[k];
    pzeta[j] = azeta[I];
    pindex[j] = k;
    pcls[j] = atom_cls[I];
}

// (B z)_k = sum_J Z_J erf(zeta_k r_kJ) / r_kJ (Eq. 4); erf(x) rounds to 1 in
// FP64 for x > 6, where the plain Z_J / r_kJ is used.
__global__ void bz_kernel(int M, int natom, const double *__restrict__ px, const double *__restrict__ py,
                          const double *__restrict__ pz, const double *__restrict__ pzeta,
                          const double *__restrict__ xyz, const double *__restrict__ Z, double *__restrict__ Bz)
{
    __shared__ double sx[SURF_ATOM_TILE], sy[SURF_ATOM_TILE], sz[SURF_ATOM_TILE], sq[SURF_ATOM_TILE];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = k < M;
    double x = 0, y = 0, z = 0, zk = 1;
    if (active) {
        x = px[k];
        y = py[k];
        z = pz[k];
        zk = pzeta[k];
    }
    double s = 0.0;
    for (int J0 = 0; J0 < natom; J0 += SURF_ATOM_TILE) {
        const int nj = min(SURF_ATOM_TILE, natom - J0);
        __syncthreads();
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
            sx[j] = xyz[3 * (J0 + j) + 0];
            sy[j] = xyz[3 * (J0 + j) + 1];
            sz[j] = xyz[3 * (J0 + j) + 2];
            sq[j] = Z[J0 + j];
        }
        __syncthreads();
        if (active) {
            for (int j = 0; j < nj; ++j) {
                const double dx = x - sx[j], dy = y - sy[j], dz = z - sz[j];
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                const double a = zk * r;
                s += sq[j] * (a > 6.0 ? 1.0 : erf(a)) / r;
            }
        }
    }
    if (active) Bz[k] = s;
}

// Tile (bi, bj), bi <= bj, of linear block t in the row-major upper triangle
// of nt x nt tiles: row b starts at b nt - b (b - 1) / 2.  The row comes from
// the quadratic's root and is then corrected to the exact integer answer.
__device__ __forceinline__ void upper_tile(long long t, int nt, int &bi, int &bj)
{
    auto start = [nt](long long b) { return b * nt - b * (b - 1) / 2; };
    const double q = 2.0 * nt + 1.0;
    long long b = (long long)((q - sqrt(fmax(q * q - 8.0 * (double)t, 0.0))) * 0.5);
    b = b < 0 ? 0 : (b > nt - 1 ? nt - 1 : b);
    while (b > 0 && start(b) > t) --b;
    while (b + 1 < nt && start(b + 1) <= t) ++b;
    bi = (int)b;
    bj = bi + (int)(t - start(b));
}

// Stored A in FP64 (Eq. 2, Eq. 3 read as zeta_k sqrt(2/pi) / S_k, Eq. 8).
// Tiles (bi, bj) with bi <= bj are computed once and written to both halves.
constexpr int AT = 32;
__global__ void a_build_kernel(int M, int lda, const double *__restrict__ px, const double *__restrict__ py,
                               const double *__restrict__ pz, const double *__restrict__ pzeta,
                               const double *__restrict__ pS, const int *__restrict__ pcls, int ncls,
                               const double *__restrict__ zp_cls, double *__restrict__ A)
{
    // zeta'_kl of Eq. 8 depends only on the two exponent classes: zp_cls holds
    // it for every class pair (up to 16 classes; more are computed per element)
    __shared__ double zp_tab[16 * 16];
    const bool tab = ncls <= 16;
    if (tab)
        for (int t = threadIdx.x; t < ncls * ncls; t += blockDim.x) zp_tab[t] = zp_cls[t];
    __syncthreads();
    const int nt = (M + AT - 1) / AT;
    int bi, bj;
    upper_tile(blockIdx.x, nt, bi, bj);
    __shared__ double tile[AT][AT + 1];
    const int tx = threadIdx.x & (AT - 1);
    const int ty = threadIdx.x / AT;  // 0 .. 7
    const int l = bj * AT + tx;
    double lx = 0, ly = 0, lz = 0, lzeta = 1;
    int lcls = 0;
    if (l < M) {
        lx = px[l];
        ly = py[l];
        lz = pz[l];
        lzeta = pzeta[l];
        lcls = pcls[l];
    }
    for (int r = ty; r < AT; r += 8) {
        const int k = bi * AT + r;
        double v = 0.0;
        if (k < M && l < M) {
            if (k == l) {
                v = pzeta[k] * 0.79788456080286535588 / pS[k];  // sqrt(2/pi)
            } else {
                const double dx = px[k] - lx, dy = py[k] - ly, dz = pz[k] - lz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                const double inv = rsqrt(d2);
                const double zk = pzeta[k];
                const double zp = tab ? zp_tab[pcls[k] * ncls + lcls] : zk * lzeta / sqrt(zk * zk + lzeta * lzeta);
                const double a = zp * (d2 * inv);
                // erf(a) rounds to 1 in FP64 for a > 6
                v = (a > 6.0) ? inv : erf(a) * inv;
            }
            A[(size_t)k * lda + l] = v;
        }
        tile[r][tx] = v;
    }
    if (bi == bj) return;
    __syncthreads();
    // transposed write: rows of tile bj, columns of tile bi
    for (int r = ty; r < AT; r += 8) {
        const int k = bj * AT + r;
        const int ll = bi * AT + tx;
        if (k < M && ll < M) A[(size_t)k * lda + ll] = tile[tx][r];
    }
}

// The same A for PCM_MIXED, evaluated in double-float arithmetic on the FP32
// pipes (the FP64 pipe, 64 times slower on this GPU, bounds a_build_kernel):
// with the points split as x = xh + xl (xh on a 2^-10 grid, so xh_k - xh_l is
// exact), d = (xh_k - xh_l) + (xl_k - xl_l) as a hi + lo pair, R^2 = |d|^2 with
// error-free products and sums, and 1/R from the FP32 reciprocal square root
// refined by one Newton step in FP32 and one in double-float.  The off-diagonal
// elements with zeta' R <= 6, where erf differs from 1 in FP64, and the
// diagonal are evaluated in FP64 as in a_build_kernel.  1/R comes out to about
// 3e-14 relative; the FP32 split of the coordinates limits the elements of the
// nearest points to ~1e-10 relative.  Writes A32 (hi) and A32lo (lo), the
// matrices of the inner FP32 GEMV and of the double-float GEMV, and A (FP64,
// = hi + lo) only when A is not null.
__global__ void a_build_df_kernel(int M, int lda, const float *__restrict__ ph, const float *__restrict__ pl,
                                  const double *__restrict__ px, const double *__restrict__ py,
                                  const double *__restrict__ pz, const double *__restrict__ pzeta,
                                  const double *__restrict__ pS, const int *__restrict__ pcls, int ncls,
                                  const double *__restrict__ zp_cls, double *__restrict__ A,
                                  float *__restrict__ A32, float *__restrict__ A32lo)
{
    __shared__ float zp_tab[16 * 16];
    __shared__ double zp_tab64[16 * 16];
    const bool tab = ncls <= 16;
    if (tab)
        for (int t = threadIdx.x; t < ncls * ncls; t += blockDim.x) {
            zp_tab64[t] = zp_cls[t];
            zp_tab[t] = (float)zp_cls[t];
        }
    __syncthreads();
    const int nt = (M + AT - 1) / AT;
    int bi, bj;
    upper_tile(blockIdx.x, nt, bi, bj);
    __shared__ float2 tile[AT][AT + 1];
    __shared__ double tile64[AT][AT + 1];
    const int tx = threadIdx.x & (AT - 1);
    const int ty = threadIdx.x / AT;  // 0 .. 7
    const int l = bj * AT + tx;
    float lxh = 0.f, lyh = 0.f, lzh = 0.f, lxl = 0.f, lyl = 0.f, lzl = 0.f;
    double lzeta = 1.0;
    int lcls = 0;
    if (l < M) {
        lxh = ph[l];
        lyh = ph[(size_t)M + l];
        lzh = ph[2 * (size_t)M + l];
        lxl = pl[l];
        lyl = pl[(size_t)M + l];
        lzl = pl[2 * (size_t)M + l];
        lzeta = pzeta[l];
        lcls = pcls[l];
    }
    for (int r = ty; r < AT; r += 8) {
        const int k = bi * AT + r;
        float h = 0.f, lo = 0.f;
        double v = 0.0;
        if (k < M && l < M) {
            if (k == l) {
                v = pzeta[k] * 0.79788456080286535588 / pS[k];  // sqrt(2/pi)
                h = (float)v;
                lo = (float)(v - (double)h);
            } else {
                float r2;
                df_rsqrt(ph[k] - lxh, pl[k] - lxl, ph[(size_t)M + k] - lyh, pl[(size_t)M + k] - lyl,
                         ph[2 * (size_t)M + k] - lzh, pl[2 * (size_t)M + k] - lzl, h, lo, r2);
                const float zp = tab ? zp_tab[pcls[k] * ncls + lcls]
                                     : (float)(pzeta[k] * lzeta / sqrt(pzeta[k] * pzeta[k] + lzeta * lzeta));
                // zeta' R in FP32 decides the branch with a margin: erf(6) rounds
                // to 1 in FP64, and FP32 moves the threshold by ~1e-6
                if (zp * (r2 * h) <= 6.001f) {  // zeta' R, R = R^2 / R
                    const double dx = px[k] - px[l], dy = py[k] - py[l], dz = pz[k] - pz[l];
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    const double inv = rsqrt(d2);
                    const double zk = pzeta[k];
                    const double zp64 = tab ? zp_tab64[pcls[k] * ncls + lcls]
                                            : zk * lzeta / sqrt(zk * zk + lzeta * lzeta);
                    const double a = zp64 * (d2 * inv);
                    const double e = (a > 6.0) ? inv : erf(a) * inv;
                    h = (float)e;
                    lo = (float)(e - (double)h);
                }
                v = (double)h + (double)lo;
            }
            if (A) A[(size_t)k * lda + l] = v;
            A32[(size_t)k * lda + l] = h;
            A32lo[(size_t)k * lda + l] = lo;
        }
        tile[r][tx] = make_float2(h, lo);
        tile64[r][tx] = v;
    }
    if (bi == bj) return;
    __syncthreads();
    for (int r = ty; r < AT; r += 8) {
        const int k = bj * AT + r;
        const int ll = bi * AT + tx;
        if (k < M && ll < M) {
            const float2 e = tile[tx][r];
            if (A) A[(size_t)k * lda + ll] = tile64[tx][r];
            A32[(size_t)k * lda + ll] = e.x;
            A32lo[(size_t)k * lda + ll] = e.y;
        }
    }
}

__global__ void dinv_kernel(int M, int lda, const double *__restrict__ A, double *__restrict__ dinv)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) dinv[k] = 1.0 / A[(size_t)k * lda + k];
}

__global__ void dinv_df_kernel(int M, int lda, const float *__restrict__ hi, const float *__restrict__ lo,
                               double *__restrict__ dinv)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) {
        const size_t i = (size_t)k * lda + k;
        dinv[k] = 1.0 / ((double)hi[i] + (double)lo[i]);
    }
}

int surface_build(pcm_ctx *c, int natom, const double *xyz, const double *Z, const double *radius, int n)
{
    // the previous surface's A may still be in use on the side stream (and
    // need not be built at all if nothing used it)
    c->op_stale = false;
    PCM_TRY(join_side(c));
    c->natom = natom;
    c->npts_sphere = n;
    c->h_xyz.assign(xyz, xyz + 3 * natom);
    c->h_Z.assign(Z, Z + natom);
    c->h_radius.assign(radius, radius + natom);
    PCM_TRY(c->xyz.alloc(3 * natom));
    PCM_TRY(c->Z.alloc(natom));
    PCM_TRY(c->radius.alloc(natom));
    PCM_CUDA(cudaMemcpyAsync(c->xyz.p, xyz, 3 * natom * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->Z.p, Z, natom * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->radius.p, radius, natom * sizeof(double), cudaMemcpyHostToDevice, c->stream));

    // exponent classes: atoms with equal zeta (Eq. 7) share a class; classes in increasing zeta
    DBuf<double> &azeta = c->sd[0];
    PCM_TRY(azeta.alloc(natom));
    atom_zeta_kernel<<<(natom + 127) / 128, 128, 0, c->stream>>>(natom, c->radius.p, c->opt.zeta, n, azeta.p);
    PCM_LAUNCHED(c);
    std::vector<double> h_azeta(natom);
    PCM_CUDA(cudaMemcpyAsync(h_azeta.data(), azeta.p, natom * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<double> uz(h_azeta);
    std::sort(uz.begin(), uz.end());
    uz.erase(std::unique(uz.begin(), uz.end()), uz.end());
    c->ncls = (int)uz.size();
    c->h_cls_zeta = uz;
    std::vector<int> h_acls(natom);
    for (int I = 0; I < natom; ++I)
        h_acls[I] = (int)(std::lower_bound(uz.begin(), uz.end(), h_azeta[I]) - uz.begin());
    DBuf<int> &acls = c->si[0];
    PCM_TRY(acls.alloc(natom));
    PCM_CUDA(cudaMemcpyAsync(acls.p, h_acls.data(), natom * sizeof(int), cudaMemcpyHostToDevice, c->stream));

    // candidates
    const long long ncand = (long long)natom * n;
    DBuf<double> &cx = c->sd[1], &cy = c->sd[2], &cz = c->sd[3], &cS = c->sd[4];
    DBuf<unsigned char> &keep = c->su8[0];
    PCM_TRY(cx.alloc(ncand));
    PCM_TRY(cy.alloc(ncand));
    PCM_TRY(cz.alloc(ncand));
    PCM_TRY(cS.alloc(ncand));
    PCM_TRY(keep.alloc(ncand));
    surface_candidates_kernel<<<(unsigned)((ncand + SURF_T - 1) / SURF_T), SURF_T, 0, c->stream>>>(
        natom, n, c->xyz.p, c->radius.p, azeta.p, c->opt.switch_drop, cx.p, cy.p, cz.p, cS.p, keep.p);
    PCM_LAUNCHED(c);

    // compaction class by class into library order
    PCM_TRY(c->flags8.alloc(ncand));
    PCM_TRY(c->idx32.alloc(ncand));
    PCM_TRY(c->iscal.alloc(64));
    std::vector<int> counts(c->ncls);
    DBuf<int> &order = c->si[1];
    PCM_TRY(order.alloc(ncand));
    int M = 0;
    c->h_cls_off.assign(c->ncls + 1, 0);
    for (int e = 0; e < c->ncls; ++e) {
        class_flags_kernel<<<(unsigned)((ncand + 255) / 256), 256, 0, c->stream>>>(ncand, n, keep.p, acls.p, e,
                                                                                  c->flags8.p);
        PCM_LAUNCHED(c);
        PCM_TRY(compact_flags(c, c->flags8.p, ncand, order.p + M, nullptr, c->iscal.p));
        int cnt = 0;
        PCM_CUDA(cudaMemcpyAsync(&cnt, c->iscal.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
        M += cnt;
        c->h_cls_off[e + 1] = M;
    }
    c->M = M;
    if (M == 0) {
        set_last_error("no surface point survives the switching threshold");
        return PCM_ERR_ARG;
    }
    PCM_TRY(c->px.alloc(M));
    PCM_TRY(c->py.alloc(M));
    PCM_TRY(c->pz.alloc(M));
    PCM_TRY(c->pzeta.alloc(M));
    PCM_TRY(c->pS.alloc(M));
    PCM_TRY(c->pindex.alloc(M));
    PCM_TRY(c->pcls.alloc(M));
    PCM_TRY(c->Bz.alloc(M));
    gather_points_kernel<<<(M + 127) / 128, 128, 0, c->stream>>>(M, n, order.p, cx.p, cy.p, cz.p, cS.p, azeta.p,
                                                                acls.p, c->px.p, c->py.p, c->pz.p, c->pzeta.p,
                                                                c->pS.p, c->pindex.p, c->pcls.p);
    PCM_LAUNCHED(c);
    PCM_TRY(c->cls_zeta.alloc(c->ncls));
    PCM_TRY(c->cls_off.alloc(c->ncls + 1));
    PCM_CUDA(cudaMemcpyAsync(c->cls_zeta.p, c->h_cls_zeta.data(), c->ncls * sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->cls_off.p, c->h_cls_off.data(), (c->ncls + 1) * sizeof(int),
                             cudaMemcpyHostToDevice, c->stream));

    bz_kernel<<<(M + 127) / 128, 128, 0, c->stream>>>(M, natom, c->px.p, c->py.p, c->pz.p, c->pzeta.p, c->xyz.p,
                                                     c->Z.p, c->Bz.p);
    PCM_LAUNCHED(c);

    PCM_TRY(points_split(c));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    // PCM_MIXED operator for this surface: matrix-free for large surfaces (its
    // FP32 product outruns the stored FP32 GEMV there) or when the stored parts
    // would crowd the device; stored otherwise, and always for batch members
    c->mf_active = false;
    if (c->opt.precision == PCM_MIXED && !c->store_a) {
        if (c->opt.operator_mode == PCM_OPERATOR_FREE) {
            c->mf_active = true;
        } else if (c->opt.operator_mode == PCM_OPERATOR_AUTO) {
            size_t fr = 0, tot = 0;
            const double need = 8.0 * (double)c->M * (double)((c->M + 31) / 32 * 32);
            const bool tight = cudaMemGetInfo(&fr, &tot) == cudaSuccess && need > 0.25 * (double)fr;
            c->mf_active = c->M > 24576 || tight;
        }
    }
    c->stats.operator_free = c->mf_active ? 1 : 0;
    c->pc_ready = false;
    c->have_c = false;
    c->aq_valid = false;
    // the stored A and what depends on it are built on the second stream when
    // first needed (pcm_esp starts it, so that it runs beside the integrals)
    c->op_stale = true;
    return PCM_OK;
}

// Stored A (Eq. 2, Eq. 3, Eq. 8) and 1/A_kk on stream s: FP64, or for
// PCM_MIXED double-float only, as its FP32 hi and lo parts (A32, A32lo); the
// RBJ set-up of that mode reads hi + lo
int a_build(pcm_ctx *c, cudaStream_t s)
{
    const int M = c->M;
    c->lda = (M + 31) / 32 * 32;
    const bool mixed = c->opt.precision == PCM_MIXED;
    PCM_TRY(zeta_pairs(c, s));
    const long long nt = (M + AT - 1) / AT;
    const long long ntiles = nt * (nt + 1) / 2;
    PCM_TRY(c->dinv.alloc(M));
    c->st_arow_ok = false;
    if (mixed) {
        PCM_TRY(c->A32.alloc((size_t)M * c->lda));
        PCM_TRY(c->A32lo.alloc((size_t)M * c->lda));
        a_build_df_kernel<<<(unsigned)ntiles, 256, 0, s>>>(M, c->lda, c->p32.p, c->p32lo.p, c->px.p, c->py.p,
                                                          c->pz.p, c->pzeta.p, c->pS.p, c->pcls.p, c->ncls,
                                                          c->zp_cls.p, nullptr, c->A32.p, c->A32lo.p);
        PCM_LAUNCHED(c);
        dinv_df_kernel<<<(M + 127) / 128, 128, 0, s>>>(M, c->lda, c->A32.p, c->A32lo.p, c->dinv.p);
    } else {
        PCM_TRY(c->A.alloc((size_t)M * c->lda));
        a_build_kernel<<<(unsigned)ntiles, 256, 0, s>>>(M, c->lda, c->px.p, c->py.p, c->pz.p, c->pzeta.p, c->pS.p,
                                                       c->pcls.p, c->ncls, c->zp_cls.p, c->A.p);
        PCM_LAUNCHED(c);
        dinv_kernel<<<(M + 127) / 128, 128, 0, s>>>(M, c->lda, c->A.p, c->dinv.p);
    }
    PCM_LAUNCHED(c);
    return PCM_OK;
}

}  // namespace pcm
