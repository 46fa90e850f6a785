// PCM_MIXED ESP over the cross-atom primitive pairs, two pairs per packed
// FP32x2 instruction, with a far-field path.
//
// Most pair-point interactions of a protein-sized surface lie where the Boys
// function has reached its asymptotic form (T = rho R^2 >= far_T(L)); there
// every Hermite integral is a derivative of 1/R times sqrt(pi)/(2 sqrt(p)),
// independent of the point's exponent (farfield.cuh), and the interaction is
// sum_n R^-(2n+1) Q_n(X, Y, Z) with per-pair polynomial coefficients.  A warp
// evaluates a slot of two pairs in that form when none of its interactions is
// near (T < far_T); otherwise it evaluates the general form (tabulated Boys
// function, (-2 rho)^n with the rho_lo correction, Hermite recurrence, U D_tuv)
// as well and keeps, per lane, the form its own T calls for.
//
// Pair data are laid out in global memory per tile of 32 pairs exactly as the
// kernel reads them from shared memory (pairs 2s and 2s+1 of slot s in the two
// lanes of float2 / float4 words): a class-independent far block and one near
// block per point class.  One thread issues the tile's two bulk copies
// (cp.async.bulk) into a ring of three shared buffers; each warp waits for the
// tile it reads next and releases it when done (pipeline.cuh).
//
// Error control as in the other FP32 kernels: coordinates split hi (2^-10
// grid) + lo so every distance is the FP32 rounding of the exact one; 1/R by
// the hardware reciprocal square root and one Newton step; the dominant
// coefficient (Q_0, the charge term; U D_000 in the general form) carries its
// lo part; every interaction is added with Kahan compensation, per lane (the
// compensation keeps the small terms that a plain FP32 running sum would drop,
// always towards a smaller magnitude for terms of one sign), and the lanes
// are added in FP64 at the end.
#include <math.h>

#include <algorithm>
#include <vector>

#include "boys.cuh"
#include "common.cuh"
#include "context.h"
#include "f2.cuh"
#include "fastmath.cuh"
#include "farfield.cuh"
#include "pipeline.cuh"

namespace pcm {

constexpr int PK_NT = 128;   // threads per block
constexpr int PK_TP = 32;    // pairs per tile
constexpr int PK_NS = 16;    // slots (two pairs each) per tile
// far block: P0, P1, P2 (float4 per slot), NC coefficient rows and the lo of
// row 0 (float2 per slot); near block: N0 (rho hi, lo), N1 (rho lo / hi,
// R^2 threshold) as float4 per slot, NH rows of hi(U D_h) and lo(U D_000)
template <int L>
struct PkLayout {
    static constexpr int NH = nherm(L);
    static constexpr int NC = far_nterms(L);
    static constexpr int FAR = 3 * 4 * PK_NS + (NC + 1) * 2 * PK_NS;
    static constexpr int NEAR = 2 * 4 * PK_NS + (NH + 1) * 2 * PK_NS;
    static_assert(FAR % 4 == 0 && NEAR % 4 == 0, "16-byte blocks");
};

// ---------------------------------------------------------------------------
// tile preparation: pair j of [jbeg, jbeg + 32 ntile) -> tile (j - jbeg) / 32;
// pairs at or beyond jend are padding (far away, zero coefficients)
// ---------------------------------------------------------------------------
template <int L>
__global__ void esp_tile_prep_kernel(int nesp, int jbeg, int jend, int ntile, int ncls,
                                     const double *__restrict__ cls_zeta, const double *__restrict__ eP,
                                     const double *__restrict__ eD, float *__restrict__ far,
                                     float *__restrict__ near)
{
    using Ly = PkLayout<L>;
    constexpr int NH = Ly::NH, NC = Ly::NC;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ntile * PK_TP) return;
    const int t = r / PK_TP, jj = r % PK_TP, s = jj >> 1, l = jj & 1;
    const int j = jbeg + r;
    float *F = far + (size_t)t * Ly::FAR;
    const bool v = j < jend;
    float xh = 1.0e4f, yh = 1.0e4f, zh = 1.0e4f, xl = 0.f, yl = 0.f, zl = 0.f;
    double p = 1.0;
    double D[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) D[h] = 0.0;
    if (v) {
        const double P[3] = {eP[j], eP[(size_t)nesp + j], eP[2 * (size_t)nesp + j]};
        double hi[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) hi[d] = rint(P[d] * 1024.0) * (1.0 / 1024.0);
        xh = (float)hi[0];
        yh = (float)hi[1];
        zh = (float)hi[2];
        xl = (float)(P[0] - hi[0]);
        yl = (float)(P[1] - hi[1]);
        zl = (float)(P[2] - hi[2]);
        p = eP[3 * (size_t)nesp + j];
#pragma unroll
        for (int h = 0; h < NH; ++h) D[h] = eD[(size_t)h * nesp + j];
    }
    F[4 * s + l] = xh;
    F[4 * s + 2 + l] = yh;
    F[64 + 4 * s + l] = zh;
    F[64 + 4 * s + 2 + l] = xl;
    F[128 + 4 * s + l] = yl;
    F[128 + 4 * s + 2 + l] = zl;
    // far-field coefficients: D_tuv sqrt(pi) / (2 sqrt(p)) mapped onto the terms
    constexpr FarContrib FC = far_contrib(L);
    double G[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) G[k] = 0.0;
    const double g = 0.88622692545275801365 / sqrt(p);
#pragma unroll
    for (int q = 0; q < FC.count; ++q) G[FC.term[q]] = fma(FC.w[q] * g, D[FC.h[q]], G[FC.term[q]]);
    float *Fg = F + 3 * 4 * PK_NS;
#pragma unroll
    for (int k = 0; k < NC; ++k) Fg[2 * PK_NS * k + 2 * s + l] = (float)G[k];
    Fg[2 * PK_NS * NC + 2 * s + l] = (float)(G[0] - (double)(float)G[0]);
    // near blocks, one per point class
    for (int e = 0; e < ncls; ++e) {
        float *N = near + ((size_t)e * ntile + t) * Ly::NEAR;
        const double z2 = cls_zeta[e] * cls_zeta[e];
        const double inv = 1.0 / (p + z2);
        const double rho = p * z2 * inv;
        const double U = sqrt(z2 * inv);
        const float rh = (float)rho;
        N[4 * s + l] = v ? rh : 1.f;
        N[4 * s + 2 + l] = v ? (float)(rho - (double)rh) : 0.f;
        N[64 + 4 * s + l] = v ? (float)((rho - (double)rh) / (double)rh) : 0.f;
        // near when R^2 < far_T / rho, i.e. T < far_T
        N[64 + 4 * s + 2 + l] = v ? (float)((double)far_T(L) / rho) : 0.f;
        float *Nd = N + 2 * 4 * PK_NS;
#pragma unroll
        for (int h = 0; h < NH; ++h) Nd[2 * PK_NS * h + 2 * s + l] = (float)(U * D[h]);
        const double u0 = U * D[0];
        Nd[2 * PK_NS * NH + 2 * s + l] = (float)(u0 - (double)(float)u0);
    }
}

// ---------------------------------------------------------------------------
// far-field value of one slot for the thread's point: sum_n R^-(2n+1) Q_n
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ f2 far_value(f2 X, f2 Y, f2 Z, f2 R2, const float2 *__restrict__ sG, int s)
{
    constexpr int NC = far_nterms(L);
    constexpr FarTerms FT = far_terms(L);
    // 1/R: hardware estimate and one Newton step, rs = r0 (1 + e/2), e = 1 - R^2 r0^2
    const f2 r0(rsqrt_fast(R2.v.x), rsqrt_fast(R2.v.y));
    const f2 em = fma2(R2 * r0, r0, f2(-1.f));
    const f2 rs = fma2(r0 * f2(-0.5f), em, r0);
    const float2 g0 = sG[s], g0l = sG[PK_NS * NC + s];
    f2 val = fma2(f2(g0.x, g0.y), rs, f2(g0l.x, g0l.y) * rs);
    if constexpr (L > 0) {
        // monomials X^a Y^b Z^c of degree 2..L, in Hermite index order
        constexpr MonoTab MT = mono_tab(L);
        f2 mono[nherm(L)];
        mono[1] = X;
        mono[2] = Y;
        mono[3] = Z;
#pragma unroll
        for (int i = 4; i < nherm(L); ++i) {
            const int a = MT.a[i], b = MT.b[i], c = MT.c[i];
            if (a > 0)
                mono[i] = mono[hidx(a - 1, b, c)] * X;
            else if (b > 0)
                mono[i] = mono[hidx(a, b - 1, c)] * Y;
            else
                mono[i] = mono[hidx(a, b, c - 1)] * Z;
        }
        const f2 rs2 = rs * rs;
        f2 Rn = rs;
#pragma unroll
        for (int n = 1; n <= L; ++n) {
            Rn = Rn * rs2;
            f2 Q(0.f);
            bool first = true;
#pragma unroll
            for (int kk = 1; kk < NC; ++kk) {
                if (FT.n[kk] != n) continue;
                const float2 g = sG[PK_NS * kk + s];
                const f2 gk(g.x, g.y);
                const int d = FT.a[kk] + FT.b[kk] + FT.c[kk];
                if (d == 0) {
                    Q = first ? gk : Q + gk;
                } else {
                    const f2 m = mono[hidx(FT.a[kk], FT.b[kk], FT.c[kk])];
                    Q = first ? gk * m : fma2(gk, m, Q);
                }
                first = false;
            }
            val = fma2(Q, Rn, val);
        }
    }
    return val;
}

// general (near) form of one slot for the thread's point: tabulated Boys
// function at T = rho R^2 (T clamped to the table's range in lanes that use
// the far form), Hermite recurrence and U D_tuv
template <int L>
__device__ __forceinline__ f2 near_value(f2 X, f2 Y, f2 Z, f2 R2, const float4 *__restrict__ sN,
                                         const float2 *__restrict__ sD, const float *__restrict__ boys, int s)
{
    constexpr int NH = nherm(L);
    const float4 n0 = sN[s];
    const f2 rh(n0.x, n0.y), rl(n0.z, n0.w);
    f2 T = fma2(rh, R2, rl * R2);
    T = f2(fminf(T.v.x, far_T(L)), fminf(T.v.y, far_T(L)));
    const f2 t = fma2(T, f2((float)BOYS_INV_DT), f2(12582912.0f));
    const int i0 = __float_as_int(t.v.x) - 0x4B400000, i1 = __float_as_int(t.v.y) - 0x4B400000;
    const f2 d = fma2(t + f2(-12582912.0f), f2(-(float)BOYS_DT), T);
    float fa[L + 1], fb[L + 1];
    boys_near32<L>(i0, d.v.x, boys, fa);
    boys_near32<L>(i1, d.v.y, boys, fb);
    const float2 D0 = sD[s], D0l = sD[PK_NS * NH + s];
    if constexpr (L == 0) {
        const f2 F0(fa[0], fb[0]);
        return fma2(f2(D0.x, D0.y), F0, f2(D0l.x, D0l.y) * F0);
    } else {
        const float4 n1 = sN[PK_NS + s];
        const f2 dr(n1.x, n1.y);
        const f2 m2r = rh * f2(-2.f);
        f2 Rn[L + 1];
        Rn[0] = f2(fa[0], fb[0]);
        f2 f = m2r;
#pragma unroll
        for (int n = 1; n <= L; ++n) {
            const f2 v = f * f2(fa[n], fb[n]);
            Rn[n] = fma2(v, dr * f2((float)n), v);
            if (n < L) f = f * m2r;
        }
        f2 R[NH];
        hermite_R<L, f2>(X, Y, Z, Rn, R);
        f2 dot = fma2(f2(D0.x, D0.y), R[0], f2(D0l.x, D0l.y) * R[0]);
#pragma unroll
        for (int h = 1; h < NH; ++h) {
            const float2 D = sD[PK_NS * h + s];
            dot = fma2(f2(D.x, D.y), R[h], dot);
        }
        return dot;
    }
}

// resident blocks per SM the register allocation aims for (without spills)
constexpr int pk_min_blocks(int L, int PPT) { return PPT == 4 ? 2 : (L == 0 ? 7 : (L == 1 ? 5 : (L == 2 ? 4 : 3))); }

template <int L, int PPT>
__device__ __forceinline__ void esp_block(const EspJob &jb, const float *__restrict__ boys, int *__restrict__ err)
{
    using Ly = PkLayout<L>;
    constexpr int BUF = Ly::FAR + Ly::NEAR;
    constexpr int NSTAGE = 3;
    __shared__ __align__(16) TileRing<NSTAGE, BUF> ring;
    const int k0 = jb.k0, k1 = jb.k1, e = jb.e, t0 = jb.t0, nt = jb.nt, ntile = jb.ntile, M = jb.M;
    const float *__restrict__ far = jb.far;
    const float *__restrict__ near = jb.near;
    const float *__restrict__ ph = jb.ph;
    const float *__restrict__ pl = jb.pl;

    if (threadIdx.x == 0) ring.init(PK_NT / 32);
    __syncthreads();
    int issued = 0;
    auto issue = [&](int j) {
        float *d = ring.data(j);
        mbar_expect_tx(ring.full_bar(j), (uint32_t)(BUF * sizeof(float)));
        bulk_g2s(d, far + (size_t)(t0 + j) * Ly::FAR, Ly::FAR * sizeof(float), ring.full_bar(j));
        bulk_g2s(d + Ly::FAR, near + ((size_t)e * ntile + t0 + j) * Ly::NEAR, Ly::NEAR * sizeof(float),
                 ring.full_bar(j));
        issued = j + 1;
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < min(NSTAGE, nt); ++j) issue(j);

    // the points, negated and duplicated into both lanes
    f2 nxh[PPT], nyh[PPT], nzh[PPT], nxl[PPT], nyl[PPT], nzl[PPT];
    f2 a32[PPT], k32[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = min(k0 + (int)threadIdx.x + q * PK_NT, k1 - 1);
        nxh[q] = f2(-ph[k]);
        nyh[q] = f2(-ph[(size_t)M + k]);
        nzh[q] = f2(-ph[2 * (size_t)M + k]);
        nxl[q] = f2(-pl[k]);
        nyl[q] = f2(-pl[(size_t)M + k]);
        nzl[q] = f2(-pl[2 * (size_t)M + k]);
        a32[q] = k32[q] = f2(0.f);
    }
    int j = 0;
    bool ok = true;
    for (; j < nt; ++j) {
        // producer: refill the buffer of tile j - 1 once every warp has released it
        if (threadIdx.x == 0 && j >= 1 && j - 1 + NSTAGE < nt) {
            if (ring.wait_empty(j - 1 + NSTAGE))
                issue(j - 1 + NSTAGE);
            else
                ok = false;
        }
        if (!__all_sync(0xffffffffu, ok && ring.wait_full(j))) {
            ok = false;
            break;
        }
        const float *tile = ring.data(j);
        const float4 *sP = reinterpret_cast<const float4 *>(tile);
        const float2 *sG = reinterpret_cast<const float2 *>(tile + 3 * 4 * PK_NS);
        const float4 *sN = reinterpret_cast<const float4 *>(tile + Ly::FAR);
        const float2 *sD = reinterpret_cast<const float2 *>(tile + Ly::FAR + 2 * 4 * PK_NS);
#pragma unroll 1
        for (int s = 0; s < PK_NS; ++s) {
            const float4 p0 = sP[s], p1 = sP[PK_NS + s], p2 = sP[2 * PK_NS + s];
            const f2 Ax(p0.x, p0.y), Ay(p0.z, p0.w), Az(p1.x, p1.y);
            const f2 Bx(p1.z, p1.w), By(p2.x, p2.y), Bz(p2.z, p2.w);
            const float4 n1 = sN[PK_NS + s];
            const float rf0 = n1.z, rf1 = n1.w;
            f2 X[PPT], Y[PPT], Z[PPT], R2[PPT];
            bool nr = false;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                X[q] = (Ax + nxh[q]) + (Bx + nxl[q]);
                Y[q] = (Ay + nyh[q]) + (By + nyl[q]);
                Z[q] = (Az + nzh[q]) + (Bz + nzl[q]);
                R2[q] = fma2(X[q], X[q], fma2(Y[q], Y[q], Z[q] * Z[q]));
                nr |= (R2[q].v.x < rf0) | (R2[q].v.y < rf1);
            }
            if (__any_sync(0xffffffffu, nr)) {
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    const f2 vf = far_value<L>(X[q], Y[q], Z[q], R2[q], sG, s);
                    const f2 vn = near_value<L>(X[q], Y[q], Z[q], R2[q], sN, sD, boys, s);
                    const f2 val(R2[q].v.x < rf0 ? vn.v.x : vf.v.x, R2[q].v.y < rf1 ? vn.v.y : vf.v.y);
                    const f2 y = val - k32[q];
                    const f2 tt = a32[q] + y;
                    k32[q] = (tt - a32[q]) - y;
                    a32[q] = tt;
                }
            } else {
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    const f2 val = far_value<L>(X[q], Y[q], Z[q], R2[q], sG, s);
                    const f2 y = val - k32[q];
                    const f2 tt = a32[q] + y;
                    k32[q] = (tt - a32[q]) - y;
                    a32[q] = tt;
                }
            }
        }
        ring.release(j);
    }
    if (!ok) {
        // a bounded wait gave up: report it; the producer lets its copies still
        // in flight land (bounded) before the block's shared memory is released
        if ((threadIdx.x & 31) == 0) atomicExch(err, 1);
        if (threadIdx.x == 0)
            for (int jj = j; jj < issued; ++jj) ring.wait_full(jj);
        return;
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int k = k0 + threadIdx.x + q * PK_NT;
        if (k < k1)
            jb.part[k] = ((double)a32[q].v.x - (double)k32[q].v.x) + ((double)a32[q].v.y - (double)k32[q].v.y);
    }
}

// One block: a run of points of one class (blk_off, blk_cls) against the
// tiles [blockIdx.y * tps, ...) of the class's cross-atom pairs; partial sums
// to part[blockIdx.y][k].
template <int L, int PPT>
__global__ void __launch_bounds__(PK_NT, pk_min_blocks(L, PPT))
    esp_kernel_f32x2(int ntile, int tps, const float *__restrict__ far, const float *__restrict__ near,
                     const int *__restrict__ blk_off, const int *__restrict__ blk_cls, const float *__restrict__ ph,
                     const float *__restrict__ pl, const float *__restrict__ boys, int M, double *__restrict__ part,
                     int *__restrict__ err)
{
    EspJob jb;
    jb.far = far;
    jb.near = near;
    jb.ph = ph;
    jb.pl = pl;
    jb.part = part + (size_t)blockIdx.y * M;
    jb.ntile = ntile;
    jb.M = M;
    jb.k0 = blk_off[blockIdx.x];
    jb.k1 = blk_off[blockIdx.x + 1];
    jb.e = blk_cls[blockIdx.x];
    jb.t0 = blockIdx.y * tps;
    jb.nt = max(0, min(ntile, jb.t0 + tps) - jb.t0);
    esp_block<L, PPT>(jb, boys, err);
}

// The same for a table of blocks of many molecules (one launch per class)
template <int L, int PPT>
__global__ void __launch_bounds__(PK_NT, pk_min_blocks(L, PPT))
    esp_jobs_kernel(const EspJob *__restrict__ jobs, const float *__restrict__ boys, int *__restrict__ err)
{
    esp_block<L, PPT>(jobs[blockIdx.x], boys, err);
}

// segments of ntile tiles for nblk point blocks: enough CTAs to fill the GPU
static void pk_plan(int ntile, int nblk, int *tps, int *rows)
{
    if (ntile <= 0) {
        *tps = 0;
        *rows = 0;
        return;
    }
    const int target = 152 * 8;
    const int ns = std::max(1, std::min(ntile, (target + nblk - 1) / nblk));
    *tps = (ntile + ns - 1) / ns;
    *rows = (ntile + *tps - 1) / *tps;
}

int esp_packed_rows(int npairs, int nblk)
{
    int tps, rows;
    pk_plan((npairs + PK_TP - 1) / PK_TP, nblk, &tps, &rows);
    return rows;
}

template <int L, int PPT>
static int esp_packed_launch(pcm_ctx *c, PairClass &pc, int jbeg, int jend, const int *blk, const int *bcls,
                             int nblk, double *part)
{
    using Ly = PkLayout<L>;
    const int ntile = (jend - jbeg + PK_TP - 1) / PK_TP;
    if (ntile <= 0) return PCM_OK;
    PCM_TRY(pc.tfar.alloc((size_t)ntile * Ly::FAR));
    PCM_TRY(pc.tnear.alloc((size_t)c->ncls * ntile * Ly::NEAR));
    PCM_TRY(device_error_flag(c));
    esp_tile_prep_kernel<L><<<(ntile * PK_TP + 127) / 128, 128, 0, c->stream>>>(
        pc.nesp, jbeg, jend, ntile, c->ncls, c->cls_zeta.p, pc.eP.p, pc.eD.p, pc.tfar.p, pc.tnear.p);
    PCM_LAUNCHED(c);
    int tps, rows;
    pk_plan(ntile, nblk, &tps, &rows);
    if (c->jobs) {
        // a batch: the blocks join one launch per class with the other molecules'
        const std::vector<int> &hoff = c->h_pblk[PPT == 4 ? 0 : 1], &hcls = c->h_pbcls[PPT == 4 ? 0 : 1];
        if ((int)hcls.size() != nblk) {
            set_last_error("batched ESP: point blocks do not match");
            return PCM_ERR_ARG;
        }
        auto &v = c->jobs->esp[L][PPT == 4 ? 1 : 0];
        for (int y = 0; y < rows; ++y)
            for (int x = 0; x < nblk; ++x) {
                EspJob jb;
                jb.far = pc.tfar.p;
                jb.near = pc.tnear.p;
                jb.ph = c->p32.p;
                jb.pl = c->p32lo.p;
                jb.part = part + (size_t)y * c->M;
                jb.ntile = ntile;
                jb.M = c->M;
                jb.k0 = hoff[x];
                jb.k1 = hoff[x + 1];
                jb.e = hcls[x];
                jb.t0 = y * tps;
                jb.nt = std::max(0, std::min(ntile, jb.t0 + tps) - jb.t0);
                jb.pad = 0;
                v.push_back(jb);
            }
        return PCM_OK;
    }
    dim3 grid(nblk, rows);
    esp_kernel_f32x2<L, PPT><<<grid, PK_NT, 0, c->stream>>>(ntile, tps, pc.tfar.p, pc.tnear.p, blk, bcls, c->p32.p,
                                                           c->p32lo.p, c->boys32.p, c->M, part, c->dev_err.p);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

int esp_packed(pcm_ctx *c, PairClass &pc, int L, int ppt, int jbeg, int jend, const int *blk, const int *bcls,
               int nblk, double *part)
{
#define PCM_PK(LL)                                                                                   \
    case LL:                                                                                         \
        return ppt == 4 ? esp_packed_launch<LL, 4>(c, pc, jbeg, jend, blk, bcls, nblk, part)         \
                        : esp_packed_launch<LL, 2>(c, pc, jbeg, jend, blk, bcls, nblk, part);
    switch (L) {
        PCM_PK(0)
        PCM_PK(1)
        PCM_PK(2)
        PCM_PK(3)
        PCM_PK(4)
    }
#undef PCM_PK
    return PCM_ERR_ARG;
}

// the packed ESP blocks of a batch (job table on the device), one launch
int esp_packed_jobs(int L, int ppt, const EspJob *jobs, int njob, const float *boys, int *err, cudaStream_t s)
{
#define PCM_PKJ(LL)                                                                                  \
    case LL:                                                                                         \
        if (ppt == 4) esp_jobs_kernel<LL, 4><<<njob, PK_NT, 0, s>>>(jobs, boys, err);               \
        else esp_jobs_kernel<LL, 2><<<njob, PK_NT, 0, s>>>(jobs, boys, err);                        \
        break;
    switch (L) {
        PCM_PKJ(0)
        PCM_PKJ(1)
        PCM_PKJ(2)
        PCM_PKJ(3)
        PCM_PKJ(4)
    default: return PCM_ERR_ARG;
    }
#undef PCM_PKJ
    PCM_CUDA(cudaGetLastError());
    return PCM_OK;
}

}  // namespace pcm
