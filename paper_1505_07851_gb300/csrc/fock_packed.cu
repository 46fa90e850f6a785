// PCM_MIXED Fock accumulation W_tuv = sum_k q_k U R_tuv(k) over the surface
// points for every primitive pair, two points per packed FP32x2 instruction,
// with the far-field path of farfield.cuh.
//
// Far from a pair (T = rho R^2 >= far_T(L)) U R_tuv equals sqrt(pi)/(2 sqrt(p))
// times the Hermite recurrence built on Rn[n] = (-1)^n (2n-1)!! R^-(2n+1),
// whatever the point's exponent.  So every interaction is accumulated in units
// of sqrt(pi)/(2 sqrt(p)): far interactions with those Rn times q_k, near ones
// (T < far_T, tabulated Boys function) with q_k cn (-2 rho)^n F_n, where
// cn = 2 U sqrt(p / pi) is a per-(pair, class) constant; the unit is applied
// once per pair at the end.  A warp takes the near form for a slot of two
// points only when one of its interactions needs it, and then selects it per
// lane before the recurrence.
//
// Points are staged per tile of 128 points of one class, negated and
// lane-interleaved (points 2s and 2s+1 of slot s in the two lanes), in global
// memory exactly as in shared memory; one thread streams the tiles into a
// ring of three buffers with bulk copies (pipeline.cuh).  Tile sums run in
// FP32 per lane (64 points) and go into double-float (FP32 hi + lo)
// accumulators after every tile.
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

constexpr int FK_NT = 128;     // threads per block
constexpr int FK_TQ = 128;     // points per tile
constexpr int FK_NS = 64;      // slots (two points each) per tile
constexpr int FK_TILE = 3 * 4 * FK_NS + 2 * FK_NS;   // floats per tile: P0, P1, P2 (float4), P3 (float2)
constexpr int FK_NC = 5;       // near constants per (class, pair): rho hi, rho lo, rho lo / hi, cn, R^2 threshold

// tiles of FK_TQ points of one class each, in point order (the last tile of a
// class padded); rebuilt with every surface
int fock_point_tiles_map(pcm_ctx *c)
{
    c->h_fk_cls.clear();
    c->h_fk_k0.clear();
    for (int e = 0; e < c->ncls; ++e)
        for (int k = c->h_cls_off[e]; k < c->h_cls_off[e + 1]; k += FK_TQ) {
            c->h_fk_cls.push_back(e);
            c->h_fk_k0.push_back(k);
        }
    c->fk_ntile = (int)c->h_fk_cls.size();
    if (c->fk_ntile == 0) return PCM_OK;
    PCM_TRY(c->fk_cls.alloc(c->fk_ntile));
    PCM_TRY(c->fk_k0.alloc(c->fk_ntile));
    PCM_CUDA(cudaMemcpyAsync(c->fk_cls.p, c->h_fk_cls.data(), c->fk_ntile * sizeof(int), cudaMemcpyHostToDevice,
                             c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->fk_k0.p, c->h_fk_k0.data(), c->fk_ntile * sizeof(int), cudaMemcpyHostToDevice,
                             c->stream));
    return PCM_OK;
}

// point tiles for one Fock call: negated split coordinates and q_k; padding
// points far away with q = 0
__global__ void fock_point_tiles_kernel(int ntile, const int *__restrict__ tile_cls, const int *__restrict__ tile_k0,
                                        const int *__restrict__ cls_off, const float *__restrict__ ph,
                                        const float *__restrict__ pl, const double *__restrict__ q, int M,
                                        float *__restrict__ tiles)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ntile * FK_TQ) return;
    const int t = r / FK_TQ, i = r % FK_TQ, s = i >> 1, l = i & 1;
    const int k = tile_k0[t] + i;
    const bool v = k < cls_off[tile_cls[t] + 1];
    float *T = tiles + (size_t)t * FK_TILE;
    T[4 * s + l] = v ? -ph[k] : -1.0e4f;
    T[4 * s + 2 + l] = v ? -ph[(size_t)M + k] : -1.0e4f;
    T[4 * FK_NS + 4 * s + l] = v ? -ph[2 * (size_t)M + k] : -1.0e4f;
    T[4 * FK_NS + 4 * s + 2 + l] = v ? (float)q[k] : 0.f;
    T[8 * FK_NS + 4 * s + l] = v ? -pl[k] : 0.f;
    T[8 * FK_NS + 4 * s + 2 + l] = v ? -pl[(size_t)M + k] : 0.f;
    T[12 * FK_NS + 2 * s + l] = v ? -pl[2 * (size_t)M + k] : 0.f;
}

// near constants of every (class, pair) of class L
template <int L>
__global__ void fock_near_prep_kernel(int npair, int ncls, const double *__restrict__ gp,
                                      const double *__restrict__ cls_zeta, float *__restrict__ nc)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npair) return;
    const double p = gp[j];
    for (int e = 0; e < ncls; ++e) {
        const double z2 = cls_zeta[e] * cls_zeta[e];
        const double inv = 1.0 / (p + z2);
        const double rho = p * z2 * inv;
        const double U = sqrt(z2 * inv);
        const float rh = (float)rho;
        float *N = nc + (size_t)e * FK_NC * npair;
        N[j] = rh;
        N[(size_t)npair + j] = (float)(rho - (double)rh);
        N[2 * (size_t)npair + j] = (float)((rho - (double)rh) / (double)rh);
        N[3 * (size_t)npair + j] = (float)(2.0 * U * sqrt(p / PCM_PI));
        N[4 * (size_t)npair + j] = (float)((double)far_T(L) / rho);
    }
}

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// resident blocks per SM the register allocation aims for (no spills at these)
constexpr int fk_min_blocks(int L, int NPT)
{
    return L == 0 ? 5 : (L == 1 ? (NPT == 2 ? 4 : 5) : (L == 2 ? (NPT == 2 ? 3 : 4) : (L == 3 ? 3 : (L == 4 ? 2 : 1))));
}

// Block x: pairs (x NPT + i) FK_NT + threadIdx.x, i < NPT; block y: the tiles
// [y tps, (y + 1) tps).  W[y][h][pair] receives that split's sum.
template <int L, int NPT>
__device__ __forceinline__ void fock_block(int bx, int by, int npair, const double *__restrict__ gp,
                                           const float *__restrict__ Phl, const float *__restrict__ nc, int ntile,
                                           int tps, const float *__restrict__ tiles,
                                           const int *__restrict__ tile_cls, const float *__restrict__ boys,
                                           double *__restrict__ W, int *__restrict__ err)
{
    constexpr int NH = nherm(L);
    constexpr int NSTAGE = 3;
    __shared__ __align__(16) TileRing<NSTAGE, FK_TILE> ring;
    const int t0 = by * tps;
    const int nt = max(0, min(ntile, t0 + tps) - t0);
    if (threadIdx.x == 0) ring.init(FK_NT / 32);
    __syncthreads();
    int issued = 0;
    auto issue = [&](int j) {
        mbar_expect_tx(ring.full_bar(j), (uint32_t)(FK_TILE * sizeof(float)));
        bulk_g2s(ring.data(j), tiles + (size_t)(t0 + j) * FK_TILE, FK_TILE * sizeof(float), ring.full_bar(j));
        issued = j + 1;
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < min(NSTAGE, nt); ++j) issue(j);

    int r[NPT];
    f2 Pxh[NPT], Pyh[NPT], Pzh[NPT], Pxl[NPT], Pyl[NPT], Pzl[NPT];
    float ah[NPT][NH], al[NPT][NH];
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
        r[i] = (bx * NPT + i) * FK_NT + threadIdx.x;
        const int rr = min(r[i], npair - 1);
        Pxh[i] = f2(Phl[rr]);
        Pyh[i] = f2(Phl[(size_t)npair + rr]);
        Pzh[i] = f2(Phl[2 * (size_t)npair + rr]);
        Pxl[i] = f2(Phl[3 * (size_t)npair + rr]);
        Pyl[i] = f2(Phl[4 * (size_t)npair + rr]);
        Pzl[i] = f2(Phl[5 * (size_t)npair + rr]);
#pragma unroll
        for (int h = 0; h < NH; ++h) ah[i][h] = al[i][h] = 0.f;
    }
    int cur = -1;
    float rh[NPT], rl[NPT], dr[NPT], cn[NPT], rf[NPT];
    int j = 0;
    bool ok = true;
    for (; j < nt; ++j) {
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
        const int e = tile_cls[t0 + j];
        if (e != cur) {
            cur = e;
            const float *N = nc + (size_t)e * FK_NC * npair;
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
                const int rr = min(r[i], npair - 1);
                rh[i] = N[rr];
                rl[i] = N[(size_t)npair + rr];
                dr[i] = N[2 * (size_t)npair + rr];
                cn[i] = N[3 * (size_t)npair + rr];
                rf[i] = N[4 * (size_t)npair + rr];
            }
        }
        const float *tile = ring.data(j);
        const float4 *sP = reinterpret_cast<const float4 *>(tile);
        const float2 *sZl = reinterpret_cast<const float2 *>(tile + 12 * FK_NS);
        f2 w32[NPT][NH];
#pragma unroll
        for (int i = 0; i < NPT; ++i)
#pragma unroll
            for (int h = 0; h < NH; ++h) w32[i][h] = f2(0.f);
#pragma unroll 1
        for (int s = 0; s < FK_NS; ++s) {
            const float4 p0 = sP[s], p1 = sP[FK_NS + s], p2 = sP[2 * FK_NS + s];
            const float2 p3 = sZl[s];
            const f2 Hx(p0.x, p0.y), Hy(p0.z, p0.w), Hz(p1.x, p1.y), Q(p1.z, p1.w);
            const f2 Lx(p2.x, p2.y), Ly(p2.z, p2.w), Lz(p3.x, p3.y);
            f2 X[NPT], Y[NPT], Z[NPT], R2[NPT];
            bool nr = false;
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
                X[i] = (Pxh[i] + Hx) + (Pxl[i] + Lx);
                Y[i] = (Pyh[i] + Hy) + (Pyl[i] + Ly);
                Z[i] = (Pzh[i] + Hz) + (Pzl[i] + Lz);
                R2[i] = fma2(X[i], X[i], fma2(Y[i], Y[i], Z[i] * Z[i]));
                nr |= (R2[i].v.x < rf[i]) | (R2[i].v.y < rf[i]);
            }
            const bool general = __any_sync(0xffffffffu, nr);
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
                // far form: q (-1)^n (2n-1)!! R^-(2n+1), 1/R with one Newton step
                const f2 r0(rsqrt_fast(R2[i].v.x), rsqrt_fast(R2[i].v.y));
                const f2 em = fma2(R2[i] * r0, r0, f2(-1.f));
                const f2 rs = fma2(r0 * f2(-0.5f), em, r0);
                f2 Rn[L + 1];
                Rn[0] = Q * rs;
                if constexpr (L > 0) {
                    const f2 rs2 = rs * rs;
#pragma unroll
                    for (int n = 1; n <= L; ++n) Rn[n] = (Rn[n - 1] * rs2) * f2(-(float)(2 * n - 1));
                }
                if (general) {
                    // near form in the lanes that need it: q cn (-2 rho)^n F_n
                    const bool n0 = R2[i].v.x < rf[i], n1 = R2[i].v.y < rf[i];
                    const f2 rhv(rh[i]);
                    f2 T = fma2(rhv, R2[i], f2(rl[i]) * R2[i]);
                    T = f2(fminf(T.v.x, far_T(L)), fminf(T.v.y, far_T(L)));
                    const f2 t = fma2(T, f2((float)BOYS_INV_DT), f2(12582912.0f));
                    const int i0 = __float_as_int(t.v.x) - 0x4B400000, i1 = __float_as_int(t.v.y) - 0x4B400000;
                    const f2 d = fma2(t + f2(-12582912.0f), f2(-(float)BOYS_DT), T);
                    float fa[L + 1], fb[L + 1];
                    boys_near32<L>(i0, d.v.x, boys, fa);
                    boys_near32<L>(i1, d.v.y, boys, fb);
                    const f2 m2r = rhv * f2(-2.f);
                    f2 f = Q * f2(cn[i]);
#pragma unroll
                    for (int n = 0; n <= L; ++n) {
                        const f2 v = f * f2(fa[n], fb[n]);
                        const f2 rn = (n == 0) ? v : fma2(v, f2((float)n * dr[i]), v);
                        Rn[n] = f2(n0 ? rn.v.x : Rn[n].v.x, n1 ? rn.v.y : Rn[n].v.y);
                        if (n < L) f = f * m2r;
                    }
                }
                if constexpr (L == 0) {
                    w32[i][0] += Rn[0];
                } else {
                    f2 R[NH];
                    hermite_R<L, f2>(X[i], Y[i], Z[i], Rn, R);
#pragma unroll
                    for (int h = 0; h < NH; ++h) w32[i][h] += R[h];
                }
            }
        }
        // fold the tile: each lane into the double-float accumulators
#pragma unroll
        for (int i = 0; i < NPT; ++i)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                float s, e2, s2, e3;
                two_sum_f(ah[i][h], w32[i][h].v.x, s, e2);
                two_sum_f(s, w32[i][h].v.y, s2, e3);
                ah[i][h] = s2;
                al[i][h] += e2 + e3;
            }
        ring.release(j);
    }
    if (!ok) {
        if ((threadIdx.x & 31) == 0) atomicExch(err, 1);
        if (threadIdx.x == 0)
            for (int jj = j; jj < issued; ++jj) ring.wait_full(jj);
        return;
    }
#pragma unroll
    for (int i = 0; i < NPT; ++i)
        if (r[i] < npair) {
            // the unit of the accumulators: sqrt(pi) / (2 sqrt(p))
            const double g = 0.88622692545275801365 / sqrt(gp[r[i]]);
#pragma unroll
            for (int h = 0; h < NH; ++h)
                W[((size_t)by * NH + h) * npair + r[i]] = g * ((double)ah[i][h] + (double)al[i][h]);
        }
}

template <int L, int NPT>
__global__ void __launch_bounds__(FK_NT, fk_min_blocks(L, NPT))
    fock_kernel_f32x2(int npair, const double *__restrict__ gp, const float *__restrict__ Phl,
                      const float *__restrict__ nc, int ntile, int tps, const float *__restrict__ tiles,
                      const int *__restrict__ tile_cls, const float *__restrict__ boys, double *__restrict__ W,
                      int *__restrict__ err)
{
    fock_block<L, NPT>(blockIdx.x, blockIdx.y, npair, gp, Phl, nc, ntile, tps, tiles, tile_cls, boys, W, err);
}

// The same for a table of blocks of many molecules (one launch per class)
template <int L, int NPT>
__global__ void __launch_bounds__(FK_NT, fk_min_blocks(L, NPT))
    fock_jobs_kernel(const FockJob *__restrict__ jobs, const float *__restrict__ boys, int *__restrict__ err)
{
    const FockJob &j = jobs[blockIdx.x];
    fock_block<L, NPT>(j.bx, j.by, j.npair, j.gp, j.Phl, j.nc, j.ntile, j.tps, j.tiles, j.tile_cls, boys, j.W, err);
}

template <int L, int NPT>
static int fock_packed_launch(pcm_ctx *c, int npair, const double *gp, const float *Phl, DBuf<float> &nbuf,
                              const double *dq, int nsplit, double *W)
{
    const int ntile = c->fk_ntile;
    PCM_TRY(c->fk_tiles.alloc((size_t)std::max(1, ntile) * FK_TILE));
    PCM_TRY(nbuf.alloc((size_t)c->ncls * FK_NC * npair));
    PCM_TRY(device_error_flag(c));
    if (ntile > 0) {
        fock_point_tiles_kernel<<<(ntile * FK_TQ + 127) / 128, 128, 0, c->stream>>>(
            ntile, c->fk_cls.p, c->fk_k0.p, c->cls_off.p, c->p32.p, c->p32lo.p, dq, c->M, c->fk_tiles.p);
        PCM_LAUNCHED(c);
    }
    fock_near_prep_kernel<L><<<(npair + 127) / 128, 128, 0, c->stream>>>(npair, c->ncls, gp, c->cls_zeta.p, nbuf.p);
    PCM_LAUNCHED(c);
    const int tps = std::max(1, (ntile + nsplit - 1) / nsplit);
    const int nb = (npair + FK_NT * NPT - 1) / (FK_NT * NPT);
    if (c->jobs) {
        // a batch: the blocks join one launch per class with the other molecules'
        auto &v = c->jobs->fock[L][NPT == 2 ? 1 : 0];
        for (int by = 0; by < nsplit; ++by)
            for (int bx = 0; bx < nb; ++bx) {
                FockJob fj;
                fj.gp = gp;
                fj.Phl = Phl;
                fj.nc = nbuf.p;
                fj.tiles = c->fk_tiles.p;
                fj.tile_cls = c->fk_cls.p;
                fj.W = W;
                fj.npair = npair;
                fj.ntile = ntile;
                fj.tps = tps;
                fj.bx = bx;
                fj.by = by;
                fj.pad = 0;
                v.push_back(fj);
            }
        return PCM_OK;
    }
    dim3 grid(nb, nsplit);
    fock_kernel_f32x2<L, NPT><<<grid, FK_NT, 0, c->stream>>>(npair, gp, Phl, nbuf.p, ntile, tps, c->fk_tiles.p,
                                                            c->fk_cls.p, c->boys32.p, W, c->dev_err.p);
    PCM_LAUNCHED(c);
    return PCM_OK;
}

// W[nsplit][nherm(L)][npair] over npair primitive pairs (exponent sums gp,
// split centres Phl: 6 x npair, hi then lo) for charges dq; every split is
// written (splits without tiles with zeros).  Two pairs per thread for L <= 2.
int fock_packed(pcm_ctx *c, int L, int npt, int npair, const double *gp, const float *Phl, DBuf<float> &nbuf,
                const double *dq, int nsplit, double *W)
{
    if (npair <= 0) return PCM_OK;
    const bool two = npt == 2 && L <= 2;
    switch (L) {
    case 0: return two ? fock_packed_launch<0, 2>(c, npair, gp, Phl, nbuf, dq, nsplit, W)
                       : fock_packed_launch<0, 1>(c, npair, gp, Phl, nbuf, dq, nsplit, W);
    case 1: return two ? fock_packed_launch<1, 2>(c, npair, gp, Phl, nbuf, dq, nsplit, W)
                       : fock_packed_launch<1, 1>(c, npair, gp, Phl, nbuf, dq, nsplit, W);
    case 2: return two ? fock_packed_launch<2, 2>(c, npair, gp, Phl, nbuf, dq, nsplit, W)
                       : fock_packed_launch<2, 1>(c, npair, gp, Phl, nbuf, dq, nsplit, W);
    case 3: return fock_packed_launch<3, 1>(c, npair, gp, Phl, nbuf, dq, nsplit, W);
    case 4: return fock_packed_launch<4, 1>(c, npair, gp, Phl, nbuf, dq, nsplit, W);
    case 5: return fock_packed_launch<5, 1>(c, npair, gp, Phl, nbuf, dq, nsplit, W);
    }
    return PCM_ERR_ARG;
}

// Launch every block collected from a batch's molecules: one launch per
// (kernel, angular momentum, points or pairs per thread).  The job tables are
// copied from the sink (kept by the caller until the stream has run them).
int launch_jobs(JobSink &sink, DBuf<EspJob> &dej, DBuf<FockJob> &dfj, const float *boys, int *err, cudaStream_t s)
{
    size_t ne = 0, nf = 0;
    for (auto &v : sink.esp)
        for (auto &w : v) ne += w.size();
    for (auto &v : sink.fock)
        for (auto &w : v) nf += w.size();
    if (ne) PCM_TRY(dej.alloc(ne));
    if (nf) PCM_TRY(dfj.alloc(nf));
    size_t o = 0;
    for (int L = 0; L < 5; ++L)
        for (int v = 0; v < 2; ++v) {
            const auto &w = sink.esp[L][v];
            if (w.empty()) continue;
            PCM_CUDA(cudaMemcpyAsync(dej.p + o, w.data(), w.size() * sizeof(EspJob), cudaMemcpyHostToDevice, s));
            PCM_TRY(esp_packed_jobs(L, v == 1 ? 4 : 2, dej.p + o, (int)w.size(), boys, err, s));
            o += w.size();
        }
    o = 0;
    for (int L = 0; L < 6; ++L)
        for (int v = 0; v < 2; ++v) {
            const auto &w = sink.fock[L][v];
            if (w.empty()) continue;
            PCM_CUDA(cudaMemcpyAsync(dfj.p + o, w.data(), w.size() * sizeof(FockJob), cudaMemcpyHostToDevice, s));
            switch (L) {
            case 0: v ? fock_jobs_kernel<0, 2><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err)
                      : fock_jobs_kernel<0, 1><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err); break;
            case 1: v ? fock_jobs_kernel<1, 2><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err)
                      : fock_jobs_kernel<1, 1><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err); break;
            case 2: v ? fock_jobs_kernel<2, 2><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err)
                      : fock_jobs_kernel<2, 1><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err); break;
            case 3: fock_jobs_kernel<3, 1><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err); break;
            case 4: fock_jobs_kernel<4, 1><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err); break;
            case 5: fock_jobs_kernel<5, 1><<<(unsigned)w.size(), FK_NT, 0, s>>>(dfj.p + o, boys, err); break;
            }
            PCM_CUDA(cudaGetLastError());
            o += w.size();
        }
    return PCM_OK;
}

}  // namespace pcm
