// Basis set-up and the primitive-pair list with the Schwarz-type screening of
// Eq. 15 (Section 4a).
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "context.h"

namespace pcm {

__host__ __device__ inline int class_index(int la, int lb) { return la * (la + 1) / 2 + lb; }

// coefficient x (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!): normalisation of the
// x^l component; the other Cartesian components differ by comp_factor().
__global__ void cnorm_kernel(int nshell, const int *__restrict__ sh_l, const int *__restrict__ sh_nprim,
                             const int *__restrict__ sh_off, const double *__restrict__ exps,
                             const double *__restrict__ coefs, double *__restrict__ cnorm)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshell) return;
    const int l = sh_l[s];
    double dfl = 1.0;
    for (int k = 2 * l - 1; k > 1; k -= 2) dfl *= k;
    for (int i = 0; i < sh_nprim[s]; ++i) {
        const double a = exps[sh_off[s] + i];
        cnorm[sh_off[s] + i] = coefs[sh_off[s] + i] * pow(2.0 * a / PCM_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfl);
    }
}

// sqrt((2l-1)!! / ((2lx-1)!! (2ly-1)!! (2lz-1)!!)) for l <= 2
__device__ inline double comp_factor(int l, int c)
{
    if (l < 2) return 1.0;
    return (c == 1 || c == 2 || c == 4) ? 1.7320508075688772935 : 1.0;  // xy, xz, yz
}

// (T-1)!! for even T >= 0
__device__ inline double dfact_even(int T)
{
    double r = 1.0;
    for (int k = T - 1; k > 1; k -= 2) r *= k;
    return r;
}

// TS: arithmetic of the Schwarz bound (FP64, or FP32 for PCM_MIXED, where a
// bound off by 1e-6 relative only moves pairs at the cutoff whose
// contributions are of the cutoff's size); the pair data are FP64 either way.
template <int LA, int LB, typename TS>
__global__ void pair_screen_kernel(long long ncand, int nsp, const long long *__restrict__ sp_cand,
                                   const int *__restrict__ spA, const int *__restrict__ spB,
                                   const int *__restrict__ sh_atom, const int *__restrict__ sh_nprim,
                                   const int *__restrict__ sh_off, const double *__restrict__ exps,
                                   const double *__restrict__ cnorm, const double *__restrict__ xyz, double thresh,
                                   int *__restrict__ o_sp, int *__restrict__ o_i, int *__restrict__ o_j,
                                   double *__restrict__ o_P, double *__restrict__ o_p, double *__restrict__ o_pref,
                                   double *__restrict__ o_Q, unsigned char *__restrict__ flag)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncand) return;
    // shell pair holding candidate g
    int lo = 0, hi = nsp - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sp_cand[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const int s = lo;
    const int A = spA[s], B = spB[s];
    int r = (int)(g - sp_cand[s]);
    int i, j;
    if (A == B) {
        const int n = sh_nprim[A];
        i = 0;
        while (r >= n - i) {
            r -= n - i;
            ++i;
        }
        j = i + r;
    } else {
        const int nb = sh_nprim[B];
        i = r / nb;
        j = r - i * nb;
    }
    const double a = exps[sh_off[A] + i], b = exps[sh_off[B] + j];
    const double *RA = xyz + 3 * sh_atom[A], *RB = xyz + 3 * sh_atom[B];
    const double p = a + b;
    // one FP64 division per candidate (the FP64 pipe runs at 1/64 of FP32 here)
    const double ip = 1.0 / p;
    double P[3], ab2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        P[d] = (a * RA[d] + b * RB[d]) * ip;
        const double t = RA[d] - RB[d];
        ab2 += t * t;
    }
    const double K = exp(-a * b * ip * ab2);
    const double pref = 2.0 * PCM_PI * ip * K;

    // Schwarz bound |c_i c_j| max_{ab} N_a N_b [ab|ab]^(1/2) from the
    // McMurchie-Davidson diagonal two-electron integral at zero separation
    //   [ab|ab] = 2 pi^(5/2) / (p^2 sqrt(2p)) K^2
    //             sum_{tuv,t'u'v'} E_tuv E_t'u'v' (-1)^(t'+u'+v') R_{t+t',u+u',v+v'}(p/2, 0),
    // R_{TUV}(alpha, 0) = (-2 alpha)^((T+U+V)/2) (T-1)!!(U-1)!!(V-1)!! / (T+U+V+1)
    // for even T, U, V and 0 otherwise.
    E1T<LA, LB, TS> Ex, Ey, Ez;
    const TS inv2p = TS(0.5 * ip);
    // 2 pi^(5/2) / (p^2 sqrt(2 p)) K^2 (2 pi^(5/2) = 2 * 17.4934...)
    const double eri_pre = 2.0 * 17.493418327624862846 * ip * ip * sqrt(0.5 * ip) * K * K;
    hermite_E1T<LA, LB, TS>(TS(P[0] - RA[0]), TS(P[0] - RB[0]), inv2p, Ex);
    hermite_E1T<LA, LB, TS>(TS(P[1] - RA[1]), TS(P[1] - RB[1]), inv2p, Ey);
    hermite_E1T<LA, LB, TS>(TS(P[2] - RA[2]), TS(P[2] - RB[2]), inv2p, Ez);
    constexpr int LL = LA + LB;
    // (-2 alpha)^n with alpha = p / 2
    TS pw[LL + 1];
    pw[0] = TS(1);
#pragma unroll
    for (int n = 1; n <= LL; ++n) pw[n] = pw[n - 1] * TS(-p);
    double qmax = 0.0;
#pragma unroll
    for (int ca = 0; ca < ncart(LA); ++ca)
#pragma unroll
        for (int cb = 0; cb < ncart(LB); ++cb) {
            const int ax = cart_e(LA, ca, 0), ay = cart_e(LA, ca, 1), az = cart_e(LA, ca, 2);
            const int bx = cart_e(LB, cb, 0), by = cart_e(LB, cb, 1), bz = cart_e(LB, cb, 2);
            TS Gx[2 * LL + 1], Gy[2 * LL + 1], Gz[2 * LL + 1];
#pragma unroll
            for (int t = 0; t <= 2 * LL; ++t) Gx[t] = Gy[t] = Gz[t] = TS(0);
            // E_t vanishes for t > i + j, so the full loops add exact zeros there
#pragma unroll
            for (int t = 0; t <= LL; ++t)
#pragma unroll
                for (int t2 = 0; t2 <= LL; ++t2) {
                    const TS sg = (t2 & 1) ? TS(-1) : TS(1);
                    Gx[t + t2] += Ex.e[ax][bx][t] * Ex.e[ax][bx][t2] * sg;
                    Gy[t + t2] += Ey.e[ay][by][t] * Ey.e[ay][by][t2] * sg;
                    Gz[t + t2] += Ez.e[az][bz][t] * Ez.e[az][bz][t2] * sg;
                }
            TS sum = TS(0);
#pragma unroll
            for (int T = 0; T <= 2 * LL; T += 2)
#pragma unroll
                for (int U = 0; U <= 2 * LL - T; U += 2)
#pragma unroll
                    for (int V = 0; V <= 2 * LL - T - U; V += 2) {
                        const int n = (T + U + V) / 2;
                        const TS R = TS(dfact_even(T) * dfact_even(U) * dfact_even(V) / (T + U + V + 1)) * pw[n];
                        sum += Gx[T] * Gy[U] * Gz[V] * R;
                    }
            const double eri = eri_pre * (double)sum;
            const double f = comp_factor(LA, ca) * comp_factor(LB, cb);
            qmax = fmax(qmax, f * f * fabs(eri));
        }
    const double Q = fabs(cnorm[sh_off[A] + i] * cnorm[sh_off[B] + j]) * sqrt(qmax);
    const bool keep = thresh <= 0.0 || Q >= thresh;
    flag[g] = keep ? 1 : 0;
    if (!keep) return;   // only kept candidates are gathered
    o_sp[g] = s;
    o_i[g] = i;
    o_j[g] = j;
    o_P[3 * g + 0] = P[0];
    o_P[3 * g + 1] = P[1];
    o_P[3 * g + 2] = P[2];
    o_p[g] = p;
    o_pref[g] = pref;
    o_Q[g] = Q;
}

__global__ void pair_gather_kernel(int n, const int *__restrict__ idx, const int *__restrict__ c_sp,
                                   const int *__restrict__ c_i, const int *__restrict__ c_j,
                                   const double *__restrict__ c_P, const double *__restrict__ c_p,
                                   const double *__restrict__ c_pref, const double *__restrict__ c_Q, int *sp, int *ia,
                                   int *ib, double *Px, double *Py, double *Pz, double *p, double *pref, double *Q,
                                   float *P32)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int g = idx[r];
    sp[r] = c_sp[g];
    ia[r] = c_i[g];
    ib[r] = c_j[g];
    Px[r] = c_P[3 * g + 0];
    Py[r] = c_P[3 * g + 1];
    Pz[r] = c_P[3 * g + 2];
    p[r] = c_p[g];
    pref[r] = c_pref[g];
    Q[r] = c_Q[g];
    // FP32 hi/lo split of the centre: hi on a 2^-10 grid, so that differences of
    // hi parts are exact in FP32
    for (int d = 0; d < 3; ++d) {
        const double v = c_P[3 * g + d];
        const double h = rint(v * 1024.0) * (1.0 / 1024.0);
        P32[(size_t)d * n + r] = (float)h;
        P32[(size_t)(3 + d) * n + r] = (float)(v - h);
    }
}

__global__ void sp_start_kernel(int nsp, const long long *__restrict__ sp_cand, const int *__restrict__ pos,
                                int *__restrict__ sp_start)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= nsp) sp_start[s] = pos[sp_cand[s]];
}

template <int LA, int LB>
static int screen_class(pcm_ctx *c, PairClass &pc)
{
    DBuf<int> &c_sp = c->si[0], &c_i = c->si[1], &c_j = c->si[2], &pos = c->si[3];
    DBuf<double> &c_P = c->sd[0], &c_p = c->sd[1], &c_pref = c->sd[2], &c_Q = c->sd[3];
    DBuf<unsigned char> &flag = c->su8[0];
    const long long n = pc.ncand;
    PCM_TRY(c_sp.alloc(n));
    PCM_TRY(c_i.alloc(n));
    PCM_TRY(c_j.alloc(n));
    PCM_TRY(c_P.alloc(3 * n));
    PCM_TRY(c_p.alloc(n));
    PCM_TRY(c_pref.alloc(n));
    PCM_TRY(c_Q.alloc(n));
    PCM_TRY(flag.alloc(n));
    PCM_TRY(pos.alloc(n + 1));
    if (n > 0) {
        const unsigned grid = (unsigned)((n + 127) / 128);
        if (c->opt.precision == PCM_MIXED)
            pair_screen_kernel<LA, LB, float><<<grid, 128, 0, c->stream>>>(
                n, pc.nsp, pc.sp_cand.p, pc.spA.p, pc.spB.p, c->sh_atom.p, c->sh_nprim.p, c->sh_off.p, c->exps.p,
                c->cnorm.p, c->xyz.p, c->opt.schwarz, c_sp.p, c_i.p, c_j.p, c_P.p, c_p.p, c_pref.p, c_Q.p, flag.p);
        else
            pair_screen_kernel<LA, LB, double><<<grid, 128, 0, c->stream>>>(
                n, pc.nsp, pc.sp_cand.p, pc.spA.p, pc.spB.p, c->sh_atom.p, c->sh_nprim.p, c->sh_off.p, c->exps.p,
                c->cnorm.p, c->xyz.p, c->opt.schwarz, c_sp.p, c_i.p, c_j.p, c_P.p, c_p.p, c_pref.p, c_Q.p, flag.p);
        PCM_LAUNCHED(c);
    }
    DBuf<int> &idx = c->si[4];
    PCM_TRY(idx.alloc(n));
    PCM_TRY(compact_flags(c, flag.p, n, idx.p, pos.p, c->iscal.p));
    int kept = 0;
    PCM_CUDA(cudaMemcpyAsync(&kept, c->iscal.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PCM_CUDA(cudaStreamSynchronize(c->stream));
    pc.npair = kept;
    PCM_TRY(pc.sp.alloc(kept));
    PCM_TRY(pc.ia.alloc(kept));
    PCM_TRY(pc.ib.alloc(kept));
    PCM_TRY(pc.Px.alloc(kept));
    PCM_TRY(pc.Py.alloc(kept));
    PCM_TRY(pc.Pz.alloc(kept));
    PCM_TRY(pc.p.alloc(kept));
    PCM_TRY(pc.pref.alloc(kept));
    PCM_TRY(pc.Q.alloc(kept));
    PCM_TRY(pc.Pxyz32.alloc(6 * (size_t)kept));
    if (kept > 0) {
        pair_gather_kernel<<<(kept + 127) / 128, 128, 0, c->stream>>>(
            kept, idx.p, c_sp.p, c_i.p, c_j.p, c_P.p, c_p.p, c_pref.p, c_Q.p, pc.sp.p, pc.ia.p, pc.ib.p, pc.Px.p,
            pc.Py.p, pc.Pz.p, pc.p.p, pc.pref.p, pc.Q.p, pc.Pxyz32.p);
        PCM_LAUNCHED(c);
    }
    PCM_TRY(pc.sp_start.alloc(pc.nsp + 1));
    sp_start_kernel<<<(pc.nsp + 1 + 127) / 128, 128, 0, c->stream>>>(pc.nsp, pc.sp_cand.p, pos.p, pc.sp_start.p);
    PCM_LAUNCHED(c);
    PCM_CUDA(cudaStreamSynchronize(c->stream));  // the scratch slots are reused by the next class
    return PCM_OK;
}

int basis_build(pcm_ctx *c, int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                const double *exps, const double *coefs)
{
    // expand sp shells into an s and a p shell that share exponents
    c->h_sh_atom.clear();
    c->h_sh_l.clear();
    c->h_sh_nprim.clear();
    c->h_sh_off.clear();
    c->h_sh_bf.clear();
    std::vector<double> ex, co;
    int off = 0, coff = 0, bf = 0;
    for (int s = 0; s < nshell; ++s) {
        const int l = shell_l[s], n = shell_nprim[s];
        if (n <= 0 || shell_atom[s] < 0 || shell_atom[s] >= c->natom) {
            set_last_error("shell %d: bad atom index or primitive count", s);
            return PCM_ERR_ARG;
        }
        if (l > 2 || l < -1) {
            set_last_error("shell %d: angular momentum %d is not supported (s, p, d, sp only)", s, l);
            return PCM_ERR_UNSUPPORTED;
        }
        for (int i = 0; i < n; ++i)
            if (!(exps[off + i] > 0.0) || !std::isfinite(exps[off + i])) {
                set_last_error("shell %d: exponent %d is not a positive finite number", s, i);
                return PCM_ERR_ARG;
            }
        const int nparts = (l == -1) ? 2 : 1;
        for (int part = 0; part < nparts; ++part) {
            const int ll = (l == -1) ? part : l;
            c->h_sh_atom.push_back(shell_atom[s]);
            c->h_sh_l.push_back(ll);
            c->h_sh_nprim.push_back(n);
            c->h_sh_off.push_back((int)ex.size());
            c->h_sh_bf.push_back(bf);
            for (int i = 0; i < n; ++i) {
                ex.push_back(exps[off + i]);
                const double cf = coefs[coff + part * n + i];
                if (!std::isfinite(cf)) {
                    set_last_error("shell %d: contraction coefficient %d is not finite", s, i);
                    return PCM_ERR_ARG;
                }
                co.push_back(cf);
            }
            bf += ncart(ll);
        }
        off += n;
        coff += nparts * n;
    }
    c->nshell = (int)c->h_sh_l.size();
    c->nbf = bf;
    const int ns = c->nshell;
    PCM_TRY(c->sh_atom.alloc(ns));
    PCM_TRY(c->sh_l.alloc(ns));
    PCM_TRY(c->sh_nprim.alloc(ns));
    PCM_TRY(c->sh_off.alloc(ns));
    PCM_TRY(c->sh_bf.alloc(ns));
    PCM_TRY(c->exps.alloc(ex.size()));
    PCM_TRY(c->cnorm.alloc(ex.size()));
    DBuf<double> &dco = c->sd[4];
    PCM_TRY(dco.alloc(co.size()));
    PCM_CUDA(cudaMemcpyAsync(c->sh_atom.p, c->h_sh_atom.data(), ns * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->sh_l.p, c->h_sh_l.data(), ns * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->sh_nprim.p, c->h_sh_nprim.data(), ns * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->sh_off.p, c->h_sh_off.data(), ns * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->sh_bf.p, c->h_sh_bf.data(), ns * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(c->exps.p, ex.data(), ex.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PCM_CUDA(cudaMemcpyAsync(dco.p, co.data(), co.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    cnorm_kernel<<<(ns + 127) / 128, 128, 0, c->stream>>>(ns, c->sh_l.p, c->sh_nprim.p, c->sh_off.p, c->exps.p, dco.p,
                                                         c->cnorm.p);
    PCM_LAUNCHED(c);

    // shell pairs by class (la >= lb); the higher-l shell (ties: lower index) comes
    // first.  They depend only on the shells' atoms, angular momenta and
    // primitive counts: a new geometry with the same shells (the next step of an
    // optimisation or a trajectory) reuses the lists already on the device.
    const bool same_layout = c->pair_layout_ok && c->pl_atom == c->h_sh_atom && c->pl_l == c->h_sh_l &&
                             c->pl_nprim == c->h_sh_nprim;
    if (!same_layout) {
        c->pair_layout_ok = false;
        for (int k = 0; k < 6; ++k) {
            c->cls[k].h_spA.clear();
            c->cls[k].h_spB.clear();
        }
        for (int sa = 0; sa < ns; ++sa)
            for (int sb = sa; sb < ns; ++sb) {
                int A = sa, B = sb;
                if (c->h_sh_l[sb] > c->h_sh_l[sa]) std::swap(A, B);
                const int k = class_index(c->h_sh_l[A], c->h_sh_l[B]);
                c->cls[k].h_spA.push_back(A);
                c->cls[k].h_spB.push_back(B);
            }
    }
    c->pairs_candidate = 0;
    c->pairs_kept = 0;
    PCM_TRY(c->iscal.alloc(64));
    static const int LA[6] = {0, 1, 1, 2, 2, 2}, LB[6] = {0, 0, 1, 0, 1, 2};
    for (int k = 0; k < 6; ++k) {
        PairClass &pc = c->cls[k];
        pc.la = LA[k];
        pc.lb = LB[k];
        pc.nsp = (int)pc.h_spA.size();
        if (!same_layout) {
            pc.csr_ready = false;
            std::vector<long long> cand(pc.nsp + 1, 0);
            for (int s = 0; s < pc.nsp; ++s) {
                const int A = pc.h_spA[s], B = pc.h_spB[s];
                const long long na = c->h_sh_nprim[A], nb = c->h_sh_nprim[B];
                cand[s + 1] = cand[s] + (A == B ? na * (na + 1) / 2 : na * nb);
            }
            pc.ncand = cand[pc.nsp];
            PCM_TRY(pc.spA.alloc(pc.nsp));
            PCM_TRY(pc.spB.alloc(pc.nsp));
            PCM_TRY(pc.sp_cand.alloc(pc.nsp + 1));
            if (pc.nsp > 0) {
                PCM_CUDA(cudaMemcpyAsync(pc.spA.p, pc.h_spA.data(), pc.nsp * sizeof(int), cudaMemcpyHostToDevice,
                                         c->stream));
                PCM_CUDA(cudaMemcpyAsync(pc.spB.p, pc.h_spB.data(), pc.nsp * sizeof(int), cudaMemcpyHostToDevice,
                                         c->stream));
            }
            PCM_CUDA(cudaMemcpyAsync(pc.sp_cand.p, cand.data(), (pc.nsp + 1) * sizeof(long long),
                                     cudaMemcpyHostToDevice, c->stream));
            // cand is read by the copy before it goes out of scope
            PCM_CUDA(cudaStreamSynchronize(c->stream));
        }
        switch (k) {
        case 0: PCM_TRY((screen_class<0, 0>(c, pc))); break;
        case 1: PCM_TRY((screen_class<1, 0>(c, pc))); break;
        case 2: PCM_TRY((screen_class<1, 1>(c, pc))); break;
        case 3: PCM_TRY((screen_class<2, 0>(c, pc))); break;
        case 4: PCM_TRY((screen_class<2, 1>(c, pc))); break;
        case 5: PCM_TRY((screen_class<2, 2>(c, pc))); break;
        }
        c->pairs_candidate += pc.ncand;
        c->pairs_kept += pc.npair;
    }
    if (!same_layout) {
        c->pl_atom = c->h_sh_atom;
        c->pl_l = c->h_sh_l;
        c->pl_nprim = c->h_sh_nprim;
        c->pair_layout_ok = true;
    }
    return PCM_OK;
}

}  // namespace pcm
