// C ABI of the C-PCM / ISWIG library (declared in include/pcm.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "common.cuh"
#include "context.h"

namespace pcm {

static thread_local std::string g_last_error;

void set_last_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

// rhs = -f (B z + c)  (Eq. 1)
__global__ void rhs_kernel(int M, double f, const double *__restrict__ Bz, const double *__restrict__ c,
                           double *__restrict__ rhs)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) rhs[k] = -f * (Bz[k] + c[k]);
}

// xyzzs[k] = (x, y, z, zeta, S)
__global__ void pack_surface_kernel(int M, const double *px, const double *py, const double *pz, const double *pzeta,
                                    const double *pS, double *out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    out[5 * k + 0] = px[k];
    out[5 * k + 1] = py[k];
    out[5 * k + 2] = pz[k];
    out[5 * k + 3] = pzeta[k];
    out[5 * k + 4] = pS[k];
}

static bool all_finite(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// bring an input array to the device (copy from host unless PCM_PTR_DEVICE)
static int to_device(pcm_ctx *c, const double *src, size_t n, DBuf<double> &stage, const double **out, int flags)
{
    if (flags & PCM_PTR_DEVICE) {
        *out = src;
        return PCM_OK;
    }
    if (!all_finite(src, n)) {
        set_last_error("input array holds a NaN or an infinity");
        return PCM_ERR_ARG;
    }
    PCM_TRY(stage.alloc(n));
    PCM_CUDA(cudaMemcpyAsync(stage.p, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    *out = stage.p;
    return PCM_OK;
}

static int finish(pcm_ctx *c, int flags)
{
    if (!(flags & PCM_ASYNC) || !(flags & PCM_PTR_DEVICE)) PCM_CUDA(cudaStreamSynchronize(c->stream));
    return PCM_OK;
}

}  // namespace pcm

using namespace pcm;

extern "C" {

const char *pcm_strerror(int status)
{
    switch (status) {
    case PCM_OK: return "ok";
    case PCM_ERR_ARG: return "invalid argument";
    case PCM_ERR_CUDA: return "CUDA error";
    case PCM_ERR_OOM: return "out of memory";
    case PCM_ERR_UNSUPPORTED: return "unsupported (angular momentum above d)";
    case PCM_ERR_NOT_CONVERGED: return "solver did not converge within its iteration cap";
    case PCM_ERR_TIMEOUT: return "a bounded device wait gave up";
    default: return "unknown status";
    }
}

const char *pcm_last_error(void) { return g_last_error.c_str(); }

int pcm_default_options(pcm_options *o)
{
    if (!o) return PCM_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->eps = 78.39;
    o->k = 0.0;
    o->zeta = 4.9;
    o->switch_drop = 1e-8;
    o->schwarz = 1e-12;
    o->rbj_block = 100;
    o->precond = PCM_PRECOND_AUTO;
    o->jacobi_below = 1000;
    o->precision = PCM_FP64;
    o->max_iter = 5000;
    o->device = 0;
    o->seed = 0;
    o->stream = nullptr;
    o->octree_leaf = 800;
    o->esp_variant = -1;
    o->fp32x2 = 1;
    o->operator_mode = PCM_OPERATOR_AUTO;
    return PCM_OK;
}

int pcm_create(pcm_ctx **out, const pcm_options *opt)
{
    if (!out) return PCM_ERR_ARG;
    *out = nullptr;
    pcm_options o;
    if (opt) o = *opt;
    else pcm_default_options(&o);
    if (!(o.eps > 1.0) || !(o.zeta > 0.0) || o.rbj_block < 1 || o.max_iter < 1 || o.switch_drop < 0.0 ||
        o.schwarz < 0.0 || (o.precision != PCM_FP64 && o.precision != PCM_MIXED) || o.precond < 0 || o.precond > 4 ||
        (o.precond == PCM_PRECOND_OCTREE && o.octree_leaf < 1) || o.esp_variant < -1 || o.esp_variant > 2 ||
        (o.fp32x2 != 0 && o.fp32x2 != 1) || o.operator_mode < 0 || o.operator_mode > 2) {
        set_last_error("invalid pcm_options");
        return PCM_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_last_error("no CUDA device is available");
        return PCM_ERR_CUDA;
    }
    if (o.device < 0 || o.device >= ndev) {
        set_last_error("device %d does not exist", o.device);
        return PCM_ERR_ARG;
    }
    DeviceGuard g(o.device);
    pcm_ctx *c = new (std::nothrow) pcm_ctx();
    if (!c) return PCM_ERR_OOM;
    c->opt = o;
    c->device = o.device;
    memset(&c->stats, 0, sizeof(c->stats));
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            set_last_error("cudaStreamCreate failed");
            return PCM_ERR_CUDA;
        }
        c->own_stream = true;
    }
    if (o.timing) {
        for (int i = 0; i < 14; ++i) {
            cudaEventCreate(&c->ev_a[i]);
            cudaEventCreate(&c->ev_b[i]);
        }
        c->have_events = true;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_side, cudaEventDisableTiming) != cudaSuccess) {
        set_last_error("cudaStreamCreate / cudaEventCreate failed");
        pcm_destroy(c);
        return PCM_ERR_CUDA;
    }
    int st = boys_build_tables(c);
    if (st != PCM_OK) {
        pcm_destroy(c);
        return st;
    }
    *out = c;
    return PCM_OK;
}

int pcm_destroy(pcm_ctx *c)
{
    if (!c) return PCM_OK;
    DeviceGuard g(c->device);
    if (c->side) cudaStreamSynchronize(c->side);
    cudaStreamSynchronize(c->stream);
    if (c->have_events)
        for (int i = 0; i < 14; ++i) {
            cudaEventDestroy(c->ev_a[i]);
            cudaEventDestroy(c->ev_b[i]);
        }
    if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
    if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_side) cudaEventDestroy(c->ev_side);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;  // device buffers free themselves
    return PCM_OK;
}

int pcm_build_surface(pcm_ctx *c, int natom, const double *xyz, const double *Z, const double *radius,
                      int pts_per_sphere, int *M_out)
{
    if (!c || natom <= 0 || !xyz || !Z || !radius || pts_per_sphere < 1) {
        set_last_error("pcm_build_surface: bad arguments");
        return PCM_ERR_ARG;
    }
    if (!all_finite(xyz, 3 * (size_t)natom) || !all_finite(Z, natom) || !all_finite(radius, natom)) {
        set_last_error("pcm_build_surface: non-finite input");
        return PCM_ERR_ARG;
    }
    for (int i = 0; i < natom; ++i)
        if (!(radius[i] > 0.0)) {
            set_last_error("pcm_build_surface: radius %d is not positive", i);
            return PCM_ERR_ARG;
        }
    DeviceGuard g(c->device);
    c->nbf = 0;
    c->nshell = 0;
    for (auto &pc : c->cls) {
        pc.nsp = 0;
        pc.npair = 0;
        pc.nesp = 0;
    }
    PCM_TRY(surface_build(c, natom, xyz, Z, radius, pts_per_sphere));
    c->stats.M = c->M;
    if (M_out) *M_out = c->M;
    return PCM_OK;
}

int pcm_get_surface(pcm_ctx *c, double *xyzzs, int *index, int flags)
{
    if (!c || c->M == 0) {
        set_last_error("pcm_get_surface: no surface");
        return PCM_ERR_ARG;
    }
    DeviceGuard g(c->device);
    const int M = c->M;
    if (xyzzs) {
        double *dst = xyzzs;
        DBuf<double> &tmp = c->sd[2];
        if (!(flags & PCM_PTR_DEVICE)) {
            PCM_TRY(tmp.alloc(5 * (size_t)M));
            dst = tmp.p;
        }
        pack_surface_kernel<<<(M + 127) / 128, 128, 0, c->stream>>>(M, c->px.p, c->py.p, c->pz.p, c->pzeta.p,
                                                                   c->pS.p, dst);
        PCM_LAUNCHED(c);
        if (!(flags & PCM_PTR_DEVICE))
            PCM_CUDA(cudaMemcpyAsync(xyzzs, dst, 5 * (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
    }
    if (index) {
        PCM_CUDA(cudaMemcpyAsync(index, c->pindex.p, M * sizeof(int),
                                 (flags & PCM_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
        PCM_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PCM_OK;
}

int pcm_set_basis(pcm_ctx *c, int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                  const double *exps, const double *coefs, int *nbf_out)
{
    if (!c || nshell <= 0 || !shell_atom || !shell_l || !shell_nprim || !exps || !coefs) {
        set_last_error("pcm_set_basis: bad arguments");
        return PCM_ERR_ARG;
    }
    if (c->M == 0) {
        set_last_error("pcm_set_basis: call pcm_build_surface first");
        return PCM_ERR_ARG;
    }
    DeviceGuard g(c->device);
    PCM_TRY(basis_build(c, nshell, shell_atom, shell_l, shell_nprim, exps, coefs));
    c->stats.nbf = c->nbf;
    c->stats.pairs_candidate = c->pairs_candidate;
    c->stats.pairs_kept = c->pairs_kept;
    c->have_c = false;
    if (nbf_out) *nbf_out = c->nbf;
    return PCM_OK;
}

int pcm_esp(pcm_ctx *c, const double *P, double *cout, double *Bzout, int flags)
{
    if (!c || !P || !cout) {
        set_last_error("pcm_esp: bad arguments");
        return PCM_ERR_ARG;
    }
    if (c->nbf == 0) {
        set_last_error("pcm_esp: call pcm_set_basis first");
        return PCM_ERR_ARG;
    }
    DeviceGuard g(c->device);
    const double *dP;
    PCM_TRY(to_device(c, P, (size_t)c->nbf * c->nbf, c->dP, &dP, flags));
    PCM_TRY(c->c_last.alloc(c->M));
    PCM_TRY(esp_compute(c, dP, c->c_last.p));
    c->have_c = true;
    const cudaMemcpyKind kind = (flags & PCM_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PCM_CUDA(cudaMemcpyAsync(cout, c->c_last.p, c->M * sizeof(double), kind, c->stream));
    if (Bzout) PCM_CUDA(cudaMemcpyAsync(Bzout, c->Bz.p, c->M * sizeof(double), kind, c->stream));
    return finish(c, flags);
}

int pcm_cg_threshold(double delta, double prev_diis_error, int flags, double *out)
{
    if (!out || std::isnan(delta) || std::isnan(prev_diis_error)) {
        set_last_error("pcm_cg_threshold: NaN threshold or NULL output");
        return PCM_ERR_ARG;
    }
    double d = delta;
    if (flags & PCM_TWO_DELTA) {
        // Section 4b-i: s * delta_2 (s = 1e4) until the previous SCF iteration's
        // DIIS error has reached 1e-3, then delta_2
        if (!(delta > 0.0)) {
            set_last_error("pcm_cg_threshold: PCM_TWO_DELTA needs delta_2 > 0");
            return PCM_ERR_ARG;
        }
        d = (prev_diis_error < 0.0 || prev_diis_error > 1e-3) ? 1e4 * delta : delta;
    } else if (!(d > 0.0)) {
        // Eq. 21 and the rule that follows it: the CG threshold that predicts an
        // energy error of 1e-3 times the previous DIIS error; delta = 1 when
        // there is no previous iteration
        if (prev_diis_error < 0.0) {
            d = 1.0;
        } else {
            d = pow(1e-3 * prev_diis_error / 0.01, 1.0 / 1.07);
            d = fmin(1.0, fmax(1e-10, d));
        }
    }
    *out = d;
    return PCM_OK;
}

int pcm_solve(pcm_ctx *c, const double *rhs, double delta, double prev_diis_error, double *q, pcm_stats *st,
              int flags)
{
    if (!c || !q || c->M == 0) {
        set_last_error("pcm_solve: bad arguments");
        return PCM_ERR_ARG;
    }
    if (!rhs && !c->have_c) {
        set_last_error("pcm_solve: rhs is NULL and no pcm_esp result is available");
        return PCM_ERR_ARG;
    }
    if (std::isnan(delta) || std::isnan(prev_diis_error)) {
        set_last_error("pcm_solve: NaN threshold");
        return PCM_ERR_ARG;
    }
    double d = 0.0;
    PCM_TRY(pcm_cg_threshold(delta, prev_diis_error, flags, &d));
    DeviceGuard g(c->device);
    const int M = c->M;
    const double f = (c->opt.eps - 1.0) / (c->opt.eps + c->opt.k);
    const double *drhs;
    PCM_TRY(c->vrhs.alloc(M));
    if (rhs) {
        PCM_TRY(to_device(c, rhs, M, c->vin, &drhs, flags));
    } else {
        rhs_kernel<<<(M + 255) / 256, 256, 0, c->stream>>>(M, f, c->Bz.p, c->c_last.p, c->vrhs.p);
        PCM_LAUNCHED(c);
        drhs = c->vrhs.p;
    }
    const bool warm = (flags & PCM_WARM) != 0;
    double *dq = q;
    if (!(flags & PCM_PTR_DEVICE)) {
        PCM_TRY(c->vx.alloc(M));
        if (warm) {
            if (!all_finite(q, M)) {
                set_last_error("pcm_solve: initial guess holds a NaN or an infinity");
                return PCM_ERR_ARG;
            }
            PCM_CUDA(cudaMemcpyAsync(c->vx.p, q, M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        }
        dq = c->vx.p;
    }
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[12], c->stream));
    int status = solver_run(c, drhs, d, dq, warm, st);
    if (c->have_events) {
        PCM_CUDA(cudaEventRecord(c->ev_b[12], c->stream));
        PCM_CUDA(cudaEventSynchronize(c->ev_b[12]));
        float ms = 0.f;
        PCM_CUDA(cudaEventElapsedTime(&ms, c->ev_a[12], c->ev_b[12]));
        c->stats.ms_solve = ms;
        if (st) st->ms_solve = ms;
    }
    if (status != PCM_OK && status != PCM_ERR_NOT_CONVERGED) return status;
    if (!(flags & PCM_PTR_DEVICE))
        PCM_CUDA(cudaMemcpyAsync(q, dq, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PCM_TRY(finish(c, flags));
    return status;
}

int pcm_fock(pcm_ctx *c, const double *q, double *dF, int flags)
{
    if (!c || !q || !dF) {
        set_last_error("pcm_fock: bad arguments");
        return PCM_ERR_ARG;
    }
    if (c->nbf == 0) {
        set_last_error("pcm_fock: call pcm_set_basis first");
        return PCM_ERR_ARG;
    }
    DeviceGuard g(c->device);
    const double *dq;
    PCM_TRY(to_device(c, q, c->M, c->vin, &dq, flags));
    double *ddF = dF;
    const size_t n2 = (size_t)c->nbf * c->nbf;
    if (!(flags & PCM_PTR_DEVICE)) {
        PCM_TRY(c->dF.alloc(n2));
        ddF = c->dF.p;
    }
    PCM_TRY(fock_compute(c, dq, ddF));
    if (!(flags & PCM_PTR_DEVICE))
        PCM_CUDA(cudaMemcpyAsync(dF, ddF, n2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return finish(c, flags);
}

int pcm_energy(pcm_ctx *c, const double *q, const double *cv, double *E, int flags)
{
    if (!c || !q || !E || c->M == 0) {
        set_last_error("pcm_energy: bad arguments");
        return PCM_ERR_ARG;
    }
    if (!cv && !c->have_c) {
        set_last_error("pcm_energy: c is NULL and no pcm_esp result is available");
        return PCM_ERR_ARG;
    }
    DeviceGuard g(c->device);
    const double *dq, *dcv;
    DBuf<double> &stq = c->sd[3], &stc = c->sd[4];
    PCM_TRY(to_device(c, q, c->M, stq, &dq, flags));
    if (cv) PCM_TRY(to_device(c, cv, c->M, stc, &dcv, flags));
    else dcv = c->c_last.p;
    PCM_TRY(energy_compute(c, dq, dcv, E));
    return PCM_OK;
}

int pcm_apply_a(pcm_ctx *c, const double *x, double *y, int flags)
{
    if (!c || !x || !y || c->M == 0) {
        set_last_error("pcm_apply_a: bad arguments");
        return PCM_ERR_ARG;
    }
    if ((flags & PCM_APPLY_FP32) && !matrix_free(c)) {
        set_last_error("pcm_apply_a: the FP32 product is the matrix-free operator of PCM_MIXED contexts");
        return PCM_ERR_UNSUPPORTED;
    }
    DeviceGuard g(c->device);
    const double *dx;
    DBuf<double> &stx = c->sd[3];
    PCM_TRY(to_device(c, x, c->M, stx, &dx, flags));
    double *dy = y;
    if (!(flags & PCM_PTR_DEVICE)) {
        PCM_TRY(c->vout.alloc(c->M));
        dy = c->vout.p;
    }
    PCM_TRY(apply_a(c, dx, dy, (flags & PCM_APPLY_FP32) != 0));
    if (!(flags & PCM_PTR_DEVICE))
        PCM_CUDA(cudaMemcpyAsync(y, dy, c->M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return finish(c, flags);
}

int pcm_gradient(pcm_ctx *c, const double *P, const double *q, double *grad, int flags)
{
    if (!c || !q || !grad || c->M == 0) {
        set_last_error("pcm_gradient: bad arguments");
        return PCM_ERR_ARG;
    }
    int terms = flags & (PCM_GRAD_B | PCM_GRAD_C | PCM_GRAD_A);
    if (terms == 0) terms = PCM_GRAD_B | PCM_GRAD_C | PCM_GRAD_A;
    if ((terms & PCM_GRAD_C) && (!P || c->nbf == 0)) {
        set_last_error("pcm_gradient: the integral term needs P and pcm_set_basis");
        return PCM_ERR_ARG;
    }
    DeviceGuard g(c->device);
    const double *dq, *dP = nullptr;
    DBuf<double> &stq = c->sd[3];
    PCM_TRY(to_device(c, q, c->M, stq, &dq, flags));
    if (terms & PCM_GRAD_C) PCM_TRY(to_device(c, P, (size_t)c->nbf * c->nbf, c->dP, &dP, flags));
    double *dg = grad;
    if (!(flags & PCM_PTR_DEVICE)) {
        PCM_TRY(c->g_out.alloc(3 * (size_t)c->natom));
        dg = c->g_out.p;
    }
    if (c->have_events) PCM_CUDA(cudaEventRecord(c->ev_a[12], c->stream));
    PCM_TRY(gradient_compute(c, dP, dq, terms, dg));
    if (c->have_events) {
        PCM_CUDA(cudaEventRecord(c->ev_b[12], c->stream));
        PCM_CUDA(cudaEventSynchronize(c->ev_b[12]));
        float ms = 0.f;
        PCM_CUDA(cudaEventElapsedTime(&ms, c->ev_a[12], c->ev_b[12]));
        c->stats.ms_grad = ms;
    }
    if (!(flags & PCM_PTR_DEVICE))
        PCM_CUDA(cudaMemcpyAsync(grad, dg, 3 * (size_t)c->natom * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return finish(c, flags);
}

int pcm_get_stats(pcm_ctx *c, pcm_stats *st)
{
    if (!c || !st) return PCM_ERR_ARG;
    *st = c->stats;
    return PCM_OK;
}

}  // extern "C"
