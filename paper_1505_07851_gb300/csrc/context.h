// Host-side context of the C-PCM library: device buffers, the surface, the
// basis and primitive-pair lists, the stored A and the preconditioner.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pcm.h"

namespace pcm {

// error plumbing -------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};
void set_last_error(const char *fmt, ...);

#define PCM_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            pcm::set_last_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? PCM_ERR_OOM : PCM_ERR_CUDA;               \
        }                                                                                     \
    } while (0)

// check a kernel launch and count it
#define PCM_LAUNCHED(ctx)                                                                      \
    do {                                                                                       \
        ++(ctx)->stats.launches;                                                               \
        PCM_CUDA(cudaGetLastError());                                                          \
    } while (0)

#define PCM_TRY(call)                  \
    do {                               \
        int s_ = (call);               \
        if (s_ != PCM_OK) return s_;   \
    } while (0)

// A device buffer that frees itself.
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    int alloc(size_t count)
    {
        if (count <= n && p) return PCM_OK;
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            set_last_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? PCM_ERR_OOM : PCM_ERR_CUDA;
        }
        n = count;
        return PCM_OK;
    }
};

// One angular-momentum class of primitive pairs (la >= lb), SoA.
struct PairClass {
    int la = 0, lb = 0;
    // shell pairs of this class (host and device)
    std::vector<int> h_spA, h_spB;          // expanded shell indices, l(A) = la, l(B) = lb
    DBuf<int> spA, spB;                    // shell pair -> shells
    DBuf<int> sp_start;                    // nsp + 1: range of kept primitive pairs per shell pair
    DBuf<long long> sp_cand;               // nsp + 1: candidate offsets
    int nsp = 0;
    long long ncand = 0;
    int npair = 0;                         // kept primitive pairs
    // kept primitive pairs
    DBuf<int> sp, ia, ib;                  // shell pair id, primitive index in A and in B
    DBuf<double> Px, Py, Pz, p, pref, Q;   // centre, exponent sum, (2 pi / p) K_AB, Schwarz bound
    // per-call ESP pairs (after the density test of Eq. 18), SoA; D has nherm(L) rows
    int nesp = 0;
    int nesp_same = 0;                     // the first nesp_same ESP pairs join primitives on one atom
    DBuf<double> eP, eD;                   // eP: 4 x nesp (Px, Py, Pz, p); eD: nherm x nesp
    DBuf<float> eX32, eC32;                // PCM_MIXED ESP: 6 x nesp split centres; ncls x (3 + 2 nherm) x nesp constants
    DBuf<float> tfar, tnear;               // PCM_MIXED packed ESP: per 32-pair tile far block, near block per class
    DBuf<float> fnear;                     // PCM_MIXED packed Fock: near constants per (class, pair)
    DBuf<float> Pxyz32;                    // 6 x npair: hi (3) and lo (3) FP32 parts of the centre (Fock, PCM_MIXED)
    DBuf<int> elist;                       // nesp: ESP pair -> kept pair index (valid after each ESP preparation)
    // shell pairs by atom for the gradient: entry 2 s + side (side 0: atom of A, 1: atom of B)
    bool csr_ready = false;
    DBuf<int> csr_off, csr_ent;            // natom + 1 offsets, 2 nsp entries
};

struct pcm_ctx_impl;

// Work of one thread block of the packed integral kernels, so that the blocks
// of many molecules can run in one launch (batches).
struct EspJob {
    const float *far, *near, *ph, *pl;   // pair tiles (far block, near blocks per class), split point coordinates
    double *part;                        // the block's row of partial sums (indexed by point)
    int ntile, M, k0, k1, e, t0, nt, pad;  // tiles of the class, points, point range, class, tile range
};

struct FockJob {
    const double *gp;                    // exponent sums of the pairs
    const float *Phl, *nc, *tiles;       // split pair centres, near constants, point tiles
    const int *tile_cls;                 // class of each point tile
    double *W;                           // accumulators [nsplit][nherm][npair]
    int npair, ntile, tps, bx, by, pad;  // pairs, point tiles, tiles per split, pair block, split
};

// Collects the blocks of the packed ESP (by L and points per thread: 2, 4)
// and Fock (by L and pairs per thread: 1, 2) kernels instead of launching them.
struct JobSink {
    std::vector<EspJob> esp[5][2];
    std::vector<FockJob> fock[6][2];
    void clear()
    {
        for (auto &v : esp)
            for (auto &w : v) w.clear();
        for (auto &v : fock)
            for (auto &w : v) w.clear();
    }
};

}  // namespace pcm

struct pcm_ctx {
    pcm_options opt;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // Boys tables
    pcm::DBuf<double> boys64;
    pcm::DBuf<float> boys32;

    // molecule
    int natom = 0;
    std::vector<double> h_xyz, h_Z, h_radius;
    pcm::DBuf<double> xyz, Z, radius;

    // surface in library order (grouped by exponent class)
    int npts_sphere = 0;
    int M = 0;
    int ncls = 0;
    std::vector<double> h_cls_zeta;        // exponent of each class (ascending)
    std::vector<int> h_cls_off;            // ncls + 1 offsets into the point list
    pcm::DBuf<double> cls_zeta;            // ncls
    std::vector<double> h_zp_cls;          // ncls x ncls: zeta' of Eq. 8 for each pair of classes
    pcm::DBuf<double> zp_cls;
    pcm::DBuf<int> cls_off;                // ncls + 1
    pcm::DBuf<double> px, py, pz, pzeta, pS, Bz;
    pcm::DBuf<int> pindex, pcls;
    pcm::DBuf<float> p32;                  // 3 x M: FP32 high parts of x, y, z (2^-10 grid)
    pcm::DBuf<float> p32lo;                // 3 x M: FP32 low parts

    // stored A (FP64), leading dimension lda
    int lda = 0;
    pcm::DBuf<double> A;
    pcm::DBuf<float> A32;                  // FP32 copy of A for the inner solves of PCM_MIXED
    pcm::DBuf<float> A32lo;                // A - A32 in FP32: A32 + A32lo is the double-float A
    pcm::DBuf<double> dinv;                // 1 / A_kk

    // basis (expanded: sp shells split into an s and a p shell)
    int nbf = 0;
    int nshell = 0;
    std::vector<int> h_sh_atom, h_sh_l, h_sh_nprim, h_sh_off, h_sh_bf;
    pcm::DBuf<int> sh_atom, sh_l, sh_nprim, sh_off, sh_bf;
    pcm::DBuf<double> exps, cnorm;         // exponent and coefficient x base normalisation per primitive
    pcm::PairClass cls[6];                 // (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
    // the shells the class lists were built for (reused while they stay the same)
    bool pair_layout_ok = false;
    std::vector<int> pl_atom, pl_l, pl_nprim;
    long long pairs_candidate = 0, pairs_kept = 0;

    // last results
    pcm::DBuf<double> c_last;
    bool have_c = false;
    // PCM_MIXED: the last solve's charges and A q = rhs - r from its final true
    // residual, so that the energy of those charges needs no further product
    pcm::DBuf<double> aq_q, aq_y;
    bool aq_valid = false;

    // preconditioner
    int pc_kind = 0;                       // resolved PCM_PRECOND_*
    bool pc_ready = false;
    int rbj_l = 0, rbj_nblk = 0;
    pcm::DBuf<int> rbj_perm;               // M: block-ordered point indices
    pcm::DBuf<int> rbj_T;                  // natom x points per sphere: candidate-index table of the RBJ set-up
    pcm::DBuf<double> rbj_inv;             // nblk x l x l inverses (padded)
    pcm::DBuf<int> rbj_bstart;             // octree: nblk + 1 block starts in rbj_perm (blocks of varying size)

    // solver work vectors and scalars
    pcm::DBuf<double> vx, vr, vz, vp, vAp, vrhs, vtmp, vro, vd;
    pcm::DBuf<float> vxs32;                // 2 x lda: FP32 hi and lo parts of a GEMV's input vector
    pcm::DBuf<double> red;                 // partial sums
    pcm::DBuf<double> scal;                // device scalars
    pcm::DBuf<int> iscal;                  // device ints (done flag, iteration count)
    pcm::DBuf<unsigned int> counter;       // last-block counters
    double *h_pinned = nullptr;            // pinned host scratch for scalars (32 doubles)
    // the PCG iteration loop as a CUDA graph (conditional WHILE node), its key
    // (what the captured launches read) and the private stream it is captured on
    cudaGraph_t pcg_graph = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    uintptr_t pcg_key[24] = {};
    cudaStream_t cap_stream = nullptr;

    // integral scratch
    pcm::DBuf<double> esp_part;            // nseg x M partial potentials (x 3 for the gradient)
    pcm::DBuf<double> fock_W;              // nsplit x nherm x npair accumulators
    pcm::DBuf<double> dP, dF;              // device copies of P and dF for host-pointer calls
    // gradient scratch
    pcm::DBuf<int> patom, arange;          // atom of each point; per-atom point range (2 x natom)
    pcm::DBuf<double> g_pt, g_atom, g_pair, g_full, g_out;  // 3 x M, natom x 3, natom x 3, 6 x npair, natom x 3
    pcm::DBuf<double> vin, vout;           // device copies of M-vectors for host-pointer calls
    pcm::DBuf<unsigned char> flags8;
    pcm::DBuf<int> idx32, scan32;
    pcm::DBuf<long long> scan64;

    // grow-only scratch reused by successive calls, so that steady-state calls
    // make no cudaMalloc/cudaFree (cudaFree synchronises the device)
    pcm::DBuf<double> sd[8];
    pcm::DBuf<int> si[8];
    pcm::DBuf<unsigned char> su8[2];

    pcm::DBuf<int> dev_err;                // device error flag (a bounded wait in a kernel gave up)
    // deferred packed integral blocks (batches): while jobs is set, the packed
    // kernels' blocks are appended there and the ESP reduction and Fock
    // epilogues wait for esp_mixed_finish / fock_mixed_finish
    pcm::JobSink *jobs = nullptr;
    std::vector<int> h_pblk[2], h_pbcls[2];   // host copies of the PCM_MIXED point blocks (4 and 2 points per thread)
    int esp_total_rows = 0;
    double *esp_out = nullptr;
    pcm::DBuf<double> fock_Wk[6];
    int fock_nsplit_k[6] = {0, 0, 0, 0, 0, 0};
    bool fock_pending[6] = {false, false, false, false, false, false};
    // matrix-free A (PCM_MIXED): FP32 coordinates, near pairs (CSR, exact values), solver scratch
    bool store_a = false;                  // keep the stored A and its FP32 parts instead (batch members)
    bool mf_active = false;                // this surface's PCM_MIXED solver is matrix-free (set per surface)
    float mf_rc2 = 0.f;
    int mf_nnz = 0;
    int pg_grid[2] = {0, 0};      // persistent inner PCG: grid (matrix-free, stored)
    size_t pg_smem[2] = {0, 0};
    pcm::DBuf<float4> mf_pts;
    pcm::DBuf<int> mf_off, mf_cnt, mf_col, mf_out, mf_iperm;
    pcm::DBuf<double> mf_val, mf_y64, mf_idot, mf_red, mf_rn;
    // stored-operator product of the persistent PCG: fixed-point accumulators,
    // max |p| per product parity, max row sum of |A32| (built once per operator)
    pcm::DBuf<unsigned long long> st_acc;
    pcm::DBuf<unsigned> st_pmax;
    pcm::DBuf<double> st_arow;
    bool st_arow_ok = false;
    pcm::DBuf<float> mf_val32, mf_p32, mf_ypart;
    pcm::DBuf<float2> mf_xs;
    pcm::DBuf<unsigned> mf_bar;
    // packed Fock: tiles of 128 points of one class (class and first point per tile), the per-call tile data
    int fk_ntile = 0;
    std::vector<int> h_fk_cls, h_fk_k0;
    pcm::DBuf<int> fk_cls, fk_k0;
    pcm::DBuf<float> fk_tiles;

    pcm_stats stats;
    cudaEvent_t ev_a[14], ev_b[14];         // timing events: 0-5 ESP classes, 6-11 Fock classes, 12 solve, 13 precond
    bool have_events = false;

    // A, its diagonal and the preconditioner are built on a second stream that
    // runs beside the basis set-up and the integrals; every use joins it first
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_side = nullptr;
    bool side_pending = false;
    bool op_stale = false;                 // the surface changed: A and its preconditioner are not built yet
    bool side_rbj = false;                 // the side work includes an RBJ set-up (status to check)
    pcm::DBuf<int> rbj_U, rbj_U2, rbj_status;
    pcm::DBuf<double> rbj_work;
};

namespace pcm {
// launchers implemented in the .cu files ------------------------------------
int boys_build_tables(pcm_ctx *c);
int surface_build(pcm_ctx *c, int natom, const double *xyz, const double *Z, const double *radius, int n);
int basis_build(pcm_ctx *c, int nshell, const int *shell_atom, const int *shell_l, const int *shell_nprim,
                const double *exps, const double *coefs);
int esp_compute(pcm_ctx *c, const double *dP, double *dc);
int fock_compute(pcm_ctx *c, const double *dq, double *ddF);
// PCM_MIXED (integrals_mixed.cu)
int points_split(pcm_ctx *c);
int esp_compute_mixed(pcm_ctx *c, double *dc);
// deferred blocks of a batch: launch every collected job, then finish each molecule
int launch_jobs(JobSink &sink, DBuf<EspJob> &dej, DBuf<FockJob> &dfj, const float *boys, int *err, cudaStream_t s);
int esp_mixed_finish(pcm_ctx *c);
int esp_packed_jobs(int L, int ppt, const EspJob *jobs, int njob, const float *boys, int *err, cudaStream_t s);
int fock_mixed_finish(pcm_ctx *c, double *ddF);
// packed FP32x2 ESP with the far-field path (esp_packed.cu): pairs [jbeg, jend) of class pc
int esp_packed(pcm_ctx *c, PairClass &pc, int L, int ppt, int jbeg, int jend, const int *blk, const int *bcls,
               int nblk, double *part);
// packed FP32x2 Fock with the far-field path (fock_packed.cu)
int fock_point_tiles_map(pcm_ctx *c);
int fock_packed(pcm_ctx *c, int L, int npt, int npair, const double *gp, const float *Phl, DBuf<float> &nbuf,
                const double *dq, int nsplit, double *W);
// matrix-free A for PCM_MIXED (matfree.cu)
struct AFree;
AFree afree(pcm_ctx *c);
int zeta_pairs(pcm_ctx *c, cudaStream_t s);
int matfree_build(pcm_ctx *c, cudaStream_t s);
int matfree_dfmv(pcm_ctx *c, const double *x, double *y, double *part, int *nparts);
int matfree_mv32(pcm_ctx *c, const double *x, double *y);
int persistent_pcg(pcm_ctx *c, const double *b, double *x, double delta, int max_iter, int *iters, int *conv,
                double *rnorm);
inline bool matrix_free(const pcm_ctx *c) { return c->mf_active; }
// the device error flag: allocated and cleared on first use; check after a synchronisation
int device_error_flag(pcm_ctx *c);
int check_device_error(pcm_ctx *c, const char *where);
int fock_mixed_class(pcm_ctx *c, int k, const double *dq, int nsplit, int ksplit, double *W, int npt);
int fock_mixed_pairs_per_thread(pcm_ctx *c, int L, long long npair);
int grad_point_mixed(pcm_ctx *c, int *total_rows);
int grad_w_mixed(pcm_ctx *c, int k, const double *dq, int nsplit, int ksplit, double *W, int npt);
int solver_prepare(pcm_ctx *c);
int operator_build_async(pcm_ctx *c);   // A, 1/A_kk, preconditioner, FP32 A on the side stream
int a_build(pcm_ctx *c, cudaStream_t s);
int join_side(pcm_ctx *c);              // wait for that work (starting it if needed); report its errors
int ensure_operator(pcm_ctx *c);        // start that work if the surface changed since
int solver_prepare_full(pcm_ctx *c);
void octree_partition(const std::vector<double> &x, const std::vector<double> &y, const std::vector<double> &z,
                      int leaf, std::vector<int> &perm, std::vector<int> &start);
int solver_run(pcm_ctx *c, const double *drhs, double delta, double *dq, bool warm, pcm_stats *st);
int energy_compute(pcm_ctx *c, const double *dq, const double *dcv, double *E);
int apply_a(pcm_ctx *c, const double *x, double *y, bool fp32);
// gradient (gradient.cu, integrals.cu)
int esp_prepare_all(pcm_ctx *c, const double *dP);
int grad_integrals(pcm_ctx *c, const double *dP, const double *dq, double *gk, double *gpair);
int gradient_compute(pcm_ctx *c, const double *dP, const double *dq, int terms, double *dgrad);

// stable compaction of n byte flags: out[j] = i of the j-th nonzero flag (if
// out != nullptr), pos[i] = number of nonzero flags before i (n + 1 entries,
// if pos != nullptr); *count_dev = total.  Scratch is taken from the context.
int compact_flags(pcm_ctx *c, const unsigned char *flags, long long n, int *out, int *pos, int *count_dev);
}  // namespace pcm
