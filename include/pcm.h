/*
 * pcm.h -- C ABI of the GB300 (sm_103a) C-PCM / ISWIG solvation hot path.
 *
 * The library computes, on one GPU, the quantities of the conductor-like
 * polarizable continuum model with ISWIG switching/Gaussian discretization
 * of Liu, Luehr, Kulik & Martinez (arXiv 1505.07851):
 *
 *   A q = -f (B z + c)                                   (Eq. 1)
 *   A_kl = erf(zeta'_kl r_kl) / r_kl                      (Eq. 2, Eq. 8)
 *   A_kk = zeta_k sqrt(2/pi) / S_k                        (Eq. 3, read as the r -> 0 limit of Eq. 2)
 *   (B z)_k = sum_J Z_J erf(zeta_k r_kJ) / r_kJ           (Eq. 4)
 *   c_k = sum_{mu nu} P_{mu nu} L^k_{mu nu}               (Eq. 5)
 *   L^k_{mu nu} = -(mu | erf(zeta_k |r - r_k|)/|r - r_k| | nu)   (Eq. 6, Eq. 12)
 *   dF_{mu nu} = sum_k q_k L^k_{mu nu}                    (Eq. 10)
 *   dG = (Bz)^T q + c^T q + q^T A q / (2 f)               (Eq. 13)
 *   d*dG/dR = z^T (dB^T/dR) q + (d*c^T/dR) q + q^T (dA/dR) q / (2 f)   (Eq. 14, Eq. 22)
 *
 * Units: atomic units (bohr, hartree).
 *
 * Conventions
 *   - Every function returns a pcm_status; PCM_OK is 0.  pcm_strerror()
 *     gives a message.  On an error nothing is written to the outputs
 *     unless stated.
 *   - A context (pcm_ctx) owns every device buffer it allocates (surface,
 *     pair lists, the stored A, preconditioner, scratch).  Arrays passed
 *     to a call are borrowed for the duration of that call only.
 *   - By default pointers are HOST pointers; the library copies them to
 *     and from the device.  With PCM_PTR_DEVICE in `flags` they are CUDA
 *     device pointers on the context's device (e.g. from PyTorch).
 *   - All GPU work is enqueued on the context's CUDA stream.  A call
 *     returns after that work has finished unless PCM_ASYNC is given
 *     (then only for device pointers; host pointers always synchronise).
 *   - A context is not thread-safe; use one context per host thread.
 *   - Surface points are numbered in the library's order: grouped by
 *     Gaussian exponent class (points of equal zeta_k together, classes in
 *     increasing zeta), and within a class by candidate index I*n + i
 *     (atom I, sphere point i).  pcm_get_surface() returns each point's
 *     candidate index.  c, Bz, rhs and q use this order.
 *   - Basis functions are Cartesian; shells in input order; within an sp
 *     shell s, px, py, pz; p: x, y, z; d: xx, xy, xz, yy, yz, zz.  Each
 *     Cartesian primitive component is normalised to unit self-overlap and
 *     multiplied by the raw contraction coefficient (no renormalisation of
 *     the contracted function).
 */
#ifndef PCM_H
#define PCM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pcm_status {
    PCM_OK = 0,
    PCM_ERR_ARG = 1,            /* invalid argument (size, pointer, NaN input, call order) */
    PCM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    PCM_ERR_OOM = 3,            /* device or host allocation failed */
    PCM_ERR_UNSUPPORTED = 4,    /* e.g. shell angular momentum above d */
    PCM_ERR_NOT_CONVERGED = 5,  /* solver hit its iteration cap; q holds the last iterate */
    PCM_ERR_TIMEOUT = 6         /* a bounded device wait gave up */
} pcm_status;

/* flags */
#define PCM_PTR_DEVICE 1        /* array arguments are device pointers */
#define PCM_ASYNC 2             /* do not synchronise the stream before returning */
#define PCM_WARM 4              /* pcm_solve: q holds the initial guess */
#define PCM_GRAD_B 8            /* pcm_gradient: include z^T (dB^T/dR) q */
#define PCM_GRAD_C 16           /* pcm_gradient: include (d*c^T/dR) q (the integrals) */
#define PCM_GRAD_A 32           /* pcm_gradient: include q^T (dA/dR) q / (2 f) (with switching) */
#define PCM_TWO_DELTA 64        /* pcm_solve: delta is delta_2 of the 2-delta threshold scheme (Section 4b-i) */
#define PCM_APPLY_FP32 128      /* pcm_apply_a: the FP32 matrix-free product (PCM_MIXED; the inner solver's elements) */

/* precision modes */
#define PCM_FP64 0              /* every step in FP64 */
#define PCM_MIXED 1             /* FP32 integrals and inner solver, FP64 accumulation, refinement with
                                   double-float (FP32 hi + lo) true residuals; energy within 1e-6 Eh */

/* preconditioners (Section 4b-ii) */
#define PCM_PRECOND_AUTO 0      /* Jacobi below `jacobi_below` points, else RBJ */
#define PCM_PRECOND_NONE 1
#define PCM_PRECOND_JACOBI 2
#define PCM_PRECOND_RBJ 3
#define PCM_PRECOND_OCTREE 4    /* block Jacobi on octree leaves of at most octree_leaf points (comparison) */

typedef struct pcm_options {
    double eps;                 /* dielectric constant, default 78.39 (Section 3) */
    double k;                   /* f = (eps - 1) / (eps + k); default 0 (Eq. 1) */
    double zeta;                /* sphere exponent of Eq. 7, default 4.9 (110 points) */
    double switch_drop;         /* drop points with S_k below this, default 1e-8 (Section 3) */
    double schwarz;             /* primitive-pair screening cutoff of Eq. 15 / Eq. 18, default 1e-12; 0 disables */
    int rbj_block;              /* RBJ block size l, default 100 (Section 3) */
    int precond;                /* PCM_PRECOND_*, default AUTO */
    int jacobi_below;           /* AUTO uses Jacobi when M is below this, default 1000 (Section 4b-ii) */
    int precision;              /* PCM_FP64 or PCM_MIXED */
    int max_iter;               /* PCG iteration cap, default 5000 */
    int device;                 /* CUDA device ordinal, default 0 */
    unsigned long long seed;    /* RBJ pivot stream seed (splitmix64), default 0 */
    void *stream;               /* cudaStream_t to use; NULL: the context creates its own */
    int timing;                 /* 1: time the integral kernels and the solve with CUDA events (stats) */
    int autotune;               /* 1: pick the FP32 integral kernels' tile shapes by timed trials (default 0) */
    int octree_leaf;            /* PCM_PRECOND_OCTREE: most points per octree leaf (block), default 800 */
    int esp_variant;            /* PCM_MIXED ESP kernel: -1 default (or the autotuner's pick), 0 pair-driven with
                                   4 points per thread, 1 with 2, 2 MS-driven (s and p classes; others default) */
    int fp32x2;                 /* PCM_MIXED: 1 (default) evaluates two primitive pairs (ESP) or two points (Fock)
                                   per packed FP32x2 instruction (FADD2/FMUL2/FFMA2; each lane rounded as the
                                   scalar instruction); 0 scalar FP32 instructions (the general form for every
                                   interaction, no far-field path) */
    int operator_mode;          /* PCM_MIXED operator A: PCM_OPERATOR_AUTO (default), _STORED or _FREE */
} pcm_options;

/* operator modes (PCM_MIXED; PCM_FP64 always stores A) */
#define PCM_OPERATOR_AUTO 0     /* matrix-free above 24576 points or when the stored parts would take more than a
                                   quarter of the free device memory, else stored */
#define PCM_OPERATOR_STORED 1   /* A stored as FP32 hi + lo parts (8 bytes per element, no FP64 copy) */
#define PCM_OPERATOR_FREE 2     /* no stored A: near pairs kept exactly, every other element 1/R recomputed */

typedef struct pcm_stats {
    int iterations;             /* PCG iterations of the last solve */
    int converged;              /* 1 if ||A q - rhs||_2 < delta was reached */
    double delta;               /* threshold used by the last solve */
    double rnorm;               /* final residual norm (recursively updated) */
    int refinements;            /* outer refinement steps (PCM_MIXED) */
    int M;                      /* surface points */
    int nbf;                    /* basis functions */
    long long pairs_candidate;  /* primitive pairs before screening */
    long long pairs_kept;       /* primitive pairs surviving Eq. 15 */
    long long pairs_esp;        /* pairs surviving the density-weighted test of Eq. 18 in the last pcm_esp */
    double integrals_esp;       /* equivalent Cartesian primitive integrals of the last pcm_esp */
    double integrals_fock;      /* equivalent Cartesian primitive integrals of the last pcm_fock */
    long long esp_class_pairs[6];   /* pairs per class (ss, ps, pp, ds, dp, dd) in the last pcm_esp */
    long long fock_class_pairs[6];  /* pairs per class in the last pcm_fock */
    double ms_esp_class[6];     /* with timing: main ESP kernel time per class (ms) */
    double ms_fock_class[6];    /* with timing: main Fock kernel time per class (ms) */
    double ms_solve;            /* with timing: device time of the last pcm_solve (ms) */
    double ms_precond;          /* with timing: build of A, its preconditioner and FP32 parts on the context's
                                   second stream after the last pcm_build_surface (ms; it overlaps the basis
                                   set-up and the integrals) */
    long long launches;         /* kernels launched by this context since its creation */
    double integrals_grad;      /* equivalent Cartesian primitive integrals of the last pcm_gradient (two passes) */
    double ms_grad;             /* with timing: device time of the last pcm_gradient (ms) */
    int operator_free;          /* 1 if the current surface's PCM_MIXED solver is matrix-free (no stored A) */
} pcm_stats;

typedef struct pcm_ctx pcm_ctx;

/* Fill `opt` with the paper's defaults (Section 3). */
int pcm_default_options(pcm_options *opt);

/* Create a context on opt->device (NULL opt: defaults).  *ctx receives the
 * handle; destroy it with pcm_destroy. */
int pcm_create(pcm_ctx **ctx, const pcm_options *opt);
int pcm_destroy(pcm_ctx *ctx);

/* Message for a status code (static storage). */
const char *pcm_strerror(int status);

/* Details of the last error raised on the calling host thread (empty if
 * none); valid until the next failing call on that thread. */
const char *pcm_last_error(void);

/* Build the ISWIG cavity surface (Eq. 7, Eq. 9, Section 3).
 * xyz: natom*3 nuclear positions (bohr); Z: natom nuclear charges;
 * radius: natom sphere radii (bohr, already scaled, e.g. 1.2 x Bondi);
 * pts_per_sphere: points per atom (Fibonacci sphere, equal weights
 * w = 4 pi / n, used in place of Lebedev points).  Host pointers.
 * Points with S_k < switch_drop are dropped; *M_out receives M.  Also
 * stores A (Eq. 2, Eq. 3) and B z (Eq. 4) for the new surface.  Invalidates
 * any preconditioner of a previous surface. */
int pcm_build_surface(pcm_ctx *ctx, int natom, const double *xyz, const double *Z,
                      const double *radius, int pts_per_sphere, int *M_out);

/* Copy the surface out: xyzzs (M*5: x, y, z, zeta_k, S_k) and index (M:
 * candidate index I*n + i).  Either may be NULL.  flags: PCM_PTR_DEVICE. */
int pcm_get_surface(pcm_ctx *ctx, double *xyzzs, int *index, int flags);

/* Set the basis (Eq. 11).  shell_atom/shell_l/shell_nprim: nshell entries,
 * shell_l in {0, 1, 2, -1 (sp)}; exps: sum(nprim) exponents; coefs: raw
 * contraction coefficients, shell after shell, an sp shell giving its
 * nprim s coefficients then its nprim p coefficients.  Host pointers.
 * Needs pcm_build_surface first (uses the atom positions).  Builds the
 * primitive-pair list with the Schwarz-type screening of Eq. 15.
 * *nbf_out receives the number of basis functions.  PCM_ERR_UNSUPPORTED
 * for l > 2. */
int pcm_set_basis(pcm_ctx *ctx, int nshell, const int *shell_atom, const int *shell_l,
                  const int *shell_nprim, const double *exps, const double *coefs, int *nbf_out);

/* Electrostatic potential of the electrons at the points, c (Eq. 5, Eq. 6):
 * c_k = -sum_{mu nu} P_{mu nu} (mu|J_k|nu).  P: nbf*nbf symmetric,
 * row-major.  c: M outputs.  Bz: optional (may be NULL) M outputs of
 * (B z)_k.  Primitive pairs are screened with |P_{mu nu}| [ij|ij]^{1/2}
 * (Eq. 18).  The context keeps c for pcm_solve(rhs = NULL). */
int pcm_esp(pcm_ctx *ctx, const double *P, double *c, double *Bz, int flags);

/* Solve A q = rhs (Eq. 1) by preconditioned CG to ||A q - rhs||_2 < delta
 * (Eq. 20).  rhs: M entries, or NULL for -f (B z + c) with c from the last
 * pcm_esp.  delta > 0: fixed threshold; delta <= 0: dynamic threshold of
 * Eq. 21 from prev_diis_error (delta = (1e-3 prev / 0.01)^(1/1.07) clamped
 * to [1e-10, 1]; prev_diis_error < 0 means first SCF step, delta = 1).
 * With PCM_TWO_DELTA, delta is delta_2 of the 2-delta scheme (see
 * pcm_cg_threshold).  q: M outputs (and the initial guess with PCM_WARM).  st: optional stats.
 * Returns PCM_ERR_NOT_CONVERGED when max_iter is reached (q is the last
 * iterate). */
int pcm_solve(pcm_ctx *ctx, const double *rhs, double delta, double prev_diis_error, double *q,
              pcm_stats *st, int flags);

/* The CG threshold pcm_solve uses for (delta, prev_diis_error, flags), with
 * no GPU work (host logic of Section 4b-i):
 *   - PCM_TWO_DELTA in flags: the 2-delta scheme, delta = delta_2 > 0; the
 *     threshold is 1e4 * delta_2 while prev_diis_error is negative (first SCF
 *     step) or above 1e-3, then delta_2;
 *   - else delta > 0: delta itself (fixed threshold);
 *   - else: Eq. 21, (1e-3 prev_diis_error / 0.01)^(1/1.07) clamped to
 *     [1e-10, 1]; 1 when prev_diis_error < 0.
 * *out receives the threshold.  PCM_ERR_ARG for NaN inputs, a NULL out, or
 * PCM_TWO_DELTA with delta <= 0. */
int pcm_cg_threshold(double delta, double prev_diis_error, int flags, double *out);

/* Solvation correction to the Fock matrix (Eq. 10, Eq. 16, Eq. 17):
 * dF_{mu nu} = -sum_k q_k (mu|J_k|nu).  q: M inputs; dF: nbf*nbf outputs,
 * symmetric, row-major. */
int pcm_fock(pcm_ctx *ctx, const double *q, double *dF, int flags);

/* Electrostatic solvation energy (Eq. 13) in hartree:
 * E = (Bz)^T q + c^T q + q^T A q / (2 f).  q, c: M inputs (c may be NULL
 * for the last pcm_esp result).  E: one host double. */
int pcm_energy(pcm_ctx *ctx, const double *q, const double *c, double *E, int flags);

/* y = A x with the context's operator (Eq. 2, Eq. 3, Eq. 8) for its current
 * surface: x, y are M-vectors in library point order.  PCM_FP64 multiplies
 * by the stored FP64 A.  PCM_MIXED with a stored operator multiplies by
 * A32 + A32lo in double-float (about 1e-14 relative).  PCM_MIXED with the
 * matrix-free operator keeps no A: pairs with zeta' R below a cutoff (the
 * diagonal included) are held with their FP64 values, every other element is
 * 1/R recomputed per product; the default product is the one the solver forms
 * true residuals and the energy with (double-float 1/R, FP64 near pairs,
 * about 1e-14 relative), PCM_APPLY_FP32 an FP32 product with the inner
 * solver's element formula (FP32 1/R with R^2 clamped at the near-pair
 * radius, the near-pair list's FP32 corrections; rows summed per column
 * chunk, whereas the inner solver sums the upper triangle's tiles in fixed
 * point: the same elements, another order of the FP32 sums; about 1e-6
 * relative).  flags: PCM_PTR_DEVICE, PCM_ASYNC, PCM_APPLY_FP32
 * (PCM_ERR_UNSUPPORTED unless the context is matrix-free). */
int pcm_apply_a(pcm_ctx *ctx, const double *x, double *y, int flags);

/* Nuclear gradient of the solvation energy at fixed density and charges
 * (Eq. 14; its integral term split as in Eq. 22), in hartree/bohr:
 *   g_I = z^T (dB^T/dR_I) q + (d*c^T/dR_I) q + q^T (dA/dR_I) q / (2 f)
 * where every surface point moves with its atom, the diagonal of A varies
 * through the switching factors S_k (Eq. 9), and d* leaves P fixed.  At the
 * solution q of Eq. 1 this is the derivative of Eq. 13 at fixed P (Eq. 13 is
 * stationary in q there); the density's own response is the caller's.
 * P: nbf*nbf symmetric (may be NULL when PCM_GRAD_C is not requested);
 * q: M charges in library order; grad: natom*3 outputs.  Needs
 * pcm_build_surface (and pcm_set_basis for the integral term).  flags:
 * PCM_PTR_DEVICE, PCM_ASYNC, and any of PCM_GRAD_B / PCM_GRAD_C / PCM_GRAD_A
 * to select terms (none of them: all three).  Primitive pairs are screened
 * as in pcm_esp (Eq. 18).  PCM_FP64: every step in FP64.  PCM_MIXED: the
 * integral kernels and the off-diagonal A term (from the FP32 copy of A)
 * run on the FP32 pipes with FP64 accumulation across tiles;
 * the nuclear B term, the switching term and every reduction stay FP64. */
int pcm_gradient(pcm_ctx *ctx, const double *P, const double *q, double *grad, int flags);

/* ------------------------------------------------------------------------
 * Batches: many molecules of uneven size in one call.
 *
 * A batch holds one context per molecule (options as for pcm_create; every
 * molecule's A, its FP32 parts under PCM_MIXED, and its preconditioner stay
 * resident).  pcm_batch_run computes, for every molecule, the ESP (Eq. 5),
 * the solve of Eq. 1 to ||A q - rhs||_2 < delta (Eq. 20; fixed delta), the
 * Fock correction (Eq. 10) and the energy (Eq. 13).  The solves of all
 * molecules run in lockstep on the device: one launch per PCG step serves
 * every molecule, the iteration loop is a CUDA graph whose loop condition the
 * device sets (per-molecule convergence), and PCM_MIXED wraps it in
 * iterative refinement as in pcm_solve.
 * ---------------------------------------------------------------------- */
typedef struct pcm_batch pcm_batch;

/* A batch of nmol molecules (opt NULL: defaults).  Destroy with pcm_batch_destroy. */
int pcm_batch_create(pcm_batch **batch, const pcm_options *opt, int nmol);
int pcm_batch_destroy(pcm_batch *batch);

/* Molecule i (0 <= i < nmol): surface as pcm_build_surface, basis as
 * pcm_set_basis (host pointers), then its preconditioner (and FP32 A). */
int pcm_batch_set_molecule(pcm_batch *batch, int i, int natom, const double *xyz, const double *Z,
                           const double *radius, int pts_per_sphere, int nshell, const int *shell_atom,
                           const int *shell_l, const int *shell_nprim, const double *exps,
                           const double *coefs);

/* Surface points and basis functions of molecule i. */
int pcm_batch_sizes(pcm_batch *batch, int i, int *M, int *nbf);

/* Run every molecule: P[i] its density (nbf_i^2, symmetric, row-major);
 * delta > 0 the residual threshold; E: nmol energies (host array, hartree);
 * q, dF: optional arrays of nmol pointers (M_i charges in library order,
 * nbf_i^2 Fock corrections), NULL or a NULL entry to skip.  flags:
 * PCM_PTR_DEVICE (P, q and dF entries are device pointers). */
int pcm_batch_run(pcm_batch *batch, const double *const *P, double delta, double *E, double *const *q,
                  double *const *dF, int flags);

/* Per-molecule statistics of the last run (iterations, convergence, final
 * residual, refinements, integrals); i = -1: batch totals (launches,
 * integrals, the largest iteration count, total points and functions). */
int pcm_batch_get_stats(pcm_batch *batch, int i, pcm_stats *st);

/* The autotuner's choices so far in this process: up to max_entries records
 * of eight ints: device; kernel family (0: ESP variant, choice 0 pair-driven
 * with 4 points per thread, 1 with 2, 2 MS-driven (one pair per thread with
 * block reductions per point); 1: Fock pairs per thread, choice 1 or 2;
 * 2 and 3: the same with scalar FP32 instructions; 4: the ESP variant of
 * batch members, choice 0 or 1 (their packed blocks run in one launch for
 * all molecules));
 * angular momentum L; size bucket floor(log2(pairs)); the choice; the trial
 * times of variants 0, 1, 2 in microseconds (0: not tried; for the Fock
 * family variants 0 and 1 are 1 and 2 pairs per thread).  Returns the number
 * of records. */
int pcm_autotune_table(int *entries, int max_entries);

/* Statistics of the context's last calls. */
int pcm_get_stats(pcm_ctx *ctx, pcm_stats *st);

/* Measured FMA throughput of the device's FP32 (which = 0), FP64 (which = 1) or
 * packed FP32x2 (which = 2, two lanes per instruction) pipe in TFLOP/s (an FMA
 * counts two per lane), from independent FMA chains timed with
 * CUDA events (the paper has no counterpart; a measurement aid for the roofline
 * of the integral kernels).  Allocates and frees 16 bytes of device memory. */
int pcm_pipe_peak(int device, int which, double *tflops);

/* The energy of pcm_energy for callers that cannot allocate device memory
 * (the paper has no counterpart; this is a library service).  A program
 * whose GPU memory belongs to its own allocator -- a framework pool that has
 * reserved the device, or an embedded solver with a fixed memory budget --
 * cannot let a library call cudaMalloc: the call may fail while the pool
 * holds the memory, and cudaMalloc/cudaFree may synchronise the device in
 * the middle of the caller's work.  This entry point allocates nothing.
 *
 *   E = (Bz)^T q + c^T q + q^T A q / (2 f)
 *
 * All pointers are DEVICE pointers on the current CUDA device, owned by the
 * caller: A (M rows, leading dimension lda >= M, row-major: the stored
 * interaction matrix of pcm_build_surface), Bz, c, q (M each) and the output
 * E (one double).  f = (eps - 1) / (eps + k).  stream: cudaStream_t (NULL:
 * legacy default stream).  The work is only enqueued: E is valid once the
 * stream reaches it.
 *
 * Scratch (the vector A q) lives in a fixed device array of 512 KiB inside
 * the library, held by every GPU that loads the library until the process
 * exits.  M above 65536 is rejected with PCM_ERR_ARG.  The first call on a
 * device looks up the array's device address (with that device current)
 * and may load the library's device code; make that first call before any
 * stream capture.  The address is kept for the process: do not use the
 * library across a device reset.  Every call shares the array: calls whose
 * kernels overlap on the GPU (other streams, other host threads) race and
 * give wrong results; serialise them.  Each call writes every element it
 * reads, so nothing in the array needs clearing between calls. */
int pcm_energy_noalloc(int M, const double *A, int lda, const double *Bz, const double *c,
                       const double *q, double f, double *E, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PCM_H */
