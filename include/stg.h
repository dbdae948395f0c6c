/*
 * stg.h -- C ABI of the GB300 staggered-fermion Dirac operator and CG solver.
 *
 * The operation (Jang, Kim, Lee, Lattice 2011, "Multi GPU Performance of
 * Conjugate Gradient Solver with Staggered Fermions in Mixed Precision"):
 *
 *   Dirac operator (Eq. 4/5), with the staggered phase folded into the links
 *   as in the paper's gauge-link preconditioning step (Sec. 2):
 *     (D chi)(x) = sum_mu s_mu(x) U_mu(x) chi(x+mu)
 *                       - s_mu(x-mu) U_mu(x-mu)^dag chi(x-mu),
 *     s_mu(x) = eta_mu(x) b_mu(x),  eta_mu(x) = (-1)^(x_0+...+x_{mu-1})
 *     (mu = x, y, z, t), b_t(x) = -1 on the last time slice (antiperiodic
 *     time boundary), +1 otherwise.  There is no factor 1/2 in D.
 *   Normal operator (Eq. 2/3) on even sites:  A = m^2 - D_eo D_oe.
 *   Linear system (Eq. 1):  b = A x, solved by CG (Fig. 1) or by mixed-
 *   precision CG (Fig. 2) with the corrected inner start of Eq. 6 and the
 *   reliable / group-wise updates of Sec. 3.2.
 *
 * Conventions shared by every entry point:
 *
 *   Lattice.  dims = {Lx, Ly, Lz, Lt}, every extent even and >= 2 (else
 *   STG_ERR_DIMS).  V = Lx Ly Lz Lt, Vh = V / 2.  Site x = (x, y, z, t) has
 *   lexicographic index lex = x + Lx (y + Ly (z + Lz t)), parity
 *   (x + y + z + t) & 1 (0 = even) and checkerboard index i = lex >> 1.
 *
 *   Canonical layouts (what callers hand over):
 *     links:  complex128 [Lt][Lz][Ly][Lx][4][3][3] row-major U_mu(x)[a][b],
 *             *without* phases or boundary signs (host memory);
 *     fields: complex128 [Vh][3] over one parity in checkerboard order
 *             (device memory), i.e. 6 doubles (re, im) x 3 colours per site.
 *   Device layouts ("field" arguments below) are the library's structure-of-
 *   arrays forms for FP64 / FP32 and per-site records for the 16-bit forms;
 *   stg_field_bytes() gives their size
 *   and stg_pack_field() / stg_unpack_field() convert.
 *
 *   Ownership.  The caller owns every buffer it passes; the library never
 *   frees or retains caller pointers beyond the call.  The library owns the
 *   gauge handle's device copies of the links and a per-handle workspace
 *   (allocated on first use, freed by stg_gauge_destroy).  Calls that use the
 *   same handle must not overlap (one host thread and one stream at a time);
 *   distinct handles are independent.  Batch sessions are the exception:
 *   each owns its workspace, and several sessions on one handle may step
 *   concurrently on different streams (stg_batch_create).
 *
 *   Streams.  Every call enqueues its GPU work on `stream` (NULL = the legacy
 *   default stream).  stg_dslash, stg_apply_A*, stg_pack_field and
 *   stg_unpack_field return once work is enqueued; stg_gauge_create and
 *   stg_cg_solve return after their results are complete.
 *
 *   Errors.  Functions never abort and never print.  They return a status;
 *   stg_last_error() gives a per-thread text for the most recent failure
 *   (including the CUDA error string for STG_ERR_CUDA).  Invalid pointers
 *   that are non-NULL cannot be detected: device pointers must point to at
 *   least the stated number of bytes on the current device, 16-byte aligned.
 */
#ifndef STG_H
#define STG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *stg_stream_t;

typedef enum stg_status {
    STG_OK = 0,
    STG_ERR_INVALID_ARG = 1,   /* NULL pointer, bad enum, bad size, NaN input */
    STG_ERR_DIMS = 2,          /* a lattice extent is odd, zero or negative   */
    STG_ERR_OOM = 3,           /* device or host allocation failed            */
    STG_ERR_CUDA = 4,          /* a CUDA runtime call failed                  */
    STG_ERR_NOT_CONVERGED = 5, /* maxiter reached; stats and x still filled   */
    STG_ERR_BREAKDOWN = 6,     /* d^dag A d <= 0 or a non-finite reduction     */
    STG_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up           */
    STG_ERR_UNSUPPORTED = 8    /* precision / reconstruction not held by handle */
} stg_status;

/* Storage precision of links and fields.  FP64 and FP32 compute in their own
 * precision; FP16 (IEEE binary16), BF16 (bfloat16) and FX16 (16-bit fixed
 * point) store 16-bit values and compute in FP32.  Fields of the 16-bit kinds
 * carry one FP32 scale per site (the largest |re| or |im| of the site's
 * colour vector); FX16 links use the fixed scale 1/32767 and so require
 * |U_ab| <= 1, which holds for SU(3).  BF16 keeps 8 significand bits (unit
 * round-off 2^-8): its Dslash error is about 3e-3, above FP16's 2e-3. */
typedef enum stg_prec { STG_FP64 = 0, STG_FP32 = 1, STG_FP16 = 2, STG_FX16 = 3, STG_BF16 = 4 } stg_prec;

typedef enum stg_cg_policy {
    STG_CG_RELIABLE = 0, /* Sec. 3.2: Eq. 6 start, reliable + group-wise update */
    STG_CG_REFINE = 1,   /* Fig. 2: plain iterative refinement, d restarted    */
    STG_CG_PLAIN = 2     /* Fig. 1 in FP64 only (sloppy precision ignored)     */
} stg_cg_policy;

typedef struct stg_cg_params {
    int policy;        /* stg_cg_policy                                        */
    int sloppy;        /* stg_prec of the inner iterations; must be FP64 or the
                          handle's sloppy precision                            */
    double delta;      /* eps^in of Sec. 3.2: an update fires when
                          |r^y| < delta * max|r^y| since the last update       */
    long maxiter;      /* bound on the total iteration count (0 = 10 N_dim,
                          N_dim = 3 Vh as in Fig. 1)                           */
    int check_every;   /* inner iterations between host checks (0 = auto)     */
    int timing;        /* 1: chunks rotate between timing the four kernels
                          of their first iteration with CUDA events recorded
                          inside the solver's graph, and timing whole chunks
                          with events around the graph launch, with and
                          without programmatic dependent launch (stats.t_*);
                          0: no events                                         */
} stg_cg_params;

typedef struct stg_cg_stats {
    long iters;            /* iterations, all precisions                        */
    long sloppy_iters;     /* of which in the sloppy (inner) precision          */
    long updates;          /* FP64 true-residual recomputations (Sec. 3.2)     */
    double true_res;       /* |b - A x| / |b| with the FP64 operator at exit   */
    double iter_res;       /* iterated residual / |b| at exit                  */
    double seconds;        /* wall time of the solve (host clock)              */
    long launches;         /* kernels enqueued by the solve (graph nodes count) */
    long timed_iters;      /* inner iterations that carried timing events       */
    double t_dslash_ms;    /* mean duration: first half-pass t = D_oe d          */
    double t_dslash_a_ms;  /* mean duration: q = m^2 d - D_eo t with d^dag q     */
    double t_update_ms;    /* mean duration: y += alpha d, r -= alpha q, |r|^2   */
    double t_xpay_ms;      /* mean duration: d = r + beta d                      */
    double t_iter_ms;      /* mean duration of one inner iteration, from events
                              around whole chunks without per-kernel events    */
    double t_iter_serial_ms; /* the same for chunks launched without
                              programmatic dependent launch (consecutive
                              kernels do not overlap): the reference that
                              calibrates the per-kernel event overhead        */
} stg_cg_stats;

typedef struct stg_gauge stg_gauge; /* opaque */

/* Library version (monotone integer). */
int stg_version(void);

/* Static text for a status code. */
const char *stg_status_string(stg_status s);

/* Per-thread text describing the most recent failing call on this thread. */
const char *stg_last_error(void);

/*
 * Build a gauge handle on the current CUDA device.
 *   dims[4]     : Lx, Ly, Lz, Lt (even, >= 2).
 *   links_host  : host complex128 [Lt][Lz][Ly][Lx][4][3][3] (canonical, no
 *                 phases), 4 V 9 complex values; read during the call only.
 *   sloppy      : low precision also held besides FP64 (STG_FP64 = none).
 *   recon       : 18 (all 9 complex entries stored) or 12 (rows 0 and 1
 *                 stored; row 2 rebuilt in the kernel as s conj(r0 x r1),
 *                 which requires every U_mu(x) to be in SU(3); Sec. 3.3
 *                 link compression).  Applies to the sloppy copy; the FP64
 *                 copy uses recon only when sloppy == STG_FP64, else 18.
 *   stream      : stream for the upload and packing (the call synchronises).
 *   out         : receives the handle.
 * Applies s_mu(x) once at pack time (the paper's link preconditioning).
 * Errors: STG_ERR_DIMS, STG_ERR_INVALID_ARG (NULL, bad recon / precision),
 * STG_ERR_OOM, STG_ERR_CUDA.
 */
stg_status stg_gauge_create(const int dims[4], const double *links_host,
                            stg_prec sloppy, int recon, stg_stream_t stream,
                            stg_gauge **out);

/* Device bytes that a handle created with these arguments keeps resident
 * (FP64 links, the sloppy links and their tile-major copies; the solver
 * workspace comes on top).  During stg_gauge_create a further 576 V bytes
 * (the canonical links) are held for the upload.  0 for invalid arguments. */
size_t stg_gauge_bytes(const int dims[4], stg_prec sloppy, int recon);

/* Free the handle, its device links and its workspace.  NULL is a no-op. */
stg_status stg_gauge_destroy(stg_gauge *g);

/* Lattice extents and Vh of a handle. */
stg_status stg_gauge_dims(const stg_gauge *g, int dims[4], long *vh);

/*
 * Bytes of one checkerboard field (Vh sites, 3 colours) in the device layout
 * of `prec`: FP64 48 Vh (three double2 planes), FP32 24 Vh (float4 plane for
 * colours 0-1, float2 plane for colour 2), FP16 / BF16 16 Vh (per site three
 * half2 / bfloat162 colours and one float scale in one 16-byte record), FX16 16 Vh (per site
 * three (re, im) pairs of 16-bit integers q, value q * s, and the float s).
 */
stg_status stg_field_bytes(const stg_gauge *g, stg_prec prec, size_t *bytes);

/*
 * Convert a canonical complex128 [Vh][3] device field to / from the device
 * layout of `prec` (rounding to nearest on the way down; FP16 stores each
 * site's colour vector divided by its largest |re| or |im| plus that scale,
 * FX16 stores rint(32767 v / max) and max / 32767).
 * Buffers must not overlap.
 */
stg_status stg_pack_field(const stg_gauge *g, stg_prec prec, const double *canon_dev,
                          void *field_dev, stg_stream_t stream);
stg_status stg_unpack_field(const stg_gauge *g, stg_prec prec, const void *field_dev,
                            double *canon_dev, stg_stream_t stream);

/*
 * One Dslash half-pass (Eq. 5): out = D_{p <- 1-p} in, with p = out_parity.
 *   in_dev  : field of parity 1-p in the device layout of prec;
 *   out_dev : field of parity p, same layout; must not alias in_dev.
 *   prec    : STG_FP64, or the handle's sloppy precision.
 * Errors: STG_ERR_INVALID_ARG, STG_ERR_UNSUPPORTED, STG_ERR_CUDA.
 */
stg_status stg_dslash(const stg_gauge *g, int out_parity, const void *in_dev,
                      void *out_dev, stg_prec prec, stg_stream_t stream);

/*
 * Several lattices in one launch: out_dev[k] = D_{p_k <- 1-p_k} in_dev[k] on
 * handle g[k] (Eq. 5), k = 0..n-1, n <= 16, p_k = out_parity[k].  The
 * handles may hold lattices of different sizes but must share the device
 * and the reconstruction (18 or 12) of their links in `prec`.  Each item's
 * output is bitwise the one of stg_dslash where that runs the one-site-per-
 * thread kernel (every precision but FX16 / 12-real, whose stg_dslash runs
 * the packed staged kernel: agreement to rounding); the group runs as one
 * grid, which fills the GPU where one small lattice would not.  Arrays
 * are host arrays of n entries; fields as for stg_dslash.  No item's output
 * may alias any item's input: an output pointer equal to any in_dev[j]
 * returns STG_ERR_INVALID_ARG (partial overlaps are not detected).  The paper applies the
 * operator to one lattice at a time; this is a serving-layer form of it.
 * Errors: STG_ERR_INVALID_ARG, STG_ERR_UNSUPPORTED, STG_ERR_CUDA.
 */
stg_status stg_dslash_group(int n, const stg_gauge *const *g, const int *out_parity,
                            const void *const *in_dev, void *const *out_dev, stg_prec prec,
                            stg_stream_t stream);

/*
 * Even-site normal operator (Eq. 3): out = m^2 in - D_eo (D_oe in).
 * in_dev / out_dev: even fields in the device layout of prec (no aliasing).
 * The odd intermediate lives in the handle's workspace.
 */
stg_status stg_apply_A(const stg_gauge *g, double mass, const void *in_dev,
                       void *out_dev, stg_prec prec, stg_stream_t stream);

/*
 * Same as stg_apply_A and, fused into the second half-pass, the CG
 * denominator d^dag A d = Re sum_x in(x)^dag out(x) accumulated in FP64
 * (Sec. 3.2: all inner products in double).  dot_dev: one device double,
 * written when the work completes; the summation order is fixed, so the
 * value is bitwise reproducible for a given lattice and precision.
 */
stg_status stg_apply_A_dot(const stg_gauge *g, double mass, const void *in_dev,
                           void *out_dev, double *dot_dev, stg_prec prec,
                           stg_stream_t stream);

/*
 * stg_apply_A_dot without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory -- a latency-bound loop that cannot absorb the device-wide
 * synchronisation of cudaMalloc / cudaFree, or a host whose device memory is
 * owned by another allocator or a fixed budget.  It computes exactly what
 * stg_apply_A_dot computes (same kernels, same summation order), with the
 * odd intermediate, block partials and counter in a 32 MiB array that the
 * library reserves statically on every device that loads it (held until the
 * process exits).
 *   Arguments as for stg_apply_A_dot; the handle must already exist (its
 *   links were allocated by stg_gauge_create).
 *   Limit: 48 Vh (FP64), 24 Vh (FP32) or 16 Vh (FP16, FX16, BF16) bytes plus 8
 *   bytes per 256 sites must fit in 32 MiB (FP64 up to 24^3x48, the others
 *   up to 32^3x64); larger lattices return STG_ERR_INVALID_ARG with a message.
 *   The first call on a device looks up the array's device address (once per
 *   device); make that first call before any stream capture.
 *   All calls on a device share the array: calls whose GPU work overlaps
 *   (other streams, unordered host threads) race and corrupt each other.
 *   Calls no cudaMalloc, cudaFree or allocating library routine.
 */
stg_status stg_apply_A_dot_noalloc(const stg_gauge *g, double mass, const void *in_dev,
                                   void *out_dev, double *dot_dev, stg_prec prec,
                                   stg_stream_t stream);

/*
 * Several right-hand sides on one gauge field (the batched path).  A batch is
 * `nrhs` (1..64) consecutive fields, each in the device layout of `prec`
 * (stg_field_bytes apart).  The multi-system kernels load every link once
 * per register block of NB systems, so the link traffic per system falls by
 * NB; NB (1, 2, 4, 8) and the thread-block size (128, 256) come from an
 * autotuner that times the candidates on the first call for a (lattice,
 * precision, reconstruction, nrhs) and caches the choice for the process
 * (and, when the environment variable STG_TUNE_CACHE names a file, in that
 * file).  prec must be FP32 or FX16 and held by the handle.
 *
 * stg_dslash_mrhs: out_k = D_{p <- 1-p} in_k for k < nrhs (Eq. 5).
 */
stg_status stg_dslash_mrhs(const stg_gauge *g, int out_parity, int nrhs, const void *in_dev,
                           void *out_dev, stg_prec prec, stg_stream_t stream);

/* out_k = m_k^2 in_k - D_eo D_oe in_k (Eq. 3) with masses[k] (host array). */
stg_status stg_apply_A_mrhs(const stg_gauge *g, int nrhs, const double *masses, const void *in_dev,
                            void *out_dev, stg_prec prec, stg_stream_t stream);

/*
 * Solve A_k x_k = b_k for k < nrhs with the mixed-precision CG of Sec. 3.2
 * (policy RELIABLE or REFINE; inner precision params->sloppy, FP32 or FX16),
 * batched: every inner iteration advances all unconverged systems with the
 * multi-system kernels, each system keeping its own alpha, beta, residual,
 * updates and convergence test (a converged system drops out of the batch).
 *   src_dev / x_dev: nrhs consecutive canonical complex128 [Vh][3] fields
 *   (x_dev holds the initial guesses on entry); masses: host array;
 *   stats: NULL or nrhs entries.
 *   params->check_every = 0 runs chunks of 8 inner iterations between host
 *   checks (a system that asks for a reliable update waits for its chunk to
 *   end, so shorter chunks shorten the batch's longest system).
 * Returns STG_OK when every system converged, else the first error;
 * STG_ERR_NOT_CONVERGED if any system reached maxiter (all x_k written).
 */
stg_status stg_cg_solve_mrhs(const stg_gauge *g, int nrhs, const double *src_dev, double *x_dev,
                             const double *masses, double tol, const stg_cg_params *params,
                             stg_cg_stats *stats, stg_stream_t stream);

/*
 * Batch session: the continuous-batching form of stg_cg_solve_mrhs.  A
 * session owns the device buffers of `max_systems` (1..64) systems on one
 * gauge handle (it shares the handle's read-only links; several sessions on
 * one handle may run concurrently on different streams) and runs on `stream`.
 * Systems join with stg_batch_add and leave when they finish: every
 * stg_batch_step runs one chunk of inner iterations (params->check_every,
 * default 16) for all systems present, performs the FP64 reliable updates of
 * the systems that asked for one, writes x of each finished system and
 * reports it.  A slot freed by a finished system can take a new system
 * before the next step, while the other systems continue.
 *   stg_batch_create: params as for stg_cg_solve (policy RELIABLE or REFINE,
 *     sloppy FP32 or FX16; NULL = defaults).
 *   stg_batch_add: src_dev / x_dev canonical complex128 [Vh][3] device fields
 *     owned by the caller until the system is reported done (x_dev holds x0 on
 *     entry and the solution after); `slot` receives the system's slot.
 *     Synchronises the session stream.  STG_ERR_INVALID_ARG when full.
 *   stg_batch_step: reports up to max_done finished systems (slot, status:
 *     STG_OK, STG_ERR_NOT_CONVERGED or STG_ERR_BREAKDOWN, and stats; stats may
 *     be NULL) and the number of systems still present in *n_active.  Returns
 *     after the chunk's work and any reported solutions are complete.
 *   stg_batch_bytes: device bytes a session of this size allocates.
 * The paper solves one system at a time; sessions are this library's
 * serving layer on top of the batched CG.
 */
typedef struct stg_batch stg_batch;
stg_status stg_batch_create(const stg_gauge *g, int max_systems, const stg_cg_params *params,
                            stg_stream_t stream, stg_batch **out);
stg_status stg_batch_destroy(stg_batch *b);
stg_status stg_batch_add(stg_batch *b, const double *src_dev, double *x_dev, double mass, double tol,
                         int *slot);
stg_status stg_batch_step(stg_batch *b, int max_done, int *done_slots, int *done_status,
                          stg_cg_stats *done_stats, int *n_done, int *n_active);
size_t stg_batch_bytes(const stg_gauge *g, int max_systems, stg_prec sloppy);

/*
 * Lattice-group session: systems on different lattices (each on its own
 * gauge handle, of any size up to max_vh sites per parity) iterate the CG of
 * Fig. 1 in lock-step, one grid per kernel for all of them: t_k = D_oe d_k,
 * q_k = m_k^2 d_k - D_eo t_k with d_k^dag q_k (Eq. 3), the update with
 * |r_k|^2, and d_k = r_k + beta_k d_k -- four launches per iteration for the
 * whole group, captured once in a CUDA graph and replayed.  Each system
 * keeps its own alpha, beta and stop flag and leaves when it converges;
 * between chunks the session performs the Sec. 3.2 reliable and group-wise
 * updates (x_k += y_k, r_k = b_k - A_k x_k in FP64 with the system's own
 * handle) and the Eq. 6 restart, as stg_batch_step does.  Small lattices
 * fill little of the GPU one launch at a time; a group fills it.
 *   stg_lgroup_create: max_systems 1..16; max_vh the largest Vh a slot will
 *     hold; sloppy the inner storage precision and recon (12 / 18) of the
 *     handles it will take; params as for stg_batch_create (NULL = RELIABLE
 *     with the precision's default delta).  Allocates its buffers on the
 *     current device.
 *   stg_lgroup_add: the handle must be on the session's device, hold links
 *     in `sloppy` with reconstruction `recon`, and have Vh <= max_vh (else
 *     STG_ERR_INVALID_ARG / STG_ERR_UNSUPPORTED); src_dev / x_dev canonical
 *     complex128 [Vh][3] device fields owned by the caller until the system
 *     is reported done, x_dev holding x0 on entry.  The handle must outlive
 *     the system's stay.  Synchronises the session stream.
 *   stg_lgroup_step / stg_lgroup_bytes / stg_lgroup_destroy: as for the
 *     batch session.
 * The paper solves one lattice at a time; this is a serving-layer form of
 * the same iteration.
 */
typedef struct stg_lgroup stg_lgroup;
stg_status stg_lgroup_create(int max_systems, long max_vh, stg_prec sloppy, int recon,
                             const stg_cg_params *params, stg_stream_t stream, stg_lgroup **out);
stg_status stg_lgroup_destroy(stg_lgroup *b);
stg_status stg_lgroup_add(stg_lgroup *b, const stg_gauge *g, const double *src_dev, double *x_dev,
                          double mass, double tol, int *slot);
stg_status stg_lgroup_step(stg_lgroup *b, int max_done, int *done_slots, int *done_status,
                           stg_cg_stats *done_stats, int *n_done, int *n_active);
size_t stg_lgroup_bytes(int max_systems, long max_vh, stg_prec sloppy);

/* The autotuner's choice (rhs_block = NB systems per thread and block,
 * threads_per_site = TPS) for this handle's lattice, `prec` and nrhs;
 * threads_per_site = 0 names the staged kernel (12-real FP32 / FX16 links
 * streamed through shared memory, one link load per site for all systems,
 * NB systems per thread and pass), threads_per_site = -1 its FX16 / 12-real
 * form with two sites per thread on packed FP32x2 arithmetic,
 * threads_per_site = -2 its form with the real and imaginary part of each
 * colour in the halves of FP32x2 registers and each tile's links rebuilt
 * once in shared memory (12-real FP32 and FX16).
 * STG_ERR_INVALID_ARG if not tuned yet.  The environment variable
 * STG_MRHS_SHAPE=<k> forces shape k (0-8: register-fed (NB, TPS); 9-11:
 * staged NB = 2, 4, 8; 12-13: staged two sites per thread, NB = 2, 4;
 * 14-15: staged on (re, im) FP32x2 pairs, NB = 2, 4) where it applies. */
stg_status stg_mrhs_tuning(const stg_gauge *g, stg_prec prec, int nrhs, int *rhs_block,
                           int *threads_per_site);

/* Fill params with the defaults: sloppy = handle's sloppy precision; RELIABLE
 * with delta = 0.05 for FP32, 0.25 for FX16 / BF16 inner iterations (0.1
 * without a handle); REFINE with delta = 0.02 for FP16 (its inner search
 * direction is too inexact to carry across an update: measured on 32^3x64,
 * m = 0.005, 2652 iterations against 8203 for RELIABLE at 0.25);
 * maxiter = 0 (10 N_dim), check_every = 0 (auto), timing = 0. */
stg_status stg_cg_params_default(const stg_gauge *g, stg_cg_params *params);

/*
 * Solve A x = b on even sites (Eq. 1, A of Eq. 3).
 *   src_dev : canonical complex128 [Vh][3] device field b.
 *   x_dev   : canonical complex128 [Vh][3] device field; on entry the
 *             initial guess x0 (zeros for the paper's start), on exit x.
 *   mass    : m >= 0; tol > 0: stop when |b - A x| <= tol |b| with the FP64
 *             operator (the relative form of Fig. 1 / Fig. 2).
 *   params  : NULL = stg_cg_params_default.
 *   stats   : may be NULL.
 * Returns STG_OK on convergence, STG_ERR_NOT_CONVERGED after maxiter (x
 * holds the last iterate, stats filled), STG_ERR_BREAKDOWN, STG_ERR_INVALID_ARG
 * (NULL, non-finite b / mass / tol), or a CUDA / OOM error.  Synchronises
 * `stream` before returning.
 */
stg_status stg_cg_solve(const stg_gauge *g, const double *src_dev, double *x_dev,
                        double mass, double tol, const stg_cg_params *params,
                        stg_cg_stats *stats, stg_stream_t stream);

/*
 * t-slab domain decomposition (Sec. 3.3 and Table 1), all slabs on the
 * current device.  The lattice is cut along t into nslabs slabs of Lt /
 * nslabs time slices; each slab keeps its own links, fields and face buffers,
 * as one rank of a multi-GPU run does.  One Dirac operation (a Dslash half-
 * pass) is the paper's sequence: boundary collect (a kernel gathers each
 * slab's first and last time slice of the input field into face buffers),
 * exchange (each face reaches the neighbouring slab's ghost buffer), and the
 * Dslash of every slab, whose t-hops out of the slab read the ghosts.  The
 * backward t-links of a slab's first slice live on the previous slab; they
 * are constant and are copied in once, at creation.  Global sums (d^dag A d,
 * |r|^2) are formed per slab and added in slab order: the two-scalar
 * allreduce of a multi-GPU CG.  There is no transport between GPUs here.
 *
 *   stg_slabs_create: dims as for stg_gauge_create (all even, > 0); nslabs
 *     1..64 with Lt % nslabs == 0 and Lt / nslabs even (STG_ERR_DIMS
 *     otherwise, before any device work); prec / recon the links' storage
 *     (any precision; 12 or 18); links_host as for stg_gauge_create.  Returns
 *     after the upload and packing are complete.
 *   stg_slabs_set_exchange: mode STG_SLAB_COPY (collect into each slab's
 *     send buffers, then one device-to-device copy per face: the message of a
 *     multi-GPU run) or STG_SLAB_DIRECT (the collect kernel stores straight
 *     into the neighbours' ghost buffers, as through peer pointers);
 *     overlap = 1 runs the interior time slices (1 .. Lt/nslabs - 2) on the
 *     caller's stream while collect and exchange run on a second stream,
 *     then the two boundary slices (Sec. 4's overlap of communication with
 *     computation).  Results are bitwise the same in every mode.
 *   Field slots: each slab holds STG_SLAB_SLOTS fields in `prec` (slots 0..5;
 *     stg_slabs_cg_solve overwrites them).  stg_slabs_load packs a canonical
 *     complex128 [Vh][3] device field of one parity (the global lattice's
 *     checkerboard order, t slowest) into slot `slot` of every slab;
 *     stg_slabs_store writes a slot back in the same form.
 *   stg_slabs_dslash: slot out = D slot in (Eq. 5) with output parity
 *     out_parity (the slot contents are one parity; slots carry no parity).
 *   stg_slabs_apply_A_dot: slot out = A slot in (Eq. 3, via slot 4 as the
 *     odd intermediate) and *dot_dev (device double) = Re sum in^dag out.
 *   stg_slabs_cg_solve: CG on the decomposed operator, stopping at
 *     |b - A x| <= tol |b| in FP64.  FP64 slabs: Fig. 1 in FP64, the true
 *     residual recomputed at the end (restarting from it otherwise).  FP32 /
 *     FX16 slabs: inner iterations in that precision (y and r in FP32) with
 *     the reliable updates of Sec. 3.2 (x += y, r = b - A x with an FP64 /
 *     18-real copy of the links that the handle then keeps) and the restart
 *     of Eq. 6, delta = 0.05 (FP32) or 0.25 (FX16); FP16 / BF16 slabs:
 *     STG_ERR_UNSUPPORTED.  src_dev / x_dev canonical [Vh][3] device fields,
 *     x_dev holding x0 on entry; maxiter 0 = 10 N_dim.  Synchronises
 *     `stream`.
 *   stg_slabs_profile: one Dirac operation (out parity 1, slot 0 -> slot 4),
 *     `reps` times each: ms[0] the collect kernel, ms[1] the exchange copies
 *     (0 in DIRECT mode), ms[2] the slabs' Dslash kernels, ms[3] the whole
 *     operation in the current mode; means per operation from CUDA events.
 *   stg_slabs_bytes: device bytes a handle of this shape allocates.
 */
typedef struct stg_slabs stg_slabs;
enum { STG_SLAB_COPY = 0, STG_SLAB_DIRECT = 1, STG_SLAB_SLOTS = 6 };
stg_status stg_slabs_create(const int dims[4], const double *links_host, int nslabs, stg_prec prec,
                            int recon, stg_stream_t stream, stg_slabs **out);
stg_status stg_slabs_destroy(stg_slabs *s);
stg_status stg_slabs_set_exchange(stg_slabs *s, int mode, int overlap);
stg_status stg_slabs_load(stg_slabs *s, int slot, const double *canon_dev, stg_stream_t stream);
stg_status stg_slabs_store(stg_slabs *s, int slot, double *canon_dev, stg_stream_t stream);
stg_status stg_slabs_dslash(stg_slabs *s, int out_parity, int in_slot, int out_slot,
                            stg_stream_t stream);
stg_status stg_slabs_apply_A_dot(stg_slabs *s, double mass, int in_slot, int out_slot, double *dot_dev,
                                 stg_stream_t stream);
stg_status stg_slabs_cg_solve(stg_slabs *s, const double *src_dev, double *x_dev, double mass,
                              double tol, long maxiter, stg_cg_stats *stats, stg_stream_t stream);
stg_status stg_slabs_profile(stg_slabs *s, int reps, double ms[4], stg_stream_t stream);
size_t stg_slabs_bytes(const int dims[4], int nslabs, stg_prec prec, int recon);

#ifdef __cplusplus
}
#endif

#endif /* STG_H */
