// Several systems A_k x_k = b_k on one gauge field (masses m_k differ):
// the multi-right-hand-side Dslash, A, and CG with per-system reliable
// updates (Sec. 3.2), plus the autotuner for the register block NB and the
// thread-block size of the multi-system Dslash.
//
// The iteration is the single-system sequence (Fig. 1) with every kernel
// batched over the active systems: the two half-passes load each link once
// per NB systems, and the vector kernels run one grid row (blockIdx.y) per
// system.  A chunk of iterations is one CUDA graph; between chunks the host
// performs the FP64 updates of the systems that asked for one, retires the
// converged ones and rewrites the device-side active list, which the
// captured kernels read, so the graph is never recaptured.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mrhs_kernels.cuh"

namespace stg {

void launch_dslash_m_f32_12(int shape, int epi, const MrhsArgs &a, cudaStream_t s);
void launch_dslash_m_f32_18(int shape, int epi, const MrhsArgs &a, cudaStream_t s);
void launch_dslash_m_fx16_12(int shape, int epi, const MrhsArgs &a, cudaStream_t s);
void launch_dslash_m_fx16_18(int shape, int epi, const MrhsArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------
// autotuner cache: process-wide, optionally mirrored in a text file named by
// the STG_TUNE_CACHE environment variable ("Lx Ly Lz Lt prec recon n shape")
// ---------------------------------------------------------------------------
struct TuneEntry {
    int dims[4];
    int prec, recon, nrhs, shape;
};

static std::mutex g_tune_mutex;
static std::vector<TuneEntry> g_tune;
static bool g_tune_loaded = false;

static bool same_key(const TuneEntry &e, const int *dims, int prec, int recon, int nrhs)
{
    return e.dims[0] == dims[0] && e.dims[1] == dims[1] && e.dims[2] == dims[2] &&
           e.dims[3] == dims[3] && e.prec == prec && e.recon == recon && e.nrhs == nrhs;
}

// shapes 0 .. kMrhsShapes - 1: register-fed (NB, TPS); then the staged
// kernel with NB = ms_nb(shape - kMrhsShapes) (12-real FP32 / FX16 links);
// then (FX16 / 12-real only) the staged kernel with two sites per thread,
// NB = msp_nb(shape - kMrhsShapes - kMrhsStagedShapes); then (12-real FP32
// or FX16) the staged kernel on (re, im) FP32x2 pairs, NB = ms_ri_nb(shape -
// kRiFirst)
constexpr int kMspFirst = kMrhsShapes + kMrhsStagedShapes;
constexpr int kMspCount = kMspShapes;  // NB = 2, 4 (mrhs_paired.cuh)
constexpr int kRiFirst = kMsRiFirst;
constexpr int kNumShapes = kRiFirst + kMsRiShapes;
static bool valid_choice(int shape) { return shape >= 0 && shape < kNumShapes; }

static bool staged_ok(const LinkField *lf)
{
    return lf->mtiled && lf->recon == 12 && (lf->prec == P32 || lf->prec == PX16);
}

static bool shape_ok(const LinkField *lf, int shape)
{
    if (shape < kMrhsShapes) return true;
    if (shape < kMspFirst) return staged_ok(lf);
    if (shape < kRiFirst) return staged_ok(lf) && lf->prec == PX16;
    return staged_ok(lf);
}

static void tune_load_file_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("STG_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    TuneEntry e;
    while (fscanf(f, "%d %d %d %d %d %d %d %d", &e.dims[0], &e.dims[1], &e.dims[2], &e.dims[3],
                  &e.prec, &e.recon, &e.nrhs, &e.shape) == 8) {
        if (valid_choice(e.shape)) g_tune.push_back(e);
    }
    fclose(f);
}

static bool tune_lookup(const int *dims, int prec, int recon, int nrhs, int *shape)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load_file_locked();
    for (const TuneEntry &e : g_tune)
        if (same_key(e, dims, prec, recon, nrhs)) {
            *shape = e.shape;
            return true;
        }
    return false;
}

static void tune_store(const int *dims, int prec, int recon, int nrhs, int shape)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    TuneEntry e = {{dims[0], dims[1], dims[2], dims[3]}, prec, recon, nrhs, shape};
    g_tune.push_back(e);
    const char *path = getenv("STG_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %d %d %d %d %d\n", dims[0], dims[1], dims[2], dims[3], prec, recon, nrhs,
            shape);
    fclose(f);
}

static int num_sms_m()
{
    static const int n = [] {
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || m <= 0) m = 148;
        return m;
    }();
    return n;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
static stg_status launch_m(const stg_gauge *g, const LinkField *lf, int shape, int epi, MrhsArgs &a,
                           cudaStream_t s)
{
    a.g = g->geom;
    a.grid_cap = 2 * num_sms_m();  // blocks resident at 128 registers; they stride over tiles
    for (int mu = 0; mu < 4; ++mu) {
        a.lf[mu] = lf->blk(a.parity, mu);
        a.lb[mu] = lf->blk(1 - a.parity, mu);
    }
    a.lt = nullptr;
    // STG_MRHS_GRID caps the staged kernels' CTA count (more tiles per CTA;
    // for tests)
    a.grid_limit = 0;
    if (const char *v = getenv("STG_MRHS_GRID")) a.grid_limit = atoi(v) > 0 ? atoi(v) : 0;
    if (shape >= kMrhsShapes) {
        if (!shape_ok(lf, shape)) {
            set_error("multi-system Dslash: the staged kernel needs the tile-major 12-real links "
                      "(FP32 or FX16; two sites per thread: FX16)");
            return STG_ERR_UNSUPPORTED;
        }
        a.lt = lf->mtiled + (size_t)a.parity * lf->mtiled_parity_bytes;
    }
    if (lf->prec == P32 && lf->recon == 12) launch_dslash_m_f32_12(shape, epi, a, s);
    else if (lf->prec == P32) launch_dslash_m_f32_18(shape, epi, a, s);
    else if (lf->prec == PX16 && lf->recon == 12) launch_dslash_m_fx16_12(shape, epi, a, s);
    else if (lf->prec == PX16) launch_dslash_m_fx16_18(shape, epi, a, s);
    else {
        set_error("multi-system Dslash: only FP32 and FX16 storage are supported");
        return STG_ERR_UNSUPPORTED;
    }
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// STG_MRHS_SHAPE=<k> forces shape k where it applies (tests, benchmarks)
static bool forced_shape(const LinkField *lf, int n, int *shape)
{
    const char *v = getenv("STG_MRHS_SHAPE");
    if (!v) return false;
    const int k = atoi(v);
    if (!valid_choice(k) || !(k < kMrhsShapes ? mrhs_tps(k) <= n : shape_ok(lf, k))) return false;
    *shape = k;
    return true;
}

// Time one EPI_NONE half-pass of all n systems for every register-fed (NB,
// threads per site) shape with TPS <= n and every staged NB (one warm-up and
// three timed launches each, CUDA events on `s`) and keep the fastest.
// `out` (n fields) is overwritten.
static stg_status tune(const stg_gauge *g, const LinkField *lf, int n, const void *in, void *out,
                       size_t fstride, cudaStream_t s, int *shape_out)
{
    if (forced_shape(lf, n, shape_out)) return STG_OK;
    if (tune_lookup(g->dims, lf->prec, lf->recon, n, shape_out) && shape_ok(lf, *shape_out))
        return STG_OK;
    cudaEvent_t e0, e1;
    STG_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    float best = 1e30f;
    int bshape = 0;
    stg_status st = STG_OK;
    for (int k = 0; k < kNumShapes && st == STG_OK; ++k) {
        if (k < kMrhsShapes) {
            if (mrhs_tps(k) > n || (mrhs_tps(k) == 1 && mrhs_nb(k) > n && mrhs_nb(k) > 1)) continue;
        } else if (k < kMspFirst) {
            // the site groups of a staged CTA share the systems: a block
            // larger than a group's share only adds idle slots
            const int nb = ms_nb(k - kMrhsShapes);
            if (!staged_ok(lf) || (nb > 2 && nb > (n + kMsGroups - 1) / kMsGroups)) continue;
        } else if (k < kRiFirst) {
            // four warps share the systems (two sites per thread)
            const int nb = k == kMspFirst ? 2 : 4;
            if (!shape_ok(lf, k) || (nb > 2 && nb > (n + 3) / 4)) continue;
        } else {
            const int nb = ms_ri_nb(k - kRiFirst);
            if (!shape_ok(lf, k) || (nb > 2 && nb > (n + kMsGroups - 1) / kMsGroups)) continue;
        }
        MrhsArgs a = {};
        a.parity = 1;
        a.in = static_cast<const char *>(in);
        a.out = static_cast<char *>(out);
        a.fstride = fstride;
        a.nrhs = n;
        st = launch_m(g, lf, k, EPI_NONE, a, s);
        if (st != STG_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && st == STG_OK; ++r) st = launch_m(g, lf, k, EPI_NONE, a, s);
        cudaEventRecord(e1, s);
        ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
            st = cuda_fail(ce, "autotune timing");
            break;
        }
        if (ms < best) {
            best = ms;
            bshape = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != STG_OK) return st;
    tune_store(g->dims, lf->prec, lf->recon, n, bshape);
    *shape_out = bshape;
    return STG_OK;
}

// ---------------------------------------------------------------------------
// device buffers of n systems
// ---------------------------------------------------------------------------
static stg_status dev_alloc(void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("multi-system workspace: allocation failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    return STG_OK;
}

void mrhs_free(MrhsWs *m)
{
    if (!m) return;
    if (m->graph) cudaGraphExecDestroy(m->graph);
    void *v[] = {m->x64, m->b64, m->r64, m->y, m->r, m->d, m->q, m->t, m->partials, m->states,
                 m->active, m->counter, m->tmp};
    for (void *p : v) cudaFree(p);
    if (m->states_host) cudaFreeHost(m->states_host);
    if (m->active_host) cudaFreeHost(m->active_host);
    delete m;
}

static int pr_of_m(int pd) { return (pd == P16 || pd == PX16) ? P32 : pd; }

size_t mrhs_bytes(const Geom &g, int n, int pd)
{
    const size_t vh = (size_t)g.Vh;
    const size_t pstride = (size_t)((g.Vh + 127) / 128) + 1024;
    return n * vh * (3 * 48 + 2 * field_site_bytes(pr_of_m(pd)) + 3 * field_site_bytes(pd)) +
           vh * 48 + n * pstride * sizeof(double) + n * (sizeof(CGState) + sizeof(int)) + 1024;
}

static stg_status mrhs_alloc(const stg_gauge *g, int n, int pd, MrhsWs **out)
{
    MrhsWs *m = new (std::nothrow) MrhsWs();
    if (!m) {
        set_error("multi-system workspace: host allocation failed");
        return STG_ERR_OOM;
    }
    const size_t vh = (size_t)g->geom.Vh;
    m->nrhs = n;
    m->pd = pd;
    m->f64 = vh * 48;
    m->fr = vh * field_site_bytes(pr_of_m(pd));
    m->fd = vh * field_site_bytes(pd);
    m->pstride = (size_t)((g->geom.Vh + 127) / 128) + 1024;  // >= both grids of the iteration
    stg_status st = STG_OK;
    char **bufs[] = {&m->x64, &m->b64, &m->r64};
    for (char **b : bufs)
        if (st == STG_OK) st = dev_alloc((void **)b, n * m->f64);
    if (st == STG_OK) st = dev_alloc((void **)&m->y, n * m->fr);
    if (st == STG_OK) st = dev_alloc((void **)&m->r, n * m->fr);
    if (st == STG_OK) st = dev_alloc((void **)&m->d, n * m->fd);
    if (st == STG_OK) st = dev_alloc((void **)&m->q, n * m->fd);
    if (st == STG_OK) st = dev_alloc((void **)&m->t, n * m->fd);
    if (st == STG_OK) st = dev_alloc(&m->tmp, m->f64);  // FP64 odd intermediate
    if (st == STG_OK) st = dev_alloc((void **)&m->partials, n * m->pstride * sizeof(double));
    if (st == STG_OK) st = dev_alloc((void **)&m->states, n * sizeof(CGState));
    if (st == STG_OK) st = dev_alloc((void **)&m->active, (n + 1) * sizeof(int));
    if (st == STG_OK) st = dev_alloc((void **)&m->counter, 256);
    if (st == STG_OK) {
        cudaError_t e = cudaMemset(m->states, 0, n * sizeof(CGState));
        if (e == cudaSuccess) e = cudaMemset(m->counter, 0, 256);
        if (e == cudaSuccess) e = cudaMemset(m->active, 0, (n + 1) * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&m->states_host, n * sizeof(CGState));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&m->active_host, (n + 1) * sizeof(int));
        if (e != cudaSuccess) st = cuda_fail(e, "multi-system workspace");
    }
    if (st != STG_OK) {
        mrhs_free(m);
        return st;
    }
    memset(m->states_host, 0, n * sizeof(CGState));
    memset(m->active_host, 0, (n + 1) * sizeof(int));
    *out = m;
    return STG_OK;
}

// one iteration of all active systems (4 launches)
static stg_status iteration_m(const stg_gauge *g, MrhsWs *m, const LinkField *lf, cudaStream_t s)
{
    MrhsArgs a = {};
    a.fstride = m->fd;
    a.nrhs = m->nrhs;
    a.nactive = m->active;
    a.active = m->active + 1;
    a.states = m->states;
    a.partials = reinterpret_cast<float2 *>(m->partials);
    a.counter = m->counter;
    a.parity = 1;
    a.in = m->d;
    a.out = m->t;
    STG_TRY(launch_m(g, lf, m->shape, EPI_GATE, a, s));
    a.parity = 0;
    a.in = m->t;
    a.out = m->q;
    a.w = m->d;
    STG_TRY(launch_m(g, lf, m->shape, EPI_A_CG, a, s));
    const int vh = g->geom.Vh;
    STG_TRY(launch_update_m(m->pd, vh, m->y, m->r, m->d, m->q, m->fr, m->fd, m->states, m->partials,
                            m->pstride, m->active + 1, m->active, m->nrhs, s));
    return launch_xpay_m(m->pd, vh, m->r, m->d, m->fr, m->fd, m->states, m->active + 1, m->active,
                         m->nrhs, s);
}

static stg_status graph_m(const stg_gauge *g, MrhsWs *m, const LinkField *lf, int iters,
                          cudaGraphExec_t *out)
{
    if (m->graph && m->graph_iters == iters) {
        *out = m->graph;
        return STG_OK;
    }
    if (m->graph) {
        cudaGraphExecDestroy(m->graph);
        m->graph = nullptr;
    }
    cudaStream_t cs;
    STG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    stg_status st = STG_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < iters && st == STG_OK; ++k) st = iteration_m(g, m, lf, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == STG_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (st == STG_OK) {
        e = cudaGraphInstantiate(&m->graph, graph, 0);
        if (e != cudaSuccess) {
            m->graph = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != STG_OK) return st;
    m->graph_iters = iters;
    *out = m->graph;
    return STG_OK;
}

static stg_status sync_states(MrhsWs *m, cudaStream_t s, bool to_host)
{
    const size_t bytes = m->nrhs * sizeof(CGState);
    if (to_host) {
        STG_CUDA(cudaMemcpyAsync(m->states_host, m->states, bytes, cudaMemcpyDeviceToHost, s));
        STG_CUDA(cudaStreamSynchronize(s));
    } else {
        STG_CUDA(cudaMemcpyAsync(m->states, m->states_host, bytes, cudaMemcpyHostToDevice, s));
    }
    return STG_OK;
}

}  // namespace stg

// ---------------------------------------------------------------------------
// batch session: systems join and leave between chunks of iterations
// ---------------------------------------------------------------------------
struct stg_batch {
    stg_gauge *g = nullptr;
    const stg::LinkField *lf = nullptr;
    int n = 0, pd = 0, pr = 0;
    stg_cg_params p;
    cudaStream_t s = nullptr;
    stg::MrhsWs *m = nullptr;
    int chunk = 16;
    long maxiter = 0;
    bool tuned = false;
    long launches = 0;
    struct Slot {
        int used = 0;              // 1 while the system occupies the slot
        double bb = 0, rr = 0, tol = 0;
        long updates = 0;
        const double *src = nullptr;
        double *x = nullptr;
        timespec t_add;
    };
    std::vector<Slot> slot;
    struct Done {
        int slot;
        int status;
        stg_cg_stats stats;
    };
    std::vector<Done> pending;   // finished, not yet reported
};

namespace stg {

static double elapsed_since(const timespec &t0)
{
    timespec t1;
    clock_gettime(CLOCK_MONOTONIC, &t1);
    return (t1.tv_sec - t0.tv_sec) + 1e-9 * (t1.tv_nsec - t0.tv_nsec);
}

static void finish(stg_batch *b, int k, int status)
{
    stg_batch::Slot &sl = b->slot[k];
    const CGState &h = b->m->states_host[k];
    stg_batch::Done d;
    d.slot = k;
    d.status = status;
    memset(&d.stats, 0, sizeof(d.stats));
    d.stats.iters = (long)h.iter;
    d.stats.sloppy_iters = (long)h.iter;
    d.stats.updates = sl.updates;
    d.stats.true_res = sl.bb > 0.0 ? sqrt(sl.rr / sl.bb) : 0.0;
    d.stats.iter_res = sl.bb > 0.0 ? sqrt(h.delta_new / sl.bb) : 0.0;
    d.stats.seconds = elapsed_since(sl.t_add);
    d.stats.launches = b->launches;
    b->pending.push_back(d);
    sl.used = 0;
}

static void rebuild_active(stg_batch *b)
{
    int nact = 0;
    for (int k = 0; k < b->n; ++k)
        if (b->slot[k].used) b->m->active_host[1 + nact++] = k;
    b->m->active_host[0] = nact;
}

static stg_status push_states(stg_batch *b)
{
    MrhsWs *m = b->m;
    for (int k = 0; k < b->n; ++k) m->states_host[k].counter = 0;
    STG_TRY(sync_states(m, b->s, false));
    STG_CUDA(cudaMemcpyAsync(m->active, m->active_host, (b->n + 1) * sizeof(int),
                             cudaMemcpyHostToDevice, b->s));
    return STG_OK;
}

stg_status batch_create(stg_gauge *g, int n, const stg_cg_params *p, cudaStream_t s, stg_batch **out)
{
    stg_batch *b = new (std::nothrow) stg_batch();
    if (!b) {
        set_error("stg_batch_create: host allocation failed");
        return STG_ERR_OOM;
    }
    b->g = g;
    b->n = n;
    b->p = *p;
    b->pd = p->sloppy;
    b->pr = pr_of_m(b->pd);
    b->lf = links_for(g, b->pd);
    b->s = s;
    b->maxiter = p->maxiter > 0 ? p->maxiter : 10L * 3L * g->geom.Vh;
    b->chunk = p->check_every > 0 ? (p->check_every > 256 ? 256 : p->check_every) : 16;
    b->slot.resize(n);
    stg_status st = mrhs_alloc(g, n, b->pd, &b->m);
    if (st != STG_OK) {
        delete b;
        return st;
    }
    *out = b;
    return STG_OK;
}

void batch_destroy(stg_batch *b)
{
    if (!b) return;
    mrhs_free(b->m);
    delete b;
}

// Admit one system: b, x0 to FP64, r = b - A x0; the system starts at the
// next chunk (or is finished at once if x0 already meets the tolerance).
stg_status batch_add(stg_batch *b, const double *src, double *x, double mass, double tol, int *slot_out)
{
    int k = -1;
    for (int j = 0; j < b->n; ++j)
        if (!b->slot[j].used) {
            k = j;
            break;
        }
    if (k < 0) {
        set_error("stg_batch_add: every slot of the session is occupied");
        return STG_ERR_INVALID_ARG;
    }
    MrhsWs *m = b->m;
    const Geom &geo = b->g->geom;
    const int vh = geo.Vh;
    cudaStream_t s = b->s;
    stg_batch::Slot &sl = b->slot[k];
    clock_gettime(CLOCK_MONOTONIC, &sl.t_add);
    sl.src = src;
    sl.x = x;
    sl.tol = tol;
    sl.updates = 0;
    STG_TRY(pack_field(geo, P64, src, m->b64 + k * m->f64, s));
    STG_TRY(pack_field(geo, P64, x, m->x64 + k * m->f64, s));
    STG_TRY(launch_norm2(P64, vh, m->b64 + k * m->f64, m->states + k, m->partials, s));
    STG_TRY(sync_states(m, s, true));
    const double bb = m->states_host[k].result;
    STG_TRY(launch_true_residual(b->g, m->x64 + k * m->f64, m->b64 + k * m->f64, m->r64 + k * m->f64,
                                 m->tmp, mass * mass, m->states + k, m->partials, s));
    STG_TRY(sync_states(m, s, true));
    const double rr = m->states_host[k].result;
    b->launches += 5;
    if (!isfinite(bb) || !isfinite(rr)) {
        set_error("stg_batch_add: non-finite source or initial residual");
        return STG_ERR_INVALID_ARG;
    }
    sl.bb = bb;
    sl.rr = rr;
    sl.used = 1;
    CGState &h = m->states_host[k];
    memset(&h, 0, sizeof(CGState));
    h.m2 = mass * mass;
    h.stop_r2 = tol * tol * bb;
    h.trig2 = b->p.policy == STG_CG_PLAIN ? 0.0 : b->p.delta * b->p.delta;
    h.track_max = (b->p.policy == STG_CG_RELIABLE) ? 1 : 0;
    h.iter_limit = b->maxiter;
    h.delta_new = h.delta_old = h.rmax2 = rr;
    if (bb == 0.0 || rr <= h.stop_r2) {
        if (bb == 0.0) STG_CUDA(cudaMemsetAsync(x, 0, m->f64, s));
        h.flag = FLAG_CONVERGED;
        finish(b, k, STG_OK);
    } else {
        STG_TRY(launch_reset(b->pd, vh, m->y + k * m->fr, m->r + k * m->fr, m->d + k * m->fd,
                             m->r64 + k * m->f64, 0.0, 1, s));
        ++b->launches;
        h.flag = FLAG_RUN;
    }
    rebuild_active(b);
    STG_TRY(push_states(b));
    *slot_out = k;
    return STG_OK;
}

// One chunk of iterations for every active system, then the FP64 updates of
// the systems that asked for one; finished systems get x written.
stg_status batch_step(stg_batch *b)
{
    MrhsWs *m = b->m;
    if (m->active_host[0] == 0) return STG_OK;
    const int vh = b->g->geom.Vh;
    cudaStream_t s = b->s;
    CGState *h = m->states_host;
    if (!b->tuned) {
        // tune NB / block size on the session's own t fields (output only)
        STG_TRY(tune(b->g, b->lf, b->n, m->d, m->t, m->fd, s, &m->shape));
        b->tuned = true;
    }
    cudaGraphExec_t graph;
    STG_TRY(graph_m(b->g, m, b->lf, b->chunk, &graph));
    STG_CUDA(cudaGraphLaunch(graph, s));
    b->launches += 4L * b->chunk;
    STG_TRY(sync_states(m, s, true));
    std::vector<int> flagged;
    for (int a = 0; a < m->active_host[0]; ++a) {
        const int k = m->active_host[1 + a];
        if (h[k].flag != FLAG_RUN) flagged.push_back(k);
    }
    if (flagged.empty()) return STG_OK;
    // Sec. 3.2 updates: x_k += y_k (FP64), r_k = b_k - A_k x_k (FP64)
    std::vector<CGState> before(flagged.size());
    for (size_t u = 0; u < flagged.size(); ++u) {
        const int k = flagged[u];
        before[u] = h[k];
        STG_TRY(launch_accumulate_x(b->pr, vh, m->x64 + k * m->f64, m->y + k * m->fr, s));
        STG_TRY(launch_true_residual(b->g, m->x64 + k * m->f64, m->b64 + k * m->f64,
                                     m->r64 + k * m->f64, m->tmp, h[k].m2, m->states + k,
                                     m->partials, s));
        b->launches += 3;
        ++b->slot[k].updates;
    }
    STG_TRY(sync_states(m, s, true));
    for (size_t u = 0; u < flagged.size(); ++u) {
        const int k = flagged[u];
        const CGState b4 = before[u];
        const double rr = h[k].result;
        h[k] = b4;  // the residual kernels touched only result and the counter
        b->slot[k].rr = rr;
        int done = -1;
        if (rr <= h[k].stop_r2) done = STG_OK;
        else if (!isfinite(rr)) done = STG_ERR_BREAKDOWN;
        else if (h[k].iter >= b->maxiter) done = STG_ERR_NOT_CONVERGED;
        if (done >= 0) {
            STG_TRY(unpack_field(b->g->geom, P64, m->x64 + k * m->f64, b->slot[k].x, s));
            ++b->launches;
            h[k].flag = FLAG_CONVERGED;
            finish(b, k, done);
            continue;
        }
        double beta = 0.0;
        if (b4.flag != FLAG_BREAKDOWN && b->p.policy == STG_CG_RELIABLE) beta = rr / b4.delta_old;
        STG_TRY(launch_reset(b->pd, vh, m->y + k * m->fr, m->r + k * m->fr, m->d + k * m->fd,
                             m->r64 + k * m->f64, beta, 1, s));
        ++b->launches;
        h[k].delta_new = rr;
        h[k].delta_old = rr;
        h[k].rmax2 = rr;
        h[k].flag = FLAG_RUN;
    }
    rebuild_active(b);
    STG_TRY(push_states(b));
    STG_CUDA(cudaStreamSynchronize(s));  // unpacked solutions are complete
    return STG_OK;
}

stg_status cg_solve_mrhs(stg_gauge *g, int n, const double *src, double *x, const double *masses,
                         double tol, const stg_cg_params *p, stg_cg_stats *stats, cudaStream_t s)
{
    // one cached session per handle for this convenience call
    Workspace *ws;
    STG_TRY(workspace_get(g, &ws));
    stg_batch *b = ws->batch;
    if (b && (b->n != n || b->pd != p->sloppy)) {
        batch_destroy(b);
        ws->batch = b = nullptr;
    }
    if (!b) {
        STG_TRY(batch_create(g, n, p, s, &b));
        ws->batch = b;
    }
    b->p = *p;
    b->s = s;
    b->launches = 0;
    b->maxiter = p->maxiter > 0 ? p->maxiter : 10L * 3L * g->geom.Vh;
    // chunks of 8 by default: a system that asks for a reliable update idles
    // until its chunk ends (measured at 16 systems on 24^3x48: FP32 inner
    // 402.4 / 399.5 / 397.5 ms at 16 / 8 / 4 iterations per chunk)
    b->chunk = p->check_every > 0 ? (p->check_every > 256 ? 256 : p->check_every) : 8;
    b->pending.clear();
    const size_t canon = (size_t)g->geom.Vh * 6;
    std::vector<int> slot_of(n, -1);
    for (int k = 0; k < n; ++k) STG_TRY(batch_add(b, src + k * canon, x + k * canon, masses[k], tol, &slot_of[k]));
    while (b->m->active_host[0] > 0) STG_TRY(batch_step(b));
    STG_CUDA(cudaStreamSynchronize(s));
    stg_status worst = STG_OK;
    for (const stg_batch::Done &d : b->pending) {
        int k = -1;
        for (int j = 0; j < n; ++j)
            if (slot_of[j] == d.slot) k = j;
        if (k < 0) continue;
        if (stats) {
            stats[k] = d.stats;
            stats[k].launches = b->launches;
        }
        if (d.status != STG_OK && worst == STG_OK) worst = (stg_status)d.status;
    }
    b->pending.clear();
    if (worst == STG_ERR_BREAKDOWN) set_error("stg_cg_solve_mrhs: non-finite true residual in a system");
    if (worst == STG_ERR_NOT_CONVERGED) set_error("stg_cg_solve_mrhs: maxiter reached before convergence of a system");
    return worst;
}

}  // namespace stg

using namespace stg;

static stg_status check_m(const stg_gauge *g, int nrhs, int prec, const LinkField **lf)
{
    if (!g || nrhs < 1 || nrhs > kMaxRhs) {
        set_error("multi-system call: NULL handle or nrhs outside [1, 64]");
        return STG_ERR_INVALID_ARG;
    }
    if (prec != STG_FP32 && prec != STG_FX16) {
        set_error("multi-system call: precision must be FP32 or FX16");
        return STG_ERR_UNSUPPORTED;
    }
    *lf = links_for(g, prec);
    if (!*lf) {
        set_error("multi-system call: the handle holds no links in this precision");
        return STG_ERR_UNSUPPORTED;
    }
    return STG_OK;
}

struct DevScope {
    int prev = -1, want;
    explicit DevScope(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~DevScope()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

extern "C" {

stg_status stg_dslash_mrhs(const stg_gauge *g, int out_parity, int nrhs, const void *in_dev,
                           void *out_dev, stg_prec prec, stg_stream_t stream)
{
    const LinkField *lf;
    STG_TRY(check_m(g, nrhs, prec, &lf));
    if (!in_dev || !out_dev || in_dev == out_dev || (out_parity != 0 && out_parity != 1)) {
        set_error("stg_dslash_mrhs: bad pointer or parity");
        return STG_ERR_INVALID_ARG;
    }
    DevScope ds(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fb = (size_t)g->geom.Vh * field_site_bytes(prec);
    int shape;
    STG_TRY(tune(g, lf, nrhs, in_dev, out_dev, fb, s, &shape));
    MrhsArgs a = {};
    a.parity = out_parity;
    a.in = static_cast<const char *>(in_dev);
    a.out = static_cast<char *>(out_dev);
    a.fstride = fb;
    a.nrhs = nrhs;
    return launch_m(g, lf, shape, EPI_NONE, a, s);
}

stg_status stg_apply_A_mrhs(const stg_gauge *gc, int nrhs, const double *masses, const void *in_dev,
                            void *out_dev, stg_prec prec, stg_stream_t stream)
{
    const LinkField *lf;
    STG_TRY(check_m(gc, nrhs, prec, &lf));
    if (!in_dev || !out_dev || in_dev == out_dev || !masses) {
        set_error("stg_apply_A_mrhs: bad pointer");
        return STG_ERR_INVALID_ARG;
    }
    for (int k = 0; k < nrhs; ++k)
        if (!isfinite(masses[k])) {
            set_error("stg_apply_A_mrhs: non-finite mass");
            return STG_ERR_INVALID_ARG;
        }
    stg_gauge *g = const_cast<stg_gauge *>(gc);
    DevScope ds(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    Workspace *ws;
    STG_TRY(workspace_get(g, &ws));
    const size_t fb = (size_t)g->geom.Vh * field_site_bytes(prec);
    if (ws->mrhs_tmp_bytes < nrhs * fb) {
        cudaFree(ws->mrhs_tmp);
        ws->mrhs_tmp = nullptr;
        ws->mrhs_tmp_bytes = 0;
        STG_TRY(dev_alloc(&ws->mrhs_tmp, nrhs * fb));
        ws->mrhs_tmp_bytes = nrhs * fb;
    }
    int shape;
    STG_TRY(tune(g, lf, nrhs, in_dev, ws->mrhs_tmp, fb, s, &shape));
    MrhsArgs a = {};
    a.parity = 1;
    a.in = static_cast<const char *>(in_dev);
    a.out = static_cast<char *>(ws->mrhs_tmp);
    a.fstride = fb;
    a.nrhs = nrhs;
    STG_TRY(launch_m(g, lf, shape, EPI_NONE, a, s));
    a.parity = 0;
    a.in = static_cast<const char *>(ws->mrhs_tmp);
    a.out = static_cast<char *>(out_dev);
    a.w = static_cast<const char *>(in_dev);
    for (int k = 0; k < nrhs; ++k) a.m2[k] = (float)(masses[k] * masses[k]);
    return launch_m(g, lf, shape, EPI_A, a, s);
}

stg_status stg_cg_solve_mrhs(const stg_gauge *gc, int nrhs, const double *src_dev, double *x_dev,
                             const double *masses, double tol, const stg_cg_params *params,
                             stg_cg_stats *stats, stg_stream_t stream)
{
    if (!gc || nrhs < 1 || nrhs > kMaxRhs || !src_dev || !x_dev || !masses || src_dev == x_dev) {
        set_error("stg_cg_solve_mrhs: NULL argument, src == x, or nrhs outside [1, 64]");
        return STG_ERR_INVALID_ARG;
    }
    if (!isfinite(tol) || !(tol > 0.0)) {
        set_error("stg_cg_solve_mrhs: tol must be finite and > 0");
        return STG_ERR_INVALID_ARG;
    }
    for (int k = 0; k < nrhs; ++k)
        if (!isfinite(masses[k]) || masses[k] < 0.0) {
            set_error("stg_cg_solve_mrhs: masses must be finite and >= 0");
            return STG_ERR_INVALID_ARG;
        }
    stg_cg_params p;
    if (params) p = *params;
    else stg_cg_params_default(gc, &p);
    if (p.policy < STG_CG_RELIABLE || p.policy > STG_CG_PLAIN || !(p.delta > 0.0 && p.delta < 1.0) ||
        p.maxiter < 0 || p.check_every < 0) {
        set_error("stg_cg_solve_mrhs: bad params");
        return STG_ERR_INVALID_ARG;
    }
    if (p.policy == STG_CG_PLAIN || p.sloppy == STG_FP64) {
        set_error("stg_cg_solve_mrhs: the batched solver runs FP32 or FX16 inner iterations "
                  "(use stg_cg_solve per system for plain FP64 CG)");
        return STG_ERR_UNSUPPORTED;
    }
    const LinkField *lf;
    STG_TRY(check_m(gc, nrhs, p.sloppy, &lf));
    stg_gauge *g = const_cast<stg_gauge *>(gc);
    DevScope ds(g->device);
    return cg_solve_mrhs(g, nrhs, src_dev, x_dev, masses, tol, &p, stats, (cudaStream_t)stream);
}

stg_status stg_batch_create(const stg_gauge *gc, int max_systems, const stg_cg_params *params,
                            stg_stream_t stream, stg_batch **out)
{
    if (!gc || !out || max_systems < 1 || max_systems > kMaxRhs) {
        set_error("stg_batch_create: NULL argument or max_systems outside [1, 64]");
        return STG_ERR_INVALID_ARG;
    }
    stg_cg_params p;
    if (params) p = *params;
    else stg_cg_params_default(gc, &p);
    if (p.policy < STG_CG_RELIABLE || p.policy > STG_CG_REFINE || !(p.delta > 0.0 && p.delta < 1.0) ||
        p.maxiter < 0 || p.check_every < 0) {
        set_error("stg_batch_create: bad params (policy RELIABLE or REFINE, 0 < delta < 1)");
        return STG_ERR_INVALID_ARG;
    }
    const LinkField *lf;
    STG_TRY(check_m(gc, max_systems, p.sloppy, &lf));
    stg_gauge *g = const_cast<stg_gauge *>(gc);
    DevScope ds(g->device);
    *out = nullptr;
    return batch_create(g, max_systems, &p, (cudaStream_t)stream, out);
}

stg_status stg_batch_destroy(stg_batch *b)
{
    if (!b) return STG_OK;
    DevScope ds(b->g->device);
    cudaStreamSynchronize(b->s);
    batch_destroy(b);
    return STG_OK;
}

stg_status stg_batch_add(stg_batch *b, const double *src_dev, double *x_dev, double mass, double tol,
                         int *slot)
{
    if (!b || !src_dev || !x_dev || !slot || src_dev == x_dev) {
        set_error("stg_batch_add: NULL argument or src == x");
        return STG_ERR_INVALID_ARG;
    }
    if (!isfinite(mass) || mass < 0.0 || !isfinite(tol) || !(tol > 0.0)) {
        set_error("stg_batch_add: mass must be finite and >= 0, tol finite and > 0");
        return STG_ERR_INVALID_ARG;
    }
    DevScope ds(b->g->device);
    return batch_add(b, src_dev, x_dev, mass, tol, slot);
}

stg_status stg_batch_step(stg_batch *b, int max_done, int *done_slots, int *done_status,
                          stg_cg_stats *done_stats, int *n_done, int *n_active)
{
    if (!b || max_done < 0 || (max_done > 0 && (!done_slots || !done_status)) || !n_done) {
        set_error("stg_batch_step: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    DevScope ds(b->g->device);
    *n_done = 0;
    stg_status st = STG_OK;
    if (b->pending.empty()) st = batch_step(b);
    int k = 0;
    while (k < max_done && !b->pending.empty()) {
        const stg_batch::Done d = b->pending.front();
        b->pending.erase(b->pending.begin());
        done_slots[k] = d.slot;
        done_status[k] = d.status;
        if (done_stats) done_stats[k] = d.stats;
        ++k;
    }
    *n_done = k;
    if (n_active) *n_active = b->m->active_host[0] + (int)b->pending.size();
    return st;
}

size_t stg_batch_bytes(const stg_gauge *g, int max_systems, stg_prec sloppy)
{
    if (!g || max_systems < 1) return 0;
    return mrhs_bytes(g->geom, max_systems, sloppy);
}

stg_status stg_mrhs_tuning(const stg_gauge *g, stg_prec prec, int nrhs, int *rhs_block,
                           int *threads_per_site)
{
    const LinkField *lf;
    STG_TRY(check_m(g, nrhs, prec, &lf));
    if (!rhs_block || !threads_per_site) {
        set_error("stg_mrhs_tuning: NULL output");
        return STG_ERR_INVALID_ARG;
    }
    int shape;
    if (!forced_shape(lf, nrhs, &shape) && !tune_lookup(g->dims, lf->prec, lf->recon, nrhs, &shape)) {
        set_error("stg_mrhs_tuning: not tuned yet for this lattice, precision and nrhs");
        return STG_ERR_INVALID_ARG;
    }
    if (shape >= kRiFirst) {
        *rhs_block = ms_ri_nb(shape - kRiFirst);
        *threads_per_site = -2;  // staged, on (re, im) FP32x2 pairs
    } else if (shape >= kMspFirst) {
        *rhs_block = shape == kMspFirst ? 2 : 4;
        *threads_per_site = -1;  // staged, two sites per thread (FX16 / 12-real)
    } else if (shape >= kMrhsShapes) {
        *rhs_block = ms_nb(shape - kMrhsShapes);
        *threads_per_site = 0;  // staged: one link load per site serves all systems
    } else {
        *rhs_block = mrhs_nb(shape);
        *threads_per_site = mrhs_tps(shape);
    }
    return STG_OK;
}

}  // extern "C"
