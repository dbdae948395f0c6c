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

void launch_dslash_m_f32(int recon, int nb, int bs, int epi, const MrhsArgs &a, cudaStream_t s);
void launch_dslash_m_fx16(int recon, int nb, int bs, int epi, const MrhsArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------
// autotuner cache: process-wide, optionally mirrored in a text file named by
// the STG_TUNE_CACHE environment variable ("Lx Ly Lz Lt prec recon n nb bs")
// ---------------------------------------------------------------------------
struct TuneEntry {
    int dims[4];
    int prec, recon, nrhs, nb, bs;
};

static std::mutex g_tune_mutex;
static std::vector<TuneEntry> g_tune;
static bool g_tune_loaded = false;

static bool same_key(const TuneEntry &e, const int *dims, int prec, int recon, int nrhs)
{
    return e.dims[0] == dims[0] && e.dims[1] == dims[1] && e.dims[2] == dims[2] &&
           e.dims[3] == dims[3] && e.prec == prec && e.recon == recon && e.nrhs == nrhs;
}

static bool valid_choice(int nb, int bs)
{
    return (nb == 1 || nb == 2 || nb == 4 || nb == 8) && (bs == 128 || bs == 256);
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
    while (fscanf(f, "%d %d %d %d %d %d %d %d %d", &e.dims[0], &e.dims[1], &e.dims[2], &e.dims[3],
                  &e.prec, &e.recon, &e.nrhs, &e.nb, &e.bs) == 9) {
        if (valid_choice(e.nb, e.bs)) g_tune.push_back(e);
    }
    fclose(f);
}

static bool tune_lookup(const int *dims, int prec, int recon, int nrhs, int *nb, int *bs)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load_file_locked();
    for (const TuneEntry &e : g_tune)
        if (same_key(e, dims, prec, recon, nrhs)) {
            *nb = e.nb;
            *bs = e.bs;
            return true;
        }
    return false;
}

static void tune_store(const int *dims, int prec, int recon, int nrhs, int nb, int bs)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    TuneEntry e = {{dims[0], dims[1], dims[2], dims[3]}, prec, recon, nrhs, nb, bs};
    g_tune.push_back(e);
    const char *path = getenv("STG_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %d %d %d %d %d %d\n", dims[0], dims[1], dims[2], dims[3], prec, recon,
            nrhs, nb, bs);
    fclose(f);
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
static stg_status launch_m(const stg_gauge *g, const LinkField *lf, int nb, int bs, int epi,
                           MrhsArgs &a, cudaStream_t s)
{
    a.g = g->geom;
    for (int mu = 0; mu < 4; ++mu) {
        a.lf[mu] = lf->blk(a.parity, mu);
        a.lb[mu] = lf->blk(1 - a.parity, mu);
    }
    if (lf->prec == P32) launch_dslash_m_f32(lf->recon, nb, bs, epi, a, s);
    else if (lf->prec == PX16) launch_dslash_m_fx16(lf->recon, nb, bs, epi, a, s);
    else {
        set_error("multi-system Dslash: only FP32 and FX16 storage are supported");
        return STG_ERR_UNSUPPORTED;
    }
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// Time one EPI_NONE half-pass of all n systems for every (NB, BS) candidate
// (one warm-up and three timed launches each, CUDA events on `s`) and keep
// the fastest.  `in` / `out` hold n fields each and are overwritten.
static stg_status tune(const stg_gauge *g, const LinkField *lf, int n, const void *in, void *out,
                       size_t fstride, cudaStream_t s, int *nb_out, int *bs_out)
{
    if (tune_lookup(g->dims, lf->prec, lf->recon, n, nb_out, bs_out)) return STG_OK;
    cudaEvent_t e0, e1;
    STG_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    float best = 1e30f;
    int bnb = 1, bbs = 256;
    stg_status st = STG_OK;
    const int nbs[4] = {1, 2, 4, 8};
    const int bss[2] = {128, 256};
    for (int u = 0; u < 4 && st == STG_OK; ++u) {
        if (nbs[u] > 1 && nbs[u] > n) break;
        for (int v = 0; v < 2 && st == STG_OK; ++v) {
            MrhsArgs a = {};
            a.parity = 1;
            a.in = static_cast<const char *>(in);
            a.out = static_cast<char *>(out);
            a.fstride = fstride;
            a.nrhs = n;
            st = launch_m(g, lf, nbs[u], bss[v], EPI_NONE, a, s);
            if (st != STG_OK) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && st == STG_OK; ++r) st = launch_m(g, lf, nbs[u], bss[v], EPI_NONE, a, s);
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
                bnb = nbs[u];
                bbs = bss[v];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != STG_OK) return st;
    tune_store(g->dims, lf->prec, lf->recon, n, bnb, bbs);
    *nb_out = bnb;
    *bs_out = bbs;
    return STG_OK;
}

// ---------------------------------------------------------------------------
// workspace of the multi-system solver
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

static stg_status mrhs_prepare(stg_gauge *g, int n, int pd, MrhsWs **out)
{
    Workspace *ws;
    STG_TRY(workspace_get(g, &ws));
    if (ws->mrhs && ws->mrhs->nrhs == n && ws->mrhs->pd == pd) {
        *out = ws->mrhs;
        return STG_OK;
    }
    if (ws->mrhs) {
        mrhs_free(ws->mrhs);
        ws->mrhs = nullptr;
    }
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
    m->pstride = (size_t)((g->geom.Vh + 127) / 128) + 64;
    stg_status st = STG_OK;
    char **bufs[] = {&m->x64, &m->b64, &m->r64};
    for (char **b : bufs)
        if (st == STG_OK) st = dev_alloc((void **)b, n * m->f64);
    if (st == STG_OK) st = dev_alloc((void **)&m->y, n * m->fr);
    if (st == STG_OK) st = dev_alloc((void **)&m->r, n * m->fr);
    if (st == STG_OK) st = dev_alloc((void **)&m->d, n * m->fd);
    if (st == STG_OK) st = dev_alloc((void **)&m->q, n * m->fd);
    if (st == STG_OK) st = dev_alloc((void **)&m->t, n * m->fd);
    if (st == STG_OK) st = dev_alloc((void **)&m->partials, n * m->pstride * sizeof(double));
    if (st == STG_OK) st = dev_alloc((void **)&m->states, n * sizeof(CGState));
    if (st == STG_OK) st = dev_alloc((void **)&m->active, (n + 1) * sizeof(int));
    if (st == STG_OK) st = dev_alloc((void **)&m->counter, 256);
    if (st == STG_OK) {
        cudaError_t e = cudaMemset(m->states, 0, n * sizeof(CGState));
        if (e == cudaSuccess) e = cudaMemset(m->counter, 0, 256);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&m->states_host, n * sizeof(CGState));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&m->active_host, (n + 1) * sizeof(int));
        if (e != cudaSuccess) st = cuda_fail(e, "multi-system workspace");
    }
    void *tmp64;
    if (st == STG_OK) st = workspace_tmp(g, P64, &tmp64);
    if (st != STG_OK) {
        mrhs_free(m);
        return st;
    }
    ws->mrhs = m;
    *out = m;
    return STG_OK;
}

// one iteration of all active systems (4 launches)
static stg_status iteration_m(stg_gauge *g, MrhsWs *m, const LinkField *lf, cudaStream_t s)
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
    STG_TRY(launch_m(g, lf, m->nb, m->bs, EPI_GATE, a, s));
    a.parity = 0;
    a.in = m->t;
    a.out = m->q;
    a.w = m->d;
    STG_TRY(launch_m(g, lf, m->nb, m->bs, EPI_A_CG, a, s));
    const int vh = g->geom.Vh;
    STG_TRY(launch_update_m(m->pd, vh, m->y, m->r, m->d, m->q, m->fr, m->fd, m->states, m->partials,
                            m->pstride, m->active + 1, m->active, m->nrhs, s));
    return launch_xpay_m(m->pd, vh, m->r, m->d, m->fr, m->fd, m->states, m->active + 1, m->active,
                         m->nrhs, s);
}

static stg_status graph_m(stg_gauge *g, MrhsWs *m, const LinkField *lf, int iters, cudaGraphExec_t *out)
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

enum { SYS_ACTIVE = 0, SYS_DONE = 1, SYS_NOT_CONVERGED = 2, SYS_BREAKDOWN = 3 };

stg_status cg_solve_mrhs(stg_gauge *g, int n, const double *src, double *x, const double *masses,
                         double tol, const stg_cg_params *p, stg_cg_stats *stats, cudaStream_t s)
{
    timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    const Geom &geo = g->geom;
    const int vh = geo.Vh;
    const int pd = p->sloppy;
    const int pr = pr_of_m(pd);
    const LinkField *lf = links_for(g, pd);
    MrhsWs *m;
    STG_TRY(mrhs_prepare(g, n, pd, &m));
    Workspace *ws = g->ws;
    const long maxiter = p->maxiter > 0 ? p->maxiter : 10L * 3L * vh;
    int chunk = p->check_every > 0 ? p->check_every : 16;
    if (chunk > 256) chunk = 256;
    const size_t canon = (size_t)vh * 6;  // doubles per canonical field

    std::vector<double> bb(n), rr(n), m2(n);
    std::vector<int> sys(n, SYS_ACTIVE);
    std::vector<long> updates(n, 0);
    long launches = 0;
    CGState *h = m->states_host;

    // b_k, x0_k into FP64 device layout; |b_k|^2
    for (int k = 0; k < n; ++k) {
        m2[k] = masses[k] * masses[k];
        STG_TRY(pack_field(geo, P64, src + k * canon, m->b64 + k * m->f64, s));
        STG_TRY(pack_field(geo, P64, x + k * canon, m->x64 + k * m->f64, s));
        STG_TRY(launch_norm2(P64, vh, m->b64 + k * m->f64, m->states + k, m->partials, s));
        launches += 3;
    }
    STG_TRY(sync_states(m, s, true));
    for (int k = 0; k < n; ++k) {
        bb[k] = h[k].result;
        if (!isfinite(bb[k])) {
            set_error("stg_cg_solve_mrhs: a source has non-finite entries");
            return STG_ERR_INVALID_ARG;
        }
    }
    // r_k = b_k - A_k x0_k
    for (int k = 0; k < n; ++k) {
        STG_TRY(launch_true_residual(g, m->x64 + k * m->f64, m->b64 + k * m->f64, m->r64 + k * m->f64,
                                     ws->tmp[P64], m2[k], m->states + k, m->partials, s));
        launches += 2;
    }
    STG_TRY(sync_states(m, s, true));
    int nact = 0;
    for (int k = 0; k < n; ++k) {
        rr[k] = h[k].result;
        const double stop = tol * tol * bb[k];
        memset(&h[k], 0, sizeof(CGState));
        h[k].m2 = m2[k];
        h[k].stop_r2 = stop;
        h[k].trig2 = p->policy == STG_CG_PLAIN ? 0.0 : p->delta * p->delta;
        h[k].track_max = (p->policy == STG_CG_RELIABLE) ? 1 : 0;
        h[k].iter_limit = maxiter;
        h[k].delta_new = h[k].delta_old = h[k].rmax2 = rr[k];
        if (bb[k] == 0.0 || rr[k] <= stop) {
            sys[k] = SYS_DONE;
            h[k].flag = FLAG_CONVERGED;
            if (bb[k] == 0.0) STG_CUDA(cudaMemsetAsync(m->x64 + k * m->f64, 0, m->f64, s));
            continue;
        }
        // y = 0, r = r64, d = r (Fig. 1 / Fig. 2 start)
        STG_TRY(launch_reset(pd, vh, m->y + k * m->fr, m->r + k * m->fr, m->d + k * m->fd,
                             m->r64 + k * m->f64, 0.0, 1, s));
        ++launches;
        h[k].flag = FLAG_RUN;
        m->active_host[1 + nact++] = k;
    }
    m->active_host[0] = nact;
    STG_TRY(sync_states(m, s, false));
    STG_CUDA(cudaMemcpyAsync(m->active, m->active_host, (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));

    stg_status status = STG_OK;
    if (nact > 0) {
        // tune NB / BS on the solver's own fields (their values are reset below)
        status = tune(g, lf, n, m->d, m->t, m->fd, s, &m->nb, &m->bs);
        if (status == STG_OK && m->tuned_nb != m->nb) {
            if (m->graph) cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
            m->tuned_nb = m->nb;
        }
        // the tuner wrote t only; d still holds r
        cudaGraphExec_t graph = nullptr;
        if (status == STG_OK) status = graph_m(g, m, lf, chunk, &graph);
        while (status == STG_OK && nact > 0) {
            cudaError_t e = cudaGraphLaunch(graph, s);
            if (e != cudaSuccess) {
                status = cuda_fail(e, "cudaGraphLaunch");
                break;
            }
            launches += 4L * chunk;
            status = sync_states(m, s, true);
            if (status != STG_OK) break;
            // systems that raised a flag: x += y, r = b - A x in FP64
            std::vector<int> flagged;
            for (int a = 0; a < nact; ++a) {
                const int k = m->active_host[1 + a];
                if (h[k].flag != FLAG_RUN) flagged.push_back(k);
            }
            if (flagged.empty()) continue;
            std::vector<CGState> before(flagged.size());
            for (size_t u = 0; u < flagged.size(); ++u) {
                const int k = flagged[u];
                before[u] = h[k];
                if (pd != P64) {
                    status = launch_accumulate_x(pr, vh, m->x64 + k * m->f64, m->y + k * m->fr, s);
                    if (status != STG_OK) break;
                }
                status = launch_true_residual(g, m->x64 + k * m->f64, m->b64 + k * m->f64,
                                              m->r64 + k * m->f64, ws->tmp[P64], m2[k], m->states + k,
                                              m->partials, s);
                if (status != STG_OK) break;
                launches += 3;
                ++updates[k];
            }
            if (status != STG_OK) break;
            status = sync_states(m, s, true);
            if (status != STG_OK) break;
            for (size_t u = 0; u < flagged.size(); ++u) {
                const int k = flagged[u];
                const CGState &b4 = before[u];
                rr[k] = h[k].result;
                // restore the iterate's scalars (the residual kernels only
                // touched result and the counter)
                h[k] = b4;
                if (rr[k] <= h[k].stop_r2) {
                    sys[k] = SYS_DONE;
                    h[k].flag = FLAG_CONVERGED;
                    continue;
                }
                if (!isfinite(rr[k])) {
                    sys[k] = SYS_BREAKDOWN;
                    continue;
                }
                if (h[k].iter >= maxiter) {
                    sys[k] = SYS_NOT_CONVERGED;
                    continue;
                }
                double beta = 0.0;
                if (b4.flag != FLAG_BREAKDOWN && p->policy == STG_CG_RELIABLE) beta = rr[k] / b4.delta_old;
                status = launch_reset(pd, vh, m->y + k * m->fr, m->r + k * m->fr, m->d + k * m->fd,
                                      m->r64 + k * m->f64, beta, 1, s);
                if (status != STG_OK) break;
                ++launches;
                h[k].delta_new = rr[k];
                h[k].delta_old = rr[k];
                h[k].rmax2 = rr[k];
                h[k].flag = FLAG_RUN;
            }
            if (status != STG_OK) break;
            nact = 0;
            for (int k = 0; k < n; ++k)
                if (sys[k] == SYS_ACTIVE) m->active_host[1 + nact++] = k;
            m->active_host[0] = nact;
            for (int k = 0; k < n; ++k) h[k].counter = 0;
            status = sync_states(m, s, false);
            if (status != STG_OK) break;
            e = cudaMemcpyAsync(m->active, m->active_host, (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) status = cuda_fail(e, "cudaMemcpyAsync(active)");
        }
    }
    if (status == STG_OK) {
        for (int k = 0; k < n && status == STG_OK; ++k) {
            status = unpack_field(geo, P64, m->x64 + k * m->f64, x + k * canon, s);
            ++launches;
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (status == STG_OK && e != cudaSuccess) status = cuda_fail(e, "cudaStreamSynchronize");
    }
    clock_gettime(CLOCK_MONOTONIC, &t1);
    const double secs = (t1.tv_sec - t0.tv_sec) + 1e-9 * (t1.tv_nsec - t0.tv_nsec);
    bool not_conv = false, broke = false;
    for (int k = 0; k < n; ++k) {
        if (stats) {
            stg_cg_stats &o = stats[k];
            memset(&o, 0, sizeof(o));
            o.iters = (long)h[k].iter;
            o.sloppy_iters = (long)h[k].iter;
            o.updates = updates[k];
            o.true_res = bb[k] > 0.0 ? sqrt(rr[k] / bb[k]) : 0.0;
            o.iter_res = bb[k] > 0.0 ? sqrt(h[k].delta_new / bb[k]) : 0.0;
            o.seconds = secs;
            o.launches = launches;
        }
        not_conv |= sys[k] == SYS_NOT_CONVERGED;
        broke |= sys[k] == SYS_BREAKDOWN;
    }
    if (status != STG_OK) return status;
    if (broke) {
        set_error("stg_cg_solve_mrhs: non-finite true residual in a system");
        return STG_ERR_BREAKDOWN;
    }
    if (not_conv) {
        set_error("stg_cg_solve_mrhs: maxiter reached before convergence of a system");
        return STG_ERR_NOT_CONVERGED;
    }
    return STG_OK;
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
    int nb, bs;
    STG_TRY(tune(g, lf, nrhs, in_dev, out_dev, fb, s, &nb, &bs));
    MrhsArgs a = {};
    a.parity = out_parity;
    a.in = static_cast<const char *>(in_dev);
    a.out = static_cast<char *>(out_dev);
    a.fstride = fb;
    a.nrhs = nrhs;
    return launch_m(g, lf, nb, bs, EPI_NONE, a, s);
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
    int nb, bs;
    STG_TRY(tune(g, lf, nrhs, in_dev, ws->mrhs_tmp, fb, s, &nb, &bs));
    MrhsArgs a = {};
    a.parity = 1;
    a.in = static_cast<const char *>(in_dev);
    a.out = static_cast<char *>(ws->mrhs_tmp);
    a.fstride = fb;
    a.nrhs = nrhs;
    STG_TRY(launch_m(g, lf, nb, bs, EPI_NONE, a, s));
    a.parity = 0;
    a.in = static_cast<const char *>(ws->mrhs_tmp);
    a.out = static_cast<char *>(out_dev);
    a.w = static_cast<const char *>(in_dev);
    for (int k = 0; k < nrhs; ++k) a.m2[k] = (float)(masses[k] * masses[k]);
    return launch_m(g, lf, nb, bs, EPI_A, a, s);
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

stg_status stg_mrhs_tuning(const stg_gauge *g, stg_prec prec, int nrhs, int *rhs_block, int *threads)
{
    const LinkField *lf;
    STG_TRY(check_m(g, nrhs, prec, &lf));
    if (!rhs_block || !threads) {
        set_error("stg_mrhs_tuning: NULL output");
        return STG_ERR_INVALID_ARG;
    }
    if (!tune_lookup(g->dims, lf->prec, lf->recon, nrhs, rhs_block, threads)) {
        set_error("stg_mrhs_tuning: not tuned yet for this lattice, precision and nrhs");
        return STG_ERR_INVALID_ARG;
    }
    return STG_OK;
}

}  // extern "C"
