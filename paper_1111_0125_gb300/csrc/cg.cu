// Conjugate gradient (Fig. 1) and mixed-precision CG (Fig. 2 with the
// corrected inner start of Eq. 6 and the reliable / group-wise updates of
// Sec. 3.2) on the even-site operator A = m^2 - D_eo D_oe.
//
// One CG iteration is a fixed sequence of four kernels whose scalars (alpha,
// beta, the residual norms and a stop flag) live in device memory:
//   1. t = D_oe d                                  (dslash, odd output)
//   2. q = m^2 d - D_eo t, d^dag q -> alpha        (dslash + fused epilogue)
//   3. y += alpha d, r -= alpha q, |r|^2 -> beta, stop / update tests
//   4. d = r + beta d
// so a chunk of iterations is captured once as a CUDA graph and replayed;
// the host only reads the state between chunks.  Once a kernel raises the
// flag, the remaining kernels of the chunk return immediately, so the
// iterate is exactly the one at which the test fired.
//
// Vector precisions: d, q, t in the sloppy precision PD; y and r in PR
// (FP32 when PD is FP16, otherwise PD).  x, b and the true residual are FP64.
#include <math.h>
#include <time.h>

#include "stg_internal.h"

namespace stg {

stg_status pack_field(const Geom &g, int prec, const double *canon, void *out, cudaStream_t s);
stg_status unpack_field(const Geom &g, int prec, const void *in, double *canon, cudaStream_t s);

static int num_sms()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

int grid_for(long n)
{
    long g = (n + kBlock - 1) / kBlock;
    long cap = (long)num_sms() * 8;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// ---------------------------------------------------------------------------
// vector kernels (grid-stride, FP64 reductions)
// ---------------------------------------------------------------------------
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_cg_update(int vh, void *y, void *r, const void *d,
                                                      const void *q, CGState *st, double *partials)
{
    if (st->flag != FLAG_RUN) return;
    typedef typename Real<PR>::T T;
    const T alpha = T(st->alpha);
    double rr = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < vh; i += gridDim.x * kBlock) {
        const auto dv = FieldIO<PD>::load(d, vh, i);
        const auto qv = FieldIO<PD>::load(q, vh, i);
        Vec3<T> yv = FieldIO<PR>::load(y, vh, i);
        Vec3<T> rv = FieldIO<PR>::load(r, vh, i);
        T n = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            yv.r[c] += alpha * T(dv.r[c]);
            yv.i[c] += alpha * T(dv.i[c]);
            rv.r[c] -= alpha * T(qv.r[c]);
            rv.i[c] -= alpha * T(qv.i[c]);
            n += rv.r[c] * rv.r[c] + rv.i[c] * rv.i[c];
        }
        FieldIO<PR>::store(y, vh, i, yv);
        FieldIO<PR>::store(r, vh, i, rv);
        rr += double(n);
    }
    double total;
    if (grid_sum<kBlock>(rr, partials, &st->counter, total)) {
        const double old = st->delta_new;
        st->delta_old = old;
        st->delta_new = total;
        st->beta = total / old;
        st->iter += 1;
        if (!isfinite(total)) st->flag = FLAG_BREAKDOWN;
        else if (total <= st->stop_r2) st->flag = FLAG_CONVERGED;
        else if (st->trig2 > 0.0 && total < st->trig2 * st->rmax2) st->flag = FLAG_UPDATE;
        else if (st->iter >= st->iter_limit) st->flag = FLAG_MAXITER;
        if (st->track_max && total > st->rmax2) st->rmax2 = total;
    }
}

template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_xpay(int vh, const void *r, void *d, const CGState *st)
{
    if (st->flag != FLAG_RUN) return;
    typedef typename Real<PR>::T T;
    const T beta = T(st->beta);
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < vh; i += gridDim.x * kBlock) {
        const Vec3<T> rv = FieldIO<PR>::load(r, vh, i);
        const auto dv = FieldIO<PD>::load(d, vh, i);
        Vec3<typename Real<PD>::T> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = rv.r[c] + beta * T(dv.r[c]);
            o.i[c] = rv.i[c] + beta * T(dv.i[c]);
        }
        FieldIO<PD>::store(d, vh, i, o);
    }
}

// x64 += y  (reliable update, Sec. 3.2: x_{k+1} = x_k + y_n in FP64)
template <int PR>
__global__ void __launch_bounds__(kBlock) k_accumulate_x(int vh, void *x64, const void *y)
{
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < vh; i += gridDim.x * kBlock) {
        Vec3<double> x = FieldIO<P64>::load(x64, vh, i);
        const auto yv = FieldIO<PR>::load(y, vh, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x.r[c] += double(yv.r[c]);
            x.i[c] += double(yv.i[c]);
        }
        FieldIO<P64>::store(x64, vh, i, x);
    }
}

// after an update: y = 0, r = (PR) r64 (group-wise update), d = r + beta d
// (Eq. 6; beta = 0 restarts the search direction as in Fig. 2)
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_reset(int vh, void *y, void *r, void *d, const void *r64,
                                                  double beta, int copy_r)
{
    typedef typename Real<PR>::T T;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < vh; i += gridDim.x * kBlock) {
        Vec3<T> rv;
        if (copy_r) {
            const Vec3<double> r64v = FieldIO<P64>::load(r64, vh, i);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rv.r[c] = T(r64v.r[c]);
                rv.i[c] = T(r64v.i[c]);
            }
            FieldIO<PR>::store(r, vh, i, rv);
            Vec3<T> z;
#pragma unroll
            for (int c = 0; c < 3; ++c) z.r[c] = z.i[c] = T(0);
            FieldIO<PR>::store(y, vh, i, z);
        } else {
            rv = FieldIO<PR>::load(r, vh, i);
        }
        Vec3<typename Real<PD>::T> o;
        if (beta != 0.0) {
            const auto dv = FieldIO<PD>::load(d, vh, i);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.r[c] = rv.r[c] + T(beta) * T(dv.r[c]);
                o.i[c] = rv.i[c] + T(beta) * T(dv.i[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.r[c] = rv.r[c];
                o.i[c] = rv.i[c];
            }
        }
        FieldIO<PD>::store(d, vh, i, o);
    }
}

template <int P>
__global__ void __launch_bounds__(kBlock) k_norm2(int vh, const void *v, CGState *st, double *partials)
{
    double s = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < vh; i += gridDim.x * kBlock) {
        const auto a = FieldIO<P>::load(v, vh, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) s += double(a.r[c]) * double(a.r[c]) + double(a.i[c]) * double(a.i[c]);
    }
    double total;
    if (grid_sum<kBlock>(s, partials, &st->counter, total)) st->result = total;
}

// ---------------------------------------------------------------------------
// dispatch over the (PD, PR) pairs used by the solver
// ---------------------------------------------------------------------------
static int pr_of(int pd) { return pd == P16 ? P32 : pd; }

#define STG_DISPATCH_PD(pd, KERNEL, ...)                                                     \
    do {                                                                                     \
        if ((pd) == P64) KERNEL<P64, P64><<<grid, kBlock, 0, s>>>(__VA_ARGS__);              \
        else if ((pd) == P32) KERNEL<P32, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);         \
        else KERNEL<P16, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                          \
    } while (0)

static stg_status norm2(const Geom &g, int prec, const void *v, Workspace *ws, cudaStream_t s)
{
    const int grid = grid_for(g.Vh);
    if (prec == P64) k_norm2<P64><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    else if (prec == P32) k_norm2<P32><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    else k_norm2<P16><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// one CG iteration on the sloppy vectors (4 launches); with `ev`, CUDA
// events are recorded before and after each kernel (5 events; external
// records, so that stream capture turns them into event-record nodes)
static stg_status iteration(stg_gauge *gg, Workspace *ws, int pd, cudaStream_t s, cudaEvent_t *ev)
{
    const Geom &g = gg->geom;
    const LinkField *lf = links_for(gg, pd);
    void *t = ws->tmp[pd];
    DslashLaunch L = {};
    L.links = lf;
    L.state = ws->state;
    L.partials = ws->partials;
    L.counter = &ws->state->counter;
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal));
    // the state flag gates every kernel, including the first half-pass
    L.out_parity = 1;
    L.in = ws->d;
    L.out = t;
    STG_TRY(launch_dslash(g, pd, EPI_GATE, L, s));
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal));
    L.out_parity = 0;
    L.in = t;
    L.out = ws->q;
    L.w = ws->d;
    STG_TRY(launch_dslash(g, pd, EPI_A_CG, L, s));
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal));
    const int grid = grid_for(g.Vh);
    STG_DISPATCH_PD(pd, k_cg_update, g.Vh, ws->y, ws->r, ws->d, ws->q, ws->state, ws->partials);
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal));
    STG_DISPATCH_PD(pd, k_xpay, g.Vh, ws->r, ws->d, ws->state);
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[4], s, cudaEventRecordExternal));
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

static stg_status cuda_check_launch()
{
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

static stg_status alloc_vec(void **p, size_t bytes)
{
    if (*p) return STG_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cg: workspace allocation failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    return STG_OK;
}

static stg_status prepare(stg_gauge *g, Workspace *ws, int pd)
{
    const size_t vh = (size_t)g->geom.Vh;
    if (ws->cg_sloppy != pd) {
        void *v[] = {ws->y, ws->r, ws->d, ws->q};
        for (void *p : v) cudaFree(p);
        ws->y = ws->r = ws->d = ws->q = nullptr;
        if (ws->graph) {
            cudaGraphExecDestroy(ws->graph);
            ws->graph = nullptr;
        }
        ws->cg_sloppy = pd;
    }
    const int pr = pr_of(pd);
    STG_TRY(alloc_vec(&ws->x64, vh * 48));
    STG_TRY(alloc_vec(&ws->b64, vh * 48));
    STG_TRY(alloc_vec(&ws->r64, vh * 48));
    STG_TRY(alloc_vec(&ws->y, vh * field_site_bytes(pr)));
    STG_TRY(alloc_vec(&ws->r, vh * field_site_bytes(pr)));
    STG_TRY(alloc_vec(&ws->d, vh * field_site_bytes(pd)));
    STG_TRY(alloc_vec(&ws->q, vh * field_site_bytes(pd)));
    void *tmp;
    STG_TRY(workspace_tmp(g, pd, &tmp));
    STG_TRY(workspace_tmp(g, P64, &tmp));
    return STG_OK;
}

// Capture `n` iterations as a graph on a private stream (capture is not
// allowed on the legacy default stream), replayed on the caller's stream.
// With timing, the first iteration of the chunk records the 5 events.
static stg_status get_graph(stg_gauge *g, Workspace *ws, int pd, int n, int timing,
                            cudaGraphExec_t *out)
{
    if (ws->graph && ws->graph_sloppy == pd && ws->graph_iters == n && ws->graph_timing == timing) {
        *out = ws->graph;
        return STG_OK;
    }
    if (ws->graph) {
        cudaGraphExecDestroy(ws->graph);
        ws->graph = nullptr;
    }
    if (timing && !ws->ev[0])
        for (int k = 0; k < 5; ++k) STG_CUDA(cudaEventCreate(&ws->ev[k]));
    cudaStream_t cs;
    STG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    stg_status st = STG_OK;
    if (e == cudaSuccess) {
        for (int k = 0; k < n && st == STG_OK; ++k)
            st = iteration(g, ws, pd, cs, (timing && k == 0) ? ws->ev : nullptr);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == STG_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (st == STG_OK) {
        e = cudaGraphInstantiate(&ws->graph, graph, 0);
        if (e != cudaSuccess) {
            ws->graph = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != STG_OK) return st;
    ws->graph_sloppy = pd;
    ws->graph_iters = n;
    ws->graph_timing = timing;
    *out = ws->graph;
    return STG_OK;
}

static stg_status read_state(Workspace *ws, cudaStream_t s)
{
    STG_CUDA(cudaMemcpyAsync(ws->state_host, ws->state, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    STG_CUDA(cudaStreamSynchronize(s));
    return STG_OK;
}

static stg_status write_state(Workspace *ws, cudaStream_t s)
{
    STG_CUDA(cudaMemcpyAsync(ws->state, ws->state_host, sizeof(CGState), cudaMemcpyHostToDevice, s));
    return STG_OK;
}

// r64 = b64 - A x64 and |r64|^2 (FP64 operator); returns |r64|^2
static stg_status true_residual(stg_gauge *g, Workspace *ws, double m2, cudaStream_t s, double *rr)
{
    const Geom &geo = g->geom;
    DslashLaunch L = {};
    L.links = &g->hi;
    L.out_parity = 1;
    L.in = ws->x64;
    L.out = ws->tmp[P64];
    STG_TRY(launch_dslash(geo, P64, EPI_NONE, L, s));
    L.out_parity = 0;
    L.in = ws->tmp[P64];
    L.out = ws->r64;
    L.w = ws->b64;
    L.v = ws->x64;
    L.m2 = m2;
    L.dot = &ws->state->result;
    L.partials = ws->partials;
    L.counter = &ws->state->counter;
    STG_TRY(launch_dslash(geo, P64, EPI_RES, L, s));
    STG_TRY(read_state(ws, s));
    *rr = ws->state_host->result;
    return STG_OK;
}

stg_status cg_solve(stg_gauge *g, const double *src, double *x, double mass, double tol,
                    const stg_cg_params *p, stg_cg_stats *stats, cudaStream_t s)
{
    timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    const Geom &geo = g->geom;
    const bool plain = (p->policy == STG_CG_PLAIN) || (p->sloppy == STG_FP64);
    const int pd = plain ? P64 : p->sloppy;
    const int pr = pr_of(pd);
    Workspace *ws;
    STG_TRY(workspace_get(g, &ws));
    STG_TRY(prepare(g, ws, pd));
    const double m2 = mass * mass;
    const long maxiter = p->maxiter > 0 ? p->maxiter : 10L * 3L * geo.Vh;
    int chunk = p->check_every > 0 ? p->check_every : (geo.Vh >= (1 << 19) ? 16 : 32);
    if (chunk > 256) chunk = 256;
    long launches = 0;
    double tsum[4] = {0.0, 0.0, 0.0, 0.0};

    // b, x0 into the FP64 device layout; |b|^2
    STG_TRY(pack_field(geo, P64, src, ws->b64, s));
    STG_TRY(pack_field(geo, P64, x, ws->x64, s));
    STG_TRY(norm2(geo, P64, ws->b64, ws, s));
    STG_TRY(read_state(ws, s));
    const double bb = ws->state_host->result;
    if (!isfinite(bb)) {
        set_error("stg_cg_solve: the source has non-finite entries");
        return STG_ERR_INVALID_ARG;
    }
    stg_cg_stats st = {};
    stg_status status = STG_OK;
    double rr = 0.0;
    if (bb == 0.0) {
        STG_CUDA(cudaMemsetAsync(x, 0, (size_t)geo.Vh * 48, s));
        STG_CUDA(cudaStreamSynchronize(s));
        if (stats) *stats = st;
        return STG_OK;
    }
    const double stop = tol * tol * bb;
    STG_TRY(true_residual(g, ws, m2, s, &rr));
    if (!isfinite(rr)) {
        set_error("stg_cg_solve: non-finite residual of the initial guess");
        return STG_ERR_INVALID_ARG;
    }

    // plain FP64 CG iterates directly on x64 / r64
    void *save_y = ws->y, *save_r = ws->r;
    if (plain) {
        ws->y = ws->x64;
        ws->r = ws->r64;
    }
    const int grid = grid_for(geo.Vh);
    CGState *h = ws->state_host;
    h->delta_new = rr;
    h->iter = 0;
    if (rr > stop) {
        // start: y = 0, r = b - A x0, d = r (Fig. 1 / Fig. 2)
        STG_DISPATCH_PD(pd, k_reset, geo.Vh, ws->y, ws->r, ws->d, ws->r64, 0.0, plain ? 0 : 1);
        status = cuda_check_launch();
        h->delta_old = rr;
        h->rmax2 = rr;
        h->stop_r2 = stop;
        h->trig2 = plain ? 0.0 : p->delta * p->delta;
        h->m2 = m2;
        h->iter_limit = maxiter;
        h->flag = FLAG_RUN;
        h->track_max = (p->policy == STG_CG_RELIABLE) ? 1 : 0;
        h->counter = 0;
        if (status == STG_OK) status = write_state(ws, s);
        cudaGraphExec_t graph = nullptr;
        if (status == STG_OK) status = get_graph(g, ws, pd, chunk, p->timing ? 1 : 0, &graph);
        int breakdowns = 0;
        while (status == STG_OK) {
            cudaError_t e = cudaGraphLaunch(graph, s);
            if (e != cudaSuccess) {
                status = cuda_fail(e, "cudaGraphLaunch");
                break;
            }
            status = read_state(ws, s);
            if (status != STG_OK) break;
            launches += 4L * chunk;
            if (p->timing) {
                // the chunk's first iteration always runs: a chunk starts with the flag down
                float ms[4];
                bool ok = true;
                for (int k = 0; k < 4 && ok; ++k)
                    ok = cudaEventElapsedTime(&ms[k], ws->ev[k], ws->ev[k + 1]) == cudaSuccess;
                if (ok) {
                    tsum[0] += ms[0]; tsum[1] += ms[1]; tsum[2] += ms[2]; tsum[3] += ms[3];
                    st.timed_iters += 1;
                } else {
                    cudaGetLastError();
                }
            }
            const int flag = h->flag;
            if (flag == FLAG_RUN) continue;
            // Sec. 3.2 update: x_{k+1} = x_k + y_n (FP64), r_{k+1} = b - A x_{k+1}
            if (!plain) {
                if (pr == P64) k_accumulate_x<P64><<<grid, kBlock, 0, s>>>(geo.Vh, ws->x64, ws->y);
                else k_accumulate_x<P32><<<grid, kBlock, 0, s>>>(geo.Vh, ws->x64, ws->y);
                status = cuda_check_launch();
                if (status != STG_OK) break;
            }
            const double delta_old = h->delta_old;
            const long long iters = h->iter;
            status = true_residual(g, ws, m2, s, &rr);
            if (status != STG_OK) break;
            st.updates += 1;
            if (rr <= stop) break;
            if (!isfinite(rr)) {
                set_error("stg_cg_solve: non-finite true residual");
                status = STG_ERR_BREAKDOWN;
                break;
            }
            if (iters >= maxiter) {
                set_error("stg_cg_solve: maxiter reached before convergence");
                status = STG_ERR_NOT_CONVERGED;
                break;
            }
            double beta = 0.0;
            if (flag == FLAG_BREAKDOWN) {
                if (++breakdowns > 3) {
                    set_error("stg_cg_solve: d^dag A d <= 0 or non-finite reduction");
                    status = STG_ERR_BREAKDOWN;
                    break;
                }
            } else if (!plain && p->policy == STG_CG_RELIABLE) {
                beta = rr / delta_old;  // Eq. 6: d^y_0 = r + beta d, d kept
            }
            // group-wise update: y = 0, r^y = r_{k+1}; then d = r + beta d
            STG_DISPATCH_PD(pd, k_reset, geo.Vh, ws->y, ws->r, ws->d, ws->r64, beta, plain ? 0 : 1);
            status = cuda_check_launch();
            if (status != STG_OK) break;
            h->delta_new = rr;
            h->delta_old = rr;
            h->rmax2 = rr;
            h->flag = FLAG_RUN;
            status = write_state(ws, s);
        }
    }
    ws->y = save_y;
    ws->r = save_r;
    if (status == STG_OK || status == STG_ERR_NOT_CONVERGED) {
        stg_status u = unpack_field(geo, P64, ws->x64, x, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (u != STG_OK) status = u;
        else if (e != cudaSuccess) status = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (st.timed_iters > 0) {
        st.t_dslash_ms = tsum[0] / st.timed_iters;
        st.t_dslash_a_ms = tsum[1] / st.timed_iters;
        st.t_update_ms = tsum[2] / st.timed_iters;
        st.t_xpay_ms = tsum[3] / st.timed_iters;
    }
    // setup: 2 packs, norm, residual (2), reset; per update: accumulate,
    // residual (2), reset; final unpack
    launches += 6 + 4L * st.updates + 1;
    st.launches = launches;
    st.iters = (long)h->iter;
    st.sloppy_iters = plain ? 0 : (long)h->iter;
    st.true_res = sqrt(rr / bb);
    st.iter_res = sqrt(h->delta_new / bb);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    st.seconds = (t1.tv_sec - t0.tv_sec) + 1e-9 * (t1.tv_nsec - t0.tv_nsec);
    if (stats) *stats = st;
    return status;
}

}  // namespace stg
