// Lattice-group CG session: systems on different lattices iterate in lock-
// step, each CG iteration (Fig. 1, with the Sec. 3.2 updates of the mixed
// solver between chunks) being four launches over all of them.
//
// A batch session (mrhs.cu) holds many systems on one gauge field; here
// every slot may sit on its own gauge handle and lattice size.  Small
// lattices (8^4 has 2048 sites per parity) fill a small part of the GPU per
// launch, so solving them one launch per lattice leaves it mostly idle;
// grouped, one grid covers the sites of every slot:
//   1. t_k = D_oe d_k                                     (all slots)
//   2. q_k = m_k^2 d_k - D_eo t_k, d_k^dag q_k -> alpha_k (all slots)
//   3. y_k += alpha_k d_k, r_k -= alpha_k q_k, |r_k|^2 -> beta_k, stop tests
//   4. d_k = r_k + beta_k d_k
// Each kernel strides over "items" of kBlock sites: item w belongs to the
// slot whose tile range holds w (ranges from a device-side table, so slots
// join and leave between chunks without recapturing the graph).  A slot
// whose CG flag is raised is skipped, as in the single-system solver.  The
// reductions are per slot: each block adds its items' block sums into
// shared-memory slots, writes one partial per slot, and the last block to
// arrive sums every slot's partials in a fixed order (no floating-point
// atomics, no waiting).
//
// The paper solves one lattice at a time; this is a serving-layer form of
// the same iteration.
#include <math.h>
#include <string.h>
#include <time.h>

#include <new>
#include <string>
#include <vector>

#include "dslash_site.cuh"

namespace stg {

constexpr int kLgMax = 16;            // systems per session
constexpr int kLgBlocksPerSM = 4;     // grid of the stride loops

struct LgEntry {
    Geom g;
    const char *links;    // sloppy link blocks: (parity, mu) at links + (4 parity + mu) blk
    size_t blk;
    char *y, *r, *d, *q, *t;
    int slot;             // index into the state array
    int first_tile;       // this entry's items are [first_tile, first_tile + tiles)
    int tiles;
};

struct LgTable {
    int n;                // entries in use
    int total_tiles;
    LgEntry e[kLgMax];
};

struct LgArgs {
    const LgTable *tab;
    CGState *states;      // indexed by slot
    float2 *partials;     // [kLgMax][gridDim.x]
    unsigned *counter;
};

// entry holding item w (entries are few; uniform over the block)
__device__ __forceinline__ int lg_entry(const LgTable *tab, int n, int w)
{
    int k = 0;
    while (k + 1 < n && w >= tab->e[k + 1].first_tile) ++k;
    return k;
}

// per-slot sums: each block adds its items into acc[], writes one partial
// per entry, and the last block to arrive sums each entry's partials in
// block order; returns true in the last block (thread 0 holds nothing
// special: totals[] is in shared memory, valid for every thread)
__device__ __forceinline__ bool lg_reduce(const LgArgs &a, int n, FF *acc, double *totals)
{
    __shared__ int is_last;
    __syncthreads();
    if ((int)threadIdx.x < n)
        a.partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] =
            make_float2(acc[threadIdx.x].hi, acc[threadIdx.x].lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(a.counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // one warp per entry, fixed order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < n; k += kBlock / 32) {
        FF s = {0.f, 0.f};
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const float2 p = __ldcg(a.partials + (size_t)k * gridDim.x + b);
            s = ff_add(s, FF{p.x, p.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
        if (lane == 0) totals[k] = (double)s.hi + (double)s.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.counter = 0u;
    return true;
}

// 1. / 2.: the two half-passes of A on every running slot
template <int P, int R, int EPI>
__global__ void __launch_bounds__(kBlock, 2) k_lg_dslash(const LgArgs a)
{
    typedef typename Real<P>::T T;
    __shared__ FF acc[kLgMax];
    __shared__ float2 smf[32];
    __shared__ double totals[kLgMax];
    const LgTable *tab = a.tab;
    const int n = tab->n, total = tab->total_tiles;
    if (EPI == EPI_A_CG && (int)threadIdx.x < kLgMax) acc[threadIdx.x] = FF{0.f, 0.f};
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int k = lg_entry(tab, n, w);
        const LgEntry &e = tab->e[k];
        CGState *st = a.states + e.slot;
        if (st->flag != FLAG_RUN) continue;  // uniform over the block
        const int parity = (EPI == EPI_GATE) ? 1 : 0;
        const char *lf[4], *lb[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            lf[mu] = e.links + (size_t)(parity * 4 + mu) * e.blk;
            lb[mu] = e.links + (size_t)((1 - parity) * 4 + mu) * e.blk;
        }
        const int vh = e.g.Vh;
        const int i = (w - e.first_tile) * kBlock + (int)threadIdx.x;
        T dot = T(0);
        if (i < vh) {
            const Vec3<T> dv = dslash_site<P, R>(e.g, lf, lb, parity, EPI == EPI_GATE ? e.d : e.t, i);
            if (EPI == EPI_GATE) {
                FieldIO<P>::store(e.t, vh, i, dv);
            } else {
                const T m2 = T(st->m2);
                const Vec3<T> d = FieldIO<P>::load_nc(e.d, vh, i);
                Vec3<T> o;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o.r[c] = m2 * d.r[c] - dv.r[c];
                    o.i[c] = m2 * d.i[c] - dv.i[c];
                }
                // d^dag q with q as stored, as the update will read it
                const Vec3<T> os = FieldIO<P>::store(e.q, vh, i, o);
#pragma unroll
                for (int c = 0; c < 3; ++c) dot += d.r[c] * os.r[c] + d.i[c] * os.i[c];
            }
        }
        if (EPI == EPI_A_CG) {
            const FF s = block_sum_ff<kBlock>(FF{float(dot), 0.f}, smf);
            if (threadIdx.x == 0) acc[k] = ff_add(acc[k], s);
        }
    }
    if (EPI == EPI_A_CG && lg_reduce(a, n, acc, totals)) {
        if ((int)threadIdx.x < n) {
            CGState *st = a.states + tab->e[threadIdx.x].slot;
            if (st->flag == FLAG_RUN) set_alpha(st, totals[threadIdx.x]);
        }
    }
}

// 3.: y += alpha d, r -= alpha q, |r|^2 -> delta, beta and the stop tests
// (the same tests as the single-system update)
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_lg_update(const LgArgs a)
{
    typedef typename Real<PR>::T T;
    __shared__ FF acc[kLgMax];
    __shared__ float2 smf[32];
    __shared__ double totals[kLgMax];
    const LgTable *tab = a.tab;
    const int n = tab->n, total = tab->total_tiles;
    if ((int)threadIdx.x < kLgMax) acc[threadIdx.x] = FF{0.f, 0.f};
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int k = lg_entry(tab, n, w);
        const LgEntry &e = tab->e[k];
        const CGState *st = a.states + e.slot;
        if (st->flag != FLAG_RUN) continue;
        const int vh = e.g.Vh;
        const int i = (w - e.first_tile) * kBlock + (int)threadIdx.x;
        T nr = T(0);
        if (i < vh) {
            const T alpha = T(st->alpha);
            const auto dv = FieldIO<PD>::load(e.d, vh, i);
            const auto qv = FieldIO<PD>::load(e.q, vh, i);
            Vec3<T> yv = FieldIO<PR>::load(e.y, vh, i);
            Vec3<T> rv = FieldIO<PR>::load(e.r, vh, i);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                yv.r[c] += alpha * T(dv.r[c]);
                yv.i[c] += alpha * T(dv.i[c]);
                rv.r[c] -= alpha * T(qv.r[c]);
                rv.i[c] -= alpha * T(qv.i[c]);
            }
            FieldIO<PR>::store(e.y, vh, i, yv);
            const Vec3<T> rs = FieldIO<PR>::store(e.r, vh, i, rv);
#pragma unroll
            for (int c = 0; c < 3; ++c) nr += rs.r[c] * rs.r[c] + rs.i[c] * rs.i[c];
        }
        FF v;
        if constexpr (PR == P64) {
            // FP64 vectors: the block's sum in FP64, carried as a rounded pair
            __shared__ double smd[32];
            const double s = block_sum<kBlock>(double(nr), smd);
            v.hi = float(s);
            v.lo = float(s - double(v.hi));
        } else {
            v = block_sum_ff<kBlock>(FF{float(nr), 0.f}, smf);
        }
        if (threadIdx.x == 0) acc[k] = ff_add(acc[k], v);
    }
    if (lg_reduce(a, n, acc, totals)) {
        if ((int)threadIdx.x < n) {
            CGState *st = a.states + tab->e[threadIdx.x].slot;
            if (st->flag == FLAG_RUN) {
                const double tot = totals[threadIdx.x];
                const double old = st->delta_new;
                st->delta_old = old;
                st->delta_new = tot;
                st->beta = tot / old;
                st->iter += 1;
                if (!isfinite(tot)) st->flag = FLAG_BREAKDOWN;
                else if (tot <= st->stop_r2) st->flag = FLAG_CONVERGED;
                else if (st->trig2 > 0.0 && tot < st->trig2 * st->rmax2) st->flag = FLAG_UPDATE;
                else if (st->iter >= st->iter_limit) st->flag = FLAG_MAXITER;
                if (st->track_max && tot > st->rmax2) st->rmax2 = tot;
            }
        }
    }
}

// 4.: d = r + beta d
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_lg_xpay(const LgArgs a)
{
    typedef typename Real<PR>::T T;
    const LgTable *tab = a.tab;
    const int n = tab->n, total = tab->total_tiles;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int k = lg_entry(tab, n, w);
        const LgEntry &e = tab->e[k];
        const CGState *st = a.states + e.slot;
        if (st->flag != FLAG_RUN) continue;
        const int vh = e.g.Vh;
        const int i = (w - e.first_tile) * kBlock + (int)threadIdx.x;
        if (i >= vh) continue;
        const T beta = T(st->beta);
        const Vec3<T> rv = FieldIO<PR>::load(e.r, vh, i);
        const auto dv = FieldIO<PD>::load(e.d, vh, i);
        Vec3<typename Real<PD>::T> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = rv.r[c] + beta * T(dv.r[c]);
            o.i[c] = rv.i[c] + beta * T(dv.i[c]);
        }
        FieldIO<PD>::store(e.d, vh, i, o);
    }
}

static int lg_pr(int pd) { return (pd == P16 || pd == PX16 || pd == PB16) ? P32 : pd; }

template <int P, int R>
static cudaError_t lg_iteration_pr(const LgArgs &a, int grid, cudaStream_t s)
{
    constexpr int PR = (P == P16 || P == PX16 || P == PB16) ? P32 : P;
    k_lg_dslash<P, R, EPI_GATE><<<grid, kBlock, 0, s>>>(a);
    k_lg_dslash<P, R, EPI_A_CG><<<grid, kBlock, 0, s>>>(a);
    k_lg_update<P, PR><<<grid, kBlock, 0, s>>>(a);
    k_lg_xpay<P, PR><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int P>
static cudaError_t lg_iteration_p(int recon, const LgArgs &a, int grid, cudaStream_t s)
{
    return recon == 18 ? lg_iteration_pr<P, 18>(a, grid, s) : lg_iteration_pr<P, 12>(a, grid, s);
}

static cudaError_t lg_iteration(int pd, int recon, const LgArgs &a, int grid, cudaStream_t s)
{
    switch (pd) {
    case P64: return lg_iteration_p<P64>(recon, a, grid, s);
    case P32: return lg_iteration_p<P32>(recon, a, grid, s);
    case P16: return lg_iteration_p<P16>(recon, a, grid, s);
    case PB16: return lg_iteration_p<PB16>(recon, a, grid, s);
    default: return lg_iteration_p<PX16>(recon, a, grid, s);
    }
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// device bytes of a session: per slot x, b, r (FP64), y, r^ (PR), d, q, t
// (PD) for max_vh sites; one FP64 odd intermediate; partials, states,
// table, counter
static size_t lg_slot_bytes(long max_vh, int pd)
{
    const size_t vh = (size_t)max_vh;
    return 3 * align256(vh * 48) + 2 * align256(vh * field_site_bytes(lg_pr(pd))) +
           3 * align256(vh * field_site_bytes(pd));
}

static size_t lg_partial_bytes(long max_vh, int grid)
{
    const size_t a = (size_t)kLgMax * grid * sizeof(float2);
    const size_t b = ((size_t)(max_vh + kBlock - 1) / kBlock + 64) * sizeof(double);
    return align256(a > b ? a : b);
}

static int lg_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 148;
    return sms * kLgBlocksPerSM;
}

size_t lgroup_bytes(int n, long max_vh, int pd)
{
    return (size_t)n * lg_slot_bytes(max_vh, pd) + align256((size_t)max_vh * 48) +
           lg_partial_bytes(max_vh, lg_grid()) + align256(kLgMax * sizeof(CGState)) +
           align256(sizeof(LgTable)) + 256;
}

}  // namespace stg

using namespace stg;

struct stg_lgroup {
    int n = 0, pd = 0, pr = 0, recon = 12, device = 0, grid = 0;
    long max_vh = 0;
    stg_cg_params p;
    cudaStream_t s = nullptr;
    int chunk = 16;
    char *slots = nullptr;        // n x lg_slot_bytes
    size_t slot_bytes = 0;
    void *tmp64 = nullptr;        // FP64 odd intermediate of the updates
    float2 *partials = nullptr;
    CGState *states = nullptr, *states_host = nullptr;
    LgTable *tab = nullptr, *tab_host = nullptr;
    unsigned *counter = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    long launches = 0;
    struct Slot {
        int used = 0;
        stg_gauge *g = nullptr;
        double bb = 0, rr = 0, tol = 0;
        long updates = 0, maxiter = 0;
        double *x = nullptr;
        timespec t_add;
    };
    std::vector<Slot> slot;
    struct Done {
        int slot;
        int status;
        stg_cg_stats stats;
    };
    std::vector<Done> pending;
    // per-slot vector pointers
    char *vec(int k, int which) const
    {
        const size_t vh = (size_t)max_vh;
        const size_t f64 = align256(vh * 48), fr = align256(vh * field_site_bytes(pr)),
                     fd = align256(vh * field_site_bytes(pd));
        char *b = slots + (size_t)k * slot_bytes;
        const size_t off[8] = {0, f64, 2 * f64, 3 * f64, 3 * f64 + fr, 3 * f64 + 2 * fr,
                               3 * f64 + 2 * fr + fd, 3 * f64 + 2 * fr + 2 * fd};
        return b + off[which];
    }
    enum { X64 = 0, B64 = 1, R64 = 2, Y = 3, R = 4, D = 5, Q = 6, T = 7 };
};

namespace stg {

static double lg_elapsed(const timespec &t0)
{
    timespec t1;
    clock_gettime(CLOCK_MONOTONIC, &t1);
    return (t1.tv_sec - t0.tv_sec) + 1e-9 * (t1.tv_nsec - t0.tv_nsec);
}

static void lg_free(stg_lgroup *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    void *v[] = {b->slots, b->tmp64, b->partials, b->states, b->tab, b->counter};
    for (void *p : v) cudaFree(p);
    if (b->states_host) cudaFreeHost(b->states_host);
    if (b->tab_host) cudaFreeHost(b->tab_host);
    delete b;
}

static stg_status lg_alloc(void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("lattice-group session: device allocation failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    return STG_OK;
}

// the table of running slots, consecutive tile ranges
static stg_status lg_push(stg_lgroup *b)
{
    LgTable &t = *b->tab_host;
    t.n = 0;
    t.total_tiles = 0;
    for (int k = 0; k < b->n; ++k) {
        const stg_lgroup::Slot &sl = b->slot[k];
        if (!sl.used) continue;
        LgEntry &e = t.e[t.n++];
        const LinkField *lf = links_for(sl.g, b->pd);
        e.g = sl.g->geom;
        e.links = lf->base;
        e.blk = lf->blk_bytes;
        e.y = b->vec(k, stg_lgroup::Y);
        e.r = b->vec(k, stg_lgroup::R);
        e.d = b->vec(k, stg_lgroup::D);
        e.q = b->vec(k, stg_lgroup::Q);
        e.t = b->vec(k, stg_lgroup::T);
        e.slot = k;
        e.first_tile = t.total_tiles;
        e.tiles = (e.g.Vh + kBlock - 1) / kBlock;
        t.total_tiles += e.tiles;
    }
    for (int k = 0; k < b->n; ++k) b->states_host[k].counter = 0;
    STG_CUDA(cudaMemcpyAsync(b->states, b->states_host, b->n * sizeof(CGState), cudaMemcpyHostToDevice,
                             b->s));
    STG_CUDA(cudaMemcpyAsync(b->tab, b->tab_host, sizeof(LgTable), cudaMemcpyHostToDevice, b->s));
    return STG_OK;
}

static stg_status lg_pull(stg_lgroup *b)
{
    STG_CUDA(cudaMemcpyAsync(b->states_host, b->states, b->n * sizeof(CGState), cudaMemcpyDeviceToHost,
                             b->s));
    STG_CUDA(cudaStreamSynchronize(b->s));
    return STG_OK;
}

static stg_status lg_graph(stg_lgroup *b, cudaGraphExec_t *out)
{
    if (b->graph && b->graph_iters == b->chunk) {
        *out = b->graph;
        return STG_OK;
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    LgArgs a;
    a.tab = b->tab;
    a.states = b->states;
    a.partials = b->partials;
    a.counter = b->counter;
    cudaStream_t cs;
    STG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    stg_status st = STG_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < b->chunk && e == cudaSuccess; ++k) e = lg_iteration(b->pd, b->recon, a, b->grid, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess) st = cuda_fail(e, "lattice-group iteration launch");
        else if (e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (st == STG_OK) {
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != STG_OK) return st;
    b->graph_iters = b->chunk;
    *out = b->graph;
    return STG_OK;
}

static void lg_finish(stg_lgroup *b, int k, int status)
{
    stg_lgroup::Slot &sl = b->slot[k];
    const CGState &h = b->states_host[k];
    stg_lgroup::Done d;
    d.slot = k;
    d.status = status;
    memset(&d.stats, 0, sizeof(d.stats));
    d.stats.iters = (long)h.iter;
    d.stats.sloppy_iters = (long)h.iter;
    d.stats.updates = sl.updates;
    d.stats.true_res = sl.bb > 0.0 ? sqrt(sl.rr / sl.bb) : 0.0;
    d.stats.iter_res = sl.bb > 0.0 ? sqrt(h.delta_new / sl.bb) : 0.0;
    d.stats.seconds = lg_elapsed(sl.t_add);
    d.stats.launches = b->launches;
    b->pending.push_back(d);
    sl.used = 0;
    sl.g = nullptr;
}

// r64 = b - A x with the slot's FP64 operator; |r64|^2 -> states[k].result
static stg_status lg_residual(stg_lgroup *b, int k, double m2)
{
    stg_lgroup::Slot &sl = b->slot[k];
    return launch_true_residual(sl.g, b->vec(k, stg_lgroup::X64), b->vec(k, stg_lgroup::B64),
                                b->vec(k, stg_lgroup::R64), b->tmp64, m2, b->states + k,
                                reinterpret_cast<double *>(b->partials), b->s);
}

static stg_status lg_add(stg_lgroup *b, stg_gauge *g, const double *src, double *x, double mass,
                         double tol, int *slot_out)
{
    int k = -1;
    for (int j = 0; j < b->n; ++j)
        if (!b->slot[j].used) {
            k = j;
            break;
        }
    if (k < 0) {
        set_error("stg_lgroup_add: every slot of the session is occupied");
        return STG_ERR_INVALID_ARG;
    }
    const Geom &geo = g->geom;
    stg_lgroup::Slot &sl = b->slot[k];
    clock_gettime(CLOCK_MONOTONIC, &sl.t_add);
    sl.g = g;
    sl.x = x;
    sl.tol = tol;
    sl.updates = 0;
    sl.maxiter = b->p.maxiter > 0 ? b->p.maxiter : 10L * 3L * geo.Vh;
    cudaStream_t s = b->s;
    STG_TRY(pack_field(geo, P64, src, b->vec(k, stg_lgroup::B64), s));
    STG_TRY(pack_field(geo, P64, x, b->vec(k, stg_lgroup::X64), s));
    STG_TRY(launch_norm2(P64, geo.Vh, b->vec(k, stg_lgroup::B64), b->states + k,
                         reinterpret_cast<double *>(b->partials), s));
    STG_TRY(lg_pull(b));
    const double bb = b->states_host[k].result;
    STG_TRY(lg_residual(b, k, mass * mass));
    STG_TRY(lg_pull(b));
    const double rr = b->states_host[k].result;
    b->launches += 5;
    if (!isfinite(bb) || !isfinite(rr)) {
        sl.g = nullptr;
        set_error("stg_lgroup_add: non-finite source or initial residual");
        return STG_ERR_INVALID_ARG;
    }
    sl.bb = bb;
    sl.rr = rr;
    sl.used = 1;
    CGState &h = b->states_host[k];
    memset(&h, 0, sizeof(CGState));
    h.m2 = mass * mass;
    h.stop_r2 = tol * tol * bb;
    h.trig2 = b->p.delta * b->p.delta;
    h.track_max = (b->p.policy == STG_CG_RELIABLE) ? 1 : 0;
    h.iter_limit = sl.maxiter;
    h.delta_new = h.delta_old = h.rmax2 = rr;
    if (bb == 0.0 || rr <= h.stop_r2) {
        if (bb == 0.0) STG_CUDA(cudaMemsetAsync(x, 0, (size_t)geo.Vh * 48, s));
        h.flag = FLAG_CONVERGED;
        lg_finish(b, k, STG_OK);
    } else {
        STG_TRY(launch_reset(b->pd, geo.Vh, b->vec(k, stg_lgroup::Y), b->vec(k, stg_lgroup::R),
                             b->vec(k, stg_lgroup::D), b->vec(k, stg_lgroup::R64), 0.0, 1, s));
        ++b->launches;
        h.flag = FLAG_RUN;
    }
    STG_TRY(lg_push(b));
    *slot_out = k;
    return STG_OK;
}

// one chunk for every running slot, then the FP64 updates of the slots that
// asked for one (Sec. 3.2), exactly as the batch session does
static stg_status lg_step(stg_lgroup *b)
{
    if (b->tab_host->n == 0) return STG_OK;
    cudaStream_t s = b->s;
    cudaGraphExec_t graph;
    STG_TRY(lg_graph(b, &graph));
    STG_CUDA(cudaGraphLaunch(graph, s));
    b->launches += 4L * b->chunk;
    STG_TRY(lg_pull(b));
    CGState *h = b->states_host;
    std::vector<int> flagged;
    for (int k = 0; k < b->n; ++k)
        if (b->slot[k].used && h[k].flag != FLAG_RUN) flagged.push_back(k);
    if (flagged.empty()) return STG_OK;
    std::vector<CGState> before(flagged.size());
    for (size_t u = 0; u < flagged.size(); ++u) {
        const int k = flagged[u];
        before[u] = h[k];
        const int vh = b->slot[k].g->geom.Vh;
        STG_TRY(launch_accumulate_x(b->pr, vh, b->vec(k, stg_lgroup::X64), b->vec(k, stg_lgroup::Y), s));
        STG_TRY(lg_residual(b, k, h[k].m2));
        b->launches += 3;
        ++b->slot[k].updates;
    }
    STG_TRY(lg_pull(b));
    for (size_t u = 0; u < flagged.size(); ++u) {
        const int k = flagged[u];
        const CGState b4 = before[u];
        const double rr = h[k].result;
        h[k] = b4;
        stg_lgroup::Slot &sl = b->slot[k];
        sl.rr = rr;
        int done = -1;
        if (rr <= h[k].stop_r2) done = STG_OK;
        else if (!isfinite(rr)) done = STG_ERR_BREAKDOWN;
        else if (h[k].iter >= sl.maxiter) done = STG_ERR_NOT_CONVERGED;
        if (done >= 0) {
            STG_TRY(unpack_field(sl.g->geom, P64, b->vec(k, stg_lgroup::X64), sl.x, s));
            ++b->launches;
            h[k].flag = FLAG_CONVERGED;
            lg_finish(b, k, done);
            continue;
        }
        double beta = 0.0;
        if (b4.flag != FLAG_BREAKDOWN && b->p.policy == STG_CG_RELIABLE) beta = rr / b4.delta_old;
        STG_TRY(launch_reset(b->pd, sl.g->geom.Vh, b->vec(k, stg_lgroup::Y), b->vec(k, stg_lgroup::R),
                             b->vec(k, stg_lgroup::D), b->vec(k, stg_lgroup::R64), beta, 1, s));
        ++b->launches;
        h[k].delta_new = rr;
        h[k].delta_old = rr;
        h[k].rmax2 = rr;
        h[k].flag = FLAG_RUN;
    }
    STG_TRY(lg_push(b));
    STG_CUDA(cudaStreamSynchronize(s));  // unpacked solutions are complete
    return STG_OK;
}

struct LgDevScope {
    int prev = -1, want;
    explicit LgDevScope(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~LgDevScope()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

}  // namespace stg

extern "C" {

stg_status stg_lgroup_create(int max_systems, long max_vh, stg_prec sloppy, int recon,
                             const stg_cg_params *params, stg_stream_t stream, stg_lgroup **out)
{
    if (!out || max_systems < 1 || max_systems > kLgMax || max_vh < 1 || max_vh > (1L << 30) ||
        (recon != 12 && recon != 18)) {
        set_error("stg_lgroup_create: NULL out, max_systems outside [1, 16], max_vh outside "
                  "[1, 2^30] or recon not 12 / 18");
        return STG_ERR_INVALID_ARG;
    }
    if (sloppy != STG_FP64 && sloppy != STG_FP32 && sloppy != STG_FP16 && sloppy != STG_FX16 &&
        sloppy != STG_BF16) {
        set_error("stg_lgroup_create: unknown precision");
        return STG_ERR_INVALID_ARG;
    }
    stg_cg_params p;
    if (params) {
        p = *params;
    } else {
        cg_params_for(sloppy, &p);  // the defaults of stg_cg_params_default
    }
    if (p.policy < STG_CG_RELIABLE || p.policy > STG_CG_REFINE || !(p.delta > 0.0 && p.delta < 1.0) ||
        p.maxiter < 0 || p.check_every < 0) {
        set_error("stg_lgroup_create: bad params (policy RELIABLE or REFINE, 0 < delta < 1)");
        return STG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    stg_lgroup *b = new (std::nothrow) stg_lgroup();
    if (!b) {
        set_error("stg_lgroup_create: host allocation failed");
        return STG_ERR_OOM;
    }
    b->n = max_systems;
    b->max_vh = max_vh;
    b->pd = sloppy;
    b->pr = lg_pr(sloppy);
    b->recon = recon;
    b->p = p;
    b->p.sloppy = sloppy;
    b->s = (cudaStream_t)stream;
    b->chunk = p.check_every > 0 ? (p.check_every > 256 ? 256 : p.check_every) : 16;
    b->slot.resize(max_systems);
    cudaGetDevice(&b->device);
    b->grid = lg_grid();
    b->slot_bytes = lg_slot_bytes(max_vh, sloppy);
    stg_status st = lg_alloc((void **)&b->slots, (size_t)max_systems * b->slot_bytes);
    if (st == STG_OK) st = lg_alloc(&b->tmp64, align256((size_t)max_vh * 48));
    if (st == STG_OK) st = lg_alloc((void **)&b->partials, lg_partial_bytes(max_vh, b->grid));
    if (st == STG_OK) st = lg_alloc((void **)&b->states, align256(kLgMax * sizeof(CGState)));
    if (st == STG_OK) st = lg_alloc((void **)&b->tab, align256(sizeof(LgTable)));
    if (st == STG_OK) st = lg_alloc((void **)&b->counter, 256);
    if (st == STG_OK) {
        cudaError_t e = cudaMemset(b->counter, 0, 256);
        if (e == cudaSuccess) e = cudaMemset(b->states, 0, kLgMax * sizeof(CGState));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&b->states_host, kLgMax * sizeof(CGState));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&b->tab_host, sizeof(LgTable));
        if (e != cudaSuccess) st = cuda_fail(e, "stg_lgroup_create");
    }
    if (st != STG_OK) {
        lg_free(b);
        return st;
    }
    memset(b->states_host, 0, kLgMax * sizeof(CGState));
    memset(b->tab_host, 0, sizeof(LgTable));
    st = lg_push(b);
    if (st != STG_OK) {
        lg_free(b);
        return st;
    }
    *out = b;
    return STG_OK;
}

stg_status stg_lgroup_destroy(stg_lgroup *b)
{
    if (!b) return STG_OK;
    LgDevScope ds(b->device);
    cudaStreamSynchronize(b->s);
    lg_free(b);
    return STG_OK;
}

stg_status stg_lgroup_add(stg_lgroup *b, const stg_gauge *gc, const double *src_dev, double *x_dev,
                          double mass, double tol, int *slot)
{
    if (!b || !gc || !src_dev || !x_dev || !slot || src_dev == x_dev) {
        set_error("stg_lgroup_add: NULL argument or src == x");
        return STG_ERR_INVALID_ARG;
    }
    if (!isfinite(mass) || mass < 0.0 || !isfinite(tol) || !(tol > 0.0)) {
        set_error("stg_lgroup_add: mass must be finite and >= 0, tol finite and > 0");
        return STG_ERR_INVALID_ARG;
    }
    if (gc->device != b->device) {
        set_error("stg_lgroup_add: the gauge handle is on another device than the session");
        return STG_ERR_INVALID_ARG;
    }
    if (gc->geom.Vh > b->max_vh) {
        set_error("stg_lgroup_add: the lattice has more sites per parity than the session's max_vh");
        return STG_ERR_INVALID_ARG;
    }
    const LinkField *lf = links_for(gc, b->pd);
    if (!lf || lf->recon != b->recon) {
        set_error("stg_lgroup_add: the handle holds no links in the session's precision and "
                  "reconstruction");
        return STG_ERR_UNSUPPORTED;
    }
    LgDevScope ds(b->device);
    return lg_add(b, const_cast<stg_gauge *>(gc), src_dev, x_dev, mass, tol, slot);
}

stg_status stg_lgroup_step(stg_lgroup *b, int max_done, int *done_slots, int *done_status,
                           stg_cg_stats *done_stats, int *n_done, int *n_active)
{
    if (!b || max_done < 0 || (max_done > 0 && (!done_slots || !done_status)) || !n_done) {
        set_error("stg_lgroup_step: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    LgDevScope ds(b->device);
    *n_done = 0;
    stg_status st = STG_OK;
    if (b->pending.empty()) st = lg_step(b);
    int k = 0;
    while (k < max_done && !b->pending.empty()) {
        const stg_lgroup::Done d = b->pending.front();
        b->pending.erase(b->pending.begin());
        done_slots[k] = d.slot;
        done_status[k] = d.status;
        if (done_stats) done_stats[k] = d.stats;
        ++k;
    }
    *n_done = k;
    if (n_active) *n_active = b->tab_host->n + (int)b->pending.size();
    return st;
}

size_t stg_lgroup_bytes(int max_systems, long max_vh, stg_prec sloppy)
{
    if (max_systems < 1 || max_systems > kLgMax || max_vh < 1) return 0;
    return lgroup_bytes(max_systems, max_vh, sloppy);
}

}  // extern "C"
