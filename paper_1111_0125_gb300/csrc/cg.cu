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

// one site per thread (setup and update-time kernels)
int grid_for(long n)
{
    long g = (n + kBlock - 1) / kBlock;
    return (int)(g < 1 ? 1 : g);
}

static int num_sms()
{
    static const int n = [] {
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || m <= 0) m = 148;
        return m;
    }();
    return n;
}

// Per-iteration vector kernels: a grid of kVecBlocksPerSM blocks per SM
// strides over the sites kVecUnroll at a time, issuing every load of the
// kVecUnroll sites before the first use, so each thread keeps ~300 bytes in
// flight and each block pays for its reduction barriers once.
constexpr int kVecBlocksPerSM = 2;

// sites per thread per pass: 4 for FP32 / 16-bit vectors, 2 for FP64 (whose
// doubled registers would spill at 4)
__host__ __device__ constexpr int vec_unroll(int pr) { return pr == P64 ? 2 : 4; }

static int grid_vec(long n, int pr)
{
    const long u = vec_unroll(pr);
    long g = (n + (long)kBlock * u - 1) / ((long)kBlock * u);
    long cap = (long)num_sms() * kVecBlocksPerSM;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// vector kernels (grid-stride, FP64 reductions)
// ---------------------------------------------------------------------------
template <int PD, int PR>
__device__ __forceinline__ void cg_update_body(int vh, void *y, void *r, const void *d, const void *q,
                                               CGState *st, double *partials)
{
    if (st->flag != FLAG_RUN) return;
    typedef typename Real<PR>::T T;
    typedef typename Real<PD>::T TD;
    constexpr int kVecUnroll = vec_unroll(PR);
    const T alpha = T(st->alpha);
    double rr64 = 0.0;
    FF rr = {0.f, 0.f};
    const int stride = gridDim.x * kBlock;
    for (int base = blockIdx.x * kBlock + threadIdx.x; base < vh; base += kVecUnroll * stride) {
        Vec3<TD> dv[kVecUnroll], qv[kVecUnroll];
        Vec3<T> yv[kVecUnroll], rv[kVecUnroll];
#pragma unroll
        for (int k = 0; k < kVecUnroll; ++k) {
            const int i = base + k * stride;
            if (i < vh) {
                dv[k] = FieldIO<PD>::load(d, vh, i);
                qv[k] = FieldIO<PD>::load(q, vh, i);
                yv[k] = FieldIO<PR>::load(y, vh, i);
                rv[k] = FieldIO<PR>::load(r, vh, i);
            }
        }
#pragma unroll
        for (int k = 0; k < kVecUnroll; ++k) {
            const int i = base + k * stride;
            if (i < vh) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    yv[k].r[c] += alpha * T(dv[k].r[c]);
                    yv[k].i[c] += alpha * T(dv[k].i[c]);
                    rv[k].r[c] -= alpha * T(qv[k].r[c]);
                    rv[k].i[c] -= alpha * T(qv[k].i[c]);
                }
                FieldIO<PR>::store(y, vh, i, yv[k]);
                const Vec3<T> rs = FieldIO<PR>::store(r, vh, i, rv[k]);
                T n = T(0);
#pragma unroll
                for (int c = 0; c < 3; ++c) n += rs.r[c] * rs.r[c] + rs.i[c] * rs.i[c];
                if constexpr (PR == P64) {
                    rr64 += n;
                } else {
                    FF t;
                    t.hi = float(n);
                    t.lo = 0.f;
                    rr = ff_add(rr, t);
                }
            }
        }
    }
    double total;
    bool last;
    if constexpr (PR == P64) last = grid_sum<kBlock>(rr64, partials, &st->counter, total);
    else last = grid_sum_ff<kBlock>(rr, reinterpret_cast<float2 *>(partials), &st->counter, total);
    if (last) {
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
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM)
k_cg_update(int vh, void *y, void *r, const void *d, const void *q, CGState *st, double *partials)
{
    pdl_wait();
    pdl_trigger();
    cg_update_body<PD, PR>(vh, y, r, d, q, st, partials);
}

// several systems: blockIdx.y is the slot in the active list
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM)
k_cg_update_m(int vh, char *y, char *r, const char *d, const char *q, size_t sr, size_t sd,
              CGState *states, double *partials, size_t pstride, const int *active,
              const int *nactive)
{
    if ((int)blockIdx.y >= *nactive) return;
    const int k = active[blockIdx.y];
    cg_update_body<PD, PR>(vh, y + k * sr, r + k * sr, d + k * sd, q + k * sd, states + k,
                           partials + k * pstride);
}

template <int PD, int PR>
__device__ __forceinline__ void xpay_body(int vh, const void *r, void *d, const CGState *st)
{
    if (st->flag != FLAG_RUN) return;
    typedef typename Real<PR>::T T;
    typedef typename Real<PD>::T TD;
    constexpr int kVecUnroll = vec_unroll(PR);
    const T beta = T(st->beta);
    const int stride = gridDim.x * kBlock;
    for (int base = blockIdx.x * kBlock + threadIdx.x; base < vh; base += kVecUnroll * stride) {
        Vec3<T> rv[kVecUnroll];
        Vec3<TD> dv[kVecUnroll];
#pragma unroll
        for (int k = 0; k < kVecUnroll; ++k) {
            const int i = base + k * stride;
            if (i < vh) {
                rv[k] = FieldIO<PR>::load(r, vh, i);
                dv[k] = FieldIO<PD>::load(d, vh, i);
            }
        }
#pragma unroll
        for (int k = 0; k < kVecUnroll; ++k) {
            const int i = base + k * stride;
            if (i < vh) {
                Vec3<TD> o;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o.r[c] = rv[k].r[c] + beta * T(dv[k].r[c]);
                    o.i[c] = rv[k].i[c] + beta * T(dv[k].i[c]);
                }
                FieldIO<PD>::store(d, vh, i, o);
            }
        }
    }
}

template <int PD, int PR>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM)
k_xpay(int vh, const void *r, void *d, const CGState *st)
{
    pdl_wait();
    pdl_trigger();
    xpay_body<PD, PR>(vh, r, d, st);
}

template <int PD, int PR>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM)
k_xpay_m(int vh, const char *r, char *d, size_t sr, size_t sd, const CGState *states,
         const int *active, const int *nactive)
{
    if ((int)blockIdx.y >= *nactive) return;
    const int k = active[blockIdx.y];
    xpay_body<PD, PR>(vh, r + k * sr, d + k * sd, states + k);
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
    double s64 = 0.0;
    FF s = {0.f, 0.f};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < vh; i += gridDim.x * kBlock) {
        const auto a = FieldIO<P>::load(v, vh, i);
        if constexpr (P == P64) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s64 += a.r[c] * a.r[c] + a.i[c] * a.i[c];
        } else {
            float n = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) n += a.r[c] * a.r[c] + a.i[c] * a.i[c];
            FF t;
            t.hi = n;
            t.lo = 0.f;
            s = ff_add(s, t);
        }
    }
    double total;
    bool last;
    if constexpr (P == P64) last = grid_sum<kBlock>(s64, partials, &st->counter, total);
    else last = grid_sum_ff<kBlock>(s, reinterpret_cast<float2 *>(partials), &st->counter, total);
    if (last) st->result = total;
}

// ---------------------------------------------------------------------------
// dispatch over the (PD, PR) pairs used by the solver
// ---------------------------------------------------------------------------
static int pr_of(int pd) { return (pd == P16 || pd == PX16 || pd == PB16) ? P32 : pd; }

#define STG_DISPATCH_PD(pd, KERNEL, ...)                                                     \
    do {                                                                                     \
        if ((pd) == P64) KERNEL<P64, P64><<<grid, kBlock, 0, s>>>(__VA_ARGS__);              \
        else if ((pd) == P32) KERNEL<P32, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);         \
        else if ((pd) == P16) KERNEL<P16, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);         \
        else if ((pd) == PB16) KERNEL<PB16, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);       \
        else KERNEL<PX16, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                         \
    } while (0)

#define STG_DISPATCH_PD_EX(pd, KERNEL, PDL, ...)                                             \
    do {                                                                                     \
        cudaError_t e_;                                                                      \
        if ((pd) == P64) e_ = launch_k(KERNEL<P64, P64>, grid, kBlock, 0, s, PDL, __VA_ARGS__);  \
        else if ((pd) == P32) e_ = launch_k(KERNEL<P32, P32>, grid, kBlock, 0, s, PDL, __VA_ARGS__); \
        else if ((pd) == P16) e_ = launch_k(KERNEL<P16, P32>, grid, kBlock, 0, s, PDL, __VA_ARGS__); \
        else if ((pd) == PB16) e_ = launch_k(KERNEL<PB16, P32>, grid, kBlock, 0, s, PDL, __VA_ARGS__); \
        else e_ = launch_k(KERNEL<PX16, P32>, grid, kBlock, 0, s, PDL, __VA_ARGS__);              \
        STG_CUDA(e_);                                                                        \
    } while (0)

static stg_status norm2(const Geom &g, int prec, const void *v, Workspace *ws, cudaStream_t s)
{
    const int grid = grid_for(g.Vh);
    if (prec == P64) k_norm2<P64><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    else if (prec == P32) k_norm2<P32><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    else if (prec == P16) k_norm2<P16><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    else if (prec == PB16) k_norm2<PB16><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    else k_norm2<PX16><<<grid, kBlock, 0, s>>>(g.Vh, v, ws->state, ws->partials);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// one CG iteration on the sloppy vectors (4 launches); with `ev`, CUDA
// events are recorded before and after each kernel (5 events; external
// records, so that stream capture turns them into event-record nodes); with
// `pdl` (never together with events), consecutive kernels overlap by
// programmatic dependent launch (each waits for its predecessor before
// reading)
static stg_status iteration(stg_gauge *gg, Workspace *ws, int pd, cudaStream_t s, cudaEvent_t *ev,
                            bool pdl)
{
    const Geom &g = gg->geom;
    const LinkField *lf = links_for(gg, pd);
    void *t = ws->tmp[pd];
    DslashLaunch L = {};
    L.links = lf;
    L.state = ws->state;
    L.partials = ws->partials;
    L.counter = &ws->state->counter;
    L.pdl = pdl;
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
    const int grid = grid_vec(g.Vh, pr_of(pd));
    STG_DISPATCH_PD_EX(pd, k_cg_update, pdl, g.Vh, ws->y, ws->r, ws->d, ws->q, ws->state, ws->partials);
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal));
    STG_DISPATCH_PD_EX(pd, k_xpay, pdl, g.Vh, ws->r, ws->d, ws->state);
    if (ev) STG_CUDA(cudaEventRecordWithFlags(ev[4], s, cudaEventRecordExternal));
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

static stg_status cuda_check_launch()
{
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// ---------------------------------------------------------------------------
// launch helpers with explicit operands (used by the multi-system solver)
// ---------------------------------------------------------------------------
int vec_grid(long n, int pd) { return grid_vec(n, pr_of(pd)); }

stg_status launch_update_m(int pd, int vh, char *y, char *r, const char *d, const char *q, size_t sr,
                           size_t sd, CGState *states, double *partials, size_t pstride,
                           const int *active, const int *nactive, int nslots, cudaStream_t s)
{
    const dim3 grid(grid_vec(vh, pr_of(pd)), nslots);
    if (pd == P64)
        k_cg_update_m<P64, P64><<<grid, kBlock, 0, s>>>(vh, y, r, d, q, sr, sd, states, partials, pstride, active, nactive);
    else if (pd == P32)
        k_cg_update_m<P32, P32><<<grid, kBlock, 0, s>>>(vh, y, r, d, q, sr, sd, states, partials, pstride, active, nactive);
    else if (pd == P16)
        k_cg_update_m<P16, P32><<<grid, kBlock, 0, s>>>(vh, y, r, d, q, sr, sd, states, partials, pstride, active, nactive);
    else if (pd == PB16)
        k_cg_update_m<PB16, P32><<<grid, kBlock, 0, s>>>(vh, y, r, d, q, sr, sd, states, partials, pstride, active, nactive);
    else
        k_cg_update_m<PX16, P32><<<grid, kBlock, 0, s>>>(vh, y, r, d, q, sr, sd, states, partials, pstride, active, nactive);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

stg_status launch_xpay_m(int pd, int vh, const char *r, char *d, size_t sr, size_t sd,
                         const CGState *states, const int *active, const int *nactive, int nslots,
                         cudaStream_t s)
{
    const dim3 grid(grid_vec(vh, pr_of(pd)), nslots);
    if (pd == P64) k_xpay_m<P64, P64><<<grid, kBlock, 0, s>>>(vh, r, d, sr, sd, states, active, nactive);
    else if (pd == P32) k_xpay_m<P32, P32><<<grid, kBlock, 0, s>>>(vh, r, d, sr, sd, states, active, nactive);
    else if (pd == P16) k_xpay_m<P16, P32><<<grid, kBlock, 0, s>>>(vh, r, d, sr, sd, states, active, nactive);
    else if (pd == PB16) k_xpay_m<PB16, P32><<<grid, kBlock, 0, s>>>(vh, r, d, sr, sd, states, active, nactive);
    else k_xpay_m<PX16, P32><<<grid, kBlock, 0, s>>>(vh, r, d, sr, sd, states, active, nactive);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

stg_status launch_reset(int pd, int vh, void *y, void *r, void *d, const void *r64, double beta,
                        int copy_r, cudaStream_t s)
{
    const int grid = grid_for(vh);
    STG_DISPATCH_PD(pd, k_reset, vh, y, r, d, r64, beta, copy_r);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

stg_status launch_accumulate_x(int pr, int vh, void *x64, const void *y, cudaStream_t s)
{
    const int grid = grid_for(vh);
    if (pr == P64) k_accumulate_x<P64><<<grid, kBlock, 0, s>>>(vh, x64, y);
    else k_accumulate_x<P32><<<grid, kBlock, 0, s>>>(vh, x64, y);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

stg_status launch_norm2(int prec, int vh, const void *v, CGState *st, double *partials, cudaStream_t s)
{
    const int grid = grid_for(vh);
    if (prec == P64) k_norm2<P64><<<grid, kBlock, 0, s>>>(vh, v, st, partials);
    else if (prec == P32) k_norm2<P32><<<grid, kBlock, 0, s>>>(vh, v, st, partials);
    else if (prec == P16) k_norm2<P16><<<grid, kBlock, 0, s>>>(vh, v, st, partials);
    else if (prec == PB16) k_norm2<PB16><<<grid, kBlock, 0, s>>>(vh, v, st, partials);
    else k_norm2<PX16><<<grid, kBlock, 0, s>>>(vh, v, st, partials);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// r64 = b64 - A x64 with the FP64 operator, |r64|^2 -> st->result (no sync)
stg_status launch_true_residual(stg_gauge *g, const void *x64, const void *b64, void *r64, void *t64,
                                double m2, CGState *st, double *partials, cudaStream_t s)
{
    DslashLaunch L = {};
    L.links = &g->hi;
    L.out_parity = 1;
    L.in = x64;
    L.out = t64;
    STG_TRY(launch_dslash(g->geom, P64, EPI_NONE, L, s));
    L.out_parity = 0;
    L.in = t64;
    L.out = r64;
    L.w = b64;
    L.v = x64;
    L.m2 = m2;
    L.dot = &st->result;
    L.partials = partials;
    L.counter = &st->counter;
    return launch_dslash(g->geom, P64, EPI_RES, L, s);
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
        for (int k = 0; k < 3; ++k)
            if (ws->graph[k]) {
                cudaGraphExecDestroy(ws->graph[k]);
                ws->graph[k] = nullptr;
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
// Variants: 0 plain, with programmatic dependent launch; 1 records the 5
// per-kernel events in its first iteration; 2 plain without dependent launch.
static stg_status get_graph(stg_gauge *g, Workspace *ws, int pd, int n, int variant,
                            cudaGraphExec_t *out)
{
    const int timed = variant;
    cudaGraphExec_t &ge = ws->graph[timed];
    if (ge && ws->graph_sloppy[timed] == pd && ws->graph_iters[timed] == n) {
        *out = ge;
        return STG_OK;
    }
    if (ge) {
        cudaGraphExecDestroy(ge);
        ge = nullptr;
    }
    if (variant == 1 && !ws->ev[0])
        for (int k = 0; k < 5; ++k) STG_CUDA(cudaEventCreate(&ws->ev[k]));
    cudaStream_t cs;
    STG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    stg_status st = STG_OK;
    if (e == cudaSuccess) {
        for (int k = 0; k < n && st == STG_OK; ++k)
            st = iteration(g, ws, pd, cs, (variant == 1 && k == 0) ? ws->ev : nullptr, variant == 0);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == STG_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (st == STG_OK) {
        e = cudaGraphInstantiate(&ge, graph, 0);
        if (e != cudaSuccess) {
            ge = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != STG_OK) return st;
    ws->graph_sloppy[timed] = pd;
    ws->graph_iters[timed] = n;
    *out = ge;
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
    double iter_sum = 0.0, serial_sum = 0.0;
    long iter_n = 0, serial_n = 0;

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
        cudaGraphExec_t graph = nullptr, graph_timed = nullptr, graph_serial = nullptr;
        if (status == STG_OK) status = get_graph(g, ws, pd, chunk, 0, &graph);
        if (status == STG_OK && p->timing) status = get_graph(g, ws, pd, chunk, 1, &graph_timed);
        if (status == STG_OK && p->timing) status = get_graph(g, ws, pd, chunk, 2, &graph_serial);
        if (status == STG_OK && p->timing && !ws->ev_chunk[0]) {
            for (int k = 0; k < 2 && status == STG_OK; ++k) {
                cudaError_t e = cudaEventCreate(&ws->ev_chunk[k]);
                if (e != cudaSuccess) status = cuda_fail(e, "cudaEventCreate");
            }
        }
        int breakdowns = 0;
        long chunk_no = 0;
        while (status == STG_OK) {
            // with timing, chunks rotate: per-kernel events; events around
            // the whole launch of a plain chunk; the same without dependent
            // launch (serial kernels)
            const int phase = (int)(chunk_no % 3);
            const bool kernel_timed = p->timing && phase == 0;
            const bool chunk_timed = p->timing && !kernel_timed;
            const bool serial = p->timing && phase == 2;
            ++chunk_no;
            cudaError_t e = cudaSuccess;
            if (chunk_timed) e = cudaEventRecord(ws->ev_chunk[0], s);
            if (e == cudaSuccess)
                e = cudaGraphLaunch(kernel_timed ? graph_timed : (serial ? graph_serial : graph), s);
            if (e == cudaSuccess && chunk_timed) e = cudaEventRecord(ws->ev_chunk[1], s);
            if (e != cudaSuccess) {
                status = cuda_fail(e, "cudaGraphLaunch");
                break;
            }
            status = read_state(ws, s);
            if (status != STG_OK) break;
            launches += 4L * chunk;
            if (chunk_timed && h->flag == FLAG_RUN) {
                // every iteration of the chunk ran in full
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ws->ev_chunk[0], ws->ev_chunk[1]) == cudaSuccess) {
                    if (serial) {
                        serial_sum += ms / chunk;
                        ++serial_n;
                    } else {
                        iter_sum += ms / chunk;
                        ++iter_n;
                    }
                } else {
                    cudaGetLastError();
                }
            }
            if (kernel_timed) {
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
            if (flag == FLAG_TIMEOUT) {
                set_error("stg_cg_solve: a bounded wait inside the Dslash kernel gave up");
                status = STG_ERR_TIMEOUT;
                break;
            }
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
    if (iter_n > 0) st.t_iter_ms = iter_sum / iter_n;
    if (serial_n > 0) st.t_iter_serial_ms = serial_sum / serial_n;
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
