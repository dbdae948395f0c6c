// extern "C" entry points declared in include/stg.h: argument checks,
// device selection, status codes and the per-thread error text.  The work
// itself is in gauge.cu (upload / layouts), dslash.cu (Eq. 5 and A of Eq. 3)
// and cg.cu (Fig. 1, Fig. 2, Eq. 6, Sec. 3.2).
#include <math.h>
#include <stdio.h>

#include <string>

#include "stg_internal.h"

namespace stg {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

stg_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : STG_ERR_CUDA;
}

stg_status gauge_create(const int dims[4], const double *links_host, int sloppy, int recon,
                        cudaStream_t s, stg_gauge **out);
void gauge_destroy(stg_gauge *g);
size_t gauge_bytes(const int dims[4], int sloppy, int recon);
stg_status pack_field(const Geom &g, int prec, const double *canon, void *out, cudaStream_t s);
stg_status unpack_field(const Geom &g, int prec, const void *in, double *canon, cudaStream_t s);
stg_status cg_solve(stg_gauge *g, const double *src, double *x, double mass, double tol,
                    const stg_cg_params *p, stg_cg_stats *stats, cudaStream_t s);

// Makes the handle's device current for the scope of a call.
struct DeviceScope {
    int prev = -1;
    int want;
    explicit DeviceScope(int dev) : want(dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

static bool valid_prec(int p)
{
    return p == STG_FP64 || p == STG_FP32 || p == STG_FP16 || p == STG_FX16 || p == STG_BF16;
}

static stg_status check_dims(const int *dims)
{
    if (!dims) {
        set_error("dims is NULL");
        return STG_ERR_INVALID_ARG;
    }
    long v = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || (dims[mu] & 1)) {
            set_error("every lattice extent must be even and >= 2");
            return STG_ERR_DIMS;
        }
        v *= dims[mu];
        if (v > (1L << 31)) {
            set_error("lattice volume above 2^31 sites");
            return STG_ERR_DIMS;
        }
    }
    return STG_OK;
}

static stg_status check_field_prec(const stg_gauge *g, int prec, const LinkField **lf)
{
    if (!valid_prec(prec)) {
        set_error("unknown precision");
        return STG_ERR_INVALID_ARG;
    }
    *lf = links_for(g, prec);
    if (!*lf) {
        set_error("the gauge handle holds no links in this precision");
        return STG_ERR_UNSUPPORTED;
    }
    return STG_OK;
}

}  // namespace stg

using namespace stg;

namespace stg {

// Defaults for inner iterations in `sloppy` (see stg_cg_params_default).
void cg_params_for(int sloppy, stg_cg_params *p)
{
    p->sloppy = sloppy;
    // eps^in (Sec. 3.2 leaves it open): the lower the inner precision, the
    // sooner the iterated residual drifts and the more often an update pays;
    // measured on 32^3x64, m = 0.005 (FP32: 0.03-0.05 best, FX16 / BF16:
    // 0.2-0.3).  IEEE FP16 (11 significand bits) is the exception: the Eq. 6
    // start carries its inner search direction into the next cycle and costs
    // it 8203 iterations at delta 0.25, while Fig. 2's restart from the true
    // residual with inner solves to 0.02 takes 2652 (FX16 with Eq. 6: 2593)
    if (sloppy == STG_FP16) {
        p->policy = STG_CG_REFINE;
        p->delta = 0.02;
    } else {
        p->policy = STG_CG_RELIABLE;
        p->delta = (sloppy == STG_FP32) ? 0.05 : (sloppy == STG_FP64 ? 0.1 : 0.25);
    }
    p->maxiter = 0;
    p->check_every = 0;
    p->timing = 0;
}

}  // namespace stg

extern "C" {

int stg_version(void) { return 1; }

const char *stg_status_string(stg_status s)
{
    switch (s) {
    case STG_OK: return "ok";
    case STG_ERR_INVALID_ARG: return "invalid argument";
    case STG_ERR_DIMS: return "invalid lattice dimensions";
    case STG_ERR_OOM: return "out of memory";
    case STG_ERR_CUDA: return "CUDA error";
    case STG_ERR_NOT_CONVERGED: return "not converged";
    case STG_ERR_BREAKDOWN: return "CG breakdown";
    case STG_ERR_TIMEOUT: return "device wait timed out";
    case STG_ERR_UNSUPPORTED: return "unsupported precision or reconstruction";
    }
    return "unknown status";
}

const char *stg_last_error(void) { return g_last_error.c_str(); }

stg_status stg_gauge_create(const int dims[4], const double *links_host, stg_prec sloppy, int recon,
                            stg_stream_t stream, stg_gauge **out)
{
    STG_TRY(check_dims(dims));
    if (!links_host || !out) {
        set_error("stg_gauge_create: NULL links or out");
        return STG_ERR_INVALID_ARG;
    }
    if (!valid_prec(sloppy) || (recon != 18 && recon != 12)) {
        set_error("stg_gauge_create: precision must be FP64/FP32/FP16/FX16/BF16 and recon 18 or 12");
        return STG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    return gauge_create(dims, links_host, sloppy, recon, (cudaStream_t)stream, out);
}

size_t stg_gauge_bytes(const int dims[4], stg_prec sloppy, int recon)
{
    if (check_dims(dims) != STG_OK || !valid_prec(sloppy) || (recon != 18 && recon != 12)) return 0;
    return gauge_bytes(dims, sloppy, recon);
}

stg_status stg_gauge_destroy(stg_gauge *g)
{
    gauge_destroy(g);
    return STG_OK;
}

stg_status stg_gauge_dims(const stg_gauge *g, int dims[4], long *vh)
{
    if (!g) {
        set_error("stg_gauge_dims: NULL handle");
        return STG_ERR_INVALID_ARG;
    }
    if (dims)
        for (int mu = 0; mu < 4; ++mu) dims[mu] = g->dims[mu];
    if (vh) *vh = g->geom.Vh;
    return STG_OK;
}

stg_status stg_field_bytes(const stg_gauge *g, stg_prec prec, size_t *bytes)
{
    if (!g || !bytes || !valid_prec(prec)) {
        set_error("stg_field_bytes: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    *bytes = (size_t)g->geom.Vh * field_site_bytes(prec);
    return STG_OK;
}

stg_status stg_pack_field(const stg_gauge *g, stg_prec prec, const double *canon_dev,
                          void *field_dev, stg_stream_t stream)
{
    if (!g || !canon_dev || !field_dev || !valid_prec(prec)) {
        set_error("stg_pack_field: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    DeviceScope ds(g->device);
    return pack_field(g->geom, prec, canon_dev, field_dev, (cudaStream_t)stream);
}

stg_status stg_unpack_field(const stg_gauge *g, stg_prec prec, const void *field_dev,
                            double *canon_dev, stg_stream_t stream)
{
    if (!g || !canon_dev || !field_dev || !valid_prec(prec)) {
        set_error("stg_unpack_field: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    DeviceScope ds(g->device);
    return unpack_field(g->geom, prec, field_dev, canon_dev, (cudaStream_t)stream);
}

stg_status stg_dslash(const stg_gauge *g, int out_parity, const void *in_dev, void *out_dev,
                      stg_prec prec, stg_stream_t stream)
{
    if (!g || !in_dev || !out_dev || (out_parity != 0 && out_parity != 1) || in_dev == out_dev) {
        set_error("stg_dslash: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    const LinkField *lf;
    STG_TRY(check_field_prec(g, prec, &lf));
    DeviceScope ds(g->device);
    DslashLaunch L = {};
    L.links = lf;
    L.out_parity = out_parity;
    L.in = in_dev;
    L.out = out_dev;
    return launch_dslash(g->geom, prec, EPI_NONE, L, (cudaStream_t)stream);
}

static stg_status apply_A_impl(const stg_gauge *gc, double mass, const void *in_dev, void *out_dev,
                               double *dot_dev, stg_prec prec, cudaStream_t s)
{
    if (!gc || !in_dev || !out_dev || in_dev == out_dev || !isfinite(mass)) {
        set_error("stg_apply_A: bad argument");
        return STG_ERR_INVALID_ARG;
    }
    const LinkField *lf;
    STG_TRY(check_field_prec(gc, prec, &lf));
    stg_gauge *g = const_cast<stg_gauge *>(gc);  // workspace is lazily created
    DeviceScope ds(g->device);
    void *tmp;
    STG_TRY(workspace_tmp(g, prec, &tmp));
    Workspace *ws = g->ws;
    DslashLaunch L = {};
    L.links = lf;
    L.out_parity = 1;
    L.in = in_dev;
    L.out = tmp;
    STG_TRY(launch_dslash(g->geom, prec, EPI_NONE, L, s));
    L.out_parity = 0;
    L.in = tmp;
    L.out = out_dev;
    L.w = in_dev;
    L.m2 = mass * mass;
    L.dot = dot_dev;
    L.partials = ws->partials;
    L.counter = &ws->state->counter;
    return launch_dslash(g->geom, prec, dot_dev ? EPI_A_DOT : EPI_A, L, s);
}

stg_status stg_apply_A(const stg_gauge *g, double mass, const void *in_dev, void *out_dev,
                       stg_prec prec, stg_stream_t stream)
{
    return apply_A_impl(g, mass, in_dev, out_dev, nullptr, prec, (cudaStream_t)stream);
}

stg_status stg_apply_A_dot(const stg_gauge *g, double mass, const void *in_dev, void *out_dev,
                           double *dot_dev, stg_prec prec, stg_stream_t stream)
{
    if (!dot_dev) {
        set_error("stg_apply_A_dot: NULL dot");
        return STG_ERR_INVALID_ARG;
    }
    return apply_A_impl(g, mass, in_dev, out_dev, dot_dev, prec, (cudaStream_t)stream);
}

stg_status stg_cg_params_default(const stg_gauge *g, stg_cg_params *p)
{
    if (!p) {
        set_error("stg_cg_params_default: NULL params");
        return STG_ERR_INVALID_ARG;
    }
    stg::cg_params_for(g ? g->sloppy : STG_FP64, p);
    return STG_OK;
}

stg_status stg_cg_solve(const stg_gauge *gc, const double *src_dev, double *x_dev, double mass,
                        double tol, const stg_cg_params *params, stg_cg_stats *stats,
                        stg_stream_t stream)
{
    if (stats) *stats = stg_cg_stats{};
    if (!gc || !src_dev || !x_dev || src_dev == x_dev) {
        set_error("stg_cg_solve: NULL handle / pointer or src == x");
        return STG_ERR_INVALID_ARG;
    }
    if (!isfinite(mass) || mass < 0.0 || !isfinite(tol) || !(tol > 0.0)) {
        set_error("stg_cg_solve: mass must be finite and >= 0, tol finite and > 0");
        return STG_ERR_INVALID_ARG;
    }
    stg_cg_params p;
    if (params) p = *params;
    else stg_cg_params_default(gc, &p);
    if (p.policy < STG_CG_RELIABLE || p.policy > STG_CG_PLAIN || !valid_prec(p.sloppy) ||
        !(p.delta > 0.0 && p.delta < 1.0) || p.maxiter < 0 || p.check_every < 0) {
        set_error("stg_cg_solve: bad params (policy, sloppy, 0 < delta < 1, maxiter >= 0)");
        return STG_ERR_INVALID_ARG;
    }
    if (p.policy == STG_CG_PLAIN) p.sloppy = STG_FP64;
    if (!links_for(gc, p.sloppy)) {
        set_error("stg_cg_solve: the handle holds no links in the sloppy precision");
        return STG_ERR_UNSUPPORTED;
    }
    stg_gauge *g = const_cast<stg_gauge *>(gc);
    DeviceScope ds(g->device);
    return cg_solve(g, src_dev, x_dev, mass, tol, &p, stats, (cudaStream_t)stream);
}

}  // extern "C"
