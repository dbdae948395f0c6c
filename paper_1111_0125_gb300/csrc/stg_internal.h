// Host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>

#include "stg.h"
#include "stg_common.cuh"

namespace stg {

constexpr int kBlock = 256;  // threads per block of every site-parallel kernel

// Launch with programmatic dependent launch when `pdl`: the kernel may start
// while its predecessor on the stream finishes; it must call pdl_wait()
// before touching anything the predecessor writes (stg_common.cuh).
template <typename... K, typename... A>
static inline cudaError_t launch_k(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   bool pdl, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Device copy of the links in one precision / reconstruction.
// Tile-major copy of FX16 or FP16 / 12-real links for the staged Dslash: for output
// parity p, tile k of kFxTile consecutive output sites and direction mu, one
// contiguous block of kFxStageBytes holds the forward links U_mu(x) (uint4
// [kFxTile] then uint2 [kFxTile]) followed by the backward links U_mu(x - mu)
// of the same output sites, each record at the output site's slot; slots past
// Vh are zero.  Every link appears twice (once per parity of output site).
constexpr int kFxTile = 1024;
constexpr unsigned kFxStageBytes = kFxTile * 48u;

// Tile-major copy of FP32 / 12-real and FX16 / 12-real links for the staged
// multi-system Dslash: for output parity p and tile k of kMTile consecutive
// output sites, one contiguous block of kMTile * 8 * L bytes holds, for mu =
// 0..3 and dir = forward, backward, the 12-real records of the tile's sites
// as planes (FP32: three float4 planes; FX16: a uint4 plane then a uint2
// plane); slots past Vh are zero.
constexpr int kMTile = 64;

struct LinkField {
    char *base = nullptr;   // 8 blocks: (parity, mu) -> base + (2 * 4 ... ) see blk()
    int prec = -1;
    int recon = 18;
    size_t blk_bytes = 0;   // bytes of one (parity, mu) block, 256-aligned
    char *tiled = nullptr;  // FX16 / 12-real only: tile-major copy (kFxTile)
    size_t tiled_parity_bytes = 0;
    char *mtiled = nullptr; // 12-real FP32 / FX16: tile-major copy (kMTile)
    size_t mtiled_parity_bytes = 0, mtile_bytes = 0;
    // test hooks of the staged FX16 kernel, read once when the handle is
    // created (STG_FX16_GRID, STG_FX16_TEST_DROP_FILL): a cap on its CTA
    // count (0 = none) and the withheld fill of the failure-detection test
    int fx_grid_cap = 0;
    int fx_drop_fill = 0;
    const char *blk(int parity, int mu) const { return base + (size_t)(parity * 4 + mu) * blk_bytes; }
};

struct Workspace;

// Workspace of the multi-system CG (mrhs.cu): n systems of every vector.
struct MrhsWs {
    int nrhs = 0, pd = -1;
    size_t f64 = 0, fr = 0, fd = 0;   // bytes of one FP64 / PR / PD field
    size_t pstride = 0;               // reduction partials per system (doubles)
    char *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
    char *y = nullptr, *r = nullptr, *d = nullptr, *q = nullptr, *t = nullptr;
    double *partials = nullptr;
    CGState *states = nullptr, *states_host = nullptr;
    int *active = nullptr, *active_host = nullptr;  // [0] = count, [1..] = systems
    unsigned *counter = nullptr;
    void *tmp = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    int shape = 0;                    // autotuned (NB, threads per site) index
};
void mrhs_free(MrhsWs *m);
void batch_destroy(stg_batch *b);
size_t mrhs_bytes(const Geom &g, int n, int pd);

}  // namespace stg

struct stg_gauge {
    int dims[4];
    stg::Geom geom;
    int device;
    int sloppy;             // stg_prec of the low-precision copy (P64 = none)
    stg::LinkField hi;      // FP64 links
    stg::LinkField lo;      // sloppy links (base == nullptr when sloppy == FP64)
    stg::Workspace *ws;     // lazily created
};

namespace stg {

// per-thread error text
void set_error(const std::string &msg);
stg_status cuda_fail(cudaError_t e, const char *what);

#define STG_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::stg::cuda_fail(e_, #call);       \
    } while (0)

#define STG_TRY(call)                                                    \
    do {                                                                 \
        stg_status s_ = (call);                                          \
        if (s_ != STG_OK) return s_;                                     \
    } while (0)

Geom make_geom(const int dims[4]);

// stg_cg_params defaults for inner iterations in `sloppy` (api.cu)
void cg_params_for(int sloppy, stg_cg_params *p);

const LinkField *links_for(const stg_gauge *g, int prec);

// Reduction scratch: partial sums (one double per block) and the state.
struct Workspace {
    double *partials = nullptr;
    size_t n_partials = 0;
    CGState *state = nullptr;      // device
    CGState *state_host = nullptr; // pinned mirror for read-back
    void *tmp[kNumPrec] = {};  // odd intermediate per precision
    // CG vectors (allocated by the solver)
    void *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *t64 = nullptr;
    void *y = nullptr, *r = nullptr, *d = nullptr, *q = nullptr;
    int cg_sloppy = -1;
    // captured chunks of iterations: [0] plain (programmatic dependent
    // launch), [1] with per-kernel events, [2] plain without dependent launch
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    int graph_sloppy[3] = {-1, -1, -1}, graph_iters[3] = {0, 0, 0};
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // per-kernel events
    cudaEvent_t ev_chunk[2] = {nullptr, nullptr};                        // around plain chunks
    stg_batch *batch = nullptr;       // session cached for stg_cg_solve_mrhs
    void *mrhs_tmp = nullptr;         // odd intermediates of stg_apply_A_mrhs
    size_t mrhs_tmp_bytes = 0;
};

stg_status workspace_get(stg_gauge *g, Workspace **out);
stg_status workspace_tmp(stg_gauge *g, int prec, void **out);
void workspace_free(Workspace *ws);

// kernels (launch only; all on `s`)
enum Epi { EPI_NONE = 0, EPI_A = 1, EPI_A_DOT = 2, EPI_A_CG = 3, EPI_RES = 4, EPI_GATE = 5 };

struct DslashLaunch {
    const LinkField *links;
    int out_parity;
    const void *in;
    void *out;
    const void *w;   // EPI_A*: the even input d (m^2 d term, d^dag q); EPI_RES: b
    const void *v;   // EPI_RES: x
    double m2;
    double *dot;     // EPI_A_DOT: result
    CGState *state;  // EPI_A_CG, EPI_GATE
    double *partials;
    unsigned *counter;
    bool pdl;        // programmatic dependent launch (inside the CG graph)
};

stg_status launch_dslash(const Geom &g, int prec, int epi, const DslashLaunch &a, cudaStream_t s);

// kernel arguments of every Dslash variant
struct DslashArgs {
    Geom g;
    const char *lf[4];  // forward link blocks  (parity p,   mu)
    const char *lb[4];  // backward link blocks (parity 1-p, mu)
    const char *lt;     // tile-major links of output parity p (FX16 / 12), or null
    int grid_cap;       // staged kernel: at most this many CTAs (0 = one per SM)
    int drop_fill;      // tests only: the staged kernel withholds the fill of
                        // its second tile's first stage, so that bounded
                        // wait runs out
    int parity;
    const void *in;
    void *out;
    const void *w;
    const void *v;
    double m2;
    double *dot;
    CGState *state;
    double *partials;
    unsigned *counter;
};

// FX16 Dslash, two sites per thread on packed FP32x2 arithmetic
void launch_dslash_fx2(int recon, int epi, const DslashArgs &a, cudaStream_t s, bool pdl);
// IEEE FP16 / 12-real with the tile-major links: the same staged kernel
void launch_dslash_f16_staged(int epi, const DslashArgs &a, cudaStream_t s, bool pdl);

int grid_for(long n);

// vector-kernel helpers with explicit operands (cg.cu)
int vec_grid(long n, int pd);
stg_status launch_update_m(int pd, int vh, char *y, char *r, const char *d, const char *q, size_t sr,
                           size_t sd, CGState *states, double *partials, size_t pstride,
                           const int *active, const int *nactive, int nslots, cudaStream_t s);
stg_status launch_xpay_m(int pd, int vh, const char *r, char *d, size_t sr, size_t sd,
                         const CGState *states, const int *active, const int *nactive, int nslots,
                         cudaStream_t s);
stg_status launch_reset(int pd, int vh, void *y, void *r, void *d, const void *r64, double beta,
                        int copy_r, cudaStream_t s);
stg_status launch_accumulate_x(int pr, int vh, void *x64, const void *y, cudaStream_t s);
stg_status launch_norm2(int prec, int vh, const void *v, CGState *st, double *partials, cudaStream_t s);
stg_status launch_true_residual(stg_gauge *g, const void *x64, const void *b64, void *r64, void *t64,
                                double m2, CGState *st, double *partials, cudaStream_t s);
stg_status pack_field(const Geom &g, int prec, const double *canon, void *out, cudaStream_t s);
stg_status unpack_field(const Geom &g, int prec, const void *in, double *canon, cudaStream_t s);

}  // namespace stg
