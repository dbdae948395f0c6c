// t-slab domain decomposition of the Dirac operator (Sec. 3.3, Table 1),
// every slab on one device.
//
// The lattice is cut along t into P slabs of Lts = Lt / P time slices.  Each
// slab is a local lattice (Lx, Ly, Lz, Lts) with its own links, fields and
// face buffers, as one rank of the paper's multi-GPU run holds its part.
// With the checkerboard index running t slowest, time slice t of one parity
// is the index range [t st, (t + 1) st), st = Lx Ly Lz / 2, in every
// structure-of-arrays plane, so a face is a few contiguous pieces.
//
// One Dirac operation (a Dslash half-pass, Eq. 5) takes the three steps of
// Table 1:
//   1. boundary collect: one kernel copies, for every slab, the input
//      field's slices t = 0 and t = Lts - 1 (bit for bit) into face buffers;
//   2. exchange: the t = 0 face goes to the previous slab's forward ghost,
//      the t = Lts - 1 face to the next slab's backward ghost (COPY: one
//      device copy per face, the message of a multi-GPU run; DIRECT: the
//      collect kernel stores into the neighbours' ghosts itself, as a kernel
//      does through peer pointers);
//   3. compute: the Dslash of every slab in one launch (blockIdx.y = slab);
//      a t-hop that leaves the slab reads the ghost, the backward t-link of
//      slice 0 comes from the ghost links (the previous slab's U_t at its
//      last slice, copied in once at creation: the links are constant).
// The interior slices 1 .. Lts - 2 read no ghost, so with `overlap` they run
// while steps 1-2 are in flight on a second stream (Sec. 4), and the two
// boundary slices follow; without overlap one launch runs the same blocks
// (interior blocks first, then boundary blocks), so every block computes the
// same sites and writes the same partial in both schedules: results are
// bitwise equal.
//
// Signs: s_mu = eta_mu b_mu (Sec. 2) is folded into the links at packing with
// the global boundary: only the slab holding global t = Lt - 1 flips its last
// slice's forward t-links.  The 12-real row-2 sign is recomputed in the
// kernel from the same rule (top / bot below).
//
// Global sums: each block writes a partial per slab; one block then sums
// each slab's partials in a fixed order and adds the slab totals in slab
// order (the two-scalar allreduce of a multi-GPU CG).  Deterministic.
#include <math.h>
#include <string.h>
#include <time.h>

#include <new>
#include <vector>

#include "dslash_site.cuh"
#include "stg_internal.h"

namespace stg {

stg_status pack_field(const Geom &g, int prec, const double *canon, void *out, cudaStream_t s);
stg_status unpack_field(const Geom &g, int prec, const void *in, double *canon, cudaStream_t s);
stg_status pack_links_flip(const Geom &g, const double2 *ucan, int prec, int recon, int t_flip,
                           LinkField *lf, cudaStream_t s);

// Field slots of every slab, each sized for FP64 (48 bytes per site): the
// user's six (slots 0-5 in the handle's precision), then four FP64 vectors
// of the CG.  The CG's inner vectors live in the user slots: y and r in PR,
// d, t and q in the handle's precision PD.
constexpr int kUserSlots = STG_SLAB_SLOTS;
constexpr int kSlabSlots = kUserSlots + 4;
constexpr int kMaxSlabs = 64;
enum SlabSlot { SL_Y = 1, SL_R = 2, SL_D = 3, SL_T = 4, SL_Q = 5, SL_B64 = 6, SL_X64 = 7, SL_R64 = 8, SL_T64 = 9 };

// the precision of y and r for inner iterations in PD
static int slab_pr(int pd) { return pd == P64 ? P64 : P32; }

static size_t sl_align(size_t n) { return (n + 255) & ~(size_t)255; }

// Element bytes of the structure-of-arrays planes of one record, in plane
// order (the layouts of FieldIO / LinkIO and k_pack_links).
static int field_planes(int prec, int e[3])
{
    if (prec == P64) { e[0] = e[1] = e[2] = 16; return 3; }
    if (prec == P32) { e[0] = 16; e[1] = 8; return 2; }
    e[0] = 16;
    return 1;
}

static int link_planes(int prec, int recon, int e[9])
{
    if (prec == P64) {
        const int n = recon == 18 ? 9 : 6;
        for (int k = 0; k < n; ++k) e[k] = 16;
        return n;
    }
    if (prec == P32) {
        const int n4 = recon == 18 ? 4 : 3;
        for (int k = 0; k < n4; ++k) e[k] = 16;
        if (recon == 18) e[4] = 8;
        return recon == 18 ? 5 : 3;
    }
    e[0] = 16;
    if (recon == 18) { e[1] = 16; e[2] = 4; return 3; }
    e[1] = 8;
    return 2;
}

// Per-slab pointers, in device memory (one entry per slab).
struct SlabDev {
    const char *lk[8];        // link blocks, index parity * 4 + mu
    const char *ghost_lk[2];  // per output parity: U_t(x - t) of the sites at slice 0 (planes of stride st)
    const char *lk64[8];      // the FP64 / 18-real links of the CG's true residual (= lk for FP64 handles)
    const char *ghost64[2];
    char *slot[kSlabSlots];   // fields (planes of stride Vh)
    char *send[2];            // COPY mode: [0] slice 0, [1] slice Lts - 1 of the collected field
    char *recv[2];            // ghosts: [0] next slab's slice 0, [1] previous slab's slice Lts - 1
    char *peer[2];            // DIRECT mode targets: previous slab's recv[0], next slab's recv[1]
    float top, bot;           // -1 where the slab holds global t = Lt - 1 (top) / t = 0 (bot), else 1
};

struct SlabArgs {
    Geom g;                   // local lattice (Lx, Ly, Lz, Lts)
    const SlabDev *sl;
    int parity;               // output parity
    int in, out, w, v;        // slots
    double m2;
    CGState *state;
    double *partials;         // [slab][pstride]
    int pstride, pbase;       // partial index of this launch's block 0
    int part;                 // 0: interior slices, 1: the two boundary slices, 2: both
    int nb_int;               // blocks of the interior part (part 2: blocks below it are interior)
    int prec, recon;          // the operator's storage
    int hi;                   // 1: the FP64 / 18-real link set (lk64, ghost64)
};

// The slab's entry, staged in shared memory once per block (every thread of
// a block works on the same slab).
__device__ __forceinline__ const SlabDev *slab_entry(const SlabDev *tab, SlabDev *sh)
{
    constexpr int kWords = sizeof(SlabDev) / 8;
    static_assert(sizeof(SlabDev) % 8 == 0, "SlabDev is copied in 8-byte words");
    if (threadIdx.x < kWords)
        reinterpret_cast<unsigned long long *>(sh)[threadIdx.x] =
            reinterpret_cast<const unsigned long long *>(tab + blockIdx.y)[threadIdx.x];
    __syncthreads();
    return sh;
}

// ---------------------------------------------------------------------------
// step 1 (and 2 in DIRECT mode): boundary collect
// ---------------------------------------------------------------------------
struct CollectArgs {
    const SlabDev *sl;
    int slot, vh, st, lts;
    int np;                   // field planes
    int e[3];                 // their element bytes
    int words;                // 8-byte words of one face
    int direct;
};

__global__ void __launch_bounds__(kBlock) k_slab_collect(const CollectArgs a)
{
    const int k = blockIdx.x * kBlock + threadIdx.x;
    if (k >= 2 * a.words) return;
    const SlabDev *S = a.sl + blockIdx.y;
    const int f = k >= a.words;            // 0: slice 0, 1: slice Lts - 1
    int w = k - f * a.words;
    const int row0 = f ? (a.lts - 1) * a.st : 0;
    const char *src = S->slot[a.slot];
    char *dst = a.direct ? S->peer[f] : S->send[f];
    size_t off_field = 0, off_face = 0;
    for (int p = 0; p < a.np; ++p) {
        const int nw = a.st * a.e[p] / 8;
        if (w < nw) {
            const uint2 v = *reinterpret_cast<const uint2 *>(src + off_field + (size_t)row0 * a.e[p] + 8 * (size_t)w);
            *reinterpret_cast<uint2 *>(dst + off_face + 8 * (size_t)w) = v;
            return;
        }
        w -= nw;
        off_field += (size_t)a.vh * a.e[p];
        off_face += (size_t)a.st * a.e[p];
    }
}

// ---------------------------------------------------------------------------
// step 3: the Dslash of every slab (Eq. 5), the same arithmetic in the same
// order as dslash_site, with the t-hops across a slab edge on the ghosts
// ---------------------------------------------------------------------------
template <int P, int R>
__device__ __forceinline__ Vec3<typename Real<P>::T> slab_site(const Geom &g, const SlabDev *S,
                                                               const char *const *lk, const char *const *gl,
                                                               int parity, const void *in, int i)
{
    typedef typename Real<P>::T T;
    const int vh = g.Vh, st = g.st, top = g.L[3] - 1;
    const Site s = site_of(g, i, parity);
    Vec3<T> acc;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.r[c] = acc.i[c] = T(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int jf, jb;
        neighbours(g, s, i, mu, jf, jb);
        const bool up = mu == 3 && s.t == top;  // x + t lies on the next slab
        const bool down = mu == 3 && s.t == 0;  // x - t lies on the previous slab
        float sf = 1.f, sb = 1.f;
        if (R == 12) {
            int e = 0;
            if (mu >= 1) e += s.x;
            if (mu >= 2) e += s.y;
            if (mu >= 3) e += s.z;
            sf = sb = (e & 1) ? -1.f : 1.f;
            if (up) sf *= S->top;
            if (down) sb *= S->bot;
        }
        const T s2f = (R == 12) ? T(sf * LinkPost<P>::row2) : T(1);
        const T s2b = (R == 12) ? T(sb * LinkPost<P>::row2) : T(1);
        const Mat3<T> uf = LinkIO<P, R>::load(lk[parity * 4 + mu], vh, i);
        const Vec3<T> vf = up ? FieldIO<P>::load_nc(S->recv[0], st, i - top * st)
                              : FieldIO<P>::load_nc(in, vh, jf);
        mul_add<R == 12>(uf, vf, acc, s2f);
        const Mat3<T> ub = down ? LinkIO<P, R>::load(gl[parity], st, i)
                                : LinkIO<P, R>::load(lk[(1 - parity) * 4 + mu], vh, jb);
        const Vec3<T> vb = down ? FieldIO<P>::load_nc(S->recv[1], st, i) : FieldIO<P>::load_nc(in, vh, jb);
        adj_mul_sub(ub, vb, acc, s2b);
    }
    if (P == PX16) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc.r[c] *= T(LinkPost<PX16>::k);
            acc.i[c] *= T(LinkPost<PX16>::k);
        }
    }
    return acc;
}

// Epilogues as in dslash.cu: EPI_NONE / EPI_GATE store D in; EPI_A_DOT /
// EPI_A_CG store m^2 w - D in and sum w^dag out; EPI_RES stores
// w - m^2 v + D in (= b - A x) and sums |out|^2.  Sums in FP64.
template <int P, int R, int EPI>
__global__ void __launch_bounds__(kBlock) k_slab_dslash(const SlabArgs a)
{
    typedef typename Real<P>::T T;
    if (EPI == EPI_GATE || EPI == EPI_A_CG) {
        if (a.state->flag != FLAG_RUN) return;  // uniform over the grid
    }
    __shared__ SlabDev sh;
    const SlabDev *S = slab_entry(a.sl, &sh);
    const int st = a.g.st, lts = a.g.L[3], vh = a.g.Vh;
    int part = a.part, blk = blockIdx.x;
    if (part == 2) {  // one launch for both parts, the same blocks as two
        part = blk < a.nb_int ? 0 : 1;
        if (part == 1) blk -= a.nb_int;
    }
    const int k = blk * kBlock + threadIdx.x;
    int i;
    bool ok;
    if (part == 0) {
        i = st + k;
        ok = i < (lts - 1) * st;
    } else {
        ok = k < 2 * st;
        i = k < st ? k : k + (lts - 2) * st;
    }
    double dot = 0.0;
    if (ok) {
        const Vec3<T> acc = slab_site<P, R>(a.g, S, a.hi ? S->lk64 : S->lk, a.hi ? S->ghost64 : S->ghost_lk,
                                            a.parity, S->slot[a.in], i);
        void *out = S->slot[a.out];
        if (EPI == EPI_NONE || EPI == EPI_GATE) {
            FieldIO<P>::store(out, vh, i, acc);
        } else if (EPI == EPI_RES) {
            const Vec3<T> b = FieldIO<P>::load_nc(S->slot[a.w], vh, i);
            const Vec3<T> x = FieldIO<P>::load_nc(S->slot[a.v], vh, i);
            const T m2 = T(a.m2);
            Vec3<T> o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.r[c] = b.r[c] - m2 * x.r[c] + acc.r[c];
                o.i[c] = b.i[c] - m2 * x.i[c] + acc.i[c];
            }
            const Vec3<T> os = FieldIO<P>::store(out, vh, i, o);
            T n = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) n += os.r[c] * os.r[c] + os.i[c] * os.i[c];
            dot = double(n);
        } else {
            const T m2 = (EPI == EPI_A_CG) ? T(a.state->m2) : T(a.m2);
            const Vec3<T> d = FieldIO<P>::load_nc(S->slot[a.w], vh, i);
            Vec3<T> o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.r[c] = m2 * d.r[c] - acc.r[c];
                o.i[c] = m2 * d.i[c] - acc.i[c];
            }
            const Vec3<T> os = FieldIO<P>::store(out, vh, i, o);
            T n = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) n += d.r[c] * os.r[c] + d.i[c] * os.i[c];
            dot = double(n);
        }
    }
    if (EPI == EPI_A_DOT || EPI == EPI_A_CG || EPI == EPI_RES) {
        __shared__ double sm[32];
        const double b = block_sum<kBlock>(dot, sm);
        if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * a.pstride + a.pbase + blockIdx.x] = b;
    }
}

// ---------------------------------------------------------------------------
// CG vector kernels on the slabs (one site per thread, blockIdx.y = slab;
// slots as in SlabSlot) and the slab-ordered sums
// ---------------------------------------------------------------------------
struct VecArgs {
    const SlabDev *sl;
    int vh;
    CGState *state;
    double *partials;
    int pstride;
};

// y += alpha d, r -= alpha q, |r|^2 partials (Fig. 1)
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_slab_update(const VecArgs a)
{
    const CGState *st = a.state;
    if (st->flag != FLAG_RUN) return;
    typedef typename Real<PR>::T T;
    const SlabDev *S = a.sl + blockIdx.y;
    const int vh = a.vh;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    double n = 0.0;
    if (i < vh) {
        const T alpha = T(st->alpha);
        const auto d = FieldIO<PD>::load(S->slot[SL_D], vh, i);
        const auto q = FieldIO<PD>::load(S->slot[SL_Q], vh, i);
        Vec3<T> y = FieldIO<PR>::load(S->slot[SL_Y], vh, i);
        Vec3<T> r = FieldIO<PR>::load(S->slot[SL_R], vh, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            y.r[c] += alpha * T(d.r[c]);
            y.i[c] += alpha * T(d.i[c]);
            r.r[c] -= alpha * T(q.r[c]);
            r.i[c] -= alpha * T(q.i[c]);
        }
        FieldIO<PR>::store(S->slot[SL_Y], vh, i, y);
        const Vec3<T> rs = FieldIO<PR>::store(S->slot[SL_R], vh, i, r);
        T m = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) m += rs.r[c] * rs.r[c] + rs.i[c] * rs.i[c];
        n = double(m);
    }
    __shared__ double sm[32];
    const double b = block_sum<kBlock>(n, sm);
    if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * a.pstride + blockIdx.x] = b;
}

// d = r + beta d
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_slab_xpay(const VecArgs a)
{
    const CGState *st = a.state;
    if (st->flag != FLAG_RUN) return;
    typedef typename Real<PR>::T T;
    typedef typename Real<PD>::T TD;
    const SlabDev *S = a.sl + blockIdx.y;
    const int vh = a.vh;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= vh) return;
    const T beta = T(st->beta);
    const Vec3<T> r = FieldIO<PR>::load(S->slot[SL_R], vh, i);
    const auto d = FieldIO<PD>::load(S->slot[SL_D], vh, i);
    Vec3<TD> o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o.r[c] = TD(r.r[c] + beta * T(d.r[c]));
        o.i[c] = TD(r.i[c] + beta * T(d.i[c]));
    }
    FieldIO<PD>::store(S->slot[SL_D], vh, i, o);
}

// start or restart of the inner iteration (Fig. 2, Eq. 6): y = 0, r = r64 in
// PR, d = r + beta d (beta = 0: d = r)
template <int PD, int PR>
__global__ void __launch_bounds__(kBlock) k_slab_reset(const VecArgs a, double beta)
{
    typedef typename Real<PR>::T T;
    typedef typename Real<PD>::T TD;
    const SlabDev *S = a.sl + blockIdx.y;
    const int vh = a.vh;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= vh) return;
    const Vec3<double> r64 = FieldIO<P64>::load(S->slot[SL_R64], vh, i);
    Vec3<T> r, z;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r.r[c] = T(r64.r[c]);
        r.i[c] = T(r64.i[c]);
        z.r[c] = z.i[c] = T(0);
    }
    FieldIO<PR>::store(S->slot[SL_Y], vh, i, z);
    const Vec3<T> rs = FieldIO<PR>::store(S->slot[SL_R], vh, i, r);
    Vec3<TD> o;
    if (beta != 0.0) {
        const auto d = FieldIO<PD>::load(S->slot[SL_D], vh, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = TD(rs.r[c] + T(beta) * T(d.r[c]));
            o.i[c] = TD(rs.i[c] + T(beta) * T(d.i[c]));
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = TD(rs.r[c]);
            o.i[c] = TD(rs.i[c]);
        }
    }
    FieldIO<PD>::store(S->slot[SL_D], vh, i, o);
}

// x64 += y (the Sec. 3.2 update: x_{k+1} = x_k + y in FP64)
template <int PR>
__global__ void __launch_bounds__(kBlock) k_slab_accumulate(const VecArgs a)
{
    const SlabDev *S = a.sl + blockIdx.y;
    const int vh = a.vh;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= vh) return;
    Vec3<double> x = FieldIO<P64>::load(S->slot[SL_X64], vh, i);
    const auto y = FieldIO<PR>::load(S->slot[SL_Y], vh, i);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        x.r[c] += double(y.r[c]);
        x.i[c] += double(y.i[c]);
    }
    FieldIO<P64>::store(S->slot[SL_X64], vh, i, x);
}

// |slot|^2 partials of an FP64 slot
__global__ void __launch_bounds__(kBlock) k_slab_norm(const VecArgs a, int slot)
{
    const SlabDev *S = a.sl + blockIdx.y;
    const int vh = a.vh;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    double n = 0.0;
    if (i < vh) {
        const Vec3<double> v = FieldIO<P64>::load(S->slot[slot], vh, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) n += v.r[c] * v.r[c] + v.i[c] * v.i[c];
    }
    __shared__ double sm[32];
    const double b = block_sum<kBlock>(n, sm);
    if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * a.pstride + blockIdx.x] = b;
}

enum SumUse { SUM_OUT = 0, SUM_ALPHA = 1, SUM_BETA = 2 };

// One block: each slab's n partials in a fixed order, then the slab totals
// in slab order.  SUM_ALPHA: alpha = delta / d^dag A d (set_alpha);
// SUM_BETA: the update's |r|^2, beta, the stop tests of Fig. 1 and the
// reliable-update trigger of Sec. 3.2 (|r|^2 < delta^2 max |r|^2);
// SUM_OUT: *out = total.
__global__ void __launch_bounds__(kBlock) k_slab_sum(const double *partials, int pstride, int n, int nslabs,
                                                     int use, CGState *st, double *out)
{
    if (use != SUM_OUT && st->flag != FLAG_RUN) return;  // uniform
    __shared__ double sm[32];
    double total = 0.0;
    for (int r = 0; r < nslabs; ++r) {
        double acc = 0.0;
        for (int k = threadIdx.x; k < n; k += kBlock) acc += partials[(size_t)r * pstride + k];
        const double sr = block_sum<kBlock>(acc, sm);
        total += sr;  // meaningful in thread 0
    }
    if (threadIdx.x != 0) return;
    if (use == SUM_OUT) {
        *out = total;
    } else if (use == SUM_ALPHA) {
        set_alpha(st, total);
    } else {
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct SlScope {
    int prev = -1, want;
    explicit SlScope(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~SlScope()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

}  // namespace stg

using namespace stg;

struct stg_slabs {
    int device = 0;
    int dims[4] = {0, 0, 0, 0};
    int P = 0, prec = 0, recon = 18;
    Geom g;                          // local lattice (Lx, Ly, Lz, Lt / P)
    std::vector<LinkField> links;    // [P], in prec / recon
    std::vector<LinkField> links64;  // [P], FP64 / 18-real, when prec is not FP64
    char *ghost = nullptr;           // [P][2 output parities] ghost t-links
    size_t ghost_bytes = 0;
    char *ghost64 = nullptr;         // the same for links64
    size_t ghost64_bytes = 0;
    char *fields = nullptr;          // [P][kSlabSlots], 48 bytes per site each
    size_t field_bytes = 0;
    char *faces = nullptr;           // [P][send 0, send 1, recv 0, recv 1], 48 bytes per face site
    size_t face_stride = 0;
    double *partials = nullptr;      // [P][pstride]
    int pstride = 0, nb_int = 0, nb_bnd = 0, nb_site = 0;
    SlabDev *dev = nullptr;          // [P]
    CGState *state = nullptr, *state_host = nullptr;
    int mode = STG_SLAB_COPY, overlap = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_t[2] = {nullptr, nullptr};
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0, graph_mode = -1, graph_overlap = -1;
    cudaStream_t graph_stream = nullptr;

    char *field(int r, int slot) const { return fields + ((size_t)r * kSlabSlots + slot) * field_bytes; }
    char *face(int r, int k) const { return faces + ((size_t)r * 4 + k) * face_stride; }
    int prev(int r) const { return (r + P - 1) % P; }
    int next(int r) const { return (r + 1) % P; }
};

namespace stg {

static void sl_free(stg_slabs *h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (LinkField &lf : h->links)
        if (lf.base) cudaFree(lf.base);
    for (LinkField &lf : h->links64)
        if (lf.base) cudaFree(lf.base);
    cudaFree(h->ghost);
    cudaFree(h->ghost64);
    cudaFree(h->fields);
    cudaFree(h->faces);
    cudaFree(h->partials);
    cudaFree(h->dev);
    cudaFree(h->state);
    if (h->state_host) cudaFreeHost(h->state_host);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (cudaEvent_t e : h->ev_t)
        if (e) cudaEventDestroy(e);
    delete h;
}

static stg_status sl_alloc(void **p, size_t n)
{
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error("stg_slabs: device allocation failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    return STG_OK;
}

struct SlabShape {
    Geom g;
    int st, nb_int, nb_bnd, nb_site, pstride;
    size_t link_blk, ghost_bytes, link64_blk, ghost64_bytes, field_bytes, face_stride;
};

static SlabShape slab_shape(const int dims[4], int P, int prec, int recon)
{
    SlabShape s;
    const int ld[4] = {dims[0], dims[1], dims[2], dims[3] / P};
    s.g = make_geom(ld);
    s.st = s.g.st;
    const int lts = ld[3];
    s.nb_int = (int)(((long)(lts - 2) * s.st + kBlock - 1) / kBlock);
    s.nb_bnd = (int)((2L * s.st + kBlock - 1) / kBlock);
    s.nb_site = (int)(((long)s.g.Vh + kBlock - 1) / kBlock);
    s.pstride = s.nb_int + s.nb_bnd > s.nb_site ? s.nb_int + s.nb_bnd : s.nb_site;
    s.link_blk = sl_align((size_t)s.g.Vh * link_bytes(prec, recon));
    s.ghost_bytes = sl_align((size_t)s.st * link_bytes(prec, recon));
    s.link64_blk = prec == P64 ? 0 : sl_align((size_t)s.g.Vh * link_bytes(P64, 18));
    s.ghost64_bytes = prec == P64 ? 0 : sl_align((size_t)s.st * link_bytes(P64, 18));
    s.field_bytes = sl_align((size_t)s.g.Vh * 48);
    s.face_stride = sl_align((size_t)s.st * 48);
    return s;
}

static size_t slabs_bytes(const int dims[4], int P, int prec, int recon)
{
    const SlabShape s = slab_shape(dims, P, prec, recon);
    size_t n = (size_t)P * 8 * s.link_blk;                  // links
    n += (size_t)P * 2 * s.ghost_bytes;                      // ghost t-links
    n += (size_t)P * (8 * s.link64_blk + 2 * s.ghost64_bytes);  // FP64 links of the CG's residual
    n += (size_t)P * kSlabSlots * s.field_bytes;             // fields
    n += (size_t)P * 4 * s.face_stride;                      // faces
    n += sl_align((size_t)P * s.pstride * sizeof(double));   // partials
    n += sl_align((size_t)P * sizeof(SlabDev)) + sl_align(sizeof(CGState));
    return n;
}

// ---------------------------------------------------------------------------
// one Dirac operation: collect, exchange, the slabs' Dslash
// ---------------------------------------------------------------------------
static stg_status sl_collect(stg_slabs *h, int slot, int prec, int direct, cudaStream_t s)
{
    CollectArgs c;
    c.sl = h->dev;
    c.slot = slot;
    c.vh = h->g.Vh;
    c.st = h->g.st;
    c.lts = h->g.L[3];
    c.np = field_planes(prec, c.e);
    c.words = (int)((size_t)h->g.st * field_site_bytes(prec) / 8);
    c.direct = direct;
    const dim3 grid((unsigned)((2L * c.words + kBlock - 1) / kBlock), (unsigned)h->P);
    k_slab_collect<<<grid, kBlock, 0, s>>>(c);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// COPY mode: slab r's slice 0 -> previous slab's forward ghost, its slice
// Lts - 1 -> next slab's backward ghost (one copy per face and neighbour)
static stg_status sl_exchange(stg_slabs *h, int prec, cudaStream_t s)
{
    const size_t bytes = (size_t)h->g.st * field_site_bytes(prec);
    for (int r = 0; r < h->P; ++r) {
        STG_CUDA(cudaMemcpyAsync(h->face(h->prev(r), 2), h->face(r, 0), bytes, cudaMemcpyDeviceToDevice, s));
        STG_CUDA(cudaMemcpyAsync(h->face(h->next(r), 3), h->face(r, 1), bytes, cudaMemcpyDeviceToDevice, s));
    }
    return STG_OK;
}

static stg_status sl_halo(stg_slabs *h, int slot, int prec, cudaStream_t s)
{
    STG_TRY(sl_collect(h, slot, prec, h->mode == STG_SLAB_DIRECT, s));
    if (h->mode == STG_SLAB_COPY) STG_TRY(sl_exchange(h, prec, s));
    return STG_OK;
}

// EPI_NONE / EPI_A_DOT for every precision; the CG's epilogues for the
// precisions it runs in (FP64, FP32, FX16)
template <int P, int R>
static void sl_launch_pr(int epi, dim3 grid, cudaStream_t s, const SlabArgs &a)
{
    switch (epi) {
    case EPI_NONE: k_slab_dslash<P, R, EPI_NONE><<<grid, kBlock, 0, s>>>(a); break;
    case EPI_A_DOT: k_slab_dslash<P, R, EPI_A_DOT><<<grid, kBlock, 0, s>>>(a); break;
    default:
        if constexpr (P == P64 || P == P32 || P == PX16) {
            if (epi == EPI_GATE) k_slab_dslash<P, R, EPI_GATE><<<grid, kBlock, 0, s>>>(a);
            else if (epi == EPI_A_CG) k_slab_dslash<P, R, EPI_A_CG><<<grid, kBlock, 0, s>>>(a);
        }
        if constexpr (P == P64) {
            if (epi == EPI_RES) k_slab_dslash<P, R, EPI_RES><<<grid, kBlock, 0, s>>>(a);
        }
        break;
    }
}

// part 0: interior slices (none when Lts = 2); part 1: slices 0 and Lts - 1;
// part 2: both in one launch
static stg_status sl_part(stg_slabs *h, int epi, SlabArgs a, int part, cudaStream_t s)
{
    const int nb = part == 2 ? h->nb_int + h->nb_bnd : (part ? h->nb_bnd : h->nb_int);
    if (nb == 0) return STG_OK;
    a.part = part;
    a.pbase = part == 1 ? h->nb_int : 0;
    a.nb_int = h->nb_int;
    const dim3 grid((unsigned)nb, (unsigned)h->P);
    const bool r12 = a.recon == 12;
    switch (a.prec) {
    case P64: if (r12) sl_launch_pr<P64, 12>(epi, grid, s, a); else sl_launch_pr<P64, 18>(epi, grid, s, a); break;
    case P32: if (r12) sl_launch_pr<P32, 12>(epi, grid, s, a); else sl_launch_pr<P32, 18>(epi, grid, s, a); break;
    case P16: if (r12) sl_launch_pr<P16, 12>(epi, grid, s, a); else sl_launch_pr<P16, 18>(epi, grid, s, a); break;
    case PB16: if (r12) sl_launch_pr<PB16, 12>(epi, grid, s, a); else sl_launch_pr<PB16, 18>(epi, grid, s, a); break;
    default: if (r12) sl_launch_pr<PX16, 12>(epi, grid, s, a); else sl_launch_pr<PX16, 18>(epi, grid, s, a); break;
    }
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

static SlabArgs sl_args(const stg_slabs *h, int parity, int in, int out, int w, int v, double m2)
{
    SlabArgs a;
    a.g = h->g;
    a.sl = h->dev;
    a.parity = parity;
    a.in = in;
    a.out = out;
    a.w = w;
    a.v = v;
    a.m2 = m2;
    a.state = h->state;
    a.partials = h->partials;
    a.pstride = h->pstride;
    a.pbase = 0;
    a.part = 0;
    a.nb_int = h->nb_int;
    a.prec = h->prec;
    a.recon = h->recon;
    a.hi = 0;
    return a;
}

// the same on the FP64 links (the FP64 / 18-real copy when the handle's
// links are in another precision)
static SlabArgs sl_args64(const stg_slabs *h, int parity, int in, int out, int w, int v, double m2)
{
    SlabArgs a = sl_args(h, parity, in, out, w, v, m2);
    a.prec = P64;
    if (h->prec != P64) {
        a.recon = 18;
        a.hi = 1;
    }
    return a;
}

static stg_status sl_dirac(stg_slabs *h, int epi, const SlabArgs &a, cudaStream_t s)
{
    if (h->overlap) {
        STG_CUDA(cudaEventRecord(h->ev_fork, s));
        STG_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        STG_TRY(sl_halo(h, a.in, a.prec, h->side));
        STG_CUDA(cudaEventRecord(h->ev_join, h->side));
        STG_TRY(sl_part(h, epi, a, 0, s));
        STG_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
        return sl_part(h, epi, a, 1, s);
    }
    STG_TRY(sl_halo(h, a.in, a.prec, s));
    return sl_part(h, epi, a, 2, s);
}

static stg_status sl_sum(stg_slabs *h, int n, int use, double *out, cudaStream_t s)
{
    k_slab_sum<<<1, kBlock, 0, s>>>(h->partials, h->pstride, n, h->P, use, h->state, out);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

static stg_status sl_read_state(stg_slabs *h, cudaStream_t s)
{
    STG_CUDA(cudaMemcpyAsync(h->state_host, h->state, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    STG_CUDA(cudaStreamSynchronize(s));
    return STG_OK;
}

static stg_status sl_write_state(stg_slabs *h, cudaStream_t s)
{
    STG_CUDA(cudaMemcpyAsync(h->state, h->state_host, sizeof(CGState), cudaMemcpyHostToDevice, s));
    return STG_OK;
}

}  // namespace stg

namespace stg {

// ---------------------------------------------------------------------------
// CG on the decomposed operator: Fig. 1 in FP64 for FP64 handles; for FP32 /
// FX16 handles, inner iterations in that precision with the reliable
// updates of Sec. 3.2 (x += y and r = b - A x with the FP64 links) and the
// restart of Eq. 6
// ---------------------------------------------------------------------------
static VecArgs sl_vec(const stg_slabs *h)
{
    VecArgs v;
    v.sl = h->dev;
    v.vh = h->g.Vh;
    v.state = h->state;
    v.partials = h->partials;
    v.pstride = h->pstride;
    return v;
}

#define SL_DISPATCH_PD(pd, KERNEL, ...)                                                          \
    do {                                                                                         \
        if ((pd) == P64) KERNEL<P64, P64><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                  \
        else if ((pd) == P32) KERNEL<P32, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);             \
        else KERNEL<PX16, P32><<<grid, kBlock, 0, s>>>(__VA_ARGS__);                             \
    } while (0)

// one inner iteration: t = D_oe d; q = m^2 d - D_eo t, d^dag q -> alpha;
// y, r update with |r|^2 -> beta and the stop / update tests; d = r + beta d
static stg_status sl_iteration(stg_slabs *h, cudaStream_t s)
{
    STG_TRY(sl_dirac(h, EPI_GATE, sl_args(h, 1, SL_D, SL_T, -1, -1, 0.0), s));
    STG_TRY(sl_dirac(h, EPI_A_CG, sl_args(h, 0, SL_T, SL_Q, SL_D, -1, 0.0), s));
    STG_TRY(sl_sum(h, h->nb_int + h->nb_bnd, SUM_ALPHA, nullptr, s));
    const VecArgs v = sl_vec(h);
    const dim3 grid((unsigned)h->nb_site, (unsigned)h->P);
    SL_DISPATCH_PD(h->prec, k_slab_update, v);
    STG_CUDA(cudaGetLastError());
    STG_TRY(sl_sum(h, h->nb_site, SUM_BETA, nullptr, s));
    SL_DISPATCH_PD(h->prec, k_slab_xpay, v);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// launches per iteration: 2 x (collect + the slabs' Dslash: one launch, or
// interior + boundary when overlapped) + 2 sums + update + xpay, plus
// 2 x 2P copies in COPY mode
static long sl_iteration_launches(const stg_slabs *h)
{
    return 2L * (1 + (h->overlap && h->nb_int ? 2 : 1)) + 4;
}

static stg_status sl_graph(stg_slabs *h, int iters)
{
    if (h->graph && h->graph_iters == iters && h->graph_mode == h->mode && h->graph_overlap == h->overlap)
        return STG_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaStream_t cs;
    STG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    stg_status st = STG_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < iters && st == STG_OK; ++k) st = sl_iteration(h, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == STG_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (st == STG_OK) {
        e = cudaGraphInstantiate(&h->graph, graph, 0);
        if (e != cudaSuccess) {
            h->graph = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != STG_OK) return st;
    h->graph_iters = iters;
    h->graph_mode = h->mode;
    h->graph_overlap = h->overlap;
    return STG_OK;
}

// r64 = b - A x64 with the FP64 links, |r64|^2 into state->result
static stg_status sl_true_residual(stg_slabs *h, double m2, cudaStream_t s, double *rr)
{
    STG_TRY(sl_dirac(h, EPI_NONE, sl_args64(h, 1, SL_X64, SL_T64, -1, -1, 0.0), s));
    STG_TRY(sl_dirac(h, EPI_RES, sl_args64(h, 0, SL_T64, SL_R64, SL_B64, SL_X64, m2), s));
    STG_TRY(sl_sum(h, h->nb_int + h->nb_bnd, SUM_OUT, &h->state->result, s));
    STG_TRY(sl_read_state(h, s));
    *rr = h->state_host->result;
    return STG_OK;
}

static stg_status sl_norm64(stg_slabs *h, int slot, cudaStream_t s, double *nn)
{
    const dim3 grid((unsigned)h->nb_site, (unsigned)h->P);
    k_slab_norm<<<grid, kBlock, 0, s>>>(sl_vec(h), slot);
    STG_CUDA(cudaGetLastError());
    STG_TRY(sl_sum(h, h->nb_site, SUM_OUT, &h->state->result, s));
    STG_TRY(sl_read_state(h, s));
    *nn = h->state_host->result;
    return STG_OK;
}

static stg_status sl_load(stg_slabs *h, int slot, int prec, const double *canon, cudaStream_t s)
{
    for (int r = 0; r < h->P; ++r)
        STG_TRY(pack_field(h->g, prec, canon + (size_t)r * h->g.Vh * 6, h->field(r, slot), s));
    return STG_OK;
}

static stg_status sl_store(stg_slabs *h, int slot, int prec, double *canon, cudaStream_t s)
{
    for (int r = 0; r < h->P; ++r)
        STG_TRY(unpack_field(h->g, prec, h->field(r, slot), canon + (size_t)r * h->g.Vh * 6, s));
    return STG_OK;
}

static stg_status sl_cg(stg_slabs *h, const double *src, double *x, double mass, double tol, long maxiter,
                        double delta, stg_cg_stats *stats, cudaStream_t s)
{
    timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    stg_cg_stats st = {};
    const bool plain = h->prec == P64;
    const int pr = slab_pr(h->prec);
    const double m2 = mass * mass;
    const long vh_total = (long)h->g.Vh * h->P;
    if (maxiter <= 0) maxiter = 10L * 3L * vh_total;
    const int chunk = vh_total >= (1L << 19) ? 16 : 32;
    const dim3 grid((unsigned)h->nb_site, (unsigned)h->P);
    STG_TRY(sl_load(h, SL_B64, P64, src, s));
    STG_TRY(sl_load(h, SL_X64, P64, x, s));
    double bb = 0.0, rr = 0.0;
    STG_TRY(sl_norm64(h, SL_B64, s, &bb));
    if (!isfinite(bb)) {
        set_error("stg_slabs_cg_solve: the source has non-finite entries");
        return STG_ERR_INVALID_ARG;
    }
    if (bb == 0.0) {
        STG_CUDA(cudaMemsetAsync(x, 0, (size_t)vh_total * 48, s));
        STG_CUDA(cudaStreamSynchronize(s));
        if (stats) *stats = st;
        return STG_OK;
    }
    const double stop = tol * tol * bb;
    STG_TRY(sl_true_residual(h, m2, s, &rr));
    if (!isfinite(rr)) {
        set_error("stg_slabs_cg_solve: non-finite residual of the initial guess");
        return STG_ERR_INVALID_ARG;
    }
    long launches = 2L * h->P + 2 + 6 + 2;  // loads, norm, residual
    stg_status status = STG_OK;
    CGState *hs = h->state_host;
    int breakdowns = 0;
    long long iters = 0;
    double beta = 0.0;
    while (status == STG_OK && rr > stop) {
        // (re)start: y = 0, r = r64, d = r + beta d (Fig. 2; Eq. 6)
        SL_DISPATCH_PD(h->prec, k_slab_reset, sl_vec(h), beta);
        STG_CUDA(cudaGetLastError());
        launches += 1;
        hs->delta_new = rr;
        hs->delta_old = rr;
        hs->rmax2 = rr;
        hs->stop_r2 = stop;
        hs->trig2 = plain ? 0.0 : delta * delta;
        hs->track_max = plain ? 0 : 1;
        hs->m2 = m2;
        hs->iter = iters;
        hs->iter_limit = maxiter;
        hs->flag = FLAG_RUN;
        hs->counter = 0;
        status = sl_write_state(h, s);
        if (status == STG_OK) status = sl_graph(h, chunk);
        while (status == STG_OK) {
            cudaError_t e = cudaGraphLaunch(h->graph, s);
            if (e != cudaSuccess) {
                status = cuda_fail(e, "cudaGraphLaunch");
                break;
            }
            launches += (long)chunk * sl_iteration_launches(h);
            status = sl_read_state(h, s);
            if (status != STG_OK || hs->flag != FLAG_RUN) break;
        }
        if (status != STG_OK) break;
        const int flag = hs->flag;
        const double delta_old = hs->delta_old;
        iters = hs->iter;
        st.iter_res = sqrt(hs->delta_new / bb);
        // x_{k+1} = x_k + y, r_{k+1} = b - A x_{k+1} (Sec. 3.2)
        if (pr == P64) k_slab_accumulate<P64><<<grid, kBlock, 0, s>>>(sl_vec(h));
        else k_slab_accumulate<P32><<<grid, kBlock, 0, s>>>(sl_vec(h));
        STG_CUDA(cudaGetLastError());
        status = sl_true_residual(h, m2, s, &rr);
        launches += 1 + 2 * 3 + 1;
        st.updates += 1;
        if (status != STG_OK || rr <= stop) break;
        if (!isfinite(rr)) {
            set_error("stg_slabs_cg_solve: non-finite true residual");
            status = STG_ERR_BREAKDOWN;
            break;
        }
        if (iters >= maxiter) {
            set_error("stg_slabs_cg_solve: maxiter reached before convergence");
            status = STG_ERR_NOT_CONVERGED;
            break;
        }
        beta = 0.0;
        if (flag == FLAG_BREAKDOWN) {
            if (++breakdowns > 3) {
                set_error("stg_slabs_cg_solve: d^dag A d <= 0 or non-finite reduction");
                status = STG_ERR_BREAKDOWN;
                break;
            }
        } else if (!plain) {
            beta = rr / delta_old;  // Eq. 6: d^y_0 = r + beta d, d kept
        }
    }
    if (status == STG_OK || status == STG_ERR_NOT_CONVERGED) {
        stg_status u = sl_store(h, SL_X64, P64, x, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (u != STG_OK) status = u;
        else if (e != cudaSuccess) status = cuda_fail(e, "cudaStreamSynchronize");
        launches += h->P;
    }
    st.iters = (long)iters;
    st.sloppy_iters = plain ? 0 : (long)iters;
    st.true_res = sqrt(rr / bb);
    if (st.updates == 0) st.iter_res = st.true_res;
    st.launches = launches;
    clock_gettime(CLOCK_MONOTONIC, &t1);
    st.seconds = (t1.tv_sec - t0.tv_sec) + 1e-9 * (t1.tv_nsec - t0.tv_nsec);
    if (stats) *stats = st;
    return status;
}

// ---------------------------------------------------------------------------
// Table 1 breakdown of one Dirac operation
// ---------------------------------------------------------------------------
static stg_status sl_profile(stg_slabs *h, int reps, double ms[4], cudaStream_t s)
{
    if (!h->ev_t[0])
        for (int k = 0; k < 2; ++k) STG_CUDA(cudaEventCreate(&h->ev_t[k]));
    const SlabArgs a = sl_args(h, 1, 0, SL_T, -1, -1, 0.0);
    float t = 0.f;
    for (int phase = 0; phase < 4; ++phase) {
        for (int round = 0; round < 2; ++round) {  // round 0 warms up
            const int n = round ? reps : 1;
            if (round) STG_CUDA(cudaEventRecord(h->ev_t[0], s));
            for (int k = 0; k < n; ++k) {
                if (phase == 0) {
                    STG_TRY(sl_collect(h, a.in, h->prec, h->mode == STG_SLAB_DIRECT, s));
                } else if (phase == 1) {
                    if (h->mode == STG_SLAB_COPY) STG_TRY(sl_exchange(h, h->prec, s));
                } else if (phase == 2) {
                    STG_TRY(sl_part(h, EPI_NONE, a, 2, s));
                } else {
                    STG_TRY(sl_dirac(h, EPI_NONE, a, s));
                }
            }
            if (round) {
                STG_CUDA(cudaEventRecord(h->ev_t[1], s));
                STG_CUDA(cudaEventSynchronize(h->ev_t[1]));
                STG_CUDA(cudaEventElapsedTime(&t, h->ev_t[0], h->ev_t[1]));
                ms[phase] = (phase == 1 && h->mode != STG_SLAB_COPY) ? 0.0 : (double)t / reps;
            }
        }
    }
    STG_CUDA(cudaStreamSynchronize(s));
    return STG_OK;
}

}  // namespace stg

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

stg_status stg_slabs_create(const int dims[4], const double *links_host, int nslabs, stg_prec prec, int recon,
                            stg_stream_t stream, stg_slabs **out)
{
    if (!out || !dims || !links_host) {
        set_error("stg_slabs_create: NULL argument");
        return STG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (prec != STG_FP64 && prec != STG_FP32 && prec != STG_FP16 && prec != STG_FX16 && prec != STG_BF16) {
        set_error("stg_slabs_create: unknown precision");
        return STG_ERR_INVALID_ARG;
    }
    if (recon != 12 && recon != 18) {
        set_error("stg_slabs_create: recon must be 12 or 18");
        return STG_ERR_INVALID_ARG;
    }
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] <= 0 || (dims[mu] & 1)) {
            set_error("stg_slabs_create: every extent must be even and positive");
            return STG_ERR_DIMS;
        }
    }
    if ((long)dims[0] * dims[1] * dims[2] * dims[3] / 2 > (1L << 30)) {
        set_error("stg_slabs_create: lattice too large");
        return STG_ERR_DIMS;
    }
    if (nslabs < 1 || nslabs > kMaxSlabs || dims[3] % nslabs != 0 || (dims[3] / nslabs) % 2 != 0) {
        set_error("stg_slabs_create: nslabs must be 1..64 and divide Lt into slabs of an even number of "
                  "time slices");
        return STG_ERR_DIMS;
    }
    stg_slabs *h = new (std::nothrow) stg_slabs();
    if (!h) {
        set_error("stg_slabs_create: host allocation failed");
        return STG_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    for (int mu = 0; mu < 4; ++mu) h->dims[mu] = dims[mu];
    h->P = nslabs;
    h->prec = prec;
    h->recon = recon;
    const SlabShape sh = slab_shape(dims, nslabs, prec, recon);
    h->g = sh.g;
    h->ghost_bytes = sh.ghost_bytes;
    h->ghost64_bytes = sh.ghost64_bytes;
    h->field_bytes = sh.field_bytes;
    h->face_stride = sh.face_stride;
    h->nb_int = sh.nb_int;
    h->nb_bnd = sh.nb_bnd;
    h->nb_site = sh.nb_site;
    h->pstride = sh.pstride;
    h->links.resize(nslabs);
    if (prec != STG_FP64) h->links64.resize(nslabs);
    const int P = nslabs, lts = h->g.L[3], st_ = h->g.st;
    const size_t vh = (size_t)h->g.Vh;

    // links of each slab, packed with the global sign rule (t_flip)
    const size_t canon_bytes = vh * 2 * 4 * 9 * sizeof(double2);
    double2 *ucan = nullptr;
    stg_status st = sl_alloc((void **)&ucan, canon_bytes);
    for (int r = 0; r < P && st == STG_OK; ++r) {
        cudaError_t e = cudaMemcpyAsync(ucan, links_host + (size_t)r * (canon_bytes / sizeof(double)), canon_bytes,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync(links)");
        const int t_flip = r == P - 1 ? lts - 1 : -1;
        if (st == STG_OK) st = pack_links_flip(h->g, ucan, prec, recon, t_flip, &h->links[r], s);
        if (st == STG_OK && prec != STG_FP64) st = pack_links_flip(h->g, ucan, P64, 18, t_flip, &h->links64[r], s);
        if (st == STG_OK) {
            e = cudaStreamSynchronize(s);  // the staging buffer is reused
            if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
        }
    }
    cudaFree(ucan);
    if (st == STG_OK) st = sl_alloc((void **)&h->ghost, (size_t)P * 2 * h->ghost_bytes);
    if (st == STG_OK && prec != STG_FP64) st = sl_alloc((void **)&h->ghost64, (size_t)P * 2 * h->ghost64_bytes);
    if (st == STG_OK) st = sl_alloc((void **)&h->fields, (size_t)P * kSlabSlots * h->field_bytes);
    if (st == STG_OK) st = sl_alloc((void **)&h->faces, (size_t)P * 4 * h->face_stride);
    if (st == STG_OK) st = sl_alloc((void **)&h->partials, (size_t)P * h->pstride * sizeof(double));
    if (st == STG_OK) st = sl_alloc((void **)&h->dev, (size_t)P * sizeof(SlabDev));
    if (st == STG_OK) st = sl_alloc((void **)&h->state, sizeof(CGState));
    if (st == STG_OK) {
        cudaError_t e = cudaMallocHost((void **)&h->state_host, sizeof(CGState));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->state, 0, sizeof(CGState), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->fields, 0, (size_t)P * kSlabSlots * h->field_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->faces, 0, (size_t)P * 4 * h->face_stride, s);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) st = cuda_fail(e, "stg_slabs_create");
    }
    // ghost t-links: for output parity p, the previous slab's block (1 - p, t)
    // at its last slice, plane by plane (planes of stride st); for each link set
    for (int set = 0; set < (prec != STG_FP64 ? 2 : 1); ++set) {
        const std::vector<LinkField> &lk = set ? h->links64 : h->links;
        char *ghost = set ? h->ghost64 : h->ghost;
        const size_t gbytes = set ? h->ghost64_bytes : h->ghost_bytes;
        int le[9];
        const int nlp = set ? link_planes(P64, 18, le) : link_planes(prec, recon, le);
        for (int r = 0; r < P && st == STG_OK; ++r) {
            for (int p = 0; p < 2 && st == STG_OK; ++p) {
                const char *src = lk[h->prev(r)].blk(1 - p, 3);
                char *dst = ghost + ((size_t)r * 2 + p) * gbytes;
                size_t off_src = 0, off_dst = 0;
                for (int k = 0; k < nlp && st == STG_OK; ++k) {
                    const size_t n = (size_t)st_ * le[k];
                    cudaError_t e = cudaMemcpyAsync(dst + off_dst, src + off_src + (size_t)(lts - 1) * n, n,
                                                    cudaMemcpyDeviceToDevice, s);
                    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync(ghost links)");
                    off_src += vh * le[k];
                    off_dst += n;
                }
            }
        }
    }
    if (st == STG_OK) {
        std::vector<SlabDev> t(P);
        for (int r = 0; r < P; ++r) {
            SlabDev &d = t[r];
            memset(&d, 0, sizeof(d));
            for (int k = 0; k < 8; ++k) d.lk[k] = h->links[r].blk(k / 4, k % 4);
            for (int p = 0; p < 2; ++p) d.ghost_lk[p] = h->ghost + ((size_t)r * 2 + p) * h->ghost_bytes;
            for (int k = 0; k < 8; ++k) d.lk64[k] = prec != STG_FP64 ? h->links64[r].blk(k / 4, k % 4) : d.lk[k];
            for (int p = 0; p < 2; ++p)
                d.ghost64[p] = prec != STG_FP64 ? h->ghost64 + ((size_t)r * 2 + p) * h->ghost64_bytes : d.ghost_lk[p];
            for (int k = 0; k < kSlabSlots; ++k) d.slot[k] = h->field(r, k);
            d.send[0] = h->face(r, 0);
            d.send[1] = h->face(r, 1);
            d.recv[0] = h->face(r, 2);
            d.recv[1] = h->face(r, 3);
            d.peer[0] = h->face(h->prev(r), 2);
            d.peer[1] = h->face(h->next(r), 3);
            d.top = (r == P - 1) ? -1.f : 1.f;
            d.bot = (r == 0) ? -1.f : 1.f;
        }
        cudaError_t e = cudaMemcpyAsync(h->dev, t.data(), (size_t)P * sizeof(SlabDev), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "stg_slabs_create");
    }
    if (st != STG_OK) {
        cudaStreamSynchronize(s);
        sl_free(h);
        return st;
    }
    *out = h;
    return STG_OK;
}

stg_status stg_slabs_destroy(stg_slabs *h)
{
    if (!h) return STG_OK;
    SlScope ds(h->device);
    cudaDeviceSynchronize();
    sl_free(h);
    return STG_OK;
}

stg_status stg_slabs_set_exchange(stg_slabs *h, int mode, int overlap)
{
    if (!h || (mode != STG_SLAB_COPY && mode != STG_SLAB_DIRECT) || (overlap != 0 && overlap != 1)) {
        set_error("stg_slabs_set_exchange: NULL handle, mode not COPY / DIRECT or overlap not 0 / 1");
        return STG_ERR_INVALID_ARG;
    }
    h->mode = mode;
    h->overlap = overlap;
    return STG_OK;
}

stg_status stg_slabs_load(stg_slabs *h, int slot, const double *canon_dev, stg_stream_t stream)
{
    if (!h || !canon_dev || slot < 0 || slot >= kUserSlots) {
        set_error("stg_slabs_load: NULL argument or slot outside 0..5");
        return STG_ERR_INVALID_ARG;
    }
    SlScope ds(h->device);
    return sl_load(h, slot, h->prec, canon_dev, (cudaStream_t)stream);
}

stg_status stg_slabs_store(stg_slabs *h, int slot, double *canon_dev, stg_stream_t stream)
{
    if (!h || !canon_dev || slot < 0 || slot >= kUserSlots) {
        set_error("stg_slabs_store: NULL argument or slot outside 0..5");
        return STG_ERR_INVALID_ARG;
    }
    SlScope ds(h->device);
    return sl_store(h, slot, h->prec, canon_dev, (cudaStream_t)stream);
}

stg_status stg_slabs_dslash(stg_slabs *h, int out_parity, int in_slot, int out_slot, stg_stream_t stream)
{
    if (!h || (out_parity != 0 && out_parity != 1) || in_slot < 0 || in_slot >= kUserSlots || out_slot < 0 ||
        out_slot >= kUserSlots || in_slot == out_slot) {
        set_error("stg_slabs_dslash: NULL handle, parity not 0 / 1, or slots outside 0..5 or equal");
        return STG_ERR_INVALID_ARG;
    }
    SlScope ds(h->device);
    return sl_dirac(h, EPI_NONE, sl_args(h, out_parity, in_slot, out_slot, -1, -1, 0.0), (cudaStream_t)stream);
}

stg_status stg_slabs_apply_A_dot(stg_slabs *h, double mass, int in_slot, int out_slot, double *dot_dev,
                                 stg_stream_t stream)
{
    if (!h || !dot_dev || in_slot < 0 || in_slot >= kUserSlots || out_slot < 0 || out_slot >= kUserSlots ||
        in_slot == out_slot || in_slot == SL_T || out_slot == SL_T || !isfinite(mass)) {
        set_error("stg_slabs_apply_A_dot: NULL argument, non-finite mass, or slots outside 0..5, equal, "
                  "or slot 4 (the odd intermediate)");
        return STG_ERR_INVALID_ARG;
    }
    SlScope ds(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    STG_TRY(sl_dirac(h, EPI_NONE, sl_args(h, 1, in_slot, SL_T, -1, -1, 0.0), s));
    STG_TRY(sl_dirac(h, EPI_A_DOT, sl_args(h, 0, SL_T, out_slot, in_slot, -1, mass * mass), s));
    return sl_sum(h, h->nb_int + h->nb_bnd, SUM_OUT, dot_dev, s);
}

stg_status stg_slabs_cg_solve(stg_slabs *h, const double *src_dev, double *x_dev, double mass, double tol,
                              long maxiter, stg_cg_stats *stats, stg_stream_t stream)
{
    if (stats) *stats = stg_cg_stats{};
    if (!h || !src_dev || !x_dev || src_dev == x_dev) {
        set_error("stg_slabs_cg_solve: NULL handle / pointer or src == x");
        return STG_ERR_INVALID_ARG;
    }
    if (!isfinite(mass) || mass < 0.0 || !isfinite(tol) || !(tol > 0.0) || maxiter < 0) {
        set_error("stg_slabs_cg_solve: mass must be finite and >= 0, tol finite and > 0, maxiter >= 0");
        return STG_ERR_INVALID_ARG;
    }
    if (h->prec != STG_FP64 && h->prec != STG_FP32 && h->prec != STG_FX16) {
        set_error("stg_slabs_cg_solve: the decomposed CG runs with FP64, FP32 or FX16 slabs");
        return STG_ERR_UNSUPPORTED;
    }
    // the reliable-update threshold of stg_cg_params_default for the precision
    const double delta = h->prec == STG_FP32 ? 0.05 : 0.25;
    SlScope ds(h->device);
    return sl_cg(h, src_dev, x_dev, mass, tol, maxiter, delta, stats, (cudaStream_t)stream);
}

stg_status stg_slabs_profile(stg_slabs *h, int reps, double ms[4], stg_stream_t stream)
{
    if (!h || !ms || reps < 1) {
        set_error("stg_slabs_profile: NULL argument or reps < 1");
        return STG_ERR_INVALID_ARG;
    }
    SlScope ds(h->device);
    return sl_profile(h, reps, ms, (cudaStream_t)stream);
}

size_t stg_slabs_bytes(const int dims[4], int nslabs, stg_prec prec, int recon)
{
    if (!dims || nslabs < 1 || nslabs > kMaxSlabs || (recon != 12 && recon != 18) || prec < STG_FP64 ||
        prec > STG_BF16)
        return 0;
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] <= 0 || (dims[mu] & 1)) return 0;
    if (dims[3] % nslabs != 0 || (dims[3] / nslabs) % 2 != 0) return 0;
    return slabs_bytes(dims, nslabs, prec, recon);
}

}  // extern "C"
