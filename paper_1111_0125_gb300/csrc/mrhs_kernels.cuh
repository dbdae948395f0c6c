// Multi-right-hand-side Dslash (Eq. 5) and its fused A epilogue (Eq. 3).
//
// One gauge field, N colour-vector fields (N consecutive device fields of
// one precision).  Each thread owns one output site and walks the right-hand
// sides in register blocks of NB: the site's eight links are loaded (and
// decoded / rebuilt) once per block and applied to NB input fields, so the
// link bytes per site and right-hand side fall from 8L to 8L / NB while the
// field bytes stay 2S (3S with the fused epilogue).  With TPS threads per
// site the register block covers NB x TPS systems per link load.  (NB, TPS)
// comes from the autotuner in mrhs.cu.
//
// The right-hand sides processed are those of a device-side list (active,
// nactive) so that the host can drop converged systems between chunks
// without recapturing the CUDA graph; inside a chunk the per-system CG flag
// is checked as well.  The fused epilogue reduces d_k^dag q_k per system in
// compensated FP32 pairs (block partials per system, last block finishes all
// systems in a fixed order).
#pragma once

#include <stdlib.h>

#include "stg_internal.h"

namespace stg {

constexpr int kMaxRhs = 64;

struct MrhsArgs {
    Geom g;
    const char *lf[4];
    const char *lb[4];
    int parity;
    const char *in;
    char *out;
    const char *w;         // EPI_A / EPI_A_CG: the even inputs d
    size_t fstride;        // bytes between consecutive right-hand-side fields
    int nrhs;              // number of systems (slots)
    const int *active;     // device list of systems to process; NULL: all
    const int *nactive;    // device count for `active`
    CGState *states;       // per system (EPI_GATE, EPI_A_CG)
    float m2[kMaxRhs];     // EPI_A: m_k^2
    float2 *partials;      // EPI_A_CG: [nrhs][gridDim.x]
    unsigned *counter;     // EPI_A_CG: arrival counter
    int grid_cap;          // blocks launched at most (they stride over site tiles)
    int grid_limit;        // staged kernels: at most this many CTAs (0 = all resident;
                           // STG_MRHS_GRID, read per call, for tests)
    const char *lt;        // staged kernel: tile-major links of the output parity
};

constexpr int kMrhsBlock = 256;

// TPS threads share one site (consecutive lanes of a warp): they load the
// same link words, which the load unit merges into one request, so the
// links come from DRAM once per site for all systems; lane `sub` of the
// group handles systems sub, sub + TPS, ... in register blocks of NB.
template <int P, int R, int NB, int TPS, int EPI>
__global__ void __launch_bounds__(kMrhsBlock) k_dslash_m(const MrhsArgs a)
{
    constexpr int BS = kMrhsBlock;
    typedef typename Real<P>::T T;
    const int vh = a.g.Vh;
    const int sub = threadIdx.x % TPS;
    const int nact = a.active ? *a.nactive : a.nrhs;
    const int per = (nact + TPS - 1) / TPS;  // systems per lane (uniform bound)
    constexpr int kTile = BS / TPS;          // sites per tile
    const int ntiles = (vh + kTile - 1) / kTile;

    __shared__ float2 red[NB][TPS][BS / 32];
    __shared__ FF sys_acc[kMaxRhs];          // this block's d^dag q per list slot
    if (EPI == EPI_A_CG) {
        for (int k = threadIdx.x; k < kMaxRhs; k += BS) sys_acc[k].hi = sys_acc[k].lo = 0.f;
        __syncthreads();
    }

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i = tile * kTile + threadIdx.x / TPS;
    const bool ok = i < vh;

    int jf[4] = {0, 0, 0, 0}, jb[4] = {0, 0, 0, 0};
    T s2f[4], s2b[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) s2f[mu] = s2b[mu] = T(1);
    if (ok) {
        const Site s = site_of(a.g, i, a.parity);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            neighbours(a.g, s, i, mu, jf[mu], jb[mu]);
            if (R == 12) {
                float sf, sb;
                link_signs(a.g, s, mu, sf, sb);
                s2f[mu] = T(sf * LinkPost<P>::row2);
                s2b[mu] = T(sb * LinkPost<P>::row2);
            }
        }
    }

    for (int k0 = 0; k0 < per; k0 += NB) {
        int rid[NB];
        bool run[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int kk = sub + TPS * (k0 + q);
            run[q] = kk < nact;
            rid[q] = run[q] ? (a.active ? a.active[kk] : kk) : 0;
            if (EPI == EPI_GATE || EPI == EPI_A_CG)
                run[q] = run[q] && a.states[rid[q]].flag == FLAG_RUN;
        }
        Vec3<T> acc[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[q].r[c] = acc[q].i[c] = T(0);
        FF dot[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) dot[q].hi = dot[q].lo = 0.f;
        if (ok) {
            // No branches in the hot loop: a slot that is not running reads
            // system rid = 0 (valid memory) and its result is dropped below,
            // so every load of the NB systems can issue before the math.
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                const Mat3<T> uf = LinkIO<P, R>::load(a.lf[mu], vh, i);
                Vec3<T> v[NB];
#pragma unroll
                for (int q = 0; q < NB; ++q) v[q] = FieldIO<P>::load_nc(a.in + rid[q] * a.fstride, vh, jf[mu]);
#pragma unroll
                for (int q = 0; q < NB; ++q) mul_add<R == 12>(uf, v[q], acc[q], s2f[mu]);
                const Mat3<T> ub = LinkIO<P, R>::load(a.lb[mu], vh, jb[mu]);
#pragma unroll
                for (int q = 0; q < NB; ++q) v[q] = FieldIO<P>::load_nc(a.in + rid[q] * a.fstride, vh, jb[mu]);
#pragma unroll
                for (int q = 0; q < NB; ++q) adj_mul_sub(ub, v[q], acc[q], s2b[mu]);
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (!run[q]) continue;
                if (P == PX16) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        acc[q].r[c] *= T(LinkPost<PX16>::k);
                        acc[q].i[c] *= T(LinkPost<PX16>::k);
                    }
                }
                char *out = a.out + rid[q] * a.fstride;
                if (EPI == EPI_NONE || EPI == EPI_GATE) {
                    FieldIO<P>::store(out, vh, i, acc[q]);
                } else {
                    const T m2 = (EPI == EPI_A_CG) ? T(a.states[rid[q]].m2) : T(a.m2[rid[q]]);
                    const Vec3<T> d = FieldIO<P>::load_nc(a.w + rid[q] * a.fstride, vh, i);
                    Vec3<T> o;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o.r[c] = m2 * d.r[c] - acc[q].r[c];
                        o.i[c] = m2 * d.i[c] - acc[q].i[c];
                    }
                    const Vec3<T> os = FieldIO<P>::store(out, vh, i, o);
                    T dq = T(0);
#pragma unroll
                    for (int c = 0; c < 3; ++c) dq += d.r[c] * os.r[c] + d.i[c] * os.i[c];
                    dot[q].hi = float(dq);
                }
            }
        }
        if (EPI == EPI_A_CG) {
            // lanes holding the same system (equal sub) are TPS apart: shuffle
            // down to offset TPS only, then add the warps into sys_acc
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
#pragma unroll
                for (int o = 16; o >= TPS; o >>= 1) dot[q] = ff_add(dot[q], ff_shfl_down(dot[q], o));
                if (lane < TPS) red[q][lane][w] = make_float2(dot[q].hi, dot[q].lo);
            }
            __syncthreads();
            if ((int)threadIdx.x < NB * TPS) {
                const int q = threadIdx.x / TPS, sb = threadIdx.x % TPS;
                const int kk = sb + TPS * (k0 + q);
                if (kk < nact) {
                    FF sum = sys_acc[kk];
#pragma unroll
                    for (int ww = 0; ww < BS / 32; ++ww) {
                        FF t;
                        t.hi = red[q][sb][ww].x;
                        t.lo = red[q][sb][ww].y;
                        sum = ff_add(sum, t);
                    }
                    sys_acc[kk] = sum;
                }
            }
            __syncthreads();
        }
    }
    }  // tiles

    if (EPI == EPI_A_CG) {
        for (int kk = threadIdx.x; kk < nact; kk += BS) {
            const int k = a.active ? a.active[kk] : kk;
            a.partials[(size_t)k * gridDim.x + blockIdx.x] = make_float2(sys_acc[kk].hi, sys_acc[kk].lo);
        }
        __threadfence();
        __syncthreads();
    }

    if (EPI == EPI_A_CG) {
        __shared__ int is_last;
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned ticket = atomicAdd(a.counter, 1u);
            is_last = (ticket == gridDim.x - 1);
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        // one warp per system (fixed summation order per system)
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int kk = w; kk < nact; kk += BS / 32) {
            const int k = a.active ? a.active[kk] : kk;
            if (a.states[k].flag != FLAG_RUN) continue;  // uniform in the warp
            FF acc = {0.f, 0.f};
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const float2 p = __ldcg(a.partials + (size_t)k * gridDim.x + b);
                FF t;
                t.hi = p.x;
                t.lo = p.y;
                acc = ff_add(acc, t);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_down(acc, o));
            if (lane == 0) {
                CGState *st = a.states + k;
                const double total = (double)acc.hi + (double)acc.lo;
                set_alpha(st, total);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *a.counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// Staged multi-system Dslash, 12-real FP32 or FX16 links from the tile-major
// copy (kMTile).  A CTA of 256 threads (two per SM) walks tiles of kMTile =
// 64 output sites; the tile's eight links (24 KB in FP32) arrive in shared
// memory by one bulk async copy into a ring of two stages and serve every
// system, so the links cost 8L / n per site and system for n systems
// instead of 8L / NB.  Thread t owns site t % 64 of the tile and, with the
// other threads of its group (t / 64, four groups), a quarter of the active
// systems, NB at a time in registers; the link is rebuilt once per NB
// systems (FX16: applied to two systems per FP32x2 instruction).
//
// Each warp adds its part of d_k^dag q_k into its own shared-memory slots,
// summed in a fixed order at the end (no barrier inside the system loop).
// The last warp to finish a tile refills that stage with the CTA's tile
// two steps ahead.  Waits on the stage barriers give up after about a
// second (g_ms_wait_timeouts; the CTA then lets its copies land), and the
// systems' reductions become NaN, which stops them.
// ---------------------------------------------------------------------------
#ifndef STG_MS_THREADS
#define STG_MS_THREADS 256
#endif
#ifndef STG_MS_STAGES
#define STG_MS_STAGES 2
#endif
#ifndef STG_MS_MINBLOCKS
#define STG_MS_MINBLOCKS 2
#endif
constexpr int kMsThreads = STG_MS_THREADS;
constexpr int kMsGroups = kMsThreads / kMTile;
constexpr int kMsWarps = kMsThreads / 32;
constexpr int kMsStages = STG_MS_STAGES;

static __device__ unsigned g_ms_wait_timeouts;

template <int P> struct MsLink;
template <> struct MsLink<P32> {
    static constexpr unsigned kRec = 48;
    __device__ __forceinline__ static Mat3<float> load(const char *blk, int a, float s2)
    {
        const float4 *p = reinterpret_cast<const float4 *>(blk);
        Mat3<float> u;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = p[k * kMTile + a];
            set_entry(u, 2 * k, v.x, v.y);
            set_entry(u, 2 * k + 1, v.z, v.w);
        }
        reconstruct_row2(u, s2);
        return u;
    }
};
template <> struct MsLink<PX16> {
    static constexpr unsigned kRec = 24;
    __device__ __forceinline__ static Mat3<float> load(const char *blk, int a, float s2)
    {
        const uint4 v = reinterpret_cast<const uint4 *>(blk)[a];
        const uint2 w = reinterpret_cast<const uint2 *>(blk + 16 * kMTile)[a];
        Mat3<float> u;
        set_entry(u, 0, fx_lo(v.x), fx_hi(v.x));
        set_entry(u, 1, fx_lo(v.y), fx_hi(v.y));
        set_entry(u, 2, fx_lo(v.z), fx_hi(v.z));
        set_entry(u, 3, fx_lo(v.w), fx_hi(v.w));
        set_entry(u, 4, fx_lo(w.x), fx_hi(w.x));
        set_entry(u, 5, fx_lo(w.y), fx_hi(w.y));
        reconstruct_row2(u, s2);
        return u;
    }
};

// Two systems in the halves of every float2 (one sm_100 FP32x2 instruction
// for both): acc += U v and acc -= U^dag v with U shared (row 2 already
// carrying its sign); the negated link entries cost no instruction.
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

__device__ __forceinline__ void mul_add2(const Mat3<float> &u, const float2 *vr, const float2 *vi,
                                         float2 *ar, float2 *ai)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ar[a] = __ffma2_rn(bc2(u.r[a][b]), vr[b], ar[a]);
            ar[a] = __ffma2_rn(bc2(-u.i[a][b]), vi[b], ar[a]);
            ai[a] = __ffma2_rn(bc2(u.r[a][b]), vi[b], ai[a]);
            ai[a] = __ffma2_rn(bc2(u.i[a][b]), vr[b], ai[a]);
        }
}

__device__ __forceinline__ void adj_mul_sub2(const Mat3<float> &u, const float2 *vr, const float2 *vi,
                                             float2 *ar, float2 *ai)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            // conj(U_ba) v_b = (u.r v.r + u.i v.i) + i (u.r v.i - u.i v.r)
            ar[a] = __ffma2_rn(bc2(-u.r[b][a]), vr[b], ar[a]);
            ar[a] = __ffma2_rn(bc2(-u.i[b][a]), vi[b], ar[a]);
            ai[a] = __ffma2_rn(bc2(-u.r[b][a]), vi[b], ai[a]);
            ai[a] = __ffma2_rn(bc2(u.i[b][a]), vr[b], ai[a]);
        }
}

// Colour vectors on FP32x2 arithmetic without moving a field value: the real
// and imaginary part of each colour sit in the two halves of one float2 (for
// FP32 as the field record holds them, for FX16 as one decoded word), so
// every entry of U enters as two broadcast products, A += (Re U) v and
// B += (Im U) v, and the complex result is Re = A.x - B.y, Im = A.y + B.x.
// Two FP32x2 instructions per complex multiply-add in place of four FMAs;
// each broadcast of U serves the NB systems of the register block (q
// innermost).
template <int NB>
__device__ __forceinline__ void mul_add_ri(const Mat3<float> &u, const float2 (*v)[3], float2 (*A)[3],
                                           float2 (*B)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 ur = bc2(u.r[a][b]), ui = bc2(u.i[a][b]);
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                A[q][a] = __ffma2_rn(ur, v[q][b], A[q][a]);
                B[q][a] = __ffma2_rn(ui, v[q][b], B[q][a]);
            }
        }
}

// acc -= U^dag v: -conj(U_ba) v_b = -(Re U_ba) v_b + i (Im U_ba) v_b enters as
// A += (-Re U_ba) v_b and B += (Im U_ba) v_b
template <int NB>
__device__ __forceinline__ void adj_mul_sub_ri(const Mat3<float> &u, const float2 (*v)[3], float2 (*A)[3],
                                               float2 (*B)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 ur = bc2(-u.r[b][a]), ui = bc2(u.i[b][a]);
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                A[q][a] = __ffma2_rn(ur, v[q][b], A[q][a]);
                B[q][a] = __ffma2_rn(ui, v[q][b], B[q][a]);
            }
        }
}

// RI: a link of the stage with row 2 taken from the tile's rebuilt rows
// (sign included), so that all three rows enter the mat-vec alike
__device__ __forceinline__ Mat3<float> ms_link_ri(const char *blk, const float4 *r4, const float2 *r2, int a)
{
    const float4 *p = reinterpret_cast<const float4 *>(blk);
    Mat3<float> u;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float4 v = p[k * kMTile + a];
        set_entry(u, 2 * k, v.x, v.y);
        set_entry(u, 2 * k + 1, v.z, v.w);
    }
    const float4 v = p[2 * kMTile + a];
    set_entry(u, 4, v.x, v.y);
    set_entry(u, 5, v.z, v.w);
    const float4 x = r4[a];
    const float2 y = r2[a];
    set_entry(u, 6, x.x, x.y);
    set_entry(u, 7, x.z, x.w);
    set_entry(u, 8, y.x, y.y);
    return u;
}

// an L1 prefetch: no register is written and no wait follows, so the load
// it starts overlaps the work issued after it
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" :: "l"(p));
}

// RI, FX16: a link decoded once per tile into FP32 (true values, row 2
// rebuilt with its sign) as four float4 planes and one float2 plane
__device__ __forceinline__ Mat3<float> ms_link_fx(const float4 *x4, const float2 *x2, int a)
{
    Mat3<float> u;
    const float4 p0 = x4[a], p1 = x4[kMTile + a], p2 = x4[2 * kMTile + a], p3 = x4[3 * kMTile + a];
    const float2 p4 = x2[a];
    set_entry(u, 0, p0.x, p0.y);
    set_entry(u, 1, p0.z, p0.w);
    set_entry(u, 2, p1.x, p1.y);
    set_entry(u, 3, p1.z, p1.w);
    set_entry(u, 4, p2.x, p2.y);
    set_entry(u, 5, p2.z, p2.w);
    set_entry(u, 6, p3.x, p3.y);
    set_entry(u, 7, p3.z, p3.w);
    set_entry(u, 8, p4.x, p4.y);
    return u;
}

// one FX16 (re, im) word as an FP32 pair: the biased values K + q from two
// byte permutes, then (K + q) s - K s in one FP32x2 FMA (K s is exact for
// the 15-bit scale, so this rounds once, like q s)
__device__ __forceinline__ float2 fx_pair(unsigned w, float2 s2, float2 ks2)
{
    const float2 b = make_float2(__int_as_float((int)__byte_perm(w, 0x4B40u, 0x5410)),
                                 __int_as_float((int)__byte_perm(w, 0x4B40u, 0x5432)));
    return __ffma2_rn(b, s2, ks2);
}

// the FX16 colour vector of site j as three (re, im) pairs
__device__ __forceinline__ void load_ri_fx(const char *f, int j, float2 *v)
{
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(f) + j);
    const float sc = __uint_as_float(u.w);
    const float2 s2 = bc2(sc), ks2 = bc2(-12615680.0f * sc);
    v[0] = fx_pair(u.x, s2, ks2);
    v[1] = fx_pair(u.y, s2, ks2);
    v[2] = fx_pair(u.z, s2, ks2);
}

// the FP32 colour vector of site j as three (re, im) pairs
__device__ __forceinline__ void load_ri(const char *f, int vh, int j, float2 *v)
{
    const float4 *p4 = reinterpret_cast<const float4 *>(f);
    const float4 x = __ldg(p4 + j);
    v[0] = make_float2(x.x, x.y);
    v[1] = make_float2(x.z, x.w);
    v[2] = __ldg(reinterpret_cast<const float2 *>(p4 + vh) + j);
}

template <int P>
__host__ __device__ constexpr unsigned ms_stage_bytes() { return kMTile * 8 * MsLink<P>::kRec; }

// RI: the mat-vecs on FP32x2 pairs of real and imaginary parts (mul_add_ri),
// with the links' row 2 (FP32) or whole links (FX16) rebuilt once per tile in
// shared memory; otherwise scalar FMAs for FP32 and system pairs for FX16
template <int P, int NB, int EPI, bool RI = false>
__global__ void __launch_bounds__(kMsThreads, STG_MS_MINBLOCKS) k_dslash_ms(const MrhsArgs a)
{
    typedef float T;
    constexpr unsigned SB = ms_stage_bytes<P>();
    constexpr unsigned LB = kMTile * MsLink<P>::kRec;  // one (mu, dir) block
    extern __shared__ __align__(128) char stage[];
    __shared__ __align__(8) unsigned long long full[kMsStages];
    __shared__ unsigned done_warps[kMsStages], issued[kMsStages];
    __shared__ int abort_flag;
    __shared__ FF sysw[kMsWarps][kMaxRhs];  // EPI_A_CG: per-warp d^dag q per list slot
    // RI: row 2 of the tile's eight links per site, rebuilt once per tile
    // (not once per register block of systems) with the link's sign
    // (FP32), or the whole FP32 links (FX16: decoded once per tile)
    constexpr int kR2 = (RI && P == P32) ? 8 * kMTile : 1;
    constexpr int kLX = (RI && P == PX16) ? 8 * kMTile : 1;
    __shared__ float4 row2s4[kR2];
    __shared__ float2 row2s2[kR2];
    __shared__ float4 lkx4[4 * kLX];
    __shared__ float2 lkx2[kLX];
    static_assert(!RI || kMsGroups == 4, "RI: site group g rebuilds the links of direction g");
    const int vh = a.g.Vh;
    const int ntiles = (vh + kMTile - 1) / kMTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int site = threadIdx.x % kMTile, grp = threadIdx.x / kMTile;
    const int nact = a.active ? *a.nactive : a.nrhs;
    const int per = (nact + kMsGroups - 1) / kMsGroups;  // list slots per group (uniform bound)

    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kMsStages; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&full[q])) : "memory");
            done_warps[q] = 0u;
            issued[q] = 0u;
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
        for (int q = 0; q < kMsStages; ++q) {
            const int tile = blockIdx.x + q * gridDim.x;
            if (tile < ntiles) {
                bulk_load(stage + (size_t)q * SB, a.lt + (size_t)tile * SB, SB, &full[q]);
                issued[q] = 1u;
            }
        }
    }
    if (EPI == EPI_A_CG)
        for (int k = threadIdx.x; k < kMsWarps * kMaxRhs; k += kMsThreads)
            sysw[k / kMaxRhs][k % kMaxRhs].hi = sysw[k / kMaxRhs][k % kMaxRhs].lo = 0.f;
    __syncthreads();
    volatile int *abort = &abort_flag;

    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
        const int st = j % kMsStages;
        const unsigned par = (unsigned)(j / kMsStages) & 1u;
        const int i = tile * kMTile + site;
        const bool ok = i < vh;
        const int iv = ok ? i : vh - 1;  // past Vh: a valid site's fields, zero links, unstored
        int jf[4], jb[4];
        T s2f[4], s2b[4];
        T sgf = T(1), sgb = T(1);  // RI: the signs of direction grp at this site
        {
            const Site s = site_of(a.g, iv, a.parity);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                neighbours(a.g, s, iv, mu, jf[mu], jb[mu]);
                if constexpr (!RI) {
                    float sf, sb;
                    link_signs(a.g, s, mu, sf, sb);
                    s2f[mu] = T(sf * LinkPost<P>::row2);
                    s2b[mu] = T(sb * LinkPost<P>::row2);
                }
            }
            if constexpr (RI) {
                float sf, sb;
                link_signs(a.g, s, grp, sf, sb);
                sgf = sf;
                sgb = sb;
            }
        }
        const bool ready = mbar_wait(smem_addr(&full[st]), par, abort, &g_ms_wait_timeouts);
        if (!__syncthreads_and(ready)) break;  // uniform over the CTA
        const char *sb = stage + (size_t)st * SB;
        if constexpr (RI) {
            // every thread rebuilds the forward and backward link of its site
            // in direction grp; the previous tile's readers have all passed
            // the barrier above
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const int l = 2 * grp + dir;
                const T sg = dir ? sgb : sgf;
                if constexpr (P == P32) {
                    const Mat3<T> u = MsLink<P>::load(sb + (size_t)l * LB, site, sg);
                    row2s4[l * kMTile + site] = make_float4(u.r[2][0], u.i[2][0], u.r[2][1], u.i[2][1]);
                    row2s2[l * kMTile + site] = make_float2(u.r[2][2], u.i[2][2]);
                } else {
                    // stored entries are q = 32767 U; row 2 from them carries
                    // 32767^2, so it takes the sign times 1/32767, then every
                    // entry takes 1/32767
                    Mat3<T> u = MsLink<P>::load(sb + (size_t)l * LB, site, sg * T(LinkPost<P>::row2));
                    constexpr T k = T(LinkPost<P>::k);
                    float4 *x4 = lkx4 + 4 * l * kMTile + site;
                    x4[0] = make_float4(k * u.r[0][0], k * u.i[0][0], k * u.r[0][1], k * u.i[0][1]);
                    x4[kMTile] = make_float4(k * u.r[0][2], k * u.i[0][2], k * u.r[1][0], k * u.i[1][0]);
                    x4[2 * kMTile] = make_float4(k * u.r[1][1], k * u.i[1][1], k * u.r[1][2], k * u.i[1][2]);
                    x4[3 * kMTile] = make_float4(k * u.r[2][0], k * u.i[2][0], k * u.r[2][1], k * u.i[2][1]);
                    lkx2[l * kMTile + site] = make_float2(k * u.r[2][2], k * u.i[2][2]);
                }
            }
            __syncthreads();
        }

        for (int k0 = 0; k0 < per; k0 += NB) {
            int rid[NB];
            bool run[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int kk = grp + kMsGroups * (k0 + q);
                run[q] = kk < nact;
                rid[q] = run[q] ? (a.active ? a.active[kk] : kk) : 0;
                if (EPI == EPI_GATE || EPI == EPI_A_CG)
                    run[q] = run[q] && a.states[rid[q]].flag == FLAG_RUN;
            }
            if (RI && (EPI == EPI_A || EPI == EPI_A_CG)) {
                // the epilogue's m^2 d reads this site's even input once per
                // system after the eight mat-vecs: start those reads into L1
                // now (measured: A of 16 systems at 24^3x48 244 -> 228 us)
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    const char *w = a.w + rid[q] * a.fstride;
                    prefetch_l1(w + (size_t)iv * 16);
                    if (P == P32) prefetch_l1(w + (size_t)vh * 16 + (size_t)iv * 8);
                }
            }
            Vec3<T> acc[NB];
            // no branches in the hot loop: a slot that is not running reads
            // system rid = 0 (valid memory) and its result is dropped below
            if constexpr (P == PX16 && !RI) {
                // systems 2p and 2p + 1 share float2 accumulators: the decode
                // of the 16-bit fields leaves the FMA pipe the busier one
                float2 ar[NB / 2][3], ai[NB / 2][3];
#pragma unroll
                for (int p2 = 0; p2 < NB / 2; ++p2)
#pragma unroll
                    for (int c = 0; c < 3; ++c) ar[p2][c] = ai[p2][c] = make_float2(0.f, 0.f);
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) {
                    // both neighbours' fields of every system in flight at once
                    Vec3<T> vf[NB], vb[NB];
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        vf[q] = FieldIO<P>::load_nc(a.in + rid[q] * a.fstride, vh, jf[mu]);
                        vb[q] = FieldIO<P>::load_nc(a.in + rid[q] * a.fstride, vh, jb[mu]);
                    }
                    const Mat3<T> uf = MsLink<P>::load(sb + (size_t)(2 * mu) * LB, site, s2f[mu]);
#pragma unroll
                    for (int p2 = 0; p2 < NB / 2; ++p2) {
                        float2 vr[3], vi[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            vr[c] = make_float2(vf[2 * p2].r[c], vf[2 * p2 + 1].r[c]);
                            vi[c] = make_float2(vf[2 * p2].i[c], vf[2 * p2 + 1].i[c]);
                        }
                        mul_add2(uf, vr, vi, ar[p2], ai[p2]);
                    }
                    const Mat3<T> ub = MsLink<P>::load(sb + (size_t)(2 * mu + 1) * LB, site, s2b[mu]);
#pragma unroll
                    for (int p2 = 0; p2 < NB / 2; ++p2) {
                        float2 vr[3], vi[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            vr[c] = make_float2(vb[2 * p2].r[c], vb[2 * p2 + 1].r[c]);
                            vi[c] = make_float2(vb[2 * p2].i[c], vb[2 * p2 + 1].i[c]);
                        }
                        adj_mul_sub2(ub, vr, vi, ar[p2], ai[p2]);
                    }
                }
#pragma unroll
                for (int p2 = 0; p2 < NB / 2; ++p2)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        acc[2 * p2].r[c] = ar[p2][c].x;
                        acc[2 * p2].i[c] = ai[p2][c].x;
                        acc[2 * p2 + 1].r[c] = ar[p2][c].y;
                        acc[2 * p2 + 1].i[c] = ai[p2][c].y;
                    }
            } else if constexpr (RI) {
                float2 A[NB][3], B[NB][3];
#pragma unroll
                for (int q = 0; q < NB; ++q)
#pragma unroll
                    for (int c = 0; c < 3; ++c) A[q][c] = B[q][c] = make_float2(0.f, 0.f);
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) {
                    // one direction's fields at a time (the accumulators
                    // take twice the registers of the scalar form)
                    float2 v[NB][3];
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        if constexpr (P == P32) load_ri(a.in + rid[q] * a.fstride, vh, jf[mu], v[q]);
                        else load_ri_fx(a.in + rid[q] * a.fstride, jf[mu], v[q]);
                    }
                    const Mat3<T> uf = (P == P32)
                        ? ms_link_ri(sb + (size_t)(2 * mu) * LB, row2s4 + 2 * mu * kMTile, row2s2 + 2 * mu * kMTile, site)
                        : ms_link_fx(lkx4 + 4 * (2 * mu) * kMTile, lkx2 + (2 * mu) * kMTile, site);
                    mul_add_ri<NB>(uf, v, A, B);
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        if constexpr (P == P32) load_ri(a.in + rid[q] * a.fstride, vh, jb[mu], v[q]);
                        else load_ri_fx(a.in + rid[q] * a.fstride, jb[mu], v[q]);
                    }
                    const Mat3<T> ub = (P == P32)
                        ? ms_link_ri(sb + (size_t)(2 * mu + 1) * LB, row2s4 + (2 * mu + 1) * kMTile,
                                     row2s2 + (2 * mu + 1) * kMTile, site)
                        : ms_link_fx(lkx4 + 4 * (2 * mu + 1) * kMTile, lkx2 + (2 * mu + 1) * kMTile, site);
                    adj_mul_sub_ri<NB>(ub, v, A, B);
                }
#pragma unroll
                for (int q = 0; q < NB; ++q)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        acc[q].r[c] = A[q][c].x - B[q][c].y;
                        acc[q].i[c] = A[q][c].y + B[q][c].x;
                    }
            } else {
                // FP32: scalar FMAs (packing the fields of two systems would
                // cost more moves than it saves; RI avoids the moves)
#pragma unroll
                for (int q = 0; q < NB; ++q)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[q].r[c] = acc[q].i[c] = T(0);
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) {
                    Vec3<T> vf[NB], vb[NB];
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        vf[q] = FieldIO<P>::load_nc(a.in + rid[q] * a.fstride, vh, jf[mu]);
                        vb[q] = FieldIO<P>::load_nc(a.in + rid[q] * a.fstride, vh, jb[mu]);
                    }
                    const Mat3<T> uf = MsLink<P>::load(sb + (size_t)(2 * mu) * LB, site, T(1));
#pragma unroll
                    for (int q = 0; q < NB; ++q) mul_add(uf, vf[q], acc[q], s2f[mu]);
                    const Mat3<T> ub = MsLink<P>::load(sb + (size_t)(2 * mu + 1) * LB, site, T(1));
#pragma unroll
                    for (int q = 0; q < NB; ++q) adj_mul_sub(ub, vb[q], acc[q], s2b[mu]);
                }
            }
            FF dot[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                dot[q].hi = dot[q].lo = 0.f;
                if (!ok || !run[q]) continue;
                if (P == PX16 && !RI) {  // RI: the links carry 1/32767 already
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        acc[q].r[c] *= T(LinkPost<PX16>::k);
                        acc[q].i[c] *= T(LinkPost<PX16>::k);
                    }
                }
                char *out = a.out + rid[q] * a.fstride;
                if (EPI == EPI_NONE || EPI == EPI_GATE) {
                    FieldIO<P>::store(out, vh, i, acc[q]);
                } else {
                    const T m2 = (EPI == EPI_A_CG) ? T(a.states[rid[q]].m2) : T(a.m2[rid[q]]);
                    const Vec3<T> d = FieldIO<P>::load_nc(a.w + rid[q] * a.fstride, vh, i);
                    Vec3<T> o;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o.r[c] = m2 * d.r[c] - acc[q].r[c];
                        o.i[c] = m2 * d.i[c] - acc[q].i[c];
                    }
                    const Vec3<T> os = FieldIO<P>::store(out, vh, i, o);
                    T dq = T(0);
#pragma unroll
                    for (int c = 0; c < 3; ++c) dq += d.r[c] * os.r[c] + d.i[c] * os.i[c];
                    dot[q].hi = float(dq);
                }
            }
            if (EPI == EPI_A_CG) {
                // a warp's 32 lanes are sites of one group: the same systems
#pragma unroll
                for (int q = 0; q < NB; ++q) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dot[q] = ff_add(dot[q], ff_shfl_down(dot[q], o));
                    const int kk = grp + kMsGroups * (k0 + q);
                    if (lane == 0 && kk < nact) sysw[warp][kk] = ff_add(sysw[warp][kk], dot[q]);
                }
            }
        }
        // release the stage: the last warp to finish refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&done_warps[st], 1u) == kMsWarps - 1) {
                done_warps[st] = 0u;
                const int next = tile + kMsStages * (int)gridDim.x;
                if (next < ntiles) {
                    __threadfence_block();
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bulk_load(stage + (size_t)st * SB, a.lt + (size_t)next * SB, SB, &full[st]);
                    issued[st] += 1u;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) {
        // after a timeout, let every copy issued into this CTA land first
#pragma unroll
        for (int q = 0; q < kMsStages; ++q)
            if (issued[q] > 0u) mbar_wait(smem_addr(&full[q]), (issued[q] - 1u) & 1u, nullptr, &g_ms_wait_timeouts);
    }

    if (EPI == EPI_A_CG) {
        for (int kk = threadIdx.x; kk < nact; kk += kMsThreads) {
            FF sum = sysw[0][kk];
#pragma unroll
            for (int w = 1; w < kMsWarps; ++w) sum = ff_add(sum, sysw[w][kk]);
            if (abort_flag) sum.hi = __int_as_float(0x7fc00000);  // the system's sum becomes NaN
            const int k = a.active ? a.active[kk] : kk;
            a.partials[(size_t)k * gridDim.x + blockIdx.x] = make_float2(sum.hi, sum.lo);
        }
        __threadfence();
        __syncthreads();
        __shared__ int is_last;
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned ticket = atomicAdd(a.counter, 1u);
            is_last = (ticket == gridDim.x - 1);
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        // one warp per system (fixed summation order per system)
        for (int kk = warp; kk < nact; kk += kMsWarps) {
            const int k = a.active ? a.active[kk] : kk;
            if (a.states[k].flag != FLAG_RUN) continue;  // uniform in the warp
            FF acc = {0.f, 0.f};
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const float2 p = __ldcg(a.partials + (size_t)k * gridDim.x + b);
                FF t;
                t.hi = p.x;
                t.lo = p.y;
                acc = ff_add(acc, t);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_down(acc, o));
            if (lane == 0) {
                CGState *st = a.states + k;
                const double total = (double)acc.hi + (double)acc.lo;
                if (!isfinite(total) && *(volatile unsigned *)&g_ms_wait_timeouts) {
                    st->pAp = total;
                    st->flag = FLAG_TIMEOUT;
                } else {
                    set_alpha(st, total);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *a.counter = 0u;
    } else if (EPI == EPI_GATE) {
        if (threadIdx.x == 0 && abort_flag)
            for (int kk = 0; kk < nact; ++kk) a.states[a.active ? a.active[kk] : kk].flag = FLAG_TIMEOUT;
    }
}

// staged shapes: NB = 2, 4, 8 systems per thread and pass
constexpr int kMrhsStagedShapes = 3;
__host__ __device__ constexpr int ms_nb(int k) { return k == 0 ? 2 : k == 1 ? 4 : 8; }

template <int P, int NB, bool RI = false>
void launch_ms_nb(int epi, const MrhsArgs &a, cudaStream_t s)
{
    constexpr unsigned smem = kMsStages * ms_stage_bytes<P>();
    // set once per instantiation (thread-safe static initialisation):
    // resident CTAs on the whole GPU
    static const int resident = [] {
        cudaFuncSetAttribute(k_dslash_ms<P, NB, EPI_NONE, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_dslash_ms<P, NB, EPI_A, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_dslash_ms<P, NB, EPI_GATE, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_dslash_ms<P, NB, EPI_A_CG, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash_ms<P, NB, EPI_A_CG, RI>, kMsThreads,
                                                          smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return sms * per_sm;
    }();
    const int ntiles = (a.g.Vh + kMTile - 1) / kMTile;
    int cap = resident;
    if (a.grid_limit > 0 && a.grid_limit < cap) cap = a.grid_limit;
    const int grid = ntiles < cap ? ntiles : cap;
    switch (epi) {
    case EPI_NONE: k_dslash_ms<P, NB, EPI_NONE, RI><<<grid, kMsThreads, smem, s>>>(a); break;
    case EPI_A: k_dslash_ms<P, NB, EPI_A, RI><<<grid, kMsThreads, smem, s>>>(a); break;
    case EPI_GATE: k_dslash_ms<P, NB, EPI_GATE, RI><<<grid, kMsThreads, smem, s>>>(a); break;
    case EPI_A_CG: k_dslash_ms<P, NB, EPI_A_CG, RI><<<grid, kMsThreads, smem, s>>>(a); break;
    }
}

template <int P>
void launch_ms(int k, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (k == 0) launch_ms_nb<P, 2>(epi, a, s);
    else if (k == 1) launch_ms_nb<P, 4>(epi, a, s);
    else launch_ms_nb<P, 8>(epi, a, s);
}

// staged kernel on (re, im) FP32x2 pairs (FP32 and FX16): NB = 2, 4; its shapes follow
// the register-fed ones, the staged ones and the two of the FX16 staged
// kernel with two sites per thread (mrhs_paired.cuh)
constexpr int kMspShapes = 2;
constexpr int kMsRiShapes = 2;
__host__ __device__ constexpr int ms_ri_nb(int k) { return k == 0 ? 2 : 4; }

template <int P>
void launch_ms_ri(int k, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (k == 0) launch_ms_nb<P, 2, true>(epi, a, s);
    else launch_ms_nb<P, 4, true>(epi, a, s);
}

// (NB, TPS) shapes the autotuner chooses from
constexpr int kMrhsShapes = 9;
constexpr int kMsRiFirst = kMrhsShapes + kMrhsStagedShapes + kMspShapes;
__host__ __device__ constexpr int mrhs_nb(int k)
{
    return k == 0 ? 1 : k == 1 ? 2 : k == 2 ? 4 : k == 3 ? 2 : k == 4 ? 1 : k == 5 ? 2 : k == 6 ? 1 : k == 7 ? 2 : 1;
}
__host__ __device__ constexpr int mrhs_tps(int k)
{
    return k == 0 ? 1 : k == 1 ? 1 : k == 2 ? 1 : k == 3 ? 2 : k == 4 ? 4 : k == 5 ? 4 : k == 6 ? 8 : k == 7 ? 8 : 16;
}

// Launch one (P, R) family with the shape index `shape` (0..kMrhsShapes-1).
template <int P, int R>
void launch_m_pr(int shape, int epi, const MrhsArgs &a, cudaStream_t s)
{
#define STG_M_EPI(K_)                                                                                  \
    do {                                                                                               \
        constexpr int NB_ = mrhs_nb(K_), TPS_ = mrhs_tps(K_);                                           \
        const long tiles_ = ((long)a.g.Vh * TPS_ + kMrhsBlock - 1) / kMrhsBlock;                      \
        const int grid = (int)(tiles_ < a.grid_cap ? tiles_ : a.grid_cap);                             \
        switch (epi) {                                                                                 \
        case EPI_NONE: k_dslash_m<P, R, NB_, TPS_, EPI_NONE><<<grid, kMrhsBlock, 0, s>>>(a); break;    \
        case EPI_A: k_dslash_m<P, R, NB_, TPS_, EPI_A><<<grid, kMrhsBlock, 0, s>>>(a); break;          \
        case EPI_GATE: k_dslash_m<P, R, NB_, TPS_, EPI_GATE><<<grid, kMrhsBlock, 0, s>>>(a); break;    \
        case EPI_A_CG: k_dslash_m<P, R, NB_, TPS_, EPI_A_CG><<<grid, kMrhsBlock, 0, s>>>(a); break;    \
        }                                                                                              \
    } while (0)
    switch (shape) {
    case 0: STG_M_EPI(0); break;
    case 1: STG_M_EPI(1); break;
    case 2: STG_M_EPI(2); break;
    case 3: STG_M_EPI(3); break;
    case 4: STG_M_EPI(4); break;
    case 5: STG_M_EPI(5); break;
    case 6: STG_M_EPI(6); break;
    case 7: STG_M_EPI(7); break;
    default: STG_M_EPI(8); break;
    }
#undef STG_M_EPI
}

}  // namespace stg
