// FX16 (16-bit fixed point) Dslash half-pass, Eq. 5, on packed FP32x2.
//
// With 16-bit storage the half-pass moves 224 bytes per site (12-real links),
// half of FP32/12, but decoding the fixed-point values and rebuilding row 2
// roughly doubles the instruction count per site, so a one-site-per-thread
// kernel runs out of issue slots before it runs out of bandwidth.  Here each
// thread computes two sites, A = i and B = i + 256 of a 512-site tile: the .x
// half of every float2 holds site A's value and the .y half site B's, and
// every FP32 operation is one sm_100 FP32x2 instruction (__ffma2_rn,
// __fadd2_rn, __fmul2_rn) for both sites.  Loads of A and B are separate and
// stay coalesced across the warp.
//
// The packed arithmetic (decode, 12-real reconstruction, mat-vecs, FX16
// encode) is in fx16_pair.cuh.
#include "fx16_pair.cuh"

#ifndef STG_FX2_MINBLOCKS
#define STG_FX2_MINBLOCKS 2
#endif

namespace stg {

// decode one 16-bit site record already in registers
template <int P = PX16>
__device__ __forceinline__ Vec3<float> fx_decode(uint4 u)
{
    const float sc = __uint_as_float(u.w);
    Vec3<float> v;
    if constexpr (P == P16) {
        v.r[0] = h_lo(u.x) * sc; v.i[0] = h_hi(u.x) * sc;
        v.r[1] = h_lo(u.y) * sc; v.i[1] = h_hi(u.y) * sc;
        v.r[2] = h_lo(u.z) * sc; v.i[2] = h_hi(u.z) * sc;
    } else {
        v.r[0] = fx_lo(u.x) * sc; v.i[0] = fx_hi(u.x) * sc;
        v.r[1] = fx_lo(u.y) * sc; v.i[1] = fx_hi(u.y) * sc;
        v.r[2] = fx_lo(u.z) * sc; v.i[2] = fx_hi(u.z) * sc;
    }
    return v;
}

// The packed epilogue over the kernel's output field (epilogue_pair)
template <int EPI, int P = PX16>
__device__ __forceinline__ f2 epilogue2(const DslashArgs &a, int iA, int iB, bool okA, bool okB,
                                        const f2 (&dr)[3], const f2 (&di)[3], float m2, uint4 wA,
                                        uint4 wB)
{
    return epilogue_pair<EPI, P>(a.out, iA, iB, okA, okB, dr, di, m2, wA, wB);
}

// the scalar epilogue of one site (same arithmetic as k_dslash's); wraw is
// the site's record of w, loaded at kernel start for the A epilogues
template <int EPI, int P = PX16>
__device__ __forceinline__ float epilogue(const DslashArgs &a, int vh, int i, const Vec3<float> &acc,
                                          float m2, uint4 wraw)
{
    float dot = 0.f;
    if (EPI == EPI_NONE || EPI == EPI_GATE) {
        FieldIO<P>::store(a.out, vh, i, acc);
    } else if (EPI == EPI_RES) {
        const Vec3<float> b = FieldIO<P>::load_nc(a.w, vh, i);
        const Vec3<float> x = FieldIO<P>::load_nc(a.v, vh, i);
        Vec3<float> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = b.r[c] - m2 * x.r[c] + acc.r[c];
            o.i[c] = b.i[c] - m2 * x.i[c] + acc.i[c];
        }
        const Vec3<float> os = FieldIO<P>::store(a.out, vh, i, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) dot += os.r[c] * os.r[c] + os.i[c] * os.i[c];
    } else {
        const Vec3<float> d = fx_decode<P>(wraw);
        Vec3<float> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = m2 * d.r[c] - acc.r[c];
            o.i[c] = m2 * d.i[c] - acc.i[c];
        }
        const Vec3<float> os = FieldIO<P>::store(a.out, vh, i, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) dot += d.r[c] * os.r[c] + d.i[c] * os.i[c];
    }
    return dot;
}

// D chi = (P - N) / 32767 of both sites, negated for the A epilogues, then
// the packed epilogue
template <int EPI, int P = PX16>
__device__ __forceinline__ f2 finish_pair(const DslashArgs &a, int iA, int iB, bool okA, bool okB,
                                          const Acc2 &A, float m2, uint4 wA, uint4 wB)
{
    const f2 k = make_float2(LinkPost<P>::k, LinkPost<P>::k);
    constexpr bool neg = (EPI == EPI_A || EPI == EPI_A_DOT || EPI == EPI_A_CG);
    f2 dr[3], di[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dr[c] = mul2(A.re[c], neg ? neg2(k) : k);
        di[c] = mul2(A.im[c], neg ? neg2(k) : k);
    }
    return epilogue2<EPI, P>(a, iA, iB, okA, okB, dr, di, m2, wA, wB);
}

template <int R, int EPI>
__global__ void __launch_bounds__(kBlock, STG_FX2_MINBLOCKS) k_dslash_fx2(const DslashArgs a)
{
    pdl_wait();
    pdl_trigger();
    if (EPI == EPI_A_CG || EPI == EPI_GATE) {
        if (a.state->flag != FLAG_RUN) return;  // uniform over the grid
    }
    const int vh = a.g.Vh;
    const int iA = blockIdx.x * (2 * kBlock) + threadIdx.x;
    const int iB = iA + kBlock;
    const bool okA = iA < vh, okB = iB < vh;
    FF dot = {0.f, 0.f};
    if (okA) {
        const int jA = iA, jB = okB ? iB : iA;  // a missing B recomputes A, unstored
        // the A epilogues read w = d at the output sites: issue those loads
        // first so their latency hides under the half-pass
        uint4 wA = make_uint4(0u, 0u, 0u, 0u), wB = wA;
        if (EPI == EPI_A || EPI == EPI_A_DOT || EPI == EPI_A_CG) {
            wA = __ldg(static_cast<const uint4 *>(a.w) + jA);
            wB = __ldg(static_cast<const uint4 *>(a.w) + jB);
        }
        const Site sA = site_of(a.g, jA, a.parity);
        const Site sB = site_of(a.g, jB, a.parity);
        Acc2 A;
#pragma unroll
        for (int c = 0; c < 3; ++c) A.re[c] = A.im[c] = make_float2(0.f, 0.f);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            int jfA, jbA, jfB, jbB;
            neighbours(a.g, sA, jA, mu, jfA, jbA);
            neighbours(a.g, sB, jB, mu, jfB, jbB);
            f2 s2f = make_float2(1.f, 1.f), s2b = make_float2(1.f, 1.f);
            if (R == 12) {
                float sfA, sbA, sfB, sbB;
                link_signs(a.g, sA, mu, sfA, sbA);
                link_signs(a.g, sB, mu, sfB, sbB);
                const float k = LinkPost<PX16>::row2;
                s2f = make_float2(sfA * k, sfB * k);
                s2b = make_float2(sbA * k, sbB * k);
            }
            Mat3x2 u;
            Vec3x2 v;
            load_link2<R>(a.lf[mu], vh, jA, jB, u);
            load_field2(a.in, jfA, jfB, v);
            fwd2<R>(u, v, s2f, A);
            load_link2<R>(a.lb[mu], vh, jbA, jbB, u);
            load_field2(a.in, jbA, jbB, v);
            bwd2<R>(u, v, s2b, A);
        }
        const float m2 = (EPI == EPI_A_CG) ? float(a.state->m2) : float(a.m2);
        f2 dA_B;
        if (EPI == EPI_RES) {
            const f2 k = make_float2(LinkPost<PX16>::k, LinkPost<PX16>::k);
            Vec3<float> accA, accB;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const f2 re = mul2(A.re[c], k);
                const f2 im = mul2(A.im[c], k);
                accA.r[c] = re.x;
                accA.i[c] = im.x;
                accB.r[c] = re.y;
                accB.i[c] = im.y;
            }
            dA_B.x = epilogue<EPI>(a, vh, iA, accA, m2, wA);
            dA_B.y = okB ? epilogue<EPI>(a, vh, iB, accB, m2, wB) : 0.f;
        } else {
            dA_B = finish_pair<EPI>(a, iA, iB, true, okB, A, m2, wA, wB);
            if (!okB) dA_B.y = 0.f;  // a missing B recomputed site A
        }
        dot.hi = dA_B.x;
        dot = ff_add(dot, FF{dA_B.y, 0.f});
    }
    if (EPI == EPI_A_DOT || EPI == EPI_A_CG || EPI == EPI_RES) {
        double total;
        if (grid_sum_ff<kBlock>(dot, reinterpret_cast<float2 *>(a.partials), a.counter, total)) {
            if (EPI == EPI_A_CG) {
                CGState *st = a.state;
                set_alpha(st, total);
            } else {
                *a.dot = total;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Staged variant (12-real links from the tile-major copy).  The eight links
// of an output site sit at that site's slot, so the links of one tile of
// kFxTile output sites and one direction mu are a single contiguous block of
// 48 KB.  One CTA of 16 warps per SM keeps a ring of kFxStages shared-memory
// stages through which the CTA's (tile, mu) items pass in order, filled by
// bulk async copies (cp.async.bulk) whose arrival an mbarrier counts in
// bytes; the threads compute two sites each exactly as k_dslash_fx2 does,
// reading the links from shared memory.  The warp that finishes reading a
// stage last (a shared-memory arrival count) refills it with the item
// kFxStages further on, so there is no producer warp and the 16 warps keep
// 128 registers each.  Up to kFxStages - 1 items of 48 KB per SM are in
// flight, independent of the registers that capped the loads in flight of
// the register-fed kernel.
//
// Each wait on an mbarrier gives up after about a second: it counts the
// event in g_fx_wait_timeouts, the CG state gets FLAG_TIMEOUT (directly, or
// through a NaN grid sum), and the CTA lets its own copies land before it
// exits.
// ---------------------------------------------------------------------------
constexpr int kFxCons = kFxTile / 2;       // threads, two sites each
constexpr int kFxConsWarps = kFxCons / 32;
constexpr int kFxCtasPerSM = 1024 / kFxTile;  // 16 warps of 128 registers per SM
#ifndef STG_FX_STAGES
#define STG_FX_STAGES 4
#endif
constexpr int kFxStages = STG_FX_STAGES;  // ring of (tile, mu) stages
constexpr unsigned kFxSmem = kFxStages * kFxStageBytes;

__device__ unsigned g_fx_wait_timeouts;

// fill ring stage st with the links of (tile, mu); one thread.  Links are
// read once per half-pass: L2 evicts them first, so the fields that the CG
// kernels re-read stay resident.
__device__ __forceinline__ void fill_stage(const char *lt, char *stage, unsigned long long *full, int st,
                                           int tile, int mu)
{
    bulk_load(stage + (size_t)st * kFxStageBytes, lt + ((size_t)tile * 4 + mu) * kFxStageBytes, kFxStageBytes,
              &full[st]);
}

template <int P, int EPI>
__global__ void __launch_bounds__(kFxCons, kFxCtasPerSM) k_dslash_fx2_staged(const DslashArgs a)
{
    extern __shared__ __align__(128) char stage[];
    __shared__ __align__(8) unsigned long long full[kFxStages];
    __shared__ unsigned done_warps[kFxStages], issued[kFxStages];
    __shared__ int abort_flag;
    const int vh = a.g.Vh;
    const int ntiles = (vh + kFxTile - 1) / kFxTile;
    const int c = threadIdx.x, lane = c & 31;
    // Before the wait only kernels two or more back have completed (the
    // predecessor triggers after its own wait); the flag's writer is one of
    // them, except for a timeout, so this read only decides whether to
    // prefetch and the check after the wait decides.
    const bool prefetch = (EPI != EPI_A_CG && EPI != EPI_GATE) ||
                          *(volatile const int *)&a.state->flag == FLAG_RUN;
    // the (tile, mu) items of this CTA in order, item q = 4 j + mu, go
    // round the ring: stage q % kFxStages, fill q / kFxStages of that stage
    if (c == 0) {
#pragma unroll
        for (int q = 0; q < kFxStages; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&full[q])) : "memory");
            done_warps[q] = 0u;
            issued[q] = 0u;
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (prefetch) {
#pragma unroll
            for (int q = 0; q < kFxStages; ++q) {
                const int tq = blockIdx.x + (q / 4) * gridDim.x;
                if (tq < ntiles) {
                    fill_stage(a.lt, stage, full, q, tq, q % 4);
                    issued[q] = 1u;
                }
            }
        }
    }
    __syncthreads();
    // the links are constant: the first fills may overlap the previous kernel
    pdl_wait();
    pdl_trigger();
    if (EPI == EPI_A_CG || EPI == EPI_GATE) {
        if (a.state->flag != FLAG_RUN) {  // uniform over the grid
            if (c == 0) {
#pragma unroll
                for (int q = 0; q < kFxStages; ++q)
                    if (issued[q]) mbar_wait(smem_addr(&full[q]), 0u, nullptr, &g_fx_wait_timeouts);
            }
            return;
        }
        if (!prefetch && c == 0) {  // the flag was lowered after the early read
#pragma unroll
            for (int q = 0; q < kFxStages; ++q) {
                const int tq = blockIdx.x + (q / 4) * gridDim.x;
                if (tq < ntiles) {
                    fill_stage(a.lt, stage, full, q, tq, q % 4);
                    issued[q] = 1u;
                }
            }
        }
        __syncthreads();
    }
    volatile int *abort = &abort_flag;
    FF dot = {0.f, 0.f};
    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
        const int iA = tile * kFxTile + c, iB = iA + kFxCons;
        const bool okA = iA < vh, okB = iB < vh;
        // slots past Vh compute on a valid site's fields (zero links), unstored
        const int jA = okA ? iA : vh - 1, jB = okB ? iB : vh - 1;
        uint4 wA = make_uint4(0u, 0u, 0u, 0u), wB = wA;
        if (EPI == EPI_A || EPI == EPI_A_DOT || EPI == EPI_A_CG) {
            wA = __ldg(static_cast<const uint4 *>(a.w) + jA);
            wB = __ldg(static_cast<const uint4 *>(a.w) + jB);
        }
        const Site sA = site_of(a.g, jA, a.parity);
        const Site sB = site_of(a.g, jB, a.parity);
        Acc2 A;
#pragma unroll
        for (int k = 0; k < 3; ++k) A.re[k] = A.im[k] = make_float2(0.f, 0.f);
        bool alive = true;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            int jfA, jbA, jfB, jbB;
            neighbours(a.g, sA, jA, mu, jfA, jbA);
            neighbours(a.g, sB, jB, mu, jfB, jbB);
            float sfA, sbA, sfB, sbB;
            link_signs(a.g, sA, mu, sfA, sbA);
            link_signs(a.g, sB, mu, sfB, sbB);
            const float k = LinkPost<P>::row2;
            const f2 s2f = make_float2(sfA * k, sfB * k);
            const f2 s2b = make_float2(sbA * k, sbB * k);
            Vec3x2 vf, vb;
            load_field2<P>(a.in, jfA, jfB, vf);
            load_field2<P>(a.in, jbA, jbB, vb);
            const int q = 4 * j + mu;          // item number
            const int sq = q % kFxStages;      // its ring stage
            const bool ready = mbar_wait(smem_addr(&full[sq]), (unsigned)(q / kFxStages) & 1u, abort,
                                         &g_fx_wait_timeouts);
            if (!__all_sync(0xffffffffu, ready)) {
                alive = false;
                break;
            }
            const char *st = stage + (size_t)sq * kFxStageBytes;
            const uint4 *f16 = reinterpret_cast<const uint4 *>(st);
            const uint2 *f8 = reinterpret_cast<const uint2 *>(st + 16 * kFxTile);
            const uint4 *b16 = reinterpret_cast<const uint4 *>(st + 24 * kFxTile);
            const uint2 *b8 = reinterpret_cast<const uint2 *>(st + 40 * kFxTile);
            const uint4 fa = f16[c], fb = f16[c + kFxCons];
            const uint2 fc = f8[c], fd = f8[c + kFxCons];
            const uint4 ba = b16[c], bb = b16[c + kFxCons];
            const uint2 bc = b8[c], bd = b8[c + kFxCons];
            // release the stage: the last warp to finish reading it refills
            // it with the item kFxStages further on
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&done_warps[sq], 1u) == kFxConsWarps - 1) {
                    done_warps[sq] = 0u;
                    const int qn = q + kFxStages;  // the item this stage holds next
                    const int tn = blockIdx.x + (qn / 4) * (int)gridDim.x;
                    if (tn < ntiles && !(a.drop_fill && qn == 4)) {
                        __threadfence_block();
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        fill_stage(a.lt, stage, full, sq, tn, qn % 4);
                        issued[sq] += 1u;
                    }
                }
            }
            Mat3x2 u;
            decode12<P>(fa, fb, fc, fd, u);
            fwd2<12>(u, vf, s2f, A);
            decode12<P>(ba, bb, bc, bd, u);
            bwd2<12>(u, vb, s2b, A);
        }
        if (!alive) {
            dot.hi = __int_as_float(0x7fc00000);  // the grid sum becomes NaN
            break;
        }
        const float m2 = (EPI == EPI_A_CG) ? float(a.state->m2) : float(a.m2);
        f2 dA_B;
        if (EPI == EPI_RES) {
            const f2 kk = make_float2(LinkPost<P>::k, LinkPost<P>::k);
            Vec3<float> accA, accB;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const f2 re = mul2(A.re[q], kk);
                const f2 im = mul2(A.im[q], kk);
                accA.r[q] = re.x;
                accA.i[q] = im.x;
                accB.r[q] = re.y;
                accB.i[q] = im.y;
            }
            dA_B.x = okA ? epilogue<EPI, P>(a, vh, iA, accA, m2, wA) : 0.f;
            dA_B.y = okB ? epilogue<EPI, P>(a, vh, iB, accB, m2, wB) : 0.f;
        } else {
            dA_B = finish_pair<EPI, P>(a, iA, iB, okA, okB, A, m2, wA, wB);
            if (!okA) dA_B.x = 0.f;
            if (!okB) dA_B.y = 0.f;
        }
        dot = ff_add(dot, FF{dA_B.x, 0.f});
        dot = ff_add(dot, FF{dA_B.y, 0.f});
    }
    __syncthreads();
    if (c == 0 && abort_flag) {
        // after a timeout, let every copy issued into this CTA land first
#pragma unroll
        for (int q = 0; q < kFxStages; ++q)
            if (issued[q]) mbar_wait(smem_addr(&full[q]), (issued[q] - 1u) & 1u, nullptr, &g_fx_wait_timeouts);
        if (EPI == EPI_GATE) a.state->flag = FLAG_TIMEOUT;  // no grid sum here
    }
    if (EPI == EPI_A_DOT || EPI == EPI_A_CG || EPI == EPI_RES) {
        double total;
        if (grid_sum_ff<kFxCons>(dot, reinterpret_cast<float2 *>(a.partials), a.counter, total)) {
            if (EPI == EPI_A_CG) {
                CGState *st = a.state;
                if (!isfinite(total) && *(volatile unsigned *)&g_fx_wait_timeouts) {
                    st->pAp = total;
                    st->flag = FLAG_TIMEOUT;
                } else {
                    set_alpha(st, total);
                }
            } else {
                *a.dot = total;
            }
        }
    }
}

template <int P, int EPI>
static void launch_staged(const DslashArgs &a, cudaStream_t s, bool pdl)
{
    // set once per instantiation (thread-safe static initialisation)
    static const int sms = [] {
        cudaFuncSetAttribute(k_dslash_fx2_staged<P, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFxSmem);
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        return n;
    }();
    // a.grid_cap (STG_FX16_GRID at handle creation) caps the CTA count, so
    // that each CTA walks more tiles (tests); a.drop_fill is the failure-
    // detection test's withheld fill (a CTA's wait for its second tile runs
    // out after about a second; no fault, no hang)
    int cap = sms * kFxCtasPerSM;
    if (a.grid_cap > 0 && a.grid_cap < cap) cap = a.grid_cap;
    const int ntiles = (a.g.Vh + kFxTile - 1) / kFxTile;
    const int grid = ntiles < cap ? ntiles : cap;
    launch_k(k_dslash_fx2_staged<P, EPI>, grid, kFxCons, kFxSmem, s, pdl, a);
}

template <int R>
static void launch_r(int epi, const DslashArgs &a, int grid, cudaStream_t s, bool pdl)
{
    switch (epi) {
    case EPI_NONE: launch_k(k_dslash_fx2<R, EPI_NONE>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_A: launch_k(k_dslash_fx2<R, EPI_A>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_A_DOT: launch_k(k_dslash_fx2<R, EPI_A_DOT>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_A_CG: launch_k(k_dslash_fx2<R, EPI_A_CG>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_RES: launch_k(k_dslash_fx2<R, EPI_RES>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_GATE: launch_k(k_dslash_fx2<R, EPI_GATE>, grid, kBlock, 0, s, pdl, a); break;
    }
}

template <int P>
static void launch_staged_p(int epi, const DslashArgs &a, cudaStream_t s, bool pdl)
{
    switch (epi) {
    case EPI_NONE: launch_staged<P, EPI_NONE>(a, s, pdl); break;
    case EPI_A: launch_staged<P, EPI_A>(a, s, pdl); break;
    case EPI_A_DOT: launch_staged<P, EPI_A_DOT>(a, s, pdl); break;
    case EPI_A_CG: launch_staged<P, EPI_A_CG>(a, s, pdl); break;
    case EPI_RES: launch_staged<P, EPI_RES>(a, s, pdl); break;
    case EPI_GATE: launch_staged<P, EPI_GATE>(a, s, pdl); break;
    }
}

// IEEE FP16 / 12-real links in the tile-major copy: the staged kernel with
// binary16 decode and encode
void launch_dslash_f16_staged(int epi, const DslashArgs &a, cudaStream_t s, bool pdl)
{
    launch_staged_p<P16>(epi, a, s, pdl);
}

void launch_dslash_fx2(int recon, int epi, const DslashArgs &a, cudaStream_t s, bool pdl)
{
    if (recon == 12 && a.lt) {
        launch_staged_p<PX16>(epi, a, s, pdl);
        return;
    }
    const int grid = (a.g.Vh + 2 * kBlock - 1) / (2 * kBlock);
    if (recon == 18) launch_r<18>(epi, a, grid, s, pdl);
    else launch_r<12>(epi, a, grid, s, pdl);
}

}  // namespace stg
