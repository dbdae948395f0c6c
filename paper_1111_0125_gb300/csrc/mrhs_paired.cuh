// Staged multi-system Dslash for FX16 / 12-real links with two sites per
// thread on packed FP32x2 arithmetic (Eq. 5, and A of Eq. 3 with the fused
// d_k^dag q_k).
//
// With several systems per gauge field the link bytes per site and system
// fall as 8L / n, so the half-pass becomes bound by its arithmetic: eight
// SU(3) mat-vecs per site and system.  This kernel keeps the staging of
// k_dslash_ms (the eight links of a 64-site tile arrive in shared memory by
// one bulk copy and serve every system) and computes like the single-system
// FX16 kernel: thread `lane` of a warp owns the site pair (lane, lane + 32)
// of the tile, decodes each link of both sites once into the halves of
// float2 registers (12-real row 2 rebuilt there too), and applies it to NB
// systems per pass with one FP32x2 instruction per product for both sites.
// The 16-bit fields decode straight into the pair halves (one byte permute
// per value and one FMA per pair), so no instruction moves values into
// pairs.  Warp w handles systems w, w + 4, ... (four warps per CTA).
//
// Stage waits give up after about a second as in k_dslash_ms; the systems'
// reductions then become NaN and the solver stops them with a timeout.
#pragma once

#include "fx16_pair.cuh"
#include "mrhs_kernels.cuh"

namespace stg {

#ifndef STG_MSP_STAGES
#define STG_MSP_STAGES 3
#endif
constexpr int kMspThreads = 128;
constexpr int kMspWarps = kMspThreads / 32;  // system groups
constexpr int kMspStages = STG_MSP_STAGES;
// kMspShapes (mrhs_kernels.cuh): NB = 2, 4
__host__ __device__ constexpr int msp_nb(int k) { return k == 0 ? 2 : 4; }

static __device__ unsigned g_msp_wait_timeouts;

template <int NB, int EPI>
__global__ void __launch_bounds__(kMspThreads, NB == 2 ? 4 : 3) k_dslash_msp(const MrhsArgs a)
{
    constexpr unsigned SB = ms_stage_bytes<PX16>();  // 64 sites x 8 links x 24 B
    constexpr unsigned LB = kMTile * 24;             // one (mu, direction) block
    extern __shared__ __align__(128) char stage[];
    __shared__ __align__(8) unsigned long long full[kMspStages];
    __shared__ unsigned done_warps[kMspStages], issued[kMspStages];
    __shared__ int abort_flag;
    __shared__ FF sysw[kMspWarps][kMaxRhs];  // EPI_A_CG: per-warp d^dag q per list slot
    const int vh = a.g.Vh;
    const int ntiles = (vh + kMTile - 1) / kMTile;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int nact = a.active ? *a.nactive : a.nrhs;
    const int per = (nact + kMspWarps - 1) / kMspWarps;  // list slots per warp (uniform bound)

    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kMspStages; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&full[q])) : "memory");
            done_warps[q] = 0u;
            issued[q] = 0u;
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
        for (int q = 0; q < kMspStages; ++q) {
            const int tile = blockIdx.x + q * gridDim.x;
            if (tile < ntiles) {
                bulk_load(stage + (size_t)q * SB, a.lt + (size_t)tile * SB, SB, &full[q]);
                issued[q] = 1u;
            }
        }
    }
    if (EPI == EPI_A_CG)
        for (int k = threadIdx.x; k < kMspWarps * kMaxRhs; k += kMspThreads)
            sysw[k / kMaxRhs][k % kMaxRhs] = FF{0.f, 0.f};
    __syncthreads();
    volatile int *abort = &abort_flag;

    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
        const int st = j % kMspStages;
        const unsigned par = (unsigned)(j / kMspStages) & 1u;
        const int iA = tile * kMTile + lane, iB = iA + 32;
        const bool okA = iA < vh, okB = iB < vh;
        // past Vh: a valid site's fields, zero links, unstored
        const int jA = okA ? iA : vh - 1, jB = okB ? iB : vh - 1;
        const Site sA = site_of(a.g, jA, a.parity);
        const Site sB = site_of(a.g, jB, a.parity);
        const bool ready = mbar_wait(smem_addr(&full[st]), par, abort, &g_msp_wait_timeouts);
        if (!__syncthreads_and(ready)) break;  // uniform over the CTA
        const char *sb = stage + (size_t)st * SB;

        for (int k0 = 0; k0 < per; k0 += NB) {
            int rid[NB];
            bool run[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int kk = grp + kMspWarps * (k0 + q);
                run[q] = kk < nact;
                rid[q] = run[q] ? (a.active ? a.active[kk] : kk) : 0;
                if (EPI == EPI_GATE || EPI == EPI_A_CG)
                    run[q] = run[q] && a.states[rid[q]].flag == FLAG_RUN;
            }
            Acc2 acc[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[q].re[c] = acc[q].im[c] = make_float2(0.f, 0.f);
            // no branches in the hot loop: a slot that is not running reads
            // system rid = 0 (valid memory) and its result is dropped below
            // one direction at a time (unrolled, the NB systems' fields of
            // all four would not fit the registers)
#pragma unroll 1
            for (int mu = 0; mu < 4; ++mu) {
                int jfA, jbA, jfB, jbB;
                neighbours(a.g, sA, jA, mu, jfA, jbA);
                neighbours(a.g, sB, jB, mu, jfB, jbB);
                float sfA, sbA, sfB, sbB;
                link_signs(a.g, sA, mu, sfA, sbA);
                link_signs(a.g, sB, mu, sfB, sbB);
                const float k2 = LinkPost<PX16>::row2;
                const f2 s2f = make_float2(sfA * k2, sfB * k2);
                const f2 s2b = make_float2(sbA * k2, sbB * k2);
                Mat3x2 u;
                {
                    const char *blk = sb + (size_t)(2 * mu) * LB;
                    const uint4 *p16 = reinterpret_cast<const uint4 *>(blk);
                    const uint2 *p8 = reinterpret_cast<const uint2 *>(blk + 16 * kMTile);
                    decode12(p16[lane], p16[lane + 32], p8[lane], p8[lane + 32], u);
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    Vec3x2 v;
                    load_field2(a.in + rid[q] * a.fstride, jfA, jfB, v);
                    fwd2<12>(u, v, s2f, acc[q]);
                }
                {
                    const char *blk = sb + (size_t)(2 * mu + 1) * LB;
                    const uint4 *p16 = reinterpret_cast<const uint4 *>(blk);
                    const uint2 *p8 = reinterpret_cast<const uint2 *>(blk + 16 * kMTile);
                    decode12(p16[lane], p16[lane + 32], p8[lane], p8[lane + 32], u);
                }
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    Vec3x2 v;
                    load_field2(a.in + rid[q] * a.fstride, jbA, jbB, v);
                    bwd2<12>(u, v, s2b, acc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                FF dot = {0.f, 0.f};
                if (run[q]) {
                    constexpr bool neg = (EPI == EPI_A || EPI == EPI_A_CG);
                    const f2 k = make_float2(neg ? -LinkPost<PX16>::k : LinkPost<PX16>::k,
                                             neg ? -LinkPost<PX16>::k : LinkPost<PX16>::k);
                    f2 dr[3], di[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        dr[c] = mul2(acc[q].re[c], k);
                        di[c] = mul2(acc[q].im[c], k);
                    }
                    char *out = a.out + rid[q] * a.fstride;
                    if (EPI == EPI_NONE || EPI == EPI_GATE) {
                        epilogue_pair<EPI_NONE>(out, iA, iB, okA, okB, dr, di, 0.f, make_uint4(0, 0, 0, 0),
                                                make_uint4(0, 0, 0, 0));
                    } else {
                        const float m2 = (EPI == EPI_A_CG) ? float(a.states[rid[q]].m2) : a.m2[rid[q]];
                        const uint4 *w = reinterpret_cast<const uint4 *>(a.w + rid[q] * a.fstride);
                        const uint4 wA = __ldg(w + jA), wB = __ldg(w + jB);
                        const f2 d2 = epilogue_pair<EPI_A_DOT>(out, iA, iB, okA, okB, dr, di, m2, wA, wB);
                        if (okA) dot = ff_add(dot, FF{d2.x, 0.f});
                        if (okB) dot = ff_add(dot, FF{d2.y, 0.f});
                    }
                }
                if (EPI == EPI_A_CG) {
                    // the warp's 32 lanes hold sites of the same system
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dot = ff_add(dot, ff_shfl_down(dot, o));
                    const int kk = grp + kMspWarps * (k0 + q);
                    if (lane == 0 && kk < nact) sysw[grp][kk] = ff_add(sysw[grp][kk], dot);
                }
            }
        }
        // release the stage: the last warp to finish refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&done_warps[st], 1u) == kMspWarps - 1) {
                done_warps[st] = 0u;
                const int next = tile + kMspStages * (int)gridDim.x;
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
        for (int q = 0; q < kMspStages; ++q)
            if (issued[q] > 0u) mbar_wait(smem_addr(&full[q]), (issued[q] - 1u) & 1u, nullptr, &g_msp_wait_timeouts);
    }

    if (EPI == EPI_A_CG) {
        for (int kk = threadIdx.x; kk < nact; kk += kMspThreads) {
            FF sum = sysw[0][kk];
#pragma unroll
            for (int w = 1; w < kMspWarps; ++w) sum = ff_add(sum, sysw[w][kk]);
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
        for (int kk = grp; kk < nact; kk += kMspWarps) {
            const int k = a.active ? a.active[kk] : kk;
            if (a.states[k].flag != FLAG_RUN) continue;  // uniform in the warp
            FF acc = {0.f, 0.f};
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const float2 p = __ldcg(a.partials + (size_t)k * gridDim.x + b);
                acc = ff_add(acc, FF{p.x, p.y});
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_down(acc, o));
            if (lane == 0) {
                CGState *st = a.states + k;
                const double total = (double)acc.hi + (double)acc.lo;
                if (!isfinite(total) && *(volatile unsigned *)&g_msp_wait_timeouts) {
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

template <int NB>
void launch_msp_nb(int epi, const MrhsArgs &a, cudaStream_t s)
{
    constexpr unsigned smem = kMspStages * ms_stage_bytes<PX16>();
    // set once per instantiation (thread-safe static initialisation):
    // resident CTAs on the whole GPU
    static const int resident = [] {
        cudaFuncSetAttribute(k_dslash_msp<NB, EPI_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_dslash_msp<NB, EPI_A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_dslash_msp<NB, EPI_GATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_dslash_msp<NB, EPI_A_CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash_msp<NB, EPI_A_CG>, kMspThreads,
                                                          smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return sms * per_sm;
    }();
    const int ntiles = (a.g.Vh + kMTile - 1) / kMTile;
    int cap = resident;
    if (a.grid_limit > 0 && a.grid_limit < cap) cap = a.grid_limit;
    const int grid = ntiles < cap ? ntiles : cap;
    switch (epi) {
    case EPI_NONE: k_dslash_msp<NB, EPI_NONE><<<grid, kMspThreads, smem, s>>>(a); break;
    case EPI_A: k_dslash_msp<NB, EPI_A><<<grid, kMspThreads, smem, s>>>(a); break;
    case EPI_GATE: k_dslash_msp<NB, EPI_GATE><<<grid, kMspThreads, smem, s>>>(a); break;
    case EPI_A_CG: k_dslash_msp<NB, EPI_A_CG><<<grid, kMspThreads, smem, s>>>(a); break;
    }
}

inline void launch_msp(int k, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (k == 0) launch_msp_nb<2>(epi, a, s);
    else launch_msp_nb<4>(epi, a, s);
}

}  // namespace stg
