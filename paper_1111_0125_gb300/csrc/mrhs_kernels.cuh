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
                for (int q = 0; q < NB; ++q) mul_add(uf, v[q], acc[q], s2f[mu]);
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
                st->pAp = total;
                if (!(total > 0.0) || !isfinite(total)) st->flag = FLAG_BREAKDOWN;
                else st->alpha = st->delta_new / total;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) *a.counter = 0u;
    }
}

// (NB, TPS) shapes the autotuner chooses from
constexpr int kMrhsShapes = 9;
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
