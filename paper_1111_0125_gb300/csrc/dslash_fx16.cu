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
// Signs are never negated in the inner loops: each colour keeps positive and
// negative real / imaginary accumulators (Pr, Nr, Pi, Ni) and D chi =
// (Pr - Nr) + i (Pi - Ni) once at the end.  Links are integer-valued floats
// (32767 U); the sum is scaled by 1/32767 at the end, and the 12-real row 2
// c = r0 x r1 enters the products with the factor s / 32767 (s the folded
// phase), i.e. U_2b = (s / 32767) conj(c_b).
#include "stg_internal.h"

#ifndef STG_FX2_MINBLOCKS
#define STG_FX2_MINBLOCKS 2
#endif

namespace stg {

typedef float2 f2;

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// biased fixed-point decode (see fx_lo / fx_hi): 1.5 * 2^23 + u, then the
// subtraction of 1.5 * 2^23 + 32768 happens once for both sites
__device__ __forceinline__ float fxb_lo(unsigned w) { return __int_as_float((int)__byte_perm(w, 0x4B40u, 0x5410)); }
__device__ __forceinline__ float fxb_hi(unsigned w) { return __int_as_float((int)__byte_perm(w, 0x4B40u, 0x5432)); }
__device__ __forceinline__ f2 unbias(float a, float b)
{
    return add2(make_float2(a, b), make_float2(-12615680.f, -12615680.f));
}

struct Mat3x2 {
    f2 r[3][3], i[3][3];
};
struct Vec3x2 {
    f2 r[3], i[3];
};

__device__ __forceinline__ void set2(Mat3x2 &u, int k, unsigned wa, unsigned wb)
{
    u.r[k / 3][k % 3] = unbias(fxb_lo(wa), fxb_lo(wb));
    u.i[k / 3][k % 3] = unbias(fxb_hi(wa), fxb_hi(wb));
}

// link of site A (index sa) and site B (index sb) of one (parity, mu) block;
// for 12-real, row 2 holds c = r0 x r1 (no conjugate, no sign, 32767^2 scale)
template <int R>
__device__ __forceinline__ void load_link2(const char *blk, int vh, int sa, int sb, Mat3x2 &u)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(blk);
    const uint4 a = ld_stream(p + sa), b = ld_stream(p + sb);
    set2(u, 0, a.x, b.x);
    set2(u, 1, a.y, b.y);
    set2(u, 2, a.z, b.z);
    set2(u, 3, a.w, b.w);
    if (R == 18) {
        const uint4 c = ld_stream(p + (size_t)vh + sa), d = ld_stream(p + (size_t)vh + sb);
        set2(u, 4, c.x, d.x);
        set2(u, 5, c.y, d.y);
        set2(u, 6, c.z, d.z);
        set2(u, 7, c.w, d.w);
        const unsigned *q = reinterpret_cast<const unsigned *>(p + (size_t)2 * vh);
        set2(u, 8, ld_stream(q + sa), ld_stream(q + sb));
    } else {
        const uint2 *q = reinterpret_cast<const uint2 *>(p + (size_t)vh);
        const uint2 c = ld_stream(q + sa), d = ld_stream(q + sb);
        set2(u, 4, c.x, d.x);
        set2(u, 5, c.y, d.y);
#pragma unroll
        for (int a2 = 0; a2 < 3; ++a2) {
            const int b2 = (a2 + 1) % 3, c2 = (a2 + 2) % 3;
            // c = r0_b r1_c - r0_c r1_b, split into positive and negative terms
            const f2 pr = fma2(u.r[0][b2], u.r[1][c2], mul2(u.i[0][c2], u.i[1][b2]));
            const f2 nr = fma2(u.i[0][b2], u.i[1][c2], mul2(u.r[0][c2], u.r[1][b2]));
            const f2 pi = fma2(u.r[0][b2], u.i[1][c2], mul2(u.i[0][b2], u.r[1][c2]));
            const f2 ni = fma2(u.r[0][c2], u.i[1][b2], mul2(u.i[0][c2], u.r[1][b2]));
            u.r[2][a2] = sub2(pr, nr);
            u.i[2][a2] = sub2(pi, ni);
        }
    }
}

__device__ __forceinline__ void load_field2(const void *f, int sa, int sb, Vec3x2 &v)
{
    const uint4 *p = static_cast<const uint4 *>(f);
    const uint4 a = __ldg(p + sa), b = __ldg(p + sb);
    const f2 sc = make_float2(__uint_as_float(a.w), __uint_as_float(b.w));
    v.r[0] = mul2(unbias(fxb_lo(a.x), fxb_lo(b.x)), sc);
    v.i[0] = mul2(unbias(fxb_hi(a.x), fxb_hi(b.x)), sc);
    v.r[1] = mul2(unbias(fxb_lo(a.y), fxb_lo(b.y)), sc);
    v.i[1] = mul2(unbias(fxb_hi(a.y), fxb_hi(b.y)), sc);
    v.r[2] = mul2(unbias(fxb_lo(a.z), fxb_lo(b.z)), sc);
    v.i[2] = mul2(unbias(fxb_hi(a.z), fxb_hi(b.z)), sc);
}

struct Acc2 {
    f2 pr[3], nr[3], pi[3], ni[3];
};

// acc += U v; for 12-real, row 2 of U is s2 conj(c)
template <int R>
__device__ __forceinline__ void fwd2(const Mat3x2 &u, const Vec3x2 &v, f2 s2, Acc2 &A)
{
    constexpr int nrow = R == 18 ? 3 : 2;
#pragma unroll
    for (int a = 0; a < nrow; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            A.pr[a] = fma2(u.r[a][b], v.r[b], A.pr[a]);
            A.nr[a] = fma2(u.i[a][b], v.i[b], A.nr[a]);
            A.pi[a] = fma2(u.r[a][b], v.i[b], A.pi[a]);
            A.pi[a] = fma2(u.i[a][b], v.r[b], A.pi[a]);
        }
    if (R == 12) {
        // sum_b conj(c_b) v_b = sum (c.r v.r + c.i v.i) + i sum (c.r v.i - c.i v.r)
        f2 wr = mul2(u.r[2][0], v.r[0]);
        f2 wp = mul2(u.r[2][0], v.i[0]);
        f2 wn = mul2(u.i[2][0], v.r[0]);
        wr = fma2(u.i[2][0], v.i[0], wr);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            wr = fma2(u.r[2][b], v.r[b], wr);
            wr = fma2(u.i[2][b], v.i[b], wr);
            wp = fma2(u.r[2][b], v.i[b], wp);
            wn = fma2(u.i[2][b], v.r[b], wn);
        }
        A.pr[2] = fma2(s2, wr, A.pr[2]);
        A.pi[2] = fma2(s2, wp, A.pi[2]);
        A.ni[2] = fma2(s2, wn, A.ni[2]);
    }
}

// acc -= U^dag v; for 12-real, conj(U_2a) = s2 c_a
template <int R>
__device__ __forceinline__ void bwd2(const Mat3x2 &u, const Vec3x2 &v, f2 s2, Acc2 &A)
{
    constexpr int nrow = R == 18 ? 3 : 2;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < nrow; ++b) {
            // conj(U_ba) v_b = (u.r v.r + u.i v.i) + i (u.r v.i - u.i v.r)
            A.nr[a] = fma2(u.r[b][a], v.r[b], A.nr[a]);
            A.nr[a] = fma2(u.i[b][a], v.i[b], A.nr[a]);
            A.ni[a] = fma2(u.r[b][a], v.i[b], A.ni[a]);
            A.pi[a] = fma2(u.i[b][a], v.r[b], A.pi[a]);
        }
    if (R == 12) {
        // s2 c_a v_2 = s2 (c.r v.r - c.i v.i) + i s2 (c.r v.i + c.i v.r)
        const f2 wr = mul2(s2, v.r[2]), wi = mul2(s2, v.i[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.nr[a] = fma2(u.r[2][a], wr, A.nr[a]);
            A.pr[a] = fma2(u.i[2][a], wi, A.pr[a]);
            A.ni[a] = fma2(u.r[2][a], wi, A.ni[a]);
            A.ni[a] = fma2(u.i[2][a], wr, A.ni[a]);
        }
    }
}

// decode one FX16 site record already in registers
__device__ __forceinline__ Vec3<float> fx_decode(uint4 u)
{
    const float sc = __uint_as_float(u.w);
    Vec3<float> v;
    v.r[0] = fx_lo(u.x) * sc; v.i[0] = fx_hi(u.x) * sc;
    v.r[1] = fx_lo(u.y) * sc; v.i[1] = fx_hi(u.y) * sc;
    v.r[2] = fx_lo(u.z) * sc; v.i[2] = fx_hi(u.z) * sc;
    return v;
}

// the scalar epilogue of one site (same arithmetic as k_dslash's); wraw is
// the site's record of w, loaded at kernel start for the A epilogues
template <int EPI>
__device__ __forceinline__ float epilogue(const DslashArgs &a, int vh, int i, const Vec3<float> &acc,
                                          float m2, uint4 wraw)
{
    float dot = 0.f;
    if (EPI == EPI_NONE || EPI == EPI_GATE) {
        FieldIO<PX16>::store(a.out, vh, i, acc);
    } else if (EPI == EPI_RES) {
        const Vec3<float> b = FieldIO<PX16>::load_nc(a.w, vh, i);
        const Vec3<float> x = FieldIO<PX16>::load_nc(a.v, vh, i);
        Vec3<float> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = b.r[c] - m2 * x.r[c] + acc.r[c];
            o.i[c] = b.i[c] - m2 * x.i[c] + acc.i[c];
        }
        const Vec3<float> os = FieldIO<PX16>::store(a.out, vh, i, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) dot += os.r[c] * os.r[c] + os.i[c] * os.i[c];
    } else {
        const Vec3<float> d = fx_decode(wraw);
        Vec3<float> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.r[c] = m2 * d.r[c] - acc.r[c];
            o.i[c] = m2 * d.i[c] - acc.i[c];
        }
        const Vec3<float> os = FieldIO<PX16>::store(a.out, vh, i, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) dot += d.r[c] * os.r[c] + d.i[c] * os.i[c];
    }
    return dot;
}

template <int R, int EPI>
__global__ void __launch_bounds__(kBlock, STG_FX2_MINBLOCKS) k_dslash_fx2(const DslashArgs a)
{
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
        for (int c = 0; c < 3; ++c) A.pr[c] = A.nr[c] = A.pi[c] = A.ni[c] = make_float2(0.f, 0.f);
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
        const f2 k = make_float2(LinkPost<PX16>::k, LinkPost<PX16>::k);
        Vec3<float> accA, accB;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const f2 re = mul2(sub2(A.pr[c], A.nr[c]), k);
            const f2 im = mul2(sub2(A.pi[c], A.ni[c]), k);
            accA.r[c] = re.x;
            accA.i[c] = im.x;
            accB.r[c] = re.y;
            accB.i[c] = im.y;
        }
        const float m2 = (EPI == EPI_A_CG) ? float(a.state->m2) : float(a.m2);
        const float dA = epilogue<EPI>(a, vh, iA, accA, m2, wA);
        float dB = 0.f;
        if (okB) dB = epilogue<EPI>(a, vh, iB, accB, m2, wB);
        dot.hi = dA;
        dot = ff_add(dot, FF{dB, 0.f});
    }
    if (EPI == EPI_A_DOT || EPI == EPI_A_CG || EPI == EPI_RES) {
        double total;
        if (grid_sum_ff<kBlock>(dot, reinterpret_cast<float2 *>(a.partials), a.counter, total)) {
            if (EPI == EPI_A_CG) {
                CGState *st = a.state;
                st->pAp = total;
                if (!(total > 0.0) || !isfinite(total)) st->flag = FLAG_BREAKDOWN;
                else st->alpha = st->delta_new / total;
            } else {
                *a.dot = total;
            }
        }
    }
}

template <int R>
static void launch_r(int epi, const DslashArgs &a, int grid, cudaStream_t s)
{
    switch (epi) {
    case EPI_NONE: k_dslash_fx2<R, EPI_NONE><<<grid, kBlock, 0, s>>>(a); break;
    case EPI_A: k_dslash_fx2<R, EPI_A><<<grid, kBlock, 0, s>>>(a); break;
    case EPI_A_DOT: k_dslash_fx2<R, EPI_A_DOT><<<grid, kBlock, 0, s>>>(a); break;
    case EPI_A_CG: k_dslash_fx2<R, EPI_A_CG><<<grid, kBlock, 0, s>>>(a); break;
    case EPI_RES: k_dslash_fx2<R, EPI_RES><<<grid, kBlock, 0, s>>>(a); break;
    case EPI_GATE: k_dslash_fx2<R, EPI_GATE><<<grid, kBlock, 0, s>>>(a); break;
    }
}

void launch_dslash_fx2(int recon, int epi, const DslashArgs &a, cudaStream_t s)
{
    const int grid = (a.g.Vh + 2 * kBlock - 1) / (2 * kBlock);
    if (recon == 18) launch_r<18>(epi, a, grid, s);
    else launch_r<12>(epi, a, grid, s);
}

}  // namespace stg
