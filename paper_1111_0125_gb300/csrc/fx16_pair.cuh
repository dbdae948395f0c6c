// Two sites (or two systems) per thread on packed FP32x2 arithmetic for the
// 16-bit storage forms FX16 (16-bit fixed point; the default template
// argument P) and IEEE FP16 (P16, per-site field scale, unscaled links): the
// .x half of every float2 holds one site's value and the .y half the
// other's, and every FP32 operation is one sm_100 FP32x2 instruction
// (__ffma2_rn, __fadd2_rn, __fmul2_rn) for both.  Shared by the single-system
// 16-bit Dslash (dslash_fx16.cu) and the staged multi-system kernel with site
// pairs (mrhs_paired.cuh).
//
// FX16 links are integer-valued floats (32767 U); a kernel scales its sum by
// 1/32767 at the end (LinkPost<P>::k), and the 12-real row 2 c = r0 x r1
// enters the products with the factor s LinkPost<P>::row2 (s the folded
// phase), i.e. U_2b = (s / 32767) conj(c_b); FP16 links carry U itself.  Each colour keeps one real and one imaginary accumulator; the
// signs of the products are carried by negated FP32x2 operands, which cost
// no instruction.
#pragma once

#include "stg_internal.h"

namespace stg {

typedef float2 f2;

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }

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

// the halves of one binary16 word as floats
__device__ __forceinline__ float h_lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))); }
__device__ __forceinline__ float h_hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

// one (re, im) word of site A (wa) and of site B (wb) as (A, B) pairs
template <int P = PX16>
__device__ __forceinline__ void word2(unsigned wa, unsigned wb, f2 &re, f2 &im)
{
    static_assert(P == PX16 || P == P16, "16-bit pair forms: FX16 and FP16");
    if constexpr (P == PX16) {
        re = unbias(fxb_lo(wa), fxb_lo(wb));
        im = unbias(fxb_hi(wa), fxb_hi(wb));
    } else {
        re = make_float2(h_lo(wa), h_lo(wb));
        im = make_float2(h_hi(wa), h_hi(wb));
    }
}

template <int P = PX16>
__device__ __forceinline__ void set2(Mat3x2 &u, int k, unsigned wa, unsigned wb)
{
    word2<P>(wa, wb, u.r[k / 3][k % 3], u.i[k / 3][k % 3]);
}

// 12-real: row 2 is c = r0 x r1 (no conjugate, no sign; FX16: 32767^2 scale);
// a / b hold rows 0-1 entries 0-3 of sites A / B, c / d entries 4-5
template <int P = PX16>
__device__ __forceinline__ void decode12(const uint4 &a, const uint4 &b, const uint2 &c, const uint2 &d,
                                         Mat3x2 &u)
{
    set2<P>(u, 0, a.x, b.x);
    set2<P>(u, 1, a.y, b.y);
    set2<P>(u, 2, a.z, b.z);
    set2<P>(u, 3, a.w, b.w);
    set2<P>(u, 4, c.x, d.x);
    set2<P>(u, 5, c.y, d.y);
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2) {
        const int b2 = (a2 + 1) % 3, c2 = (a2 + 2) % 3;
        // c = r0_b r1_c - r0_c r1_b as one FMA chain per part (the negated
        // operands cost no instruction)
        const f2 nrc = make_float2(-u.r[0][c2].x, -u.r[0][c2].y);
        const f2 nib = make_float2(-u.i[0][b2].x, -u.i[0][b2].y);
        const f2 nic = make_float2(-u.i[0][c2].x, -u.i[0][c2].y);
        f2 re = mul2(u.r[0][b2], u.r[1][c2]);
        re = fma2(nib, u.i[1][c2], re);
        re = fma2(nrc, u.r[1][b2], re);
        re = fma2(u.i[0][c2], u.i[1][b2], re);
        f2 im = mul2(u.r[0][b2], u.i[1][c2]);
        im = fma2(u.i[0][b2], u.r[1][c2], im);
        im = fma2(nrc, u.i[1][b2], im);
        im = fma2(nic, u.r[1][b2], im);
        u.r[2][a2] = re;
        u.i[2][a2] = im;
    }
}

// link of site A (index sa) and site B (index sb) of one (parity, mu) block
template <int R>
__device__ __forceinline__ void load_link2(const char *blk, int vh, int sa, int sb, Mat3x2 &u)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(blk);
    const uint4 a = ld_stream(p + sa), b = ld_stream(p + sb);
    if (R == 18) {
        set2(u, 0, a.x, b.x);
        set2(u, 1, a.y, b.y);
        set2(u, 2, a.z, b.z);
        set2(u, 3, a.w, b.w);
        const uint4 c = ld_stream(p + (size_t)vh + sa), d = ld_stream(p + (size_t)vh + sb);
        set2(u, 4, c.x, d.x);
        set2(u, 5, c.y, d.y);
        set2(u, 6, c.z, d.z);
        set2(u, 7, c.w, d.w);
        const unsigned *q = reinterpret_cast<const unsigned *>(p + (size_t)2 * vh);
        set2(u, 8, ld_stream(q + sa), ld_stream(q + sb));
    } else {
        const uint2 *q = reinterpret_cast<const uint2 *>(p + (size_t)vh);
        decode12(a, b, ld_stream(q + sa), ld_stream(q + sb), u);
    }
}

// value = (u - 1.5 * 2^23 - 32768) s: the offset removed by one add and the
// scale applied by one multiply per pair.  (One FMA, (K + q) s - K s with
// K s precomputed, is exact for the 15-bit scales of fx_scale and saves an
// instruction, but measured about 1% slower on the half-pass: it puts the
// multiply K s on the critical path of every neighbour.)
// (FP16: the binary16 value times the site's scale, as FieldIO<P16>)
template <int P = PX16>
__device__ __forceinline__ void load_field2(const void *f, int sa, int sb, Vec3x2 &v)
{
    const uint4 *p = static_cast<const uint4 *>(f);
    const uint4 a = __ldg(p + sa), b = __ldg(p + sb);
    const f2 sc = make_float2(__uint_as_float(a.w), __uint_as_float(b.w));
    f2 r, i;
    word2<P>(a.x, b.x, r, i);
    v.r[0] = mul2(r, sc);
    v.i[0] = mul2(i, sc);
    word2<P>(a.y, b.y, r, i);
    v.r[1] = mul2(r, sc);
    v.i[1] = mul2(i, sc);
    word2<P>(a.z, b.z, r, i);
    v.r[2] = mul2(r, sc);
    v.i[2] = mul2(i, sc);
}

// D chi accumulated as (re, im) per colour; the signs of the products sit
// on the operands (negated FP32x2 operands cost no instruction)
struct Acc2 {
    f2 re[3], im[3];
};

__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }

// acc += U v; for 12-real, row 2 of U is s2 conj(c)
template <int R>
__device__ __forceinline__ void fwd2(const Mat3x2 &u, const Vec3x2 &v, f2 s2, Acc2 &A)
{
    constexpr int nrow = R == 18 ? 3 : 2;
#pragma unroll
    for (int a = 0; a < nrow; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            A.re[a] = fma2(u.r[a][b], v.r[b], A.re[a]);
            A.re[a] = fma2(neg2(u.i[a][b]), v.i[b], A.re[a]);
            A.im[a] = fma2(u.r[a][b], v.i[b], A.im[a]);
            A.im[a] = fma2(u.i[a][b], v.r[b], A.im[a]);
        }
    if (R == 12) {
        // sum_b conj(c_b) v_b = sum (c.r v.r + c.i v.i) + i sum (c.r v.i - c.i v.r)
        f2 wr = mul2(u.r[2][0], v.r[0]);
        f2 wi = mul2(u.r[2][0], v.i[0]);
        wr = fma2(u.i[2][0], v.i[0], wr);
        wi = fma2(neg2(u.i[2][0]), v.r[0], wi);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            wr = fma2(u.r[2][b], v.r[b], wr);
            wr = fma2(u.i[2][b], v.i[b], wr);
            wi = fma2(u.r[2][b], v.i[b], wi);
            wi = fma2(neg2(u.i[2][b]), v.r[b], wi);
        }
        A.re[2] = fma2(s2, wr, A.re[2]);
        A.im[2] = fma2(s2, wi, A.im[2]);
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
            A.re[a] = fma2(neg2(u.r[b][a]), v.r[b], A.re[a]);
            A.re[a] = fma2(neg2(u.i[b][a]), v.i[b], A.re[a]);
            A.im[a] = fma2(neg2(u.r[b][a]), v.i[b], A.im[a]);
            A.im[a] = fma2(u.i[b][a], v.r[b], A.im[a]);
        }
    if (R == 12) {
        // s2 c_a v_2 = s2 (c.r v.r - c.i v.i) + i s2 (c.r v.i + c.i v.r)
        const f2 wr = mul2(s2, v.r[2]), wi = mul2(s2, v.i[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.re[a] = fma2(neg2(u.r[2][a]), wr, A.re[a]);
            A.re[a] = fma2(u.i[2][a], wi, A.re[a]);
            A.im[a] = fma2(neg2(u.r[2][a]), wi, A.im[a]);
            A.im[a] = fma2(neg2(u.i[2][a]), wr, A.im[a]);
        }
    }
}

// decode the FX16 records of sites A and B into .x / .y: (K + q) s - K s as
// one FMA per pair with K s precomputed, exact (one rounding, bitwise q * s)
// because fx_scale keeps 15 significant bits and K = 1.5 * 2^23 + 32768 has 9
// (FP16: the binary16 values times the sites' scales, as FieldIO<P16>)
template <int P = PX16>
__device__ __forceinline__ void decode_fx2(const uint4 &a, const uint4 &b, f2 (&r)[3], f2 (&im)[3])
{
    const f2 sc = make_float2(__uint_as_float(a.w), __uint_as_float(b.w));
    if constexpr (P == P16) {
        f2 x, y;
        word2<P>(a.x, b.x, x, y);
        r[0] = mul2(x, sc);
        im[0] = mul2(y, sc);
        word2<P>(a.y, b.y, x, y);
        r[1] = mul2(x, sc);
        im[1] = mul2(y, sc);
        word2<P>(a.z, b.z, x, y);
        r[2] = mul2(x, sc);
        im[2] = mul2(y, sc);
        return;
    }
    const f2 nks = mul2(sc, make_float2(-12615680.f, -12615680.f));
    r[0] = fma2(make_float2(fxb_lo(a.x), fxb_lo(b.x)), sc, nks);
    im[0] = fma2(make_float2(fxb_hi(a.x), fxb_hi(b.x)), sc, nks);
    r[1] = fma2(make_float2(fxb_lo(a.y), fxb_lo(b.y)), sc, nks);
    im[1] = fma2(make_float2(fxb_hi(a.y), fxb_hi(b.y)), sc, nks);
    r[2] = fma2(make_float2(fxb_lo(a.z), fxb_lo(b.z)), sc, nks);
    im[2] = fma2(make_float2(fxb_hi(a.z), fxb_hi(b.z)), sc, nks);
}

// encode sites A (.x) and B (.y) as FX16 records (the scale and the
// NaN-propagating maximum of FieldIO<PX16>::store; the scaled value plus the
// offset rounded once by one FMA)
// (FP16: the scale is the site's largest |component| and the record holds
// the components over it in binary16, as FieldIO<P16>::store)
template <int P = PX16>
__device__ __forceinline__ void encode_fx2(const f2 (&r)[3], const f2 (&im)[3], uint4 &ua, uint4 &ub)
{
    if constexpr (P == P16) {
        float mA = 0.f, mB = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mA = fmaxf(mA, fmaxf(fabsf(r[c].x), fabsf(im[c].x)));
            mB = fmaxf(mB, fmaxf(fabsf(r[c].y), fabsf(im[c].y)));
        }
        const f2 inv = make_float2(mA > 0.f ? 1.0f / mA : 0.f, mB > 0.f ? 1.0f / mB : 0.f);
        unsigned wa[3], wb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const f2 sr = mul2(r[c], inv), si = mul2(im[c], inv);
            wa[c] = f2_to_h2(sr.x, si.x);
            wb[c] = f2_to_h2(sr.y, si.y);
        }
        ua = make_uint4(wa[0], wa[1], wa[2], __float_as_uint(mA));
        ub = make_uint4(wb[0], wb[1], wb[2], __float_as_uint(mB));
        return;
    }
    float mA = 0.f, mB = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        mA = fmax_nan(mA, fmax_nan(fabsf(r[c].x), fabsf(im[c].x)));
        mB = fmax_nan(mB, fmax_nan(fabsf(r[c].y), fabsf(im[c].y)));
    }
    const float sA = fx_scale(mA), sB = fx_scale(mB);
    const f2 k = make_float2(mA > 0.f ? 1.0f / sA : 0.f, mB > 0.f ? 1.0f / sB : 0.f);
    const f2 off = make_float2(12615680.f, 12615680.f);
    unsigned wa[3], wb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const f2 br = fma2(r[c], k, off), bi = fma2(im[c], k, off);
        wa[c] = __byte_perm(__float_as_uint(br.x), __float_as_uint(bi.x), 0x5410);
        wb[c] = __byte_perm(__float_as_uint(br.y), __float_as_uint(bi.y), 0x5410);
    }
    ua = make_uint4(wa[0], wa[1], wa[2], __float_as_uint(sA));
    ub = make_uint4(wb[0], wb[1], wb[2], __float_as_uint(sB));
}

// The packed epilogue of sites A (.x) and B (.y): dr / di hold D chi, or
// -D chi for the A epilogues (nacc), which then form q = m^2 w - D chi as
// one FMA.  Stores the sites that exist; returns the pair of site terms of
// Re w^dag q (q as stored) for EPI_A_DOT / EPI_A_CG.  EPI_RES is not packed.
template <int EPI, int P = PX16>
__device__ __forceinline__ f2 epilogue_pair(void *out_field, int iA, int iB, bool okA, bool okB,
                                            const f2 (&dr)[3], const f2 (&di)[3], float m2, uint4 wA,
                                            uint4 wB)
{
    uint4 *out = static_cast<uint4 *>(out_field);
    f2 dot = make_float2(0.f, 0.f);
    if (EPI == EPI_NONE || EPI == EPI_GATE) {
        uint4 ua, ub;
        encode_fx2<P>(dr, di, ua, ub);
        if (okA) out[iA] = ua;
        if (okB) out[iB] = ub;
    } else {
        f2 wr[3], wi[3], qr[3], qi[3];
        decode_fx2<P>(wA, wB, wr, wi);
        const f2 mm = make_float2(m2, m2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            qr[c] = fma2(mm, wr[c], dr[c]);
            qi[c] = fma2(mm, wi[c], di[c]);
        }
        uint4 ua, ub;
        encode_fx2<P>(qr, qi, ua, ub);
        if (okA) out[iA] = ua;
        if (okB) out[iB] = ub;
        if (EPI == EPI_A_DOT || EPI == EPI_A_CG) {
            f2 sr[3], si[3];
            decode_fx2<P>(ua, ub, sr, si);
            dot = mul2(wr[0], sr[0]);
            dot = fma2(wi[0], si[0], dot);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                dot = fma2(wr[c], sr[c], dot);
                dot = fma2(wi[c], si[c], dot);
            }
        }
    }
    return dot;
}

}  // namespace stg
