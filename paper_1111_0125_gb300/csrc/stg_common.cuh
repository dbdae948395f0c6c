// Device-side building blocks shared by the library's kernels: lattice
// geometry on the even/odd checkerboard, the structure-of-arrays field and
// link layouts per precision, SU(3) algebra, and a deterministic FP64
// grid reduction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stg {

// P16: IEEE binary16 storage; PX16: 16-bit fixed point (int16 with a per-
// site FP32 scale for fields, a fixed 1/32767 for links).  Both compute in FP32.
enum Prec { P64 = 0, P32 = 1, P16 = 2, PX16 = 3, PB16 = 4 };
constexpr int kNumPrec = 5;  // arrays indexed by precision

// ---------------------------------------------------------------------------
// Geometry.  Site (x, y, z, t), lex = x + Lx (y + Ly (z + Lz t)), parity
// (x+y+z+t) & 1, checkerboard index i = lex >> 1 (Lx even).  Within one
// parity the y, z and t neighbours are at i +- sy, sz, st; the x neighbour
// keeps the row (i - x/2) and moves x/2 by the parity-dependent hop.
// ---------------------------------------------------------------------------
// Division by a runtime constant d through a multiply-high (the round-up
// method of Granlund and Montgomery): for n < 2^31,
//   n / d = (umulhi(n, m) + n) >> s,  s = ceil(log2 d),
//   m = floor(2^32 (2^s - d) / d) + 1   (m = s = 0 for d = 1).
struct FastDiv {
    unsigned d, m, s;
    __host__ __device__ __forceinline__ unsigned div(unsigned n) const
    {
#ifdef __CUDA_ARCH__
        return (__umulhi(n, m) + n) >> s;
#else
        return (unsigned)(((unsigned long long)n * m >> 32) + n) >> s;
#endif
    }
};

inline FastDiv make_fastdiv(unsigned d)
{
    FastDiv f;
    f.d = d;
    if (d <= 1) {
        f.m = 0;
        f.s = 0;
        return f;
    }
    unsigned l = 0;
    while ((1ull << l) < d) ++l;
    f.s = l;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    return f;
}

struct Geom {
    int L[4];  // Lx, Ly, Lz, Lt
    int Lxh;   // Lx / 2
    int Vh;    // sites per parity
    int sy, sz, st;
    FastDiv dxh, dy, dz;  // division by Lx/2, Ly, Lz
};

struct Site {
    int x, y, z, t;
    int row;  // i - x/2, start of the x-row on the checkerboard
};

__device__ __forceinline__ Site site_of(const Geom &g, int i, int parity)
{
    Site s;
    const int r = (int)g.dxh.div((unsigned)i);
    s.row = r * g.Lxh;
    const int xh = i - s.row;
    const int r2 = (int)g.dy.div((unsigned)r);
    s.y = r - r2 * g.L[1];
    s.t = (int)g.dz.div((unsigned)r2);
    s.z = r2 - s.t * g.L[2];
    s.x = 2 * xh + ((parity + s.y + s.z + s.t) & 1);
    return s;
}

// checkerboard index of x + mu (fwd) and x - mu (bwd) in the opposite parity
__device__ __forceinline__ void neighbours(const Geom &g, const Site &s, int i, int mu,
                                           int &jf, int &jb)
{
    if (mu == 0) {
        int xf = (s.x + 1 == g.L[0]) ? 0 : s.x + 1;
        int xb = (s.x == 0) ? g.L[0] - 1 : s.x - 1;
        jf = s.row + (xf >> 1);
        jb = s.row + (xb >> 1);
    } else if (mu == 1) {
        jf = (s.y == g.L[1] - 1) ? i - (g.L[1] - 1) * g.sy : i + g.sy;
        jb = (s.y == 0) ? i + (g.L[1] - 1) * g.sy : i - g.sy;
    } else if (mu == 2) {
        jf = (s.z == g.L[2] - 1) ? i - (g.L[2] - 1) * g.sz : i + g.sz;
        jb = (s.z == 0) ? i + (g.L[2] - 1) * g.sz : i - g.sz;
    } else {
        jf = (s.t == g.L[3] - 1) ? i - (g.L[3] - 1) * g.st : i + g.st;
        jb = (s.t == 0) ? i + (g.L[3] - 1) * g.st : i - g.st;
    }
}

// s_mu = eta_mu * b_mu for the link leaving x (fwd) and the link leaving
// x - mu (bwd).  eta_mu(x - mu) = eta_mu(x) since eta_mu ignores x_mu.
__device__ __forceinline__ void link_signs(const Geom &g, const Site &s, int mu,
                                           float &sf, float &sb)
{
    int e = 0;
    if (mu >= 1) e += s.x;
    if (mu >= 2) e += s.y;
    if (mu >= 3) e += s.z;
    float eta = (e & 1) ? -1.f : 1.f;
    sf = eta;
    sb = eta;
    if (mu == 3) {
        if (s.t == g.L[3] - 1) sf = -sf;
        if (s.t == 0) sb = -sb;
    }
}

// ---------------------------------------------------------------------------
// Precision traits
// ---------------------------------------------------------------------------
template <int P> struct Real { typedef float T; };
template <> struct Real<P64> { typedef double T; };

// Bytes per site of one checkerboard field in the device layout.
__host__ __device__ constexpr int field_site_bytes(int p)
{
    return p == P64 ? 48 : (p == P32 ? 24 : 16);  // P16, PX16 and PB16: 16
}

// Bytes of one link in the device layout.
__host__ __device__ constexpr int link_bytes(int p, int recon)
{
    return p == P64 ? (recon == 18 ? 144 : 96)
         : p == P32 ? (recon == 18 ? 72 : 48)
                    : (recon == 18 ? 36 : 24);  // P16, PX16 and PB16
}

// ---------------------------------------------------------------------------
// Colour vectors (3 complex) and their device layouts
//   P64: three double2 planes [3][Vh]
//   P32: float4 plane (c0, c1) then float2 plane (c2)
//   P16: one 16-byte record per site {half2 c0, half2 c1, half2 c2, f32 scale}
// ---------------------------------------------------------------------------
template <typename T> struct Vec3 {
    T r[3], i[3];
};

template <int P> struct FieldIO;

// load_nc goes through the read-only data path and is only used for data
// that no thread of the same kernel writes; load is a plain global load.
template <typename V, bool NC> __device__ __forceinline__ V ld(const V *p)
{
    if (NC) return __ldg(p);
    return *p;
}

template <> struct FieldIO<P64> {
    template <bool NC = false>
    __device__ __forceinline__ static Vec3<double> load(const void *f, int vh, int s)
    {
        const double2 *p = static_cast<const double2 *>(f);
        Vec3<double> v;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 a = ld<double2, NC>(p + (size_t)c * vh + s);
            v.r[c] = a.x;
            v.i[c] = a.y;
        }
        return v;
    }
    __device__ __forceinline__ static Vec3<double> load_nc(const void *f, int vh, int s)
    {
        return load<true>(f, vh, s);
    }
    // store returns the value as a later load will see it
    __device__ __forceinline__ static Vec3<double> store(void *f, int vh, int s, const Vec3<double> &v)
    {
        double2 *p = static_cast<double2 *>(f);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[(size_t)c * vh + s] = make_double2(v.r[c], v.i[c]);
        return v;
    }
};

template <> struct FieldIO<P32> {
    template <bool NC = false>
    __device__ __forceinline__ static Vec3<float> load(const void *f, int vh, int s)
    {
        const float4 *p4 = static_cast<const float4 *>(f);
        const float2 *p2 = reinterpret_cast<const float2 *>(p4 + vh);
        float4 a = ld<float4, NC>(p4 + s);
        float2 b = ld<float2, NC>(p2 + s);
        Vec3<float> v;
        v.r[0] = a.x; v.i[0] = a.y;
        v.r[1] = a.z; v.i[1] = a.w;
        v.r[2] = b.x; v.i[2] = b.y;
        return v;
    }
    __device__ __forceinline__ static Vec3<float> load_nc(const void *f, int vh, int s)
    {
        return load<true>(f, vh, s);
    }
    __device__ __forceinline__ static Vec3<float> store(void *f, int vh, int s, const Vec3<float> &v)
    {
        float4 *p4 = static_cast<float4 *>(f);
        float2 *p2 = reinterpret_cast<float2 *>(p4 + vh);
        p4[s] = make_float4(v.r[0], v.i[0], v.r[1], v.i[1]);
        p2[s] = make_float2(v.r[2], v.i[2]);
        return v;
    }
};

__device__ __forceinline__ float2 h2_to_f2(unsigned u)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

__device__ __forceinline__ unsigned f2_to_h2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned *>(&h);
}

// the two 16-bit floating-point storage forms: IEEE binary16 (P16) and
// bfloat16 (PB16), two values per 32-bit word
struct CodecF16 {
    __device__ __forceinline__ static float2 dec(unsigned u) { return h2_to_f2(u); }
    __device__ __forceinline__ static unsigned enc(float a, float b) { return f2_to_h2(a, b); }
};
struct CodecBF16 {
    __device__ __forceinline__ static float2 dec(unsigned u)
    {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    }
    __device__ __forceinline__ static unsigned enc(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<unsigned *>(&h);
    }
};

// one 16-byte record per site: three colours as 16-bit float pairs scaled by
// 1 / (largest |re| or |im| of the site), and that scale as an FP32
template <class C> struct FieldIO16 {
    template <bool NC = false>
    __device__ __forceinline__ static Vec3<float> load(const void *f, int vh, int s)
    {
        uint4 u = ld<uint4, NC>(static_cast<const uint4 *>(f) + s);
        float sc = __uint_as_float(u.w);
        float2 a = C::dec(u.x), b = C::dec(u.y), c = C::dec(u.z);
        Vec3<float> v;
        v.r[0] = a.x * sc; v.i[0] = a.y * sc;
        v.r[1] = b.x * sc; v.i[1] = b.y * sc;
        v.r[2] = c.x * sc; v.i[2] = c.y * sc;
        return v;
    }
    __device__ __forceinline__ static Vec3<float> load_nc(const void *f, int vh, int s)
    {
        return load<true>(f, vh, s);
    }
    __device__ __forceinline__ static Vec3<float> store(void *f, int vh, int s, const Vec3<float> &v)
    {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) m = fmaxf(m, fmaxf(fabsf(v.r[c]), fabsf(v.i[c])));
        float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4 u;
        u.x = C::enc(v.r[0] * inv, v.i[0] * inv);
        u.y = C::enc(v.r[1] * inv, v.i[1] * inv);
        u.z = C::enc(v.r[2] * inv, v.i[2] * inv);
        u.w = __float_as_uint(m);
        static_cast<uint4 *>(f)[s] = u;
        float2 a = C::dec(u.x), b = C::dec(u.y), c = C::dec(u.z);
        Vec3<float> o;
        o.r[0] = a.x * m; o.i[0] = a.y * m;
        o.r[1] = b.x * m; o.i[1] = b.y * m;
        o.r[2] = c.x * m; o.i[2] = c.y * m;
        return o;
    }
};

template <> struct FieldIO<P16> : FieldIO16<CodecF16> {};
template <> struct FieldIO<PB16> : FieldIO16<CodecBF16> {};

// 16-bit fixed point: a component q in [-32767, 32767] is kept as the
// unsigned offset u = q + 32768.  Decoding puts u into the low mantissa bits
// of 1.5 * 2^23 (one byte permute) and subtracts 1.5 * 2^23 + 32768, which
// is exact in FP32.
__device__ __forceinline__ float fx_lo(unsigned w)
{
    return __int_as_float((int)__byte_perm(w, 0x4B40u, 0x5410)) - 12615680.0f;
}
__device__ __forceinline__ float fx_hi(unsigned w)
{
    return __int_as_float((int)__byte_perm(w, 0x4B40u, 0x5432)) - 12615680.0f;
}
// Encoding: x (already scaled by 1 / s) plus 1.5 * 2^23 + 32768 rounds to
// the nearest integer in FP32, leaving rint(x) + 32768 in the low 16 bits;
// one byte permute packs the (re, im) pair.  No clamp is needed: with s from
// fx_scale and k = RN(1 / s), |x| <= 32767 (1 + 2^-21) < 32767.5 for every
// finite component, so rint(x) + 32768 stays in [1, 65535].
__device__ __forceinline__ unsigned fx_pack(float re, float im)
{
    const unsigned a = __float_as_uint(re + 12615680.0f);
    const unsigned b = __float_as_uint(im + 12615680.0f);
    return __byte_perm(a, b, 0x5410);
}

// maximum that returns NaN when either operand is NaN (max.NaN, sm_80+): a
// NaN component makes the site's scale NaN, so it decodes as NaN instead of
// turning into a finite fixed-point value
__device__ __forceinline__ float fmax_nan(float a, float b)
{
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// PX16 field: one 16-byte record {3 words of (re, im) fixed point, f32 s}
// with value = q * s and s = max |component| / 32767 of the site, rounded up
// to 15 significant bits.  With s that short, K s is exact in FP32 for the
// decode's 9-bit offset K = 1.5 * 2^23 + 32768, so a decoder may form q s
// from the biased value (K + q) as one FMA, (K + q) s - K s, with the same
// single rounding as q s (the packed Dslash kernels do).
__device__ __forceinline__ float fx_scale(float m)
{
    const float s = m * (1.0f / 32767.0f);
    return __uint_as_float((__float_as_uint(s) + 0x1FFu) & ~0x1FFu);
}

template <> struct FieldIO<PX16> {
    template <bool NC = false>
    __device__ __forceinline__ static Vec3<float> load(const void *f, int vh, int s)
    {
        uint4 u = ld<uint4, NC>(static_cast<const uint4 *>(f) + s);
        const float sc = __uint_as_float(u.w);
        Vec3<float> v;
        v.r[0] = fx_lo(u.x) * sc; v.i[0] = fx_hi(u.x) * sc;
        v.r[1] = fx_lo(u.y) * sc; v.i[1] = fx_hi(u.y) * sc;
        v.r[2] = fx_lo(u.z) * sc; v.i[2] = fx_hi(u.z) * sc;
        return v;
    }
    __device__ __forceinline__ static Vec3<float> load_nc(const void *f, int vh, int s)
    {
        return load<true>(f, vh, s);
    }
    __device__ __forceinline__ static Vec3<float> store(void *f, int vh, int s, const Vec3<float> &v)
    {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) m = fmax_nan(m, fmax_nan(fabsf(v.r[c]), fabsf(v.i[c])));
        const float sc = fx_scale(m);
        const float k = m > 0.f ? 1.0f / sc : 0.f;
        uint4 u;
        u.x = fx_pack(v.r[0] * k, v.i[0] * k);
        u.y = fx_pack(v.r[1] * k, v.i[1] * k);
        u.z = fx_pack(v.r[2] * k, v.i[2] * k);
        u.w = __float_as_uint(sc);
        static_cast<uint4 *>(f)[s] = u;
        Vec3<float> o;
        o.r[0] = fx_lo(u.x) * sc; o.i[0] = fx_hi(u.x) * sc;
        o.r[1] = fx_lo(u.y) * sc; o.i[1] = fx_hi(u.y) * sc;
        o.r[2] = fx_lo(u.z) * sc; o.i[2] = fx_hi(u.z) * sc;
        return o;
    }
};

// ---------------------------------------------------------------------------
// Links.  One block per (parity, mu) holding Vh links as planes:
//   P64/18: 9 double2 planes (entries 00..22);  P64/12: 6 (rows 0, 1)
//   P32/18: 4 float4 planes (00,01)(02,10)(11,12)(20,21) + float2 plane 22
//   P32/12: 3 float4 planes (00,01)(02,10)(11,12)
//   P16/18: 2 uint4 planes of 4 half2 + one 4-byte half2 plane (22)
//   P16/12: 1 uint4 plane (00,01,02,10) + one uint2 plane (11,12)
// For recon 12 the loader returns row 2 = conj(row0 x row1); the true row 2
// of the stored s U is s times that (det(s U) = s for U in SU(3)), and the
// mat-vecs apply s (times 1/32767 for PX16) to row 2's contribution.
// ---------------------------------------------------------------------------
template <typename T> struct Mat3 {
    T r[3][3], i[3][3];
};

template <typename T>
__device__ __forceinline__ void set_entry(Mat3<T> &u, int k, T re, T im)
{
    u.r[k / 3][k % 3] = re;
    u.i[k / 3][k % 3] = im;
}

template <typename T>
__device__ __forceinline__ void reconstruct_row2(Mat3<T> &u, T s)
{
    // (r0 x r1)_a = r0_{a+1} r1_{a+2} - r0_{a+2} r1_{a+1}, then s * conj(.)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        T re = (u.r[0][b] * u.r[1][c] - u.i[0][b] * u.i[1][c])
             - (u.r[0][c] * u.r[1][b] - u.i[0][c] * u.i[1][b]);
        T im = (u.r[0][b] * u.i[1][c] + u.i[0][b] * u.r[1][c])
             - (u.r[0][c] * u.i[1][b] + u.i[0][c] * u.r[1][b]);
        u.r[2][a] = s * re;
        u.i[2][a] = -s * im;
    }
}

// Link loads: every link is read exactly once per half-pass, so they bypass
// L1 (no_allocate) and leave it to the neighbour colour vectors, which are
// read eight times each.
__device__ __forceinline__ uint4 ld_stream(const uint4 *p)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint2 ld_stream(const uint2 *p)
{
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned ld_stream(const unsigned *p)
{
    unsigned v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4 *p)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_stream(const float2 *p)
{
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_stream(const double2 *p)
{
    double2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

template <int P, int R> struct LinkIO;

template <int R> struct LinkIO<P64, R> {
    __device__ __forceinline__ static Mat3<double> load(const char *blk, int vh, int s)
    {
        const double2 *p = reinterpret_cast<const double2 *>(blk);
        Mat3<double> u;
        constexpr int n = R == 18 ? 9 : 6;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            double2 a = ld_stream(p + (size_t)k * vh + s);
            set_entry(u, k, a.x, a.y);
        }
        if (R == 12) reconstruct_row2(u, 1.0);
        return u;
    }
};

template <int R> struct LinkIO<P32, R> {
    __device__ __forceinline__ static Mat3<float> load(const char *blk, int vh, int s)
    {
        const float4 *p = reinterpret_cast<const float4 *>(blk);
        Mat3<float> u;
        constexpr int n4 = R == 18 ? 4 : 3;
#pragma unroll
        for (int k = 0; k < n4; ++k) {
            float4 a = ld_stream(p + (size_t)k * vh + s);
            set_entry(u, 2 * k, a.x, a.y);
            set_entry(u, 2 * k + 1, a.z, a.w);
        }
        if (R == 18) {
            float2 b = ld_stream(reinterpret_cast<const float2 *>(p + (size_t)4 * vh) + s);
            set_entry(u, 8, b.x, b.y);
        } else {
            reconstruct_row2(u, 1.0f);
        }
        return u;
    }
};

// 16-bit float links (|U_ab| <= 1, no scale): entries as float pairs
template <class C, int R> struct LinkIO16 {
    __device__ __forceinline__ static Mat3<float> load(const char *blk, int vh, int s)
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(blk);
        Mat3<float> u;
        uint4 a = ld_stream(p + s);
        float2 e0 = C::dec(a.x), e1 = C::dec(a.y), e2 = C::dec(a.z), e3 = C::dec(a.w);
        set_entry(u, 0, e0.x, e0.y);
        set_entry(u, 1, e1.x, e1.y);
        set_entry(u, 2, e2.x, e2.y);
        set_entry(u, 3, e3.x, e3.y);
        if (R == 18) {
            uint4 b = ld_stream(p + (size_t)vh + s);
            float2 f0 = C::dec(b.x), f1 = C::dec(b.y), f2 = C::dec(b.z), f3 = C::dec(b.w);
            set_entry(u, 4, f0.x, f0.y);
            set_entry(u, 5, f1.x, f1.y);
            set_entry(u, 6, f2.x, f2.y);
            set_entry(u, 7, f3.x, f3.y);
            unsigned c = ld_stream(reinterpret_cast<const unsigned *>(p + (size_t)2 * vh) + s);
            float2 g = C::dec(c);
            set_entry(u, 8, g.x, g.y);
        } else {
            uint2 b = ld_stream(reinterpret_cast<const uint2 *>(p + (size_t)vh) + s);
            float2 f0 = C::dec(b.x), f1 = C::dec(b.y);
            set_entry(u, 4, f0.x, f0.y);
            set_entry(u, 5, f1.x, f1.y);
            reconstruct_row2(u, 1.0f);
        }
        return u;
    }
};

template <int R> struct LinkIO<P16, R> : LinkIO16<CodecF16, R> {};
template <int R> struct LinkIO<PB16, R> : LinkIO16<CodecBF16, R> {};

// PX16 links: entries q = rint(32767 U_ab) as offsets, no per-link scale.
// load returns 32767 * U (integer-valued floats); the kernel multiplies its
// accumulated sum by 1/32767 once per site (LinkPost).  Row 2 of a 12-real
// link is s conj(r0 x r1) / 32767, which keeps it on the same 32767 scale.
template <int R> struct LinkIO<PX16, R> {
    __device__ __forceinline__ static Mat3<float> load(const char *blk, int vh, int s)
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(blk);
        Mat3<float> u;
        uint4 a = ld_stream(p + s);
        set_entry(u, 0, fx_lo(a.x), fx_hi(a.x));
        set_entry(u, 1, fx_lo(a.y), fx_hi(a.y));
        set_entry(u, 2, fx_lo(a.z), fx_hi(a.z));
        set_entry(u, 3, fx_lo(a.w), fx_hi(a.w));
        if (R == 18) {
            uint4 b = ld_stream(p + (size_t)vh + s);
            set_entry(u, 4, fx_lo(b.x), fx_hi(b.x));
            set_entry(u, 5, fx_lo(b.y), fx_hi(b.y));
            set_entry(u, 6, fx_lo(b.z), fx_hi(b.z));
            set_entry(u, 7, fx_lo(b.w), fx_hi(b.w));
            unsigned c = ld_stream(reinterpret_cast<const unsigned *>(p + (size_t)2 * vh) + s);
            set_entry(u, 8, fx_lo(c), fx_hi(c));
        } else {
            uint2 b = ld_stream(reinterpret_cast<const uint2 *>(p + (size_t)vh) + s);
            set_entry(u, 4, fx_lo(b.x), fx_hi(b.x));
            set_entry(u, 5, fx_lo(b.y), fx_hi(b.y));
            reconstruct_row2(u, 1.0f);
        }
        return u;
    }
};

// factor applied to the accumulated D chi of a site (1/32767 for PX16 links)
// and, for 12-real links, the extra factor of row 2's contribution
template <int P> struct LinkPost {
    static constexpr float k = 1.0f;
    static constexpr float row2 = 1.0f;
};
template <> struct LinkPost<PX16> {
    static constexpr float k = 1.0f / 32767.0f;
    static constexpr float row2 = 1.0f / 32767.0f;
};

// a * b + c with one rounding, in the precision of T
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

// acc += U v, with row 2 of U scaled by s2 (the 12-real sign; 1 for 18-real).
// Every product goes into its accumulator by one FMA (two per real part of
// a complex product): written as acc += (a b - c d), the compiler would need
// a multiply, an FMA and an add, which costs the ALU-bound FP64 operator a
// third more FP64 instructions.
// SCALED_ROW2: row 2 carries the factor s2 (12-real links); otherwise s2
// must be 1 and row 2 accumulates like rows 0 and 1.
template <bool SCALED_ROW2 = true, typename T>
__device__ __forceinline__ void mul_add(const Mat3<T> &u, const Vec3<T> &v, Vec3<T> &acc, T s2)
{
    constexpr int nrow = SCALED_ROW2 ? 2 : 3;
#pragma unroll
    for (int a = 0; a < nrow; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            acc.r[a] = fmat(u.r[a][b], v.r[b], acc.r[a]);
            acc.r[a] = fmat(-u.i[a][b], v.i[b], acc.r[a]);
            acc.i[a] = fmat(u.r[a][b], v.i[b], acc.i[a]);
            acc.i[a] = fmat(u.i[a][b], v.r[b], acc.i[a]);
        }
    if (SCALED_ROW2) {
        T wr = u.r[2][0] * v.r[0], wi = u.r[2][0] * v.i[0];
        wr = fmat(-u.i[2][0], v.i[0], wr);
        wi = fmat(u.i[2][0], v.r[0], wi);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            wr = fmat(u.r[2][b], v.r[b], wr);
            wr = fmat(-u.i[2][b], v.i[b], wr);
            wi = fmat(u.r[2][b], v.i[b], wi);
            wi = fmat(u.i[2][b], v.r[b], wi);
        }
        acc.r[2] = fmat(s2, wr, acc.r[2]);
        acc.i[2] = fmat(s2, wi, acc.i[2]);
    }
}

// acc -= U^dag v, (U^dag)_{ab} = conj(U_{ba}), row 2 of U scaled by s2
template <typename T>
__device__ __forceinline__ void adj_mul_sub(const Mat3<T> &u, const Vec3<T> &v, Vec3<T> &acc, T s2)
{
    const T v2r = s2 * v.r[2], v2i = s2 * v.i[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            // conj(U_ba) v_b = (u.r v.r + u.i v.i) + i (u.r v.i - u.i v.r)
            acc.r[a] = fmat(-u.r[b][a], v.r[b], acc.r[a]);
            acc.r[a] = fmat(-u.i[b][a], v.i[b], acc.r[a]);
            acc.i[a] = fmat(-u.r[b][a], v.i[b], acc.i[a]);
            acc.i[a] = fmat(u.i[b][a], v.r[b], acc.i[a]);
        }
        acc.r[a] = fmat(-u.r[2][a], v2r, acc.r[a]);
        acc.r[a] = fmat(-u.i[2][a], v2i, acc.r[a]);
        acc.i[a] = fmat(-u.r[2][a], v2i, acc.i[a]);
        acc.i[a] = fmat(u.i[2][a], v2r, acc.i[a]);
    }
}

// ---------------------------------------------------------------------------
// Solver state in device memory.  Kernels of one CG iteration read the
// scalars they need from here, so an iteration is a fixed launch sequence
// that can be captured once in a CUDA graph.
// ---------------------------------------------------------------------------
enum CGFlag { FLAG_RUN = 0, FLAG_CONVERGED = 1, FLAG_UPDATE = 2, FLAG_BREAKDOWN = 3,
              FLAG_MAXITER = 4, FLAG_TIMEOUT = 5 };

// ---------------------------------------------------------------------------
// mbarrier waits with a time limit (bulk async copies into shared memory)
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0u;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete.  Gives up when
// another thread of the CTA has given up (`abort`, unless null) or after
// kWaitLimitNs; the first to give up raises `abort` and counts the event in
// `timeouts`.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, volatile int *abort,
                                          unsigned *timeouts)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (abort && *abort) return false;
        if (global_ns() - t0 > kWaitLimitNs) {
            if (abort) *abort = 1;
            atomicAdd(timeouts, 1u);
            return false;
        }
    }
}

// One bulk async copy global -> shared of `bytes` (16-byte aligned, a
// multiple of 16) completing on the mbarrier `bar`, which this thread arms
// with the byte count.  The source is streamed once: L2 evicts it first.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    const unsigned b = smem_addr(bar);
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
                 "[%0], [%1], %2, [%3], %4;"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(b), "l"(pol)
                 : "memory");
}

// Programmatic dependent launch: pdl_wait() returns once the preceding
// kernel of the stream has completed and its writes are visible (at once when
// the kernel was launched without the attribute); pdl_trigger() lets the next
// kernel be scheduled.  Every kernel calls pdl_trigger() only after its
// pdl_wait(), so when a kernel starts, all kernels before its immediate
// predecessor have completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

struct CGState {
    double delta_new;  // r^dag r (iterated residual of the current precision)
    double delta_old;
    double pAp;        // d^dag A d
    double alpha, beta;
    double rmax2;      // largest |r|^2 since the last update (or at reset)
    double stop_r2;    // tol^2 |b|^2: iterated-residual stopping point
    double trig2;      // delta^2: reliable-update trigger (0 = never)
    double m2;         // mass^2
    double result;     // slot for stand-alone reductions
    long long iter;        // iterations done (all precisions)
    long long iter_limit;  // stop when iter reaches this
    int flag;
    int track_max;     // 1: rmax2 follows the running maximum (Sec. 3.2)
    unsigned counter;  // arrival counter of the last-block reduction
    unsigned pad;
};

// alpha = delta / d^dag A d (Fig. 1), with a breakdown test.  For the exact
// operator d^dag A d >= m^2 |d|^2, and |d|^2 >= |r|^2 = delta because d = r +
// beta d_old with d_old orthogonal to r, so alpha <= 1 / m^2.  A
// non-positive or non-finite d^dag A d, or a step 16 times beyond that bound,
// means the low-precision iteration has lost the operator's positivity: the
// flag makes the solver take a reliable update and restart from the true
// residual before y is spoiled by the step.
__device__ __forceinline__ void set_alpha(CGState *st, double pAp)
{
    st->pAp = pAp;
    const double alpha = st->delta_new / pAp;
    if (!(pAp > 0.0) || !isfinite(pAp) || !(alpha * st->m2 <= 16.0)) st->flag = FLAG_BREAKDOWN;
    else st->alpha = alpha;
}

// ---------------------------------------------------------------------------
// Deterministic grid-wide FP64 sum: block partials, then the last block to
// arrive sums them in a fixed order.  No floating-point atomics, no waiting:
// the arrival counter only elects the block that finishes the sum.
// ---------------------------------------------------------------------------
template <int BS>
__device__ __forceinline__ double block_sum(double v, double *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = (lane < BS / 32) ? sm[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

// Compensated FP32 ("float-float") sums for FP32 data.  On GB300 one warp-
// wide FP64 instruction occupies the FP64 pipe for ~16 cycles, so the
// per-thread, warp and block levels add (hi, lo) pairs with an exact two-sum
// in FP32 (~2^-44 relative), the partials are float2, and only the final
// total becomes a double.  FP64 data keeps the FP64 path above.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    FF r;
    r.hi = s;
    r.lo = e + (a.lo + b.lo);
    return r;
}

__device__ __forceinline__ FF ff_shfl_down(FF a, int o)
{
    FF b;
    b.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
    return b;
}

template <int BS>
__device__ __forceinline__ FF block_sum_ff(FF v, float2 *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_down(v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = make_float2(v.hi, v.lo);
    __syncthreads();
    FF s = {0.f, 0.f};
    if (w == 0) {
        if (lane < BS / 32) {
            s.hi = sm[lane].x;
            s.lo = sm[lane].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
    }
    return s;  // valid in thread 0
}

template <int BS>
__device__ __forceinline__ bool grid_sum_ff(FF v, float2 *partials, unsigned *counter, double &total)
{
    __shared__ float2 smf[32];
    __shared__ int is_last_ff;
    FF s = block_sum_ff<BS>(v, smf);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = make_float2(s.hi, s.lo);
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        is_last_ff = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last_ff) return false;
    __threadfence();
    FF acc = {0.f, 0.f};
    for (int k = threadIdx.x; k < (int)gridDim.x; k += BS) {
        const float2 p = __ldcg(partials + k);
        FF q;
        q.hi = p.x;
        q.lo = p.y;
        acc = ff_add(acc, q);
    }
    FF t = block_sum_ff<BS>(acc, smf);
    if (threadIdx.x == 0) {
        total = (double)t.hi + (double)t.lo;
        *counter = 0u;
        return true;
    }
    return false;
}

// Returns true in thread 0 of the last block, with the grid total in `total`.
template <int BS>
__device__ __forceinline__ bool grid_sum(double v, double *partials, unsigned *counter,
                                         double &total)
{
    __shared__ double sm[32];
    __shared__ int is_last;
    double s = block_sum<BS>(v, sm);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += BS) acc += __ldcg(partials + k);
    total = block_sum<BS>(acc, sm);
    if (threadIdx.x == 0) {
        *counter = 0u;
        return true;
    }
    return false;
}

}  // namespace stg
