// Gauge handle: upload of the canonical links, the paper's link
// preconditioning (staggered phase and time-boundary sign folded into each
// link, Sec. 2 after Eq. 5), re-layout into per-(parity, mu) structure-of-
// arrays planes for coalesced 128-bit loads (the paper's host-side
// "rearranging data for the coalesced access", Sec. 3.3, done here on the
// GPU), and conversion of fields between the canonical and device layouts.
#include <stdio.h>
#include <stdlib.h>

#include <new>
#include <type_traits>

#include "stg_internal.h"

namespace stg {

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

Geom make_geom(const int dims[4])
{
    Geom g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
    g.Lxh = dims[0] / 2;
    g.Vh = (int)((long)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    g.sy = g.Lxh;
    g.sz = g.Lxh * dims[1];
    g.st = g.Lxh * dims[1] * dims[2];
    g.dxh = make_fastdiv((unsigned)g.Lxh);
    g.dy = make_fastdiv((unsigned)dims[1]);
    g.dz = make_fastdiv((unsigned)dims[2]);
    return g;
}

// ---------------------------------------------------------------------------
// link packing: one thread per (site, mu) of the canonical array
// ---------------------------------------------------------------------------
// t_flip: the time slice whose forward t-links carry the antiperiodic sign
// (Lt - 1 for a whole lattice; for a t-slab, its last slice when the slab
// holds global t = Lt - 1, else -1: none)
template <int P, int R>
__global__ void k_pack_links(Geom g, const double2 *__restrict__ ucan, char *base, size_t blk_bytes, int t_flip)
{
    const long n = (long)g.Vh * 2 * 4;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int mu = (int)(k & 3);
    const int lex = (int)(k >> 2);
    int r = lex;
    const int x = r % g.L[0]; r /= g.L[0];
    const int y = r % g.L[1]; r /= g.L[1];
    const int z = r % g.L[2];
    const int t = r / g.L[2];
    const int parity = (x + y + z + t) & 1;
    const int i = lex >> 1;
    int e = 0;
    if (mu >= 1) e += x;
    if (mu >= 2) e += y;
    if (mu >= 3) e += z;
    double s = (e & 1) ? -1.0 : 1.0;
    if (mu == 3 && t == t_flip) s = -s;
    const double2 *src = ucan + (size_t)k * 9;
    double2 u[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double2 v = src[q];
        u[q] = make_double2(s * v.x, s * v.y);
    }
    char *blk = base + (size_t)(parity * 4 + mu) * blk_bytes;
    const int vh = g.Vh;
    if (P == P64) {
        double2 *p = reinterpret_cast<double2 *>(blk);
        const int ne = R == 18 ? 9 : 6;
        for (int q = 0; q < ne; ++q) p[(size_t)q * vh + i] = u[q];
    } else if (P == P32) {
        float4 *p = reinterpret_cast<float4 *>(blk);
        const int n4 = R == 18 ? 4 : 3;
        for (int q = 0; q < n4; ++q)
            p[(size_t)q * vh + i] = make_float4((float)u[2 * q].x, (float)u[2 * q].y,
                                                (float)u[2 * q + 1].x, (float)u[2 * q + 1].y);
        if (R == 18)
            reinterpret_cast<float2 *>(p + (size_t)4 * vh)[i] = make_float2((float)u[8].x, (float)u[8].y);
    } else if (P == PX16) {
        // entries of a unitary link are bounded by 1: q = rint(32767 U), no scale
        const float k = 32767.0f;
        uint4 *p = reinterpret_cast<uint4 *>(blk);
        uint4 a;
        a.x = fx_pack(k * (float)u[0].x, k * (float)u[0].y);
        a.y = fx_pack(k * (float)u[1].x, k * (float)u[1].y);
        a.z = fx_pack(k * (float)u[2].x, k * (float)u[2].y);
        a.w = fx_pack(k * (float)u[3].x, k * (float)u[3].y);
        p[i] = a;
        if (R == 18) {
            uint4 b;
            b.x = fx_pack(k * (float)u[4].x, k * (float)u[4].y);
            b.y = fx_pack(k * (float)u[5].x, k * (float)u[5].y);
            b.z = fx_pack(k * (float)u[6].x, k * (float)u[6].y);
            b.w = fx_pack(k * (float)u[7].x, k * (float)u[7].y);
            p[(size_t)vh + i] = b;
            reinterpret_cast<unsigned *>(p + (size_t)2 * vh)[i] = fx_pack(k * (float)u[8].x, k * (float)u[8].y);
        } else {
            uint2 b;
            b.x = fx_pack(k * (float)u[4].x, k * (float)u[4].y);
            b.y = fx_pack(k * (float)u[5].x, k * (float)u[5].y);
            reinterpret_cast<uint2 *>(p + (size_t)vh)[i] = b;
        }
    } else {
        // 16-bit floats (P16 binary16, PB16 bfloat16): |U_ab| <= 1, no scale
        typedef typename std::conditional<P == PB16, CodecBF16, CodecF16>::type C16;
        uint4 *p = reinterpret_cast<uint4 *>(blk);
        uint4 a;
        a.x = C16::enc((float)u[0].x, (float)u[0].y);
        a.y = C16::enc((float)u[1].x, (float)u[1].y);
        a.z = C16::enc((float)u[2].x, (float)u[2].y);
        a.w = C16::enc((float)u[3].x, (float)u[3].y);
        p[i] = a;
        if (R == 18) {
            uint4 b;
            b.x = C16::enc((float)u[4].x, (float)u[4].y);
            b.y = C16::enc((float)u[5].x, (float)u[5].y);
            b.z = C16::enc((float)u[6].x, (float)u[6].y);
            b.w = C16::enc((float)u[7].x, (float)u[7].y);
            p[(size_t)vh + i] = b;
            reinterpret_cast<unsigned *>(p + (size_t)2 * vh)[i] = C16::enc((float)u[8].x, (float)u[8].y);
        } else {
            uint2 b;
            b.x = C16::enc((float)u[4].x, (float)u[4].y);
            b.y = C16::enc((float)u[5].x, (float)u[5].y);
            reinterpret_cast<uint2 *>(p + (size_t)vh)[i] = b;
        }
    }
}

stg_status pack_links_flip(const Geom &g, const double2 *ucan, int prec, int recon, int t_flip,
                           LinkField *lf, cudaStream_t s)
{
    lf->prec = prec;
    lf->recon = recon;
    lf->blk_bytes = align256((size_t)g.Vh * link_bytes(prec, recon));
    cudaError_t e = cudaMalloc((void **)&lf->base, lf->blk_bytes * 8);
    if (e != cudaSuccess) {
        lf->base = nullptr;
        set_error("stg_gauge_create: device allocation of the links failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    const long n = (long)g.Vh * 8;
    const int grid = (int)((n + 255) / 256);
#define STG_PACK(P_, R_) k_pack_links<P_, R_><<<grid, 256, 0, s>>>(g, ucan, lf->base, lf->blk_bytes, t_flip)
    if (prec == P64) { if (recon == 18) STG_PACK(P64, 18); else STG_PACK(P64, 12); }
    else if (prec == P32) { if (recon == 18) STG_PACK(P32, 18); else STG_PACK(P32, 12); }
    else if (prec == P16) { if (recon == 18) STG_PACK(P16, 18); else STG_PACK(P16, 12); }
    else if (prec == PB16) { if (recon == 18) STG_PACK(PB16, 18); else STG_PACK(PB16, 12); }
    else { if (recon == 18) STG_PACK(PX16, 18); else STG_PACK(PX16, 12); }
#undef STG_PACK
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

static stg_status pack_links(const Geom &g, const double2 *ucan, int prec, int recon,
                             LinkField *lf, cudaStream_t s)
{
    return pack_links_flip(g, ucan, prec, recon, g.L[3] - 1, lf, s);
}

// Tile-major copy of FX16 / 12-real links (see kFxTile): one thread per
// (output parity, tile, mu, slot).  The forward record is the link block
// (p, mu) at the output site, the backward record the block (1 - p, mu) at
// the backward neighbour; both are copied bit for bit.
__global__ void k_tile_links_fx12(Geom g, const char *base, size_t blk_bytes, char *tiled, int ntiles)
{
    const long n = 2L * ntiles * 4 * kFxTile;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int a = (int)(k % kFxTile);
    long r = k / kFxTile;
    const int mu = (int)(r % 4);
    r /= 4;
    const int tile = (int)(r % ntiles);
    const int p = (int)(r / ntiles);
    const int i = tile * kFxTile + a;
    uint4 f16 = make_uint4(0u, 0u, 0u, 0u), b16 = f16;
    uint2 f8 = make_uint2(0u, 0u), b8 = f8;
    if (i < g.Vh) {
        const Site s = site_of(g, i, p);
        int jf, jb;
        neighbours(g, s, i, mu, jf, jb);
        const char *bf = base + (size_t)(p * 4 + mu) * blk_bytes;
        const char *bb = base + (size_t)((1 - p) * 4 + mu) * blk_bytes;
        f16 = reinterpret_cast<const uint4 *>(bf)[i];
        f8 = reinterpret_cast<const uint2 *>(bf + (size_t)g.Vh * 16)[i];
        b16 = reinterpret_cast<const uint4 *>(bb)[jb];
        b8 = reinterpret_cast<const uint2 *>(bb + (size_t)g.Vh * 16)[jb];
    }
    char *blk = tiled + (((size_t)p * ntiles + tile) * 4 + mu) * kFxStageBytes;
    reinterpret_cast<uint4 *>(blk)[a] = f16;
    reinterpret_cast<uint2 *>(blk + 16 * kFxTile)[a] = f8;
    reinterpret_cast<uint4 *>(blk + 24 * kFxTile)[a] = b16;
    reinterpret_cast<uint2 *>(blk + 40 * kFxTile)[a] = b8;
}

static stg_status tile_links(const Geom &g, LinkField *lf, cudaStream_t s)
{
    const int ntiles = (g.Vh + kFxTile - 1) / kFxTile;
    lf->tiled_parity_bytes = (size_t)ntiles * 4 * kFxStageBytes;
    cudaError_t e = cudaMalloc((void **)&lf->tiled, 2 * lf->tiled_parity_bytes);
    if (e != cudaSuccess) {
        lf->tiled = nullptr;
        set_error("stg_gauge_create: device allocation of the tile-major links failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    const long n = 2L * ntiles * 4 * kFxTile;
    k_tile_links_fx12<<<(int)((n + 255) / 256), 256, 0, s>>>(g, lf->base, lf->blk_bytes, lf->tiled, ntiles);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// Tile-major copy for the staged multi-system Dslash (see kMTile): one
// thread per (output parity, tile, mu, dir, slot); records copied bit for
// bit from the link blocks (forward: block (p, mu) at the site; backward:
// block (1 - p, mu) at the backward neighbour).
template <int P>
__global__ void k_mtile_links(Geom g, const char *base, size_t blk_bytes, char *mtiled, int ntiles)
{
    constexpr int L = P == P32 ? 48 : 24;
    const long n = 2L * ntiles * 8 * kMTile;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int a = (int)(k % kMTile);
    long r = k / kMTile;
    const int md = (int)(r % 8);  // mu * 2 + dir
    r /= 8;
    const int tile = (int)(r % ntiles);
    const int p = (int)(r / ntiles);
    const int mu = md >> 1, dir = md & 1;
    const int i = tile * kMTile + a;
    char *blk = mtiled + ((size_t)p * ntiles + tile) * ((size_t)kMTile * 8 * L) + (size_t)md * kMTile * L;
    const int vh = g.Vh;
    int src = i, sp = p;
    const bool ok = i < vh;
    if (ok && dir == 1) {
        const Site s = site_of(g, i, p);
        int jf, jb;
        neighbours(g, s, i, mu, jf, jb);
        src = jb;
        sp = 1 - p;
    }
    const char *from = base + (size_t)(sp * 4 + mu) * blk_bytes;
    if (P == P32) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) v = reinterpret_cast<const float4 *>(from)[(size_t)q * vh + src];
            reinterpret_cast<float4 *>(blk)[q * kMTile + a] = v;
        }
    } else {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        uint2 w = make_uint2(0u, 0u);
        if (ok) {
            v = reinterpret_cast<const uint4 *>(from)[src];
            w = reinterpret_cast<const uint2 *>(from + (size_t)vh * 16)[src];
        }
        reinterpret_cast<uint4 *>(blk)[a] = v;
        reinterpret_cast<uint2 *>(blk + 16 * kMTile)[a] = w;
    }
}

static stg_status mtile_links(const Geom &g, LinkField *lf, cudaStream_t s)
{
    const int ntiles = (g.Vh + kMTile - 1) / kMTile;
    lf->mtile_bytes = (size_t)kMTile * 8 * (lf->prec == P32 ? 48 : 24);
    lf->mtiled_parity_bytes = (size_t)ntiles * lf->mtile_bytes;
    cudaError_t e = cudaMalloc((void **)&lf->mtiled, 2 * lf->mtiled_parity_bytes);
    if (e != cudaSuccess) {
        lf->mtiled = nullptr;
        set_error("stg_gauge_create: device allocation of the multi-system tile-major links failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    const long n = 2L * ntiles * 8 * kMTile;
    const int grid = (int)((n + 255) / 256);
    if (lf->prec == P32) k_mtile_links<P32><<<grid, 256, 0, s>>>(g, lf->base, lf->blk_bytes, lf->mtiled, ntiles);
    else k_mtile_links<PX16><<<grid, 256, 0, s>>>(g, lf->base, lf->blk_bytes, lf->mtiled, ntiles);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// STG_MRHS_TILED=0 at gauge creation leaves out the multi-system copy (the
// autotuner then only has the register-fed multi-system kernels).
static bool want_mtiled()
{
    const char *v = getenv("STG_MRHS_TILED");
    return !(v && v[0] == '0');
}

// The staged FX16 / FP16 12-real Dslash is the default; STG_FX16_TILED=0 at
// gauge creation keeps the register-fed (FX16) or one-site (FP16) kernel (no
// tile-major copy).
static bool want_tiled()
{
    const char *v = getenv("STG_FX16_TILED");
    return !(v && v[0] == '0');
}

// Test hooks of the staged kernel, read here once per handle so that no
// launch reads the environment: STG_FX16_GRID=n caps its CTA count (every
// CTA then walks more tiles through its ring); STG_FX16_TEST_DROP_FILL=1
// withholds one stage fill, so that a bounded wait runs out (the failure-
// detection test).
static void read_fx_hooks(LinkField *lf)
{
    const char *v = getenv("STG_FX16_GRID");
    lf->fx_grid_cap = v ? atoi(v) : 0;
    if (lf->fx_grid_cap < 0) lf->fx_grid_cap = 0;
    const char *d = getenv("STG_FX16_TEST_DROP_FILL");
    lf->fx_drop_fill = (d && d[0] == '1') ? 1 : 0;
}

// ---------------------------------------------------------------------------
// field packing
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_pack_field(int vh, const double2 *__restrict__ canon, void *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    typedef typename Real<P>::T T;
    Vec3<T> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double2 a = canon[(size_t)i * 3 + c];
        v.r[c] = T(a.x);
        v.i[c] = T(a.y);
    }
    FieldIO<P>::store(out, vh, i, v);
}

template <int P>
__global__ void k_unpack_field(int vh, const void *in, double2 *__restrict__ canon)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    const auto v = FieldIO<P>::load(in, vh, i);
#pragma unroll
    for (int c = 0; c < 3; ++c) canon[(size_t)i * 3 + c] = make_double2(double(v.r[c]), double(v.i[c]));
}

stg_status pack_field(const Geom &g, int prec, const double *canon, void *out, cudaStream_t s)
{
    const int grid = (g.Vh + 255) / 256;
    const double2 *c = reinterpret_cast<const double2 *>(canon);
    if (prec == P64) k_pack_field<P64><<<grid, 256, 0, s>>>(g.Vh, c, out);
    else if (prec == P32) k_pack_field<P32><<<grid, 256, 0, s>>>(g.Vh, c, out);
    else if (prec == P16) k_pack_field<P16><<<grid, 256, 0, s>>>(g.Vh, c, out);
    else if (prec == PB16) k_pack_field<PB16><<<grid, 256, 0, s>>>(g.Vh, c, out);
    else k_pack_field<PX16><<<grid, 256, 0, s>>>(g.Vh, c, out);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

stg_status unpack_field(const Geom &g, int prec, const void *in, double *canon, cudaStream_t s)
{
    const int grid = (g.Vh + 255) / 256;
    double2 *c = reinterpret_cast<double2 *>(canon);
    if (prec == P64) k_unpack_field<P64><<<grid, 256, 0, s>>>(g.Vh, in, c);
    else if (prec == P32) k_unpack_field<P32><<<grid, 256, 0, s>>>(g.Vh, in, c);
    else if (prec == P16) k_unpack_field<P16><<<grid, 256, 0, s>>>(g.Vh, in, c);
    else if (prec == PB16) k_unpack_field<PB16><<<grid, 256, 0, s>>>(g.Vh, in, c);
    else k_unpack_field<PX16><<<grid, 256, 0, s>>>(g.Vh, in, c);
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
const LinkField *links_for(const stg_gauge *g, int prec)
{
    if (prec == P64) return &g->hi;
    if (g->lo.base && g->lo.prec == prec) return &g->lo;
    return nullptr;
}

size_t gauge_bytes(const int dims[4], int sloppy, int recon)
{
    const Geom g = make_geom(dims);
    const size_t vh = (size_t)g.Vh;
    const int recon_hi = (sloppy == P64) ? recon : 18;
    size_t n = 8 * align256(vh * link_bytes(P64, recon_hi));
    if (sloppy != P64) n += 8 * align256(vh * link_bytes(sloppy, recon));
    if ((sloppy == PX16 || sloppy == P16) && recon == 12 && want_tiled())
        n += 2 * (size_t)((g.Vh + kFxTile - 1) / kFxTile) * 4 * kFxStageBytes;
    if ((sloppy == P32 || sloppy == PX16) && recon == 12 && want_mtiled())
        n += 2 * (size_t)((g.Vh + kMTile - 1) / kMTile) * kMTile * 8 * (sloppy == P32 ? 48 : 24);
    return n;
}

stg_status gauge_create(const int dims[4], const double *links_host, int sloppy, int recon,
                        cudaStream_t s, stg_gauge **out)
{
    stg_gauge *g = new (std::nothrow) stg_gauge();
    if (!g) {
        set_error("stg_gauge_create: host allocation failed");
        return STG_ERR_OOM;
    }
    for (int mu = 0; mu < 4; ++mu) g->dims[mu] = dims[mu];
    g->geom = make_geom(dims);
    g->sloppy = sloppy;
    g->ws = nullptr;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaGetDevice");
    }
    const size_t canon_bytes = (size_t)g->geom.Vh * 2 * 4 * 9 * sizeof(double2);
    double2 *ucan = nullptr;
    stg_status st = STG_OK;
    e = cudaMalloc((void **)&ucan, canon_bytes);
    if (e != cudaSuccess) {
        delete g;
        set_error("stg_gauge_create: device staging allocation failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemcpyAsync(ucan, links_host, canon_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync(links)");
    const int recon_hi = (sloppy == P64) ? recon : 18;
    if (st == STG_OK) st = pack_links(g->geom, ucan, P64, recon_hi, &g->hi, s);
    if (st == STG_OK && sloppy != P64) st = pack_links(g->geom, ucan, sloppy, recon, &g->lo, s);
    if (st == STG_OK && (sloppy == PX16 || sloppy == P16) && recon == 12 && want_tiled()) {
        st = tile_links(g->geom, &g->lo, s);
        read_fx_hooks(&g->lo);
    }
    if (st == STG_OK && (sloppy == P32 || sloppy == PX16) && recon == 12 && want_mtiled())
        st = mtile_links(g->geom, &g->lo, s);
    e = cudaStreamSynchronize(s);
    if (st == STG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    cudaFree(ucan);
    if (st != STG_OK) {
        if (g->hi.base) cudaFree(g->hi.base);
        if (g->lo.base) cudaFree(g->lo.base);
        if (g->lo.tiled) cudaFree(g->lo.tiled);
        if (g->lo.mtiled) cudaFree(g->lo.mtiled);
        delete g;
        return st;
    }
    *out = g;
    return STG_OK;
}

void gauge_destroy(stg_gauge *g)
{
    if (!g) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    if (g->ws) workspace_free(g->ws);
    if (g->hi.base) cudaFree(g->hi.base);
    if (g->lo.base) cudaFree(g->lo.base);
    if (g->lo.tiled) cudaFree(g->lo.tiled);
    if (g->lo.mtiled) cudaFree(g->lo.mtiled);
    if (cur >= 0 && cur != g->device) cudaSetDevice(cur);
    delete g;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
stg_status workspace_get(stg_gauge *g, Workspace **out)
{
    if (g->ws) {
        *out = g->ws;
        return STG_OK;
    }
    Workspace *ws = new (std::nothrow) Workspace();
    if (!ws) {
        set_error("workspace: host allocation failed");
        return STG_ERR_OOM;
    }
    ws->n_partials = (size_t)((g->geom.Vh + kBlock - 1) / kBlock) + 64;
    cudaError_t e = cudaMalloc((void **)&ws->partials, ws->n_partials * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ws->state, sizeof(CGState));
    if (e == cudaSuccess) e = cudaMemset(ws->state, 0, sizeof(CGState));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ws->state_host, sizeof(CGState));
    if (e != cudaSuccess) {
        workspace_free(ws);
        set_error("workspace: allocation failed");
        return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "workspace");
    }
    g->ws = ws;
    *out = ws;
    return STG_OK;
}

stg_status workspace_tmp(stg_gauge *g, int prec, void **out)
{
    if (prec < 0 || prec >= kNumPrec) {
        set_error("workspace: unknown precision");
        return STG_ERR_INVALID_ARG;
    }
    Workspace *ws;
    STG_TRY(workspace_get(g, &ws));
    if (!ws->tmp[prec]) {
        size_t n = (size_t)g->geom.Vh * field_site_bytes(prec);
        cudaError_t e = cudaMalloc(&ws->tmp[prec], n);
        if (e != cudaSuccess) {
            ws->tmp[prec] = nullptr;
            set_error("workspace: allocation of the odd intermediate failed");
            return e == cudaErrorMemoryAllocation ? STG_ERR_OOM : cuda_fail(e, "cudaMalloc");
        }
    }
    *out = ws->tmp[prec];
    return STG_OK;
}

void workspace_free(Workspace *ws)
{
    if (!ws) return;
    batch_destroy(ws->batch);
    cudaFree(ws->mrhs_tmp);
    for (int k = 0; k < 3; ++k)
        if (ws->graph[k]) cudaGraphExecDestroy(ws->graph[k]);
    for (int k = 0; k < 5; ++k)
        if (ws->ev[k]) cudaEventDestroy(ws->ev[k]);
    for (int k = 0; k < 2; ++k)
        if (ws->ev_chunk[k]) cudaEventDestroy(ws->ev_chunk[k]);
    cudaFree(ws->partials);
    cudaFree(ws->state);
    if (ws->state_host) cudaFreeHost(ws->state_host);
    for (int p = 0; p < kNumPrec; ++p) cudaFree(ws->tmp[p]);
    void *v[] = {ws->x64, ws->b64, ws->r64, ws->t64, ws->y, ws->r, ws->d, ws->q};
    for (void *p : v) cudaFree(p);
    delete ws;
}

}  // namespace stg
