// stg_apply_A_dot_noalloc: the even-site normal operator with the fused
// d^dag A d reduction, for callers that cannot allocate device memory.
//
// Who needs it.  stg_apply_A_dot keeps its scratch (the odd intermediate
// D_oe d, the per-block partial sums and the arrival counter) in a
// workspace that the library allocates with cudaMalloc on first use.  Some
// callers cannot let a library allocate: a latency-bound loop cannot absorb
// the implicit device-wide synchronisation of cudaMalloc / cudaFree, and a
// host whose device memory is owned by another allocator or a fixed HBM
// budget forbids allocations it did not make.  This entry point allocates
// nothing: its scratch is the file-scope device array below, which the CUDA
// module reserves once per device when the library is loaded there and
// keeps until the process exits.
//
// Limit.  kScratchBytes = 32 MiB holds, besides the counter and the block
// partials, the odd intermediate of Vh sites: 48 Vh bytes in FP64, 24 Vh in
// FP32, 16 Vh in FP16 / FX16 / BF16.  Up to 24^3x48 fits in FP64 and 32^3x64 in the
// others; larger lattices are rejected with STG_ERR_INVALID_ARG and a message.
//
// Sharing.  Every call on a device uses the same array and leaves its
// contents behind; each call clears the counter itself.  Two calls whose GPU
// work overlaps on one device (different streams, or different host threads
// without ordering) race on the array and corrupt each other's results.
#include <math.h>

#include <mutex>
#include <string>

#include "stg_internal.h"

namespace stg {

static constexpr size_t kScratchBytes = (size_t)32 << 20;
static constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_scratch_mutex;
static void *g_scratch_addr[kMaxDevices];

static size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

// Device address of the scratch array on `device` (which must be current).
// Looked up once per device; the host-side symbol is only a stand-in and
// must never be handed to a kernel.
static stg_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_error("stg_apply_A_dot_noalloc: device ordinal out of range");
        return STG_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return STG_OK;
}

}  // namespace stg

using namespace stg;

extern "C" stg_status stg_apply_A_dot_noalloc(const stg_gauge *g, double mass, const void *in_dev,
                                              void *out_dev, double *dot_dev, stg_prec prec,
                                              stg_stream_t stream)
{
    if (!g || !in_dev || !out_dev || !dot_dev || in_dev == out_dev || !isfinite(mass)) {
        set_error("stg_apply_A_dot_noalloc: NULL or aliased pointer, or non-finite mass");
        return STG_ERR_INVALID_ARG;
    }
    if (prec != STG_FP64 && prec != STG_FP32 && prec != STG_FP16 && prec != STG_FX16 && prec != STG_BF16) {
        set_error("stg_apply_A_dot_noalloc: unknown precision");
        return STG_ERR_INVALID_ARG;
    }
    const LinkField *lf = links_for(g, prec);
    if (!lf) {
        set_error("stg_apply_A_dot_noalloc: the gauge handle holds no links in this precision");
        return STG_ERR_UNSUPPORTED;
    }
    const Geom &geo = g->geom;
    // every EPI_A_DOT launch writes one partial (8 bytes) per thread block
    // and uses at most ceil(Vh / kBlock) blocks: one site per thread in
    // k_dslash, two in k_dslash_fx2, and at most one block per 1024-site
    // tile in the staged FX16 kernel
    const size_t n_blocks = (size_t)(geo.Vh + kBlock - 1) / kBlock;
    const size_t off_partials = 256;  // the counter lives in the first 256 bytes
    const size_t off_tmp = off_partials + round256(n_blocks * sizeof(double));
    const size_t need = off_tmp + round256((size_t)geo.Vh * field_site_bytes(prec));
    if (need > kScratchBytes) {
        set_error("stg_apply_A_dot_noalloc: this lattice needs " + std::to_string(need) +
                  " bytes of scratch in this precision; the fixed scratch holds " +
                  std::to_string(kScratchBytes) + " bytes (use stg_apply_A_dot)");
        return STG_ERR_INVALID_ARG;
    }

    int prev = -1;
    cudaError_t de = cudaGetDevice(&prev);
    if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
    if (prev != g->device) {
        // the scratch address below is cached per device: it must be looked
        // up with the handle's device current
        de = cudaSetDevice(g->device);
        if (de != cudaSuccess) return cuda_fail(de, "cudaSetDevice(handle device)");
    }
    unsigned char *base = nullptr;
    stg_status st = scratch_address(g->device, &base);
    cudaStream_t s = (cudaStream_t)stream;
    if (st == STG_OK) {
        // the array keeps the previous call's contents: the arrival counter
        // must start at zero
        cudaError_t e = cudaMemsetAsync(base, 0, 256, s);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(scratch counter)");
    }
    if (st == STG_OK) {
        void *tmp = base + off_tmp;
        DslashLaunch L = {};
        L.links = lf;
        L.out_parity = 1;
        L.in = in_dev;
        L.out = tmp;
        st = launch_dslash(geo, prec, EPI_NONE, L, s);
        if (st == STG_OK) {
            L.out_parity = 0;
            L.in = tmp;
            L.out = out_dev;
            L.w = in_dev;
            L.m2 = mass * mass;
            L.dot = dot_dev;
            L.partials = reinterpret_cast<double *>(base + off_partials);
            L.counter = reinterpret_cast<unsigned *>(base);
            st = launch_dslash(geo, prec, EPI_A_DOT, L, s);
        }
    }
    if (prev != g->device) {
        de = cudaSetDevice(prev);
        if (de != cudaSuccess && st == STG_OK) st = cuda_fail(de, "cudaSetDevice(restore)");
    }
    return st;
}
