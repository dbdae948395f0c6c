// Several lattices in one launch: the Dslash half-pass (Eq. 5) of up to
// kGroupMax (gauge field, colour field) pairs, of equal or different lattice
// sizes, as one grid.  Each item owns a contiguous range of thread blocks
// (one output site per thread, as k_dslash); a block finds its item by the
// block ranges, which travel in the kernel's parameter space.  Small
// lattices (a few thousand sites each) leave most of the GPU idle in a
// launch of their own; grouped, they fill it in one launch.  The per-site
// arithmetic is dslash_site, so an item's output is bitwise the one of
// stg_dslash wherever that runs the one-site-per-thread kernel (FX16 /
// 12-real runs the packed staged kernel instead: equal to rounding).
//
// The paper applies the operator to one lattice at a time; this is a
// serving-layer form of the same operation.
#include "dslash_site.cuh"

namespace stg {

constexpr int kGroupMax = 16;

struct GroupItem {
    Geom g;
    const char *lf[4];
    const char *lb[4];
    const void *in;
    void *out;
    int parity;
    int first_block;  // the item's blocks are [first_block, next item's first_block)
};

struct GroupArgs {
    int n;
    GroupItem it[kGroupMax];
};
static_assert(sizeof(GroupArgs) <= 4000, "the group must fit the kernel parameter space");

template <int P, int R>
__global__ void __launch_bounds__(kBlock) k_dslash_group(const __grid_constant__ GroupArgs ga)
{
    int p = 0;
    while (p + 1 < ga.n && (int)blockIdx.x >= ga.it[p + 1].first_block) ++p;
    const GroupItem &t = ga.it[p];
    const int i = ((int)blockIdx.x - t.first_block) * kBlock + (int)threadIdx.x;
    if (i >= t.g.Vh) return;
    const auto acc = dslash_site<P, R>(t.g, t.lf, t.lb, t.parity, t.in, i);
    FieldIO<P>::store(t.out, t.g.Vh, i, acc);
}

template <int P>
static void launch_group_p(int recon, const GroupArgs &ga, int blocks, cudaStream_t s)
{
    if (recon == 18) k_dslash_group<P, 18><<<blocks, kBlock, 0, s>>>(ga);
    else k_dslash_group<P, 12><<<blocks, kBlock, 0, s>>>(ga);
}

}  // namespace stg

using namespace stg;

extern "C" stg_status stg_dslash_group(int n, const stg_gauge *const *g, const int *out_parity,
                                       const void *const *in_dev, void *const *out_dev, stg_prec prec,
                                       stg_stream_t stream)
{
    if (n < 1 || n > kGroupMax || !g || !out_parity || !in_dev || !out_dev) {
        set_error("stg_dslash_group: n outside [1, 16] or NULL array");
        return STG_ERR_INVALID_ARG;
    }
    GroupArgs ga = {};
    ga.n = n;
    long blocks = 0;
    int device = -1, recon = 0;
    for (int k = 0; k < n; ++k) {
        const stg_gauge *gk = g[k];
        if (!gk || !in_dev[k] || !out_dev[k] || (out_parity[k] != 0 && out_parity[k] != 1)) {
            set_error("stg_dslash_group: NULL handle or field, or parity not 0/1");
            return STG_ERR_INVALID_ARG;
        }
        const LinkField *lf = links_for(gk, prec);
        if (!lf) {
            set_error("stg_dslash_group: a handle holds no links in this precision");
            return STG_ERR_UNSUPPORTED;
        }
        if (k == 0) {
            device = gk->device;
            recon = lf->recon;
        } else if (gk->device != device || lf->recon != recon) {
            set_error("stg_dslash_group: handles on different devices or with different reconstruction");
            return STG_ERR_INVALID_ARG;
        }
        // an output that aliases any item's input would be overwritten
        // while other threads still read it as a neighbour
        for (int j = 0; j < n; ++j)
            if (out_dev[k] == in_dev[j]) {
                set_error("stg_dslash_group: an item's output aliases an item's input");
                return STG_ERR_INVALID_ARG;
            }
        GroupItem &t = ga.it[k];
        t.g = gk->geom;
        for (int mu = 0; mu < 4; ++mu) {
            t.lf[mu] = lf->blk(out_parity[k], mu);
            t.lb[mu] = lf->blk(1 - out_parity[k], mu);
        }
        t.in = in_dev[k];
        t.out = out_dev[k];
        t.parity = out_parity[k];
        t.first_block = (int)blocks;
        blocks += (gk->geom.Vh + kBlock - 1) / kBlock;
    }
    if (blocks > 0x7fffffffL) {
        set_error("stg_dslash_group: too many sites for one launch");
        return STG_ERR_INVALID_ARG;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    cudaStream_t s = (cudaStream_t)stream;
    switch (prec) {
    case STG_FP64: launch_group_p<P64>(recon, ga, (int)blocks, s); break;
    case STG_FP32: launch_group_p<P32>(recon, ga, (int)blocks, s); break;
    case STG_FP16: launch_group_p<P16>(recon, ga, (int)blocks, s); break;
    case STG_FX16: launch_group_p<PX16>(recon, ga, (int)blocks, s); break;
    case STG_BF16: launch_group_p<PB16>(recon, ga, (int)blocks, s); break;
    default:
        if (cur != device && cur >= 0) cudaSetDevice(cur);
        set_error("stg_dslash_group: unknown precision");
        return STG_ERR_INVALID_ARG;
    }
    const cudaError_t e = cudaGetLastError();
    if (cur != device && cur >= 0) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "stg_dslash_group launch");
    return STG_OK;
}
