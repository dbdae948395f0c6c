// Staggered Dslash half-pass (Eq. 5) and its fused epilogues.
//
// One thread per output site of parity p.  Per site the kernel reads the
// four forward links U_mu(x) (parity p block, index i), the four backward
// links U_mu(x - mu) (parity 1-p block, at the neighbour's index), and the
// eight neighbour colour vectors of parity 1-p, then writes one colour
// vector.  Every link is read exactly once per half-pass; each neighbour
// vector is shared by eight sites and is served from L1/L2 after its first
// read, so the compulsory HBM traffic is 8 links + 1 input + 1 output per
// site.  The work is bandwidth-bound (0.36 flop/byte in FP64, 0.9 in
// FP32/12), so there are no tensor cores here: the 3x3 complex mat-vecs run
// on the FP32 / FP64 pipes in registers.
//
// Reductions of FP64 data sum in FP64; those of FP32 / 16-bit data use the
// compensated FP32 pairs of grid_sum_ff (the FP64 pipe is ~1/64 of FP32 here).
//
// Epilogues (all fused into the second half-pass of A, Eq. 3):
//   EPI_NONE  out = D in
//   EPI_GATE  out = D in, skipped when the CG state flag is raised
//   EPI_A     out = m^2 w - D in                     (w = the even input d)
//   EPI_A_DOT as EPI_A, plus Re sum w^dag out in FP64 -> *dot
//   EPI_A_CG  as EPI_A_DOT inside CG: alpha = delta / d^dag A d -> state
//   EPI_RES   out = w - m^2 v + D in = b - A x, plus |out|^2 in FP64 -> *dot
#include "dslash_site.cuh"

namespace stg {

template <int P, int R, int EPI>
__global__ void __launch_bounds__(kBlock) k_dslash(const DslashArgs a)
{
    typedef typename Real<P>::T T;
    pdl_wait();
    pdl_trigger();
    if (EPI == EPI_A_CG || EPI == EPI_GATE) {
        if (a.state->flag != FLAG_RUN) return;  // uniform over the grid
    }
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const int vh = a.g.Vh;
    T dot = T(0);
    if (i < vh) {
        const Vec3<T> acc = dslash_site<P, R>(a.g, a.lf, a.lb, a.parity, a.in, i);
        if (EPI == EPI_NONE || EPI == EPI_GATE) {
            FieldIO<P>::store(a.out, vh, i, acc);
        } else if (EPI == EPI_RES) {
            const Vec3<T> b = FieldIO<P>::load_nc(a.w, vh, i);
            const Vec3<T> x = FieldIO<P>::load_nc(a.v, vh, i);
            const T m2 = T(a.m2);
            Vec3<T> o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.r[c] = b.r[c] - m2 * x.r[c] + acc.r[c];
                o.i[c] = b.i[c] - m2 * x.i[c] + acc.i[c];
            }
            const Vec3<T> os = FieldIO<P>::store(a.out, vh, i, o);
#pragma unroll
            for (int c = 0; c < 3; ++c) dot += os.r[c] * os.r[c] + os.i[c] * os.i[c];
        } else {
            const T m2 = (EPI == EPI_A_CG) ? T(a.state->m2) : T(a.m2);
            const Vec3<T> d = FieldIO<P>::load_nc(a.w, vh, i);
            Vec3<T> o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.r[c] = m2 * d.r[c] - acc.r[c];
                o.i[c] = m2 * d.i[c] - acc.i[c];
            }
            // d^dag q with q as stored, i.e. as the CG update will read it
            const Vec3<T> os = FieldIO<P>::store(a.out, vh, i, o);
#pragma unroll
            for (int c = 0; c < 3; ++c) dot += d.r[c] * os.r[c] + d.i[c] * os.i[c];
        }
    }
    if (EPI == EPI_A_DOT || EPI == EPI_A_CG || EPI == EPI_RES) {
        double total;
        bool last;
        if constexpr (P == P64) {
            last = grid_sum<kBlock>(double(dot), a.partials, a.counter, total);
        } else {
            FF v;
            v.hi = float(dot);
            v.lo = 0.f;
            last = grid_sum_ff<kBlock>(v, reinterpret_cast<float2 *>(a.partials), a.counter, total);
        }
        if (last) {
            if (EPI == EPI_A_CG) {
                CGState *st = a.state;
                set_alpha(st, total);
            } else {
                *a.dot = total;
            }
        }
    }
}

template <int P, int R>
static void launch_pr(int epi, const DslashArgs &a, int grid, cudaStream_t s, bool pdl)
{
    switch (epi) {
    case EPI_NONE: launch_k(k_dslash<P, R, EPI_NONE>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_A: launch_k(k_dslash<P, R, EPI_A>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_A_DOT: launch_k(k_dslash<P, R, EPI_A_DOT>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_A_CG: launch_k(k_dslash<P, R, EPI_A_CG>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_RES: launch_k(k_dslash<P, R, EPI_RES>, grid, kBlock, 0, s, pdl, a); break;
    case EPI_GATE: launch_k(k_dslash<P, R, EPI_GATE>, grid, kBlock, 0, s, pdl, a); break;
    }
}

stg_status launch_dslash(const Geom &g, int prec, int epi, const DslashLaunch &L, cudaStream_t s)
{
    DslashArgs a;
    a.g = g;
    a.parity = L.out_parity;
    for (int mu = 0; mu < 4; ++mu) {
        a.lf[mu] = L.links->blk(L.out_parity, mu);
        a.lb[mu] = L.links->blk(1 - L.out_parity, mu);
    }
    a.lt = L.links->tiled ? L.links->tiled + (size_t)L.out_parity * L.links->tiled_parity_bytes : nullptr;
    a.grid_cap = L.links->fx_grid_cap;
    a.drop_fill = L.links->fx_drop_fill;
    a.in = L.in;
    a.out = L.out;
    a.w = L.w;
    a.v = L.v;
    a.m2 = L.m2;
    a.dot = L.dot;
    a.state = L.state;
    a.partials = L.partials;
    a.counter = L.counter;
    const int grid = (g.Vh + kBlock - 1) / kBlock;
    const int recon = L.links->recon;
    if (prec != L.links->prec) {
        set_error("dslash: link precision does not match the field precision");
        return STG_ERR_UNSUPPORTED;
    }
    if (prec == PX16) {  // two sites per thread on packed FP32x2 (dslash_fx16.cu)
        launch_dslash_fx2(recon, epi, a, s, L.pdl);
        STG_CUDA(cudaGetLastError());
        return STG_OK;
    }
    if (prec == P16 && recon == 12 && a.lt) {  // the same staged kernel, binary16 records
        launch_dslash_f16_staged(epi, a, s, L.pdl);
        STG_CUDA(cudaGetLastError());
        return STG_OK;
    }
    if (prec == P64) {
        if (recon == 18) launch_pr<P64, 18>(epi, a, grid, s, L.pdl);
        else launch_pr<P64, 12>(epi, a, grid, s, L.pdl);
    } else if (prec == P32) {
        if (recon == 18) launch_pr<P32, 18>(epi, a, grid, s, L.pdl);
        else launch_pr<P32, 12>(epi, a, grid, s, L.pdl);
    } else {
        if (prec == PB16) {
            if (recon == 18) launch_pr<PB16, 18>(epi, a, grid, s, L.pdl);
            else launch_pr<PB16, 12>(epi, a, grid, s, L.pdl);
        } else if (recon == 18) {
            launch_pr<P16, 18>(epi, a, grid, s, L.pdl);
        } else {
            launch_pr<P16, 12>(epi, a, grid, s, L.pdl);
        }
    }
    STG_CUDA(cudaGetLastError());
    return STG_OK;
}

}  // namespace stg
