// The Dslash half-pass (Eq. 5) at one output site, shared by the one-site-
// per-thread kernels (dslash.cu) and the multi-lattice group launch
// (group.cu): the four forward links at the site, the four backward links at
// the neighbours, the eight neighbour colour vectors, and for FX16 links the
// scale 1/32767 applied once to the sum.
#pragma once

#include "stg_internal.h"

namespace stg {

template <int P, int R>
__device__ __forceinline__ Vec3<typename Real<P>::T> dslash_site(const Geom &g, const char *const *lf,
                                                                 const char *const *lb, int parity,
                                                                 const void *in, int i)
{
    typedef typename Real<P>::T T;
    const int vh = g.Vh;
    const Site s = site_of(g, i, parity);
    Vec3<T> acc;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.r[c] = acc.i[c] = T(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int jf, jb;
        neighbours(g, s, i, mu, jf, jb);
        float sf = 1.f, sb = 1.f;
        if (R == 12) link_signs(g, s, mu, sf, sb);
        const T s2f = (R == 12) ? T(sf * LinkPost<P>::row2) : T(1);
        const T s2b = (R == 12) ? T(sb * LinkPost<P>::row2) : T(1);
        const Mat3<T> uf = LinkIO<P, R>::load(lf[mu], vh, i);
        const Vec3<T> vf = FieldIO<P>::load_nc(in, vh, jf);
        mul_add<R == 12>(uf, vf, acc, s2f);
        const Mat3<T> ub = LinkIO<P, R>::load(lb[mu], vh, jb);
        const Vec3<T> vb = FieldIO<P>::load_nc(in, vh, jb);
        adj_mul_sub(ub, vb, acc, s2b);
    }
    if (P == PX16) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc.r[c] *= T(LinkPost<PX16>::k);
            acc.i[c] *= T(LinkPost<PX16>::k);
        }
    }
    return acc;
}

}  // namespace stg
