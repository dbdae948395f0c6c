// Multi-system Dslash instantiations: F32 storage, 12-real links.
#include "mrhs_kernels.cuh"

namespace stg {

void launch_dslash_m_f32_12(int shape, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (shape >= kMsRiFirst) launch_ms_ri<P32>(shape - kMsRiFirst, epi, a, s);
    else if (shape >= kMrhsShapes) launch_ms<P32>(shape - kMrhsShapes, epi, a, s);
    else launch_m_pr<P32, 12>(shape, epi, a, s);
}

}  // namespace stg
