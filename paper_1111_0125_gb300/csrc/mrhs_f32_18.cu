// Multi-system Dslash instantiations: F32 storage, 18-real links.
#include "mrhs_kernels.cuh"

namespace stg {

void launch_dslash_m_f32_18(int shape, int epi, const MrhsArgs &a, cudaStream_t s)
{
    launch_m_pr<P32, 18>(shape, epi, a, s);
}

}  // namespace stg
