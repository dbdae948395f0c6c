// Multi-right-hand-side Dslash instantiations for FP32 storage.
#include "mrhs_kernels.cuh"

namespace stg {

void launch_dslash_m_f32(int recon, int nb, int bs, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (recon == 18) launch_m_pr<P32, 18>(nb, bs, epi, a, s);
    else launch_m_pr<P32, 12>(nb, bs, epi, a, s);
}

}  // namespace stg
