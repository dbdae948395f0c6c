// Multi-right-hand-side Dslash instantiations for FX16 (16-bit fixed point)
// storage.
#include "mrhs_kernels.cuh"

namespace stg {

void launch_dslash_m_fx16(int recon, int nb, int bs, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (recon == 18) launch_m_pr<PX16, 18>(nb, bs, epi, a, s);
    else launch_m_pr<PX16, 12>(nb, bs, epi, a, s);
}

}  // namespace stg
