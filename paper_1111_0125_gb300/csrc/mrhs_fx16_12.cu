// Multi-system Dslash instantiations: FX16 storage, 12-real links.
#include "mrhs_paired.cuh"

namespace stg {

void launch_dslash_m_fx16_12(int shape, int epi, const MrhsArgs &a, cudaStream_t s)
{
    if (shape >= kMsRiFirst) launch_ms_ri<PX16>(shape - kMsRiFirst, epi, a, s);
    else if (shape >= kMrhsShapes + kMrhsStagedShapes)
        launch_msp(shape - kMrhsShapes - kMrhsStagedShapes, epi, a, s);
    else if (shape >= kMrhsShapes) launch_ms<PX16>(shape - kMrhsShapes, epi, a, s);
    else launch_m_pr<PX16, 12>(shape, epi, a, s);
}

}  // namespace stg
