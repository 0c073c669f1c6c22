// Instantiations of the stream-and-collide kernel for LBGK with Guo forcing,
// D2Q9 and D3Q19 (Eq. lbgk, Eq. guo_force).
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_bgk(int lattice, int store, const StepParams& p, bool mask, bool aa,
                            cudaStream_t s)
{
    return launch_step_model<MODEL_BGK, 3u>(lattice, store, p, mask, aa, s);
}
}  // namespace lbm
