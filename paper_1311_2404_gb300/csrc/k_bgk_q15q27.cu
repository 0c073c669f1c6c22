// Instantiations of the LBGK stream-and-collide kernel on D3Q15 and D3Q27.
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_bgk_q15q27(int lattice, int store, const StepParams& p, bool mask,
                                   bool aa, cudaStream_t s)
{
    return launch_step_model<MODEL_BGK, 12u>(lattice, store, p, mask, aa, s);
}
}  // namespace lbm
