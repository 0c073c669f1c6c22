// Instantiations of the stream-and-collide kernel for the ELBM collision
// model, D3Q19.
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_elbm3(int store, const StepParams& p, bool mask, bool aa, cudaStream_t s)
{
    return launch_step_model<MODEL_ELBM, 1>(1, store, p, mask, aa, s);
}
}  // namespace lbm
