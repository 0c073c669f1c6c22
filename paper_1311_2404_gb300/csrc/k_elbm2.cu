// Instantiations of the stream-and-collide kernel for the ELBM collision
// model, D2Q9 (the D3Q19 ones are in k_elbm3.cu so the two compile in
// parallel).
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_elbm2(int store, const StepParams& p, bool mask, bool aa, cudaStream_t s)
{
    return launch_step_model<MODEL_ELBM, 0>(0, store, p, mask, aa, s);
}
}  // namespace lbm
