// Instantiations of the stream-and-collide kernel for the MRT collision model.
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_mrt(int lattice, int store, const StepParams& p, bool mask, bool aa,
                           cudaStream_t s)
{
    return launch_step_model<MODEL_MRT, 2u>(lattice, store, p, mask, aa, s);
}
}  // namespace lbm
