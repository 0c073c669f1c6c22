// Instantiations of the stream-and-collide kernel for the BGK collision model.
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_bgk(int lattice, int store, const StepParams& p, bool mask, bool aa,
                           cudaStream_t s)
{
    return launch_step_model<MODEL_BGK>(lattice, store, p, mask, aa, s);
}
}  // namespace lbm
