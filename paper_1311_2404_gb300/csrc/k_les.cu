// Instantiations of the stream-and-collide kernel for the regularized LBGK
// and the Smagorinsky LES collision models.
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_reg(int lattice, int store, const StepParams& p, bool mask, bool aa,
                            cudaStream_t s)
{
    return launch_step_model<MODEL_REG, 3u>(lattice, store, p, mask, aa, s);
}
cudaError_t launch_step_smag(int lattice, int store, const StepParams& p, bool mask, bool aa,
                             cudaStream_t s)
{
    return launch_step_model<MODEL_SMAG, 3u>(lattice, store, p, mask, aa, s);
}
}  // namespace lbm
