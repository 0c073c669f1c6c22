// Instantiations of the regularized and Smagorinsky LBGK kernels on D3Q15
// and D3Q27.
#include "step_kernel.cuh"

namespace lbm {
cudaError_t launch_step_reg_q15q27(int lattice, int store, const StepParams& p, bool mask,
                                   bool aa, cudaStream_t s)
{
    return launch_step_model<MODEL_REG, 12u>(lattice, store, p, mask, aa, s);
}
cudaError_t launch_step_smag_q15q27(int lattice, int store, const StepParams& p, bool mask,
                                    bool aa, cudaStream_t s)
{
    return launch_step_model<MODEL_SMAG, 12u>(lattice, store, p, mask, aa, s);
}
}  // namespace lbm
