// Instantiations of the ELBM stream-and-collide kernel (Eqs. elbm,
// alpha_cond).  The ELBM kernels are the slowest to compile, so this source
// is compiled once per (lattice, storage group): ELBM_LAT is the lattice
// code and ELBM_STORES the storage mask of the object being built.
#include "step_kernel.cuh"

#if !defined(ELBM_LAT) || !defined(ELBM_STORES)
#error "compile with -DELBM_LAT=<lattice code> -DELBM_STORES=<storage mask>"
#endif

namespace lbm {
template <int LAT, unsigned STORES>
cudaError_t launch_step_elbm_part(int store, const StepParams& p, bool mask, bool aa,
                                  cudaStream_t s)
{
    return launch_step_model<MODEL_ELBM, (1u << LAT), STORES>(LAT, store, p, mask, aa, s);
}
template cudaError_t launch_step_elbm_part<ELBM_LAT, ELBM_STORES>(int, const StepParams&, bool,
                                                                  bool, cudaStream_t);
}  // namespace lbm
