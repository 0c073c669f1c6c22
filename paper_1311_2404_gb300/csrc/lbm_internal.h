// Host-side declarations shared by the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kReduceBlocks = 1024;   // FP64 partial sums: kReduceBlocks x 5 doubles

// Every device allocation the library makes goes through dev_alloc, so that
// lbm_debug_fail_allocations can make the next ones fail (out of memory)
// without calling cudaMalloc: the error paths are tested on the host.
cudaError_t dev_alloc(void** p, size_t bytes);
// p for device memory, the mapped device address of pinned host memory, or
// nullptr for pageable host memory (which must be staged)
const void* kernel_view(const void* p);

cudaError_t launch_step_bgk(int lattice, int store, const StepParams& p, bool mask, bool aa,
                            cudaStream_t s);
cudaError_t launch_step_mrt(int lattice, int store, const StepParams& p, bool mask, bool aa,
                            cudaStream_t s);
// One contiguous run of a ghost-layer exchange (16-byte units).
struct HaloSeg {
    const uint4* src;
    uint4* dst;
    long long n16;
};
cudaError_t launch_halo_copy(const HaloSeg* segs_dev, int nseg, long long max_n16,
                             cudaStream_t s);
cudaError_t launch_step_reg(int lattice, int store, const StepParams& p, bool mask, bool aa,
                            cudaStream_t s);
cudaError_t launch_step_bgk_q15q27(int lattice, int store, const StepParams& p, bool mask,
                                   bool aa, cudaStream_t s);
cudaError_t launch_step_reg_q15q27(int lattice, int store, const StepParams& p, bool mask,
                                   bool aa, cudaStream_t s);
cudaError_t launch_step_smag_q15q27(int lattice, int store, const StepParams& p, bool mask,
                                    bool aa, cudaStream_t s);
cudaError_t launch_step_smag(int lattice, int store, const StepParams& p, bool mask, bool aa,
                             cudaStream_t s);
cudaError_t launch_diagnostics(int f64, const void* u, int D, int nx, int ny, int nz, int nxp,
                               long long sq, double* partials, double* out, cudaStream_t s);
// ELBM: one object per (lattice code LAT, storage mask STORES); see k_elbm.cu
template <int LAT, unsigned STORES>
cudaError_t launch_step_elbm_part(int store, const StepParams& p, bool mask, bool aa,
                                  cudaStream_t s);
// storage groups of the ELBM objects: {F64}, {F32, F32S}, {F16S, BF16S}
constexpr unsigned kElbmStoreGroup[5] = {1u, 6u, 6u, 24u, 24u};

// nearwall_segs (optional, needs nxp % 32 == 0): incremented once per
// 32-node row segment holding a fluid node with a solid upstream neighbour.
// sector (a power of two, 0 for none): nodes per 32-byte sector of a direction
// plane; solid nodes sharing an x-aligned sector with a fluid node get
// NODE_FILL.
cudaError_t launch_flags(int lattice, const uint8_t* dense, uint32_t* words, uint8_t* flags,
                         int nx, int ny, int nz, int nxp, int max_code, int* bad,
                         unsigned* nearwall_segs, int sector, cudaStream_t s);
cudaError_t launch_init(int lattice, int store, const void* rho, const void* u, int field_f32,
                        void* A, int nx, int ny, int nz, int nxp, long long sq, int entropic,
                        int feq_variant, int opposite_slots, cudaStream_t s);
// `add` is added to every value in FP64 (1 for the rho field, which holds
// rho - 1)
cudaError_t launch_pack(int src_f64, const void* src, int dst_f32, void* dst, int nfields, int nx,
                        int ny, int nz, int nxp, long long sq, double add, cudaStream_t s);
cudaError_t launch_reduce(int f64, const void* rho, const void* u, const uint32_t* nodes, int D,
                          int nx, int ny, int nz, int nxp, long long sq, double* partials,
                          double* out, cudaStream_t s);
cudaError_t launch_sum_ctr(const unsigned long long* rep, double* out, cudaStream_t s);

}  // namespace lbm
