// Ghost-layer exchange between subdomains (Sec. 3.6): the collect and
// distribute kernels.  A subdomain is a slab of whole rows of the slowest
// axis (z layers on D3Q19, y rows on D2Q9) with one ghost row on each side.
// After a step, the populations that leave a slab across a face (the
// directions with a component toward the neighbour, 5 of 19 or 3 of 9) are
// collected from its boundary row into a linear send buffer, moved to the
// neighbour's receive buffer, and distributed into the neighbour's ghost
// row, where the next step's pull reads them.  In the structure-of-arrays
// layout one direction of one row is a contiguous run, so both kernels copy
// whole runs: each is a table of (source, destination, length) segments.
#include <cstdint>

#include "lbm_internal.h"

namespace lbm {

__global__ void __launch_bounds__(256) k_halo_copy(const HaloSeg* __restrict__ segs)
{
    const HaloSeg sg = segs[blockIdx.y];
    const uint4* __restrict__ src = sg.src;
    uint4* __restrict__ dst = sg.dst;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < sg.n16;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

cudaError_t launch_halo_copy(const HaloSeg* segs_dev, int nseg, long long max_n16,
                             cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    long long bx = (max_n16 + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    k_halo_copy<<<dim3((unsigned)bx, (unsigned)nseg, 1), 256, 0, s>>>(segs_dev);
    return cudaGetLastError();
}

}  // namespace lbm
