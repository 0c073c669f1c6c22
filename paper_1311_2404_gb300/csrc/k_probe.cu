// Peak rate of the FP64 pipe, the unit that bounds the entropic (ELBM)
// collision's alpha solve (Eq. alpha_cond is solved in FP64, whose
// instruction rate on this GPU is a small fraction of FP32's).  The probe
// runs independent chains of FP64 fused multiply-adds in every thread of a
// full grid and reports the executed warp instructions per second, the same
// unit as the FP64-pipe instruction count of a profiled kernel.  A
// measurement aid for the roofline of the ELBM kernel; no counterpart in the
// paper.
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kProbeThreads = 256;

__device__ double g_probe_sink;     // target of a store the compiler cannot drop

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // x converges to b / (1 - a) = 0.1, so this store never happens, but the
    // compiler cannot know that
    if (s == 12345.678) g_probe_sink = s;
}

}  // namespace

extern "C" int lbm_probe_fp64_rate(void* cuda_stream, double* warp_inst_per_s, double* flops)
{
    if (!warp_inst_per_s || !flops) return LBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kProbeThreads, 0) !=
            cudaSuccess)
        return LBM_ECUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 14;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LBM_ECUDA;
    }
    int rc = LBM_OK;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == LBM_OK; ++rep) {   // the first run warms up
        cudaEventRecord(e0, s);
        k_fp64_fma<<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = LBM_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) return rc;
    const double fma_thread = (double)blocks * kProbeThreads * iters * kChains;
    *warp_inst_per_s = fma_thread / 32.0 / (best * 1e-3);
    *flops = 2.0 * fma_thread / (best * 1e-3);
    return LBM_OK;
}
