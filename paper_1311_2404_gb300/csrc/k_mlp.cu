// Training and inference kernels of the ELBM alpha surrogate (not in the
// paper): an 8 -> 32 -> 32 -> 1 tanh network mapping eight invariants of
// (f, f_eq - f) to alpha_guess = s2 + scale * out, where s2 is the
// second-order small-deviation guess written in the features
// (t_3 = X[0], t_4 = X[1], eps = X[4]):
//   s2 = 2 + (t_3 eps - 2 t_4 eps^2) / 3 + 4 t_3^2 eps^2 / 9,
// so the network learns what that expansion misses.
//
// Training is minibatch Adam (Kingma & Ba 2015) on the loss
// mean_b (out_b - t_b)^2, t_b = (alpha_b - s2_b) / scale, entirely on
// the GPU:
//   k_fwd_bwd   one thread per sample: forward and backward pass in
//               registers, activations in shared memory, then the CTA sums
//               the per-sample gradient contributions of its samples in a
//               fixed order into one partial row per CTA;
//   k_reduce    sums the partial rows in a fixed order (deterministic);
//   k_adam      updates the FP32 master parameters.
// Parameter layout (1394 floats): mean[8], inv_std[8], W1[32][8], b1[32],
// W2[32][32], b2[32], W3[32], b3, scale; entries 16..1392 are trained.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int NIN = 8, NH = 32;
constexpr int O_W1 = 16, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH, O_SCALE = O_B3 + 1, NPARAM = O_SCALE + 1;
constexpr int TRAIN_LO = O_W1, NTRAIN = O_SCALE - O_W1;   // 1377 trained entries
constexpr int BS = 64;                                    // samples per CTA

// second-order guess s2 from a feature row (FP64)
__device__ __forceinline__ double series2_of(const float* __restrict__ x)
{
    const double t3 = x[0], t4 = x[1], eps = x[4];
    return 2.0 + (t3 * eps - 2.0 * t4 * eps * eps) / 3.0 + 4.0 * t3 * t3 * eps * eps / 9.0;
}

__global__ void k_forward(const float* __restrict__ X, int n, const float* __restrict__ P,
                          float* __restrict__ alpha)
{
    __shared__ float sp[NPARAM];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) sp[k] = P[k];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    float z[NIN], h1[NH];
#pragma unroll
    for (int k = 0; k < NIN; ++k) z[k] = (X[(size_t)b * NIN + k] - sp[k]) * sp[8 + k];
#pragma unroll 4
    for (int o = 0; o < NH; ++o) {
        float s = sp[O_B1 + o];
#pragma unroll
        for (int k = 0; k < NIN; ++k) s = fmaf(sp[O_W1 + o * NIN + k], z[k], s);
        h1[o] = tanhf(s);
    }
    float out = sp[O_B3];
    for (int o = 0; o < NH; ++o) {
        float s = sp[O_B2 + o];
#pragma unroll
        for (int k = 0; k < NH; ++k) s = fmaf(sp[O_W2 + o * NH + k], h1[k], s);
        out = fmaf(sp[O_W3 + o], tanhf(s), out);
    }
    alpha[b] = (float)(series2_of(X + (size_t)b * NIN) + (double)(sp[O_SCALE] * out));
}

// idx: sample indices of this minibatch (nullptr: identity); B = minibatch size
__global__ void __launch_bounds__(BS) k_fwd_bwd(const float* __restrict__ X,
                                                const float* __restrict__ t,
                                                const int* __restrict__ idx, int B,
                                                const float* __restrict__ P,
                                                float* __restrict__ part,
                                                float* __restrict__ part_loss)
{
    __shared__ float sp[NPARAM];
    __shared__ float sZ[BS][NIN], sH1[BS][NH], sH2[BS][NH], sA1[BS][NH], sA2[BS][NH], sdo[BS],
        sl[BS];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) sp[k] = P[k];
    __syncthreads();
    const int lb = threadIdx.x;
    const int b = blockIdx.x * BS + lb;
    if (b < B) {
        const int s = idx ? idx[b] : b;
        float z[NIN], h1[NH], h2[NH];
#pragma unroll
        for (int k = 0; k < NIN; ++k) z[k] = (X[(size_t)s * NIN + k] - sp[k]) * sp[8 + k];
        for (int o = 0; o < NH; ++o) {
            float a = sp[O_B1 + o];
#pragma unroll
            for (int k = 0; k < NIN; ++k) a = fmaf(sp[O_W1 + o * NIN + k], z[k], a);
            h1[o] = tanhf(a);
        }
        float out = sp[O_B3];
        for (int o = 0; o < NH; ++o) {
            float a = sp[O_B2 + o];
#pragma unroll
            for (int k = 0; k < NH; ++k) a = fmaf(sp[O_W2 + o * NH + k], h1[k], a);
            h2[o] = tanhf(a);
            out = fmaf(sp[O_W3 + o], h2[o], out);
        }
        const float r = out - t[s];
        const float dout = 2.0f * r / (float)B;
        float a2[NH];
#pragma unroll
        for (int o = 0; o < NH; ++o) a2[o] = dout * sp[O_W3 + o] * (1.0f - h2[o] * h2[o]);
        for (int k = 0; k < NH; ++k) {
            float g = 0.f;
#pragma unroll
            for (int o = 0; o < NH; ++o) g = fmaf(sp[O_W2 + o * NH + k], a2[o], g);
            sA1[lb][k] = g * (1.0f - h1[k] * h1[k]);
        }
#pragma unroll
        for (int k = 0; k < NIN; ++k) sZ[lb][k] = z[k];
#pragma unroll
        for (int o = 0; o < NH; ++o) {
            sH1[lb][o] = h1[o];
            sH2[lb][o] = h2[o];
            sA2[lb][o] = a2[o];
        }
        sdo[lb] = dout;
        sl[lb] = r * r;
    } else {
#pragma unroll
        for (int k = 0; k < NIN; ++k) sZ[lb][k] = 0.f;
        for (int o = 0; o < NH; ++o) sH1[lb][o] = sH2[lb][o] = sA1[lb][o] = sA2[lb][o] = 0.f;
        sdo[lb] = 0.f;
        sl[lb] = 0.f;
    }
    __syncthreads();
    // per-CTA partial gradient: fixed summation order over the CTA's samples
    float* row = part + (size_t)blockIdx.x * NTRAIN;
    for (int e = threadIdx.x; e < NTRAIN; e += blockDim.x) {
        const int q = e + TRAIN_LO;
        float acc = 0.f;
        if (q < O_B1) {
            const int o = (q - O_W1) / NIN, k = (q - O_W1) % NIN;
            for (int j = 0; j < BS; ++j) acc = fmaf(sA1[j][o], sZ[j][k], acc);
        } else if (q < O_W2) {
            const int o = q - O_B1;
            for (int j = 0; j < BS; ++j) acc += sA1[j][o];
        } else if (q < O_B2) {
            const int o = (q - O_W2) / NH, k = (q - O_W2) % NH;
            for (int j = 0; j < BS; ++j) acc = fmaf(sA2[j][o], sH1[j][k], acc);
        } else if (q < O_W3) {
            const int o = q - O_B2;
            for (int j = 0; j < BS; ++j) acc += sA2[j][o];
        } else if (q < O_B3) {
            const int k = q - O_W3;
            for (int j = 0; j < BS; ++j) acc = fmaf(sdo[j], sH2[j][k], acc);
        } else {
            for (int j = 0; j < BS; ++j) acc += sdo[j];
        }
        row[e] = acc;
    }
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int j = 0; j < BS; ++j) s += sl[j];
        part_loss[blockIdx.x] = s;
    }
}

__global__ void k_reduce(const float* __restrict__ part, const float* __restrict__ part_loss,
                         int nblk, int B, float* __restrict__ grad, float* __restrict__ loss_acc)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < NTRAIN) {
        float s = 0.f;
        for (int k = 0; k < nblk; ++k) s += part[(size_t)k * NTRAIN + e];
        grad[TRAIN_LO + e] = s;
    }
    if (e == 0) {
        float s = 0.f;
        for (int k = 0; k < nblk; ++k) s += part_loss[k];
        loss_acc[0] += s / (float)B;
        loss_acc[1] += 1.0f;
    }
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x + TRAIN_LO;
    if (e >= O_SCALE) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    P[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_targets(const float* __restrict__ X, const double* __restrict__ alpha, int n,
                          float scale, float* __restrict__ t)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) t[b] = (float)((alpha[b] - series2_of(X + (size_t)b * NIN)) / (double)scale);
}

thread_local std::string g_mlp_err;

int mfail(int code, const char* what, cudaError_t e = cudaSuccess)
{
    g_mlp_err = what;
    if (e != cudaSuccess) g_mlp_err += std::string(": ") + cudaGetErrorString(e);
    return code;
}

bool is_dev(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return lbm::dev_alloc(&p, n); }
    template <class T> T* as() { return static_cast<T*>(p); }
};

}  // namespace

#define MCK(call, what)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return mfail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, (what), e_); \
    } while (0)

extern "C" {

const char* lbm_mlp_last_error(void) { return g_mlp_err.c_str(); }

int lbm_mlp_forward(const float* X_dev, int n, const float* params, float* alpha_dev,
                    void* stream)
{
    if (!X_dev || !alpha_dev || !params || n < 1) return mfail(LBM_EINVAL, "bad arguments");
    if (!is_dev(X_dev) || !is_dev(alpha_dev)) return mfail(LBM_EINVAL, "X, alpha must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf P;
    MCK(P.alloc(NPARAM * 4), "allocate parameters");
    MCK(cudaMemcpyAsync(P.p, params, NPARAM * 4, cudaMemcpyDefault, s), "upload parameters");
    k_forward<<<(n + 255) / 256, 256, 0, s>>>(X_dev, n, P.as<float>(), alpha_dev);
    MCK(cudaGetLastError(), "forward kernel");
    MCK(cudaStreamSynchronize(s), "synchronise");
    return LBM_OK;
}

int lbm_mlp_grad(const float* X_dev, const float* t_dev, int n, const float* params, float* loss,
                 float* grad, void* stream)
{
    if (!X_dev || !t_dev || !params || !loss || !grad || n < 1)
        return mfail(LBM_EINVAL, "bad arguments");
    if (!is_dev(X_dev) || !is_dev(t_dev)) return mfail(LBM_EINVAL, "X, t must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nblk = (n + BS - 1) / BS;
    DevBuf P, G, part, pl, la;
    MCK(P.alloc(NPARAM * 4), "allocate");
    MCK(G.alloc(NPARAM * 4), "allocate");
    MCK(part.alloc((size_t)nblk * NTRAIN * 4), "allocate");
    MCK(pl.alloc((size_t)nblk * 4), "allocate");
    MCK(la.alloc(8), "allocate");
    MCK(cudaMemcpyAsync(P.p, params, NPARAM * 4, cudaMemcpyDefault, s), "upload parameters");
    MCK(cudaMemsetAsync(G.p, 0, NPARAM * 4, s), "clear");
    MCK(cudaMemsetAsync(la.p, 0, 8, s), "clear");
    k_fwd_bwd<<<nblk, BS, 0, s>>>(X_dev, t_dev, nullptr, n, P.as<float>(), part.as<float>(),
                                  pl.as<float>());
    k_reduce<<<(NTRAIN + 255) / 256, 256, 0, s>>>(part.as<float>(), pl.as<float>(), nblk, n,
                                                  G.as<float>(), la.as<float>());
    MCK(cudaGetLastError(), "gradient kernels");
    float lh[2];
    MCK(cudaMemcpyAsync(grad, G.p, NPARAM * 4, cudaMemcpyDefault, s), "copy gradient");
    MCK(cudaMemcpyAsync(lh, la.p, 8, cudaMemcpyDeviceToHost, s), "copy loss");
    MCK(cudaStreamSynchronize(s), "synchronise");
    *loss = lh[0];
    return LBM_OK;
}

int lbm_mlp_train(const float* X_dev, const double* alpha_dev, int n, const double* cfg,
                  float* params, float* loss_out, void* stream)
{
    if (!X_dev || !alpha_dev || !cfg || !params || n < 1) return mfail(LBM_EINVAL, "bad arguments");
    if (!is_dev(X_dev) || !is_dev(alpha_dev)) return mfail(LBM_EINVAL, "X, alpha must be device memory");
    const int epochs = (int)cfg[0];
    const int batch = (int)cfg[1];
    const float lr = (float)cfg[2];
    const uint64_t seed = (uint64_t)cfg[3];
    if (epochs < 1 || batch < 1 || !(lr > 0)) return mfail(LBM_EINVAL, "bad training config");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int B = batch < n ? batch : n;
    const int nblk = (B + BS - 1) / BS;
    DevBuf P, G, M, V, part, pl, la, T, I;
    MCK(P.alloc(NPARAM * 4), "allocate");
    MCK(G.alloc(NPARAM * 4), "allocate");
    MCK(M.alloc(NPARAM * 4), "allocate");
    MCK(V.alloc(NPARAM * 4), "allocate");
    MCK(part.alloc((size_t)nblk * NTRAIN * 4), "allocate");
    MCK(pl.alloc((size_t)nblk * 4), "allocate");
    MCK(la.alloc(8), "allocate");
    MCK(T.alloc((size_t)n * 4), "allocate");
    MCK(I.alloc((size_t)n * 4), "allocate");
    MCK(cudaMemcpyAsync(P.p, params, NPARAM * 4, cudaMemcpyHostToDevice, s), "upload parameters");
    MCK(cudaMemsetAsync(M.p, 0, NPARAM * 4, s), "clear");
    MCK(cudaMemsetAsync(V.p, 0, NPARAM * 4, s), "clear");
    MCK(cudaMemsetAsync(G.p, 0, NPARAM * 4, s), "clear");
    k_targets<<<(n + 255) / 256, 256, 0, s>>>(X_dev, alpha_dev, n, params[O_SCALE], T.as<float>());
    MCK(cudaGetLastError(), "target kernel");
    std::vector<int> perm(n);
    for (int k = 0; k < n; ++k) perm[k] = k;
    std::mt19937_64 rng(seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    long long step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int k = n - 1; k > 0; --k) {   // Fisher-Yates
            const int j = (int)(rng() % (uint64_t)(k + 1));
            std::swap(perm[k], perm[j]);
        }
        MCK(cudaMemcpyAsync(I.p, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s),
            "upload permutation");
        MCK(cudaMemsetAsync(la.p, 0, 8, s), "clear loss");
        for (int off = 0; off + B <= n; off += B) {
            ++step;
            k_fwd_bwd<<<nblk, BS, 0, s>>>(X_dev, T.as<float>(), I.as<int>() + off, B,
                                          P.as<float>(), part.as<float>(), pl.as<float>());
            k_reduce<<<(NTRAIN + 255) / 256, 256, 0, s>>>(part.as<float>(), pl.as<float>(), nblk,
                                                          B, G.as<float>(), la.as<float>());
            const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
            k_adam<<<(NTRAIN + 255) / 256, 256, 0, s>>>(P.as<float>(), G.as<float>(),
                                                        M.as<float>(), V.as<float>(), lr, b1, b2,
                                                        eps, c1, c2);
        }
        MCK(cudaGetLastError(), "training kernels");
        float lh[2];
        MCK(cudaMemcpyAsync(lh, la.p, 8, cudaMemcpyDeviceToHost, s), "copy loss");
        MCK(cudaStreamSynchronize(s), "synchronise");
        // copy out the host permutation buffer only after the stream is idle
        if (loss_out) loss_out[ep] = lh[1] > 0 ? lh[0] / lh[1] : 0.f;
    }
    MCK(cudaMemcpyAsync(params, P.p, NPARAM * 4, cudaMemcpyDeviceToHost, s), "copy parameters");
    MCK(cudaStreamSynchronize(s), "synchronise");
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Gradient without allocation.  Some callers cannot call cudaMalloc: for
// example a training loop embedded in an application whose own caching
// allocator already holds nearly all free device memory, or host code on a
// real-time path where an allocation (which can synchronise the device) is
// not allowed.  lbm_mlp_grad_static runs the same forward/backward and
// reduction kernels as lbm_mlp_grad, with all its scratch in the file-scope
// array below instead of cudaMalloc'd buffers.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxSamples = 4096;                     // per call
constexpr int kStaticBlocks = kStaticMaxSamples / BS;       // partial rows
constexpr int kPad = 1408;                                  // NPARAM rounded up
constexpr size_t kOffP = 0, kOffG = kPad, kOffPart = 2 * kPad,
                 kOffPl = kOffPart + (size_t)kStaticBlocks * NTRAIN,
                 kOffLa = kOffPl + kStaticBlocks, kStaticFloats = kOffLa + 8;

// 364 KB on every GPU that loads the library, held until the process exits.
static __device__ __align__(256) float g_mlp_scratch[kStaticFloats];

// Device address of g_mlp_scratch on the current device (the host-side name
// g_mlp_scratch is only a stand-in and must never be passed to a kernel).
// Looked up on every call: the lookup allocates nothing, and an address
// cached across calls would go stale when the device's context is torn
// down and re-created (cudaDeviceReset), which reloads the module.
float* static_scratch(int* err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = 1;
        return nullptr;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mlp_scratch);
    if (e != cudaSuccess) {
        *err = 2;
        g_mlp_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return nullptr;
    }
    return static_cast<float*>(p);
}

}  // namespace

extern "C" int lbm_mlp_grad_static(const float* X_dev, const float* t_dev, int n,
                                   const float* params, float* loss, float* grad, void* stream)
{
    if (!X_dev || !t_dev || !params || !loss || !grad || n < 1)
        return mfail(LBM_EINVAL, "bad arguments");
    if (n > kStaticMaxSamples)
        return mfail(LBM_EINVAL, "lbm_mlp_grad_static: n exceeds the 4096-sample maximum of "
                                 "its static scratch (split the batch)");
    if (!is_dev(X_dev) || !is_dev(t_dev)) return mfail(LBM_EINVAL, "X, t must be device memory");
    int err = 0;
    float* base = static_scratch(&err);
    if (!base) {
        if (err == 1) return mfail(LBM_ECUDA, "no current CUDA device");
        return LBM_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* P = base + kOffP;
    float* G = base + kOffG;
    float* part = base + kOffPart;
    float* pl = base + kOffPl;
    float* la = base + kOffLa;
    const int nblk = (n + BS - 1) / BS;
    // the gradient's untrained entries and the loss accumulator must start at
    // zero; every other slot is overwritten by this call
    MCK(cudaMemcpyAsync(P, params, NPARAM * 4, cudaMemcpyDefault, s), "upload parameters");
    MCK(cudaMemsetAsync(G, 0, NPARAM * 4, s), "clear gradient");
    MCK(cudaMemsetAsync(la, 0, 8, s), "clear loss");
    k_fwd_bwd<<<nblk, BS, 0, s>>>(X_dev, t_dev, nullptr, n, P, part, pl);
    k_reduce<<<(NTRAIN + 255) / 256, 256, 0, s>>>(part, pl, nblk, n, G, la);
    MCK(cudaGetLastError(), "gradient kernels");
    float lh[2];
    MCK(cudaMemcpyAsync(grad, G, NPARAM * 4, cudaMemcpyDefault, s), "copy gradient");
    MCK(cudaMemcpyAsync(lh, la, 8, cudaMemcpyDeviceToHost, s), "copy loss");
    MCK(cudaStreamSynchronize(s), "synchronise");
    *loss = lh[0];
    return LBM_OK;
}

}  // extern "C"
