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
#include <cuda_bf16.h>
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

// ---- tensor-core forward/backward ------------------------------------------
//
// The same per-CTA partial rows as k_fwd_bwd, computed with BF16 tensor-core
// MMA (mma.sync m16n8k16, FP32 accumulation).  The network is evaluated with
// its trained entries (16 .. 1392) rounded to BF16, the rounding the ELBM
// kernel applies on load (quantisation-aware training: the gradient is that
// of the loss of the BF16-rounded network, applied to the FP32 master copy).
// Those weights are exact BF16 operands; activations and back-propagated
// gradients are FP32 values carried as an unevaluated BF16 pair hi + lo
// (hi = bf16(x), lo = bf16(x - hi), 16 significant bits), so that a product
// of an activation and a weight is two MMAs and a product of two activation
// values three (hi hi, hi lo, lo hi).
//
// One warp takes a tile of 16 samples, a CTA of TC_WARPS warps the 64
// samples of one partial row.  Per tile (m = sample, row of every MMA):
//   A1 = Z W1^T + b1 (K = 8, padded to 16), H1 = tanh A1
//   A2 = H1 W2^T + b2 (K = 32),             H2 = tanh A2
//   out = H2 W3 + b3 (a row sum over the lanes of a quad), r = out - t
//   D2 = (2 r / B) W3 (1 - H2^2),   D1 = (D2 W2) (1 - H1^2)  (K = 32)
//   dW2 = D2^T H1, dW1 = D1^T Z (K = the 16 samples), the bias and W3
//   gradients as fixed-order sums over the tile.
// The accumulator layout of two adjacent 8-column tiles of an m16n8 product
// is the A-operand layout of an m16k16 product, so H1 and D2 feed the next
// MMA from registers; the weight-gradient MMAs, whose reduction runs over the
// samples, read the transposed operands from a per-warp staging area in
// shared memory.  Warps combine their partial sums in a fixed order.
constexpr int TC_WARPS = 4;                                // 16 samples each
static_assert(TC_WARPS * 16 == BS, "one partial row per CTA, as k_fwd_bwd");

__device__ __forceinline__ unsigned bf16x2_bits(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// (a, b) -> hi pair and lo pair; a in the low half
__device__ __forceinline__ void split_bf16(float a, float b, unsigned& hi, unsigned& lo)
{
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    hi = bf16x2_bits(ah, bh);
    lo = bf16x2_bits(__float2bfloat16_rn(a - __bfloat162float(ah)),
                     __float2bfloat16_rn(b - __bfloat162float(bh)));
}

// d += A (16 x 16, row) * B (16 x 8, col), BF16 operands, FP32 accumulator
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A operand (hi and lo pairs) of an m16k16 product from the accumulators of
// two adjacent 8-column tiles c0 (columns 0..7) and c1 (8..15)
__device__ __forceinline__ void frag_from_acc(const float (&c0)[4], const float (&c1)[4],
                                              unsigned (&hi)[4], unsigned (&lo)[4])
{
    split_bf16(c0[0], c0[1], hi[0], lo[0]);
    split_bf16(c0[2], c0[3], hi[1], lo[1]);
    split_bf16(c1[0], c1[1], hi[2], lo[2]);
    split_bf16(c1[2], c1[3], hi[3], lo[3]);
}

__global__ void __launch_bounds__(TC_WARPS * 32) k_fwd_bwd_tc(const float* __restrict__ X,
                                                              const float* __restrict__ t,
                                                              const int* __restrict__ idx,
                                                              int B, const float* __restrict__ P,
                                                              float* __restrict__ part,
                                                              float* __restrict__ part_loss)
{
    // the network with its trained entries rounded to BF16 (FP32 values)
    __shared__ float sp[NPARAM];
    // weight operands as BF16 pairs: W1 [o][k] (k padded to 16), W2 [o][k],
    // W2 transposed [k][o]
    __shared__ __align__(16) unsigned sW1[NH][8], sW2[NH][NH / 2], sW2T[NH][NH / 2];
    // per-warp staging of one tile: Z, H1, D1, D2 (FP32, [sample][column])
    __shared__ float sZ[TC_WARPS][16][NIN], sH1[TC_WARPS][16][NH], sD1[TC_WARPS][16][NH],
        sD2[TC_WARPS][16][NH];
    __shared__ float sRow[NTRAIN + 1];   // the CTA's partial row and loss
    const int tid = threadIdx.x;
    for (int k = tid; k < NPARAM; k += blockDim.x) {
        const float v = P[k];
        sp[k] = (k >= O_W1 && k < O_SCALE) ? __bfloat162float(__float2bfloat16_rn(v)) : v;
    }
    __syncthreads();
    for (int e = tid; e < NH * 8; e += blockDim.x) {
        const int o = e / 8, k2 = 2 * (e % 8);
        sW1[o][e % 8] = k2 < NIN ? bf16x2_bits(__float2bfloat16_rn(sp[O_W1 + o * NIN + k2]),
                                               __float2bfloat16_rn(sp[O_W1 + o * NIN + k2 + 1]))
                                 : 0u;
    }
    for (int e = tid; e < NH * NH / 2; e += blockDim.x) {
        const int r = e / (NH / 2), c2 = 2 * (e % (NH / 2));
        sW2[r][e % (NH / 2)] = bf16x2_bits(__float2bfloat16_rn(sp[O_W2 + r * NH + c2]),
                                           __float2bfloat16_rn(sp[O_W2 + r * NH + c2 + 1]));
        sW2T[r][e % (NH / 2)] = bf16x2_bits(__float2bfloat16_rn(sp[O_W2 + c2 * NH + r]),
                                            __float2bfloat16_rn(sp[O_W2 + (c2 + 1) * NH + r]));
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, q = lane & 3;   // fragment row group and column pair
    const int r0 = g, r1 = g + 8;            // this lane's two sample rows of the tile
    const int tb = blockIdx.x * BS + warp * 16;
    const bool v0 = tb + r0 < B, v1 = tb + r1 < B;
    const int s0 = v0 ? (idx ? idx[tb + r0] : tb + r0) : 0;
    const int s1 = v1 ? (idx ? idx[tb + r1] : tb + r1) : 0;
    // ---- Z: features 2q, 2q + 1 of rows r0, r1 (zero for absent samples)
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (v0) {
        const float2 x = *reinterpret_cast<const float2*>(X + (size_t)s0 * NIN + 2 * q);
        z[0] = (x.x - sp[2 * q]) * sp[8 + 2 * q];
        z[1] = (x.y - sp[2 * q + 1]) * sp[8 + 2 * q + 1];
    }
    if (v1) {
        const float2 x = *reinterpret_cast<const float2*>(X + (size_t)s1 * NIN + 2 * q);
        z[2] = (x.x - sp[2 * q]) * sp[8 + 2 * q];
        z[3] = (x.y - sp[2 * q + 1]) * sp[8 + 2 * q + 1];
    }
    sZ[warp][r0][2 * q] = z[0];
    sZ[warp][r0][2 * q + 1] = z[1];
    sZ[warp][r1][2 * q] = z[2];
    sZ[warp][r1][2 * q + 1] = z[3];
    // ---- layer 1: columns 8 j + 2 q + (0, 1) of rows r0 (c[0..1]), r1 (c[2..3])
    float h1[4][4];
    {
        unsigned ah[4], al[4];
        split_bf16(z[0], z[1], ah[0], al[0]);
        split_bf16(z[2], z[3], ah[1], al[1]);
        ah[2] = ah[3] = al[2] = al[3] = 0u;   // k = 8 .. 15: padding
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 8 * j + 2 * q;
            float acc[4] = {sp[O_B1 + c], sp[O_B1 + c + 1], sp[O_B1 + c], sp[O_B1 + c + 1]};
            const unsigned b0 = sW1[8 * j + g][q];
            mma_bf16(acc, ah, b0, 0u);
            mma_bf16(acc, al, b0, 0u);
#pragma unroll
            for (int e = 0; e < 4; ++e) h1[j][e] = tanhf(acc[e]);
        }
    }
    // ---- layer 2
    float h2[4][4];
    {
        unsigned ah[2][4], al[2][4];
        frag_from_acc(h1[0], h1[1], ah[0], al[0]);
        frag_from_acc(h1[2], h1[3], ah[1], al[1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 8 * j + 2 * q;
            float acc[4] = {sp[O_B2 + c], sp[O_B2 + c + 1], sp[O_B2 + c], sp[O_B2 + c + 1]};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const unsigned b0 = sW2[8 * j + g][8 * ks + q], b1 = sW2[8 * j + g][8 * ks + 4 + q];
                mma_bf16(acc, ah[ks], b0, b1);
                mma_bf16(acc, al[ks], b0, b1);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) h2[j][e] = tanhf(acc[e]);
        }
    }
    // ---- output and residual of rows r0, r1 (sums over the quad's lanes)
    float o0 = 0.f, o1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = 8 * j + 2 * q;
        o0 = fmaf(sp[O_W3 + c], h2[j][0], o0);
        o0 = fmaf(sp[O_W3 + c + 1], h2[j][1], o0);
        o1 = fmaf(sp[O_W3 + c], h2[j][2], o1);
        o1 = fmaf(sp[O_W3 + c + 1], h2[j][3], o1);
    }
    o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
    o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
    o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
    o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
    const float res0 = v0 ? o0 + sp[O_B3] - t[s0] : 0.f;
    const float res1 = v1 ? o1 + sp[O_B3] - t[s1] : 0.f;
    const float dout0 = 2.0f * res0 / (float)B, dout1 = 2.0f * res1 / (float)B;
    // ---- D2 and the per-lane sums for b2, W3 (columns 8 j + 2 q + e)
    float d2[4][4], gb2[8], gw3[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = 8 * j + 2 * q;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float w = sp[O_W3 + c + e];
            d2[j][e] = dout0 * w * (1.0f - h2[j][e] * h2[j][e]);
            d2[j][2 + e] = dout1 * w * (1.0f - h2[j][2 + e] * h2[j][2 + e]);
            gb2[2 * j + e] = d2[j][e] + d2[j][2 + e];
            gw3[2 * j + e] = fmaf(dout1, h2[j][2 + e], dout0 * h2[j][e]);
            sD2[warp][r0][c + e] = d2[j][e];
            sD2[warp][r1][c + e] = d2[j][2 + e];
            sH1[warp][r0][c + e] = h1[j][e];
            sH1[warp][r1][c + e] = h1[j][2 + e];
        }
    }
    // ---- D1 = (D2 W2) (1 - H1^2), and the per-lane sums for b1
    float gb1[8];
    {
        unsigned ah[2][4], al[2][4];
        frag_from_acc(d2[0], d2[1], ah[0], al[0]);
        frag_from_acc(d2[2], d2[3], ah[1], al[1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 8 * j + 2 * q;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const unsigned b0 = sW2T[8 * j + g][8 * ks + q],
                               b1 = sW2T[8 * j + g][8 * ks + 4 + q];
                mma_bf16(acc, ah[ks], b0, b1);
                mma_bf16(acc, al[ks], b0, b1);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float a = acc[e] * (1.0f - h1[j][e] * h1[j][e]);
                const float b = acc[2 + e] * (1.0f - h1[j][2 + e] * h1[j][2 + e]);
                gb1[2 * j + e] = a + b;
                sD1[warp][r0][c + e] = a;
                sD1[warp][r1][c + e] = b;
            }
        }
    }
    __syncwarp();
    // ---- weight gradients, K = the tile's 16 samples.  A (rows o, columns
    // samples) from the staged D, B (rows samples, columns k) from the staged
    // activations; the operand pairs run along the samples.
    auto frag_T = [&](const float (*D)[NH], int o, unsigned& hi, unsigned& lo, int sm) {
        split_bf16(D[sm][o], D[sm + 1][o], hi, lo);
    };
    float gW2[2][4][4], gW1[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        unsigned ah[4], al[4];
        const int o = 16 * mt + g;
        frag_T(sD2[warp], o, ah[0], al[0], 2 * q);
        frag_T(sD2[warp], o + 8, ah[1], al[1], 2 * q);
        frag_T(sD2[warp], o, ah[2], al[2], 2 * q + 8);
        frag_T(sD2[warp], o + 8, ah[3], al[3], 2 * q + 8);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            unsigned bh0, bl0, bh1, bl1;
            frag_T(sH1[warp], 8 * j + g, bh0, bl0, 2 * q);
            frag_T(sH1[warp], 8 * j + g, bh1, bl1, 2 * q + 8);
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16(acc, ah, bh0, bh1);
            mma_bf16(acc, ah, bl0, bl1);
            mma_bf16(acc, al, bh0, bh1);
#pragma unroll
            for (int e = 0; e < 4; ++e) gW2[mt][j][e] = acc[e];
        }
        frag_T(sD1[warp], o, ah[0], al[0], 2 * q);
        frag_T(sD1[warp], o + 8, ah[1], al[1], 2 * q);
        frag_T(sD1[warp], o, ah[2], al[2], 2 * q + 8);
        frag_T(sD1[warp], o + 8, ah[3], al[3], 2 * q + 8);
        unsigned zh0, zl0, zh1, zl1;
        split_bf16(sZ[warp][2 * q][g], sZ[warp][2 * q + 1][g], zh0, zl0);
        split_bf16(sZ[warp][2 * q + 8][g], sZ[warp][2 * q + 9][g], zh1, zl1);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(acc, ah, zh0, zh1);
        mma_bf16(acc, ah, zl0, zl1);
        mma_bf16(acc, al, zh0, zh1);
#pragma unroll
        for (int e = 0; e < 4; ++e) gW1[mt][e] = acc[e];
    }
    // ---- column sums over the 8 row groups (b1, b2, W3), fixed order
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int m = 4; m < 32; m <<= 1) {
            gb1[k] += __shfl_xor_sync(0xffffffffu, gb1[k], m);
            gb2[k] += __shfl_xor_sync(0xffffffffu, gb2[k], m);
            gw3[k] += __shfl_xor_sync(0xffffffffu, gw3[k], m);
        }
    }
    // b3 and the loss: rows r0, r1 summed over the groups (the quad's lanes
    // hold the same values; lane q = 0 of each group contributes)
    float gb3 = q == 0 ? dout0 + dout1 : 0.f;
    float ls = q == 0 ? res0 * res0 + res1 * res1 : 0.f;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        gb3 += __shfl_xor_sync(0xffffffffu, gb3, m);
        ls += __shfl_xor_sync(0xffffffffu, ls, m);
    }
    // ---- the CTA's row: warps add their sums in order 0, 1, ...
    for (int w = 0; w < TC_WARPS; ++w) {
        if (warp == w) {
            auto put = [&](int q_abs, float v) {
                float* dst = &sRow[q_abs - TRAIN_LO];
                *dst = (w == 0) ? v : *dst + v;
            };
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int o = 16 * mt + g + (e >= 2 ? 8 : 0);
                    const int kk = 2 * q + (e & 1);
                    put(O_W1 + o * NIN + kk, gW1[mt][e]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) put(O_W2 + o * NH + 8 * j + kk, gW2[mt][j][e]);
                }
            }
            if (g == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int c = 8 * j + 2 * q + e;
                        put(O_B1 + c, gb1[2 * j + e]);
                        put(O_B2 + c, gb2[2 * j + e]);
                        put(O_W3 + c, gw3[2 * j + e]);
                    }
                }
            }
            if (lane == 0) {
                put(O_B3, gb3);
                sRow[NTRAIN] = (w == 0) ? ls : sRow[NTRAIN] + ls;
            }
        }
        __syncthreads();
    }
    float* row = part + (size_t)blockIdx.x * NTRAIN;
    for (int e = tid; e < NTRAIN; e += blockDim.x) row[e] = sRow[e];
    if (tid == 0) part_loss[blockIdx.x] = sRow[NTRAIN];
}

// Sum of the partial rows, in a fixed order: a CTA of RED_GROUPS x 32
// threads takes 32 consecutive entries; group k of a column sums rows k,
// k + RED_GROUPS, ... (the 32 columns of one row are one coalesced read),
// then the column's group sums are added in group order.  CTA 0 also sums
// the partial losses (row order).
constexpr int RED_GROUPS = 8;
constexpr int RED_THREADS = 32 * RED_GROUPS;
constexpr int RED_BLOCKS = (NTRAIN + 31) / 32;

__global__ void __launch_bounds__(RED_THREADS) k_reduce(const float* __restrict__ part,
                                                        const float* __restrict__ part_loss,
                                                        int nblk, int B, float* __restrict__ grad,
                                                        float* __restrict__ loss_acc)
{
    __shared__ float sg[RED_GROUPS][32];
    const int col = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + col;
    float s = 0.f;
    if (e < NTRAIN)
        for (int k = grp; k < nblk; k += RED_GROUPS) s += part[(size_t)k * NTRAIN + e];
    sg[grp][col] = s;
    __syncthreads();
    if (grp == 0 && e < NTRAIN) {
        float t = sg[0][col];
        for (int k = 1; k < RED_GROUPS; ++k) t += sg[k][col];
        grad[TRAIN_LO + e] = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float l = 0.f;
        for (int k = 0; k < nblk; ++k) l += part_loss[k];
        loss_acc[0] += l / (float)B;
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

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    cudaError_t create()
    {
        const cudaError_t e = cudaEventCreate(&a);
        return e != cudaSuccess ? e : cudaEventCreate(&b);
    }
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

static int mlp_grad_impl(const float* X_dev, const float* t_dev, int n, const float* params,
                         float* loss, float* grad, bool tc, void* stream)
{
    if (!X_dev || !t_dev || !params || !loss || !grad || n < 1)
        return mfail(LBM_EINVAL, "bad arguments");
    if (!is_dev(X_dev) || !is_dev(t_dev)) return mfail(LBM_EINVAL, "X, t must be device memory");
    if (tc && (reinterpret_cast<uintptr_t>(X_dev) & 7u))
        return mfail(LBM_EINVAL, "X must be 8-byte aligned for the tensor-core kernel");
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
    if (tc)
        k_fwd_bwd_tc<<<nblk, TC_WARPS * 32, 0, s>>>(X_dev, t_dev, nullptr, n, P.as<float>(),
                                                     part.as<float>(), pl.as<float>());
    else
        k_fwd_bwd<<<nblk, BS, 0, s>>>(X_dev, t_dev, nullptr, n, P.as<float>(), part.as<float>(),
                                      pl.as<float>());
    k_reduce<<<RED_BLOCKS, RED_THREADS, 0, s>>>(part.as<float>(), pl.as<float>(), nblk, n,
                                                  G.as<float>(), la.as<float>());
    MCK(cudaGetLastError(), "gradient kernels");
    float lh[2];
    MCK(cudaMemcpyAsync(grad, G.p, NPARAM * 4, cudaMemcpyDefault, s), "copy gradient");
    MCK(cudaMemcpyAsync(lh, la.p, 8, cudaMemcpyDeviceToHost, s), "copy loss");
    MCK(cudaStreamSynchronize(s), "synchronise");
    *loss = lh[0];
    return LBM_OK;
}

int lbm_mlp_grad(const float* X_dev, const float* t_dev, int n, const float* params, float* loss,
                 float* grad, void* stream)
{
    return mlp_grad_impl(X_dev, t_dev, n, params, loss, grad, false, stream);
}

int lbm_mlp_grad_tc(const float* X_dev, const float* t_dev, int n, const float* params,
                    float* loss, float* grad, void* stream)
{
    return mlp_grad_impl(X_dev, t_dev, n, params, loss, grad, true, stream);
}

int lbm_mlp_train_cfg(const float* X_dev, const double* alpha_dev, int n, const lbm_mlp_cfg* cfg,
                      float* params, float* loss_out, lbm_train_stats* stats, void* stream)
{
    if (!X_dev || !alpha_dev || !cfg || !params || n < 1) return mfail(LBM_EINVAL, "bad arguments");
    if (!is_dev(X_dev) || !is_dev(alpha_dev)) return mfail(LBM_EINVAL, "X, alpha must be device memory");
    const int epochs = cfg->epochs;
    const int batch = cfg->batch;
    const float lr = (float)cfg->lr;
    if (epochs < 1 || batch < 1 || !(lr > 0)) return mfail(LBM_EINVAL, "bad training config");
    if (cfg->kernel != LBM_MLP_FP32 && cfg->kernel != LBM_MLP_BF16_TC)
        return mfail(LBM_EINVAL, "kernel is LBM_MLP_FP32 or LBM_MLP_BF16_TC");
    if (cfg->reserved != 0) return mfail(LBM_EINVAL, "lbm_mlp_cfg.reserved must be 0");
    const bool tc = cfg->kernel == LBM_MLP_BF16_TC;
    // the tensor-core kernel reads each sample's feature pairs as 8-byte loads
    if (tc && (reinterpret_cast<uintptr_t>(X_dev) & 7u))
        return mfail(LBM_EINVAL, "X must be 8-byte aligned for the tensor-core kernel");
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
    EventPair ev;
    MCK(ev.create(), "create events");
    MCK(cudaMemcpyAsync(P.p, params, NPARAM * 4, cudaMemcpyHostToDevice, s), "upload parameters");
    MCK(cudaMemsetAsync(M.p, 0, NPARAM * 4, s), "clear");
    MCK(cudaMemsetAsync(V.p, 0, NPARAM * 4, s), "clear");
    MCK(cudaMemsetAsync(G.p, 0, NPARAM * 4, s), "clear");
    k_targets<<<(n + 255) / 256, 256, 0, s>>>(X_dev, alpha_dev, n, params[O_SCALE], T.as<float>());
    MCK(cudaGetLastError(), "target kernel");
    std::vector<int> perm(n);
    for (int k = 0; k < n; ++k) perm[k] = k;
    std::mt19937_64 rng(cfg->seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    long long step = 0;
    double gpu_ms = 0.0;
    float last = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int k = n - 1; k > 0; --k) {   // Fisher-Yates
            const int j = (int)(rng() % (uint64_t)(k + 1));
            std::swap(perm[k], perm[j]);
        }
        MCK(cudaMemcpyAsync(I.p, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s),
            "upload permutation");
        MCK(cudaMemsetAsync(la.p, 0, 8, s), "clear loss");
        // the epoch's training launches, timed on the stream
        MCK(cudaEventRecord(ev.a, s), "record event");
        for (int off = 0; off + B <= n; off += B) {
            ++step;
            if (tc)
                k_fwd_bwd_tc<<<nblk, TC_WARPS * 32, 0, s>>>(X_dev, T.as<float>(),
                                                             I.as<int>() + off, B, P.as<float>(),
                                                             part.as<float>(), pl.as<float>());
            else
                k_fwd_bwd<<<nblk, BS, 0, s>>>(X_dev, T.as<float>(), I.as<int>() + off, B,
                                              P.as<float>(), part.as<float>(), pl.as<float>());
            k_reduce<<<RED_BLOCKS, RED_THREADS, 0, s>>>(part.as<float>(), pl.as<float>(), nblk,
                                                          B, G.as<float>(), la.as<float>());
            const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
            k_adam<<<(NTRAIN + 255) / 256, 256, 0, s>>>(P.as<float>(), G.as<float>(),
                                                        M.as<float>(), V.as<float>(), lr, b1, b2,
                                                        eps, c1, c2);
        }
        MCK(cudaGetLastError(), "training kernels");
        MCK(cudaEventRecord(ev.b, s), "record event");
        float lh[2];
        MCK(cudaMemcpyAsync(lh, la.p, 8, cudaMemcpyDeviceToHost, s), "copy loss");
        MCK(cudaStreamSynchronize(s), "synchronise");
        // the host permutation buffer is reused only after the stream is idle
        float ms = 0.f;
        MCK(cudaEventElapsedTime(&ms, ev.a, ev.b), "event time");
        gpu_ms += ms;
        last = lh[1] > 0 ? lh[0] / lh[1] : 0.f;
        if (loss_out) loss_out[ep] = last;
    }
    MCK(cudaMemcpyAsync(params, P.p, NPARAM * 4, cudaMemcpyDeviceToHost, s), "copy parameters");
    MCK(cudaStreamSynchronize(s), "synchronise");
    if (stats) {
        stats->steps = (int)step;
        stats->reserved = 0;
        stats->gpu_ms = gpu_ms;
        stats->samples_per_s = gpu_ms > 0 ? (double)step * B / (gpu_ms * 1e-3) : 0.0;
        stats->final_loss = last;
    }
    return LBM_OK;
}

int lbm_mlp_train(const float* X_dev, const double* alpha_dev, int n, const double* cfg,
                  float* params, float* loss_out, void* stream)
{
    if (!cfg) return mfail(LBM_EINVAL, "bad arguments");
    lbm_mlp_cfg c{};
    c.epochs = (int)cfg[0];
    c.batch = (int)cfg[1];
    c.lr = cfg[2];
    c.seed = (unsigned long long)cfg[3];
    c.kernel = LBM_MLP_FP32;
    return lbm_mlp_train_cfg(X_dev, alpha_dev, n, &c, params, loss_out, nullptr, stream);
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
    k_reduce<<<RED_BLOCKS, RED_THREADS, 0, s>>>(part, pl, nblk, n, G, la);
    MCK(cudaGetLastError(), "gradient kernels");
    float lh[2];
    MCK(cudaMemcpyAsync(grad, G, NPARAM * 4, cudaMemcpyDefault, s), "copy gradient");
    MCK(cudaMemcpyAsync(lh, la, 8, cudaMemcpyDeviceToHost, s), "copy loss");
    MCK(cudaStreamSynchronize(s), "synchronise");
    *loss = lh[0];
    return LBM_OK;
}

}  // extern "C"
