// Device-side building blocks of the stream-and-collide kernels: lattice
// tables, storage codecs and the per-node collision operators.
//
// Every operator works on deviations d_i = f_i - w_i held in registers (the
// round-off-minimising formulation the paper studies in Sec. 3.7): mass is
// rho = 1 + sum d_i and momentum j = sum e_i d_i since sum w_i = 1 and
// sum w_i e_i = 0.  Storage types that keep f_i itself convert on load/store.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices (Sec. 2, Fig. lattices, Table bgkweights).  Own ordering: rest
// first, then opposite pairs (2k-1, 2k), so opp(i) = i + 1 for odd i and
// i - 1 for even i > 0.
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int D = 2, Q = 9;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

struct D3Q19 {
    static constexpr int D = 3, Q = 19;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

// ---------------------------------------------------------------------------
// Storage codecs.  load() returns the deviation d = f - w in the compute type
// R; store() takes it back.  *_S codecs keep d itself (Sec. 3.7 round-off
// minimisation; FP16/BF16 extend it to half-width storage).
// ---------------------------------------------------------------------------
// Half-width stores default to dithered rounding: round-to-nearest of a value
// that is nearly the same at a lattice location from one step to the next
// commits nearly the same rounding error every step, a bias that grows
// linearly in time (3.2e-3 relative velocity error after 1000 steps of the
// 256^3 vortex).  Adding to the bits that the narrowing drops an offset drawn
// from a multiplicative hash of the value's own 32 bits (salted with node and
// direction) and then truncating rounds up with probability equal to the
// dropped fraction, like stochastic rounding: the errors lose their bias
// (6e-4 on the same vortex).  The offset needs no counter, so CUDA-graph
// replay and the batched kernel see identical results.  FP16 values below its
// normal range (|d| < 2^-14) are dithered on the fixed subnormal grid 2^-24
// instead (a stochastic floor of |d| 2^24); a flow started from rest keeps
// most deviations there for many steps, and truncating them would bias every
// store toward zero.  Inf and NaN are narrowed unchanged.
__device__ __forceinline__ unsigned dither_hash(unsigned bits, unsigned salt)
{
    return bits * 0x9E3779B1u + salt;
}
constexpr unsigned kSaltNode = 0x85EBCA77u, kSaltDir = 0xC2B2AE3Du;

struct StoreF64 {
    using T = double;
    using R = double;
    static constexpr bool kHalf = false;
    __device__ static R load(const T* p, double w) { return __ldg(p) - w; }
    __device__ static void store(T* p, R d, double w) { *p = d + w; }
    __device__ static T encode(R d, double w) { return d + w; }
    __device__ static T encode_dither(R d, unsigned) { return d; }
};
struct StoreF32 {
    using T = float;
    using R = float;
    static constexpr bool kHalf = false;
    __device__ static R load(const T* p, double w) { return __ldg(p) - (float)w; }
    __device__ static void store(T* p, R d, double w) { *p = d + (float)w; }
    __device__ static T encode(R d, double w) { return d + (float)w; }
    __device__ static T encode_dither(R d, unsigned) { return d; }
};
struct StoreF32S {
    using T = float;
    using R = float;
    static constexpr bool kHalf = false;
    __device__ static R load(const T* p, double) { return __ldg(p); }
    __device__ static void store(T* p, R d, double) { *p = d; }
    __device__ static T encode(R d, double) { return d; }
    __device__ static T encode_dither(R d, unsigned) { return d; }
};
struct StoreF16S {
    using T = __half;
    using R = float;
    static constexpr bool kHalf = true;
    __device__ static R load(const T* p, double) { return __half2float(__ldg(p)); }
    __device__ static void store(T* p, R d, double) { *p = __float2half_rn(d); }
    __device__ static T encode(R d, double) { return __float2half_rn(d); }
    __device__ static T encode_dither(R d, unsigned salt)
    {
        const unsigned b = __float_as_uint(d), a = b & 0x7fffffffu;
        const unsigned h = dither_hash(b, salt);
        if (a >= 0x7f800000u) return __float2half_rn(d);                  // Inf, NaN
        if (a >= 0x38800000u)                                              // normal range
            return __float2half_rz(__uint_as_float((b + (h >> 19)) & ~0x1fffu));  // 13 bits
        // subnormal: k = floor(|d| 2^24 + r), r uniform in [0, 1); k <= 1024
        // is the half's magnitude bit pattern (1024 = 2^-14, the smallest normal)
        const float r = __uint_as_float(0x3f800000u | (h >> 9)) - 1.0f;
        const unsigned k = __float2uint_rz(fmaf(__uint_as_float(a), 16777216.0f, r));
        return __ushort_as_half((unsigned short)(k | ((b >> 16) & 0x8000u)));
    }
};
struct StoreBF16S {
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool kHalf = true;
    __device__ static R load(const T* p, double) { return __bfloat162float(__ldg(p)); }
    __device__ static void store(T* p, R d, double) { *p = __float2bfloat16_rn(d); }
    __device__ static T encode(R d, double) { return __float2bfloat16_rn(d); }
    __device__ static T encode_dither(R d, unsigned salt)
    {
        const unsigned b = __float_as_uint(d);
        if ((b & 0x7fffffffu) >= 0x7f800000u) return __float2bfloat16_rn(d);   // Inf, NaN
        return __float2bfloat16_rz(
            __uint_as_float((b + (dither_hash(b, salt) >> 16)) & 0xffff0000u));  // 16 bits, exact
    }
};

// ---------------------------------------------------------------------------
// Kernel parameters (passed by value).
// ---------------------------------------------------------------------------
enum { MODEL_BGK = 0, MODEL_MRT = 1, MODEL_ELBM = 2, MODEL_REG = 3, MODEL_SMAG = 4 };
enum { FLAG_SOLID = 1, FLAG_NEAR_WALL = 2 };
enum { STATUS_NAN = 1u, STATUS_NOCONV = 2u, STATUS_TIMEOUT = 4u };
// ELBM per-node outcome, shared meaning with the counters of the ABI
enum { ALPHA_CONV = 0, ALPHA_SKIP = 1, ALPHA_CLAMP = 2, ALPHA_NOCONV = 3, ALPHA_GUARDED = 5 };
enum { MLP_NPARAM = 1394 };

struct StepParams {
    const void* A;             // post-collision distributions at t (read)
    void* B;                   // post-collision distributions at t+1 (written)
    const uint8_t* flags;      // node-type map (FLAG_*) or nullptr
    void* rho;                 // output fields (compute type), padded layout
    void* u;                   // [D][sq]
    double* alpha_out;         // ELBM per-node alpha or nullptr
    unsigned int* status;      // STATUS_* bits
    unsigned long long* elbm_ctr;  // 6 counters or nullptr
    float* pairs_X;            // ELBM training-pair capture (nullptr = off)
    double* pairs_y;
    int* pairs_count;
    int pairs_cap, pairs_stride;
    int nx, ny, nz, nxp;       // logical sizes, padded row length
    long long sq;              // elements between direction planes
    int out;                   // write rho/u (and alpha) this step
    int has_force;
    int round_nearest;         // half-width stores: 1 round to nearest, 0 dither
    int aa_pushpull;           // AA pattern: 1 = pull/push step (even t), 0 = in-place step
    double omega;              // 1/tau
    double F[3];               // body force
    double mrt_c[19];          // s_k / |M_k|^2
    double mrt_cf[19];         // (1 - s_k/2) / |M_k|^2
    // the same, rounded once on the host for the FP32 kernels (a per-node
    // double -> float conversion runs on the GPU's FP64 pipe)
    float omega_f;
    float F_f[3];
    double tau, smag_cs2;      // tau0 and C_S^2 (Smagorinsky)
    float tau_f, smag_cs2_f;
    float mrt_c_f[19];
    float mrt_cf_f[19];
    // ELBM
    int alpha_mode, max_iter, guard_steps, feq_variant;
    double tol, skip_eps, guard_tol;
    const float* mlp;          // MLP_NPARAM floats (BF16-rounded weights)
};

// Parameter in the compute type: the FP32 copy for float, FP64 for double.
template <class R>
__host__ __device__ __forceinline__ R sel(float f, double d);
template <>
__host__ __device__ __forceinline__ float sel<float>(float f, double) { return f; }
template <>
__host__ __device__ __forceinline__ double sel<double>(float, double d) { return d; }

}  // namespace lbm
