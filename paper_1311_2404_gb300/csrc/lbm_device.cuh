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

// D3Q15: rest, three axis pairs, four body-diagonal pairs.
struct D3Q15 {
    static constexpr int D = 3, Q = 15;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int i) {
        constexpr int t[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

// D3Q27: the D3Q19 set (same order) followed by four body-diagonal pairs.
struct D3Q27 {
    static constexpr int D = 3, Q = 27;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0,
                               1, -1, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1,
                               1, -1, 1, -1, -1, 1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int i) {
        constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1,
                               1, -1, -1, 1, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

// Compile-time checks of a velocity set: rest first, opposite pairs
// (2k+1, 2k+2), zero mean velocity, links of each length counted.
template <class L>
__host__ __device__ constexpr bool lattice_ok(int n1, int n2, int n3)
{
    if (L::ex(0) || L::ey(0) || L::ez(0)) return false;
    int c[4] = {1, 0, 0, 0}, sx = 0, sy = 0, sz = 0;
    for (int i = 1; i < L::Q; ++i) {
        const int o = L::opp(i);
        if (L::ex(o) != -L::ex(i) || L::ey(o) != -L::ey(i) || L::ez(o) != -L::ez(i)) return false;
        c[L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i)] += 1;
        sx += L::ex(i); sy += L::ey(i); sz += L::ez(i);
        for (int k = 1; k < i; ++k)
            if (L::ex(k) == L::ex(i) && L::ey(k) == L::ey(i) && L::ez(k) == L::ez(i)) return false;
    }
    return sx == 0 && sy == 0 && sz == 0 && c[1] == n1 && c[2] == n2 && c[3] == n3;
}
static_assert(lattice_ok<D2Q9>(4, 4, 0), "D2Q9 table");
static_assert(lattice_ok<D3Q15>(6, 0, 8), "D3Q15 table");
static_assert(lattice_ok<D3Q19>(6, 12, 0), "D3Q19 table");
static_assert(lattice_ok<D3Q27>(6, 12, 8), "D3Q27 table");

// ---------------------------------------------------------------------------
// Storage codecs.  load() returns the deviation d = f - w in the compute type
// R; store() takes it back.  *_S codecs keep d itself (Sec. 3.7 round-off
// minimisation; FP16/BF16 extend it to half-width storage).
// ---------------------------------------------------------------------------
// Half-width stores default to stochastic rounding: round-to-nearest of a
// value that is nearly the same at a lattice location from one step to the
// next commits nearly the same rounding error every step, a bias that grows
// linearly in time (3.2e-3 relative velocity error after 1000 steps of the
// 256^3 vortex).  The narrowing uses the conversion with stochastic rounding
// (cvt.rs, sm_100 family): it rounds up with probability equal to the
// fraction the narrowing drops, subnormals and values below the smallest
// subnormal included, and passes Inf and NaN through.  Its random bits come
// from a multiplicative hash of each value's own 32 bits with an odd
// multiplier per direction, salted with the node index and the time step:
//   hash = bits * M_dir + n * kSaltNode + t * kSaltStep   (mod 2^32).
// The step term matters at a steady state, where the same value recurs at a
// node step after step: a hash of the value and the node alone would repeat
// the same rounding every step (a fixed point of the rounded map, short of
// the true steady state), while t * kSaltStep walks the hash's top bits
// through a Weyl sequence, so the rounding errors average out over steps.
// t is read on the device (step_salt below), so CUDA-graph replay, the
// batched kernel and subdomain runs reproduce results exactly.  With the
// direction a compile-time constant the hash is one integer multiply-add per
// value.  Two values share one conversion; each element takes 13 (FP16) or
// 16 (BF16) high bits of its own hash (the instruction reads bits 16.. of
// the word for the first element, bits 0.. for the second).
__host__ __device__ constexpr unsigned dither_mul(int dir)
{
    return 0x9E3779B1u + (unsigned)dir * 0x3C6EF372u;   // odd for every dir
}
__device__ __forceinline__ unsigned dither_hash(unsigned bits, unsigned salt, int dir)
{
    return bits * dither_mul(dir) + salt;
}
constexpr unsigned kSaltNode = 0x85EBCA77u;
constexpr unsigned kSaltStep = 0x9E3779B9u;   // 2^32 (sqrt(5) - 1) / 2, odd

// random word for a pair: high 16 bits of a's hash in the high half, of b's
// hash in the low half, shifted right by `sh` so that a field of 16 - sh bits
// starts at each half's bit 0 with the hash's top bits
template <int sh>
__device__ __forceinline__ unsigned pair_rbits(float a, float b, unsigned sa, unsigned sb, int da,
                                               int db)
{
    const unsigned ha = dither_hash(__float_as_uint(a), sa, da);
    const unsigned hb = dither_hash(__float_as_uint(b), sb, db);
    return __byte_perm(hb, ha, 0x7632) >> sh;
}

struct StoreF64 {
    using T = double;
    using R = double;
    static constexpr bool kHalf = false;
    __device__ static R load(const T* p, double w) { return __ldg(p) - w; }
    __device__ static void store(T* p, R d, double w) { *p = d + w; }
    __device__ static T encode(R d, double w) { return d + w; }
};
struct StoreF32 {
    using T = float;
    using R = float;
    static constexpr bool kHalf = false;
    __device__ static R load(const T* p, double w) { return __ldg(p) - (float)w; }
    __device__ static void store(T* p, R d, double w) { *p = d + (float)w; }
    __device__ static T encode(R d, double w) { return d + (float)w; }
};
struct StoreF32S {
    using T = float;
    using R = float;
    static constexpr bool kHalf = false;
    __device__ static R load(const T* p, double) { return __ldg(p); }
    __device__ static void store(T* p, R d, double) { *p = d; }
    __device__ static T encode(R d, double) { return d; }
};
struct StoreF16S {
    using T = __half;
    using R = float;
    static constexpr bool kHalf = true;
    __device__ static R load(const T* p, double) { return __half2float(__ldg(p)); }
    __device__ static void store(T* p, R d, double) { *p = __float2half_rn(d); }
    __device__ static T encode(R d, double) { return __float2half_rn(d); }
    // a (node salt sa, direction da) in the high half, b in the low half,
    // stochastic rounding
    __device__ static unsigned encode_pair(R a, R b, unsigned sa, unsigned sb, int da, int db)
    {
        unsigned out;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;"
            : "=r"(out) : "f"(a), "f"(b), "r"(pair_rbits<3>(a, b, sa, sb, da, db)));
        return out;
    }
    __device__ static T hi(unsigned pk) { return __ushort_as_half((unsigned short)(pk >> 16)); }
    __device__ static T lo(unsigned pk) { return __ushort_as_half((unsigned short)(pk & 0xffffu)); }
    // two x-adjacent nodes (p 4-byte aligned): the lower address first
    __device__ static void load2(const T* p, R& a, R& b)
    {
        const __half2 h = __ldg(reinterpret_cast<const __half2*>(p));
        a = __low2float(h);
        b = __high2float(h);
    }
};
struct StoreBF16S {
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool kHalf = true;
    __device__ static R load(const T* p, double) { return __bfloat162float(__ldg(p)); }
    __device__ static void store(T* p, R d, double) { *p = __float2bfloat16_rn(d); }
    __device__ static T encode(R d, double) { return __float2bfloat16_rn(d); }
    __device__ static unsigned encode_pair(R a, R b, unsigned sa, unsigned sb, int da, int db)
    {
        unsigned out;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;"
            : "=r"(out) : "f"(a), "f"(b), "r"(pair_rbits<0>(a, b, sa, sb, da, db)));
        return out;
    }
    __device__ static T hi(unsigned pk)
    {
        return __ushort_as_bfloat16((unsigned short)(pk >> 16));
    }
    __device__ static T lo(unsigned pk)
    {
        return __ushort_as_bfloat16((unsigned short)(pk & 0xffffu));
    }
    __device__ static void load2(const T* p, R& a, R& b)
    {
        const __nv_bfloat162 h = __ldg(reinterpret_cast<const __nv_bfloat162*>(p));
        a = __low2float(h);
        b = __high2float(h);
    }
};

// Stochastically rounded stores of one node's q deviations (half-width
// codecs): opposite directions (2k+1, 2k+2) share one conversion, the rest
// population pairs with itself.  dst(i) is the address of direction i.  Each
// value's random field comes from its own hash, so the rounding of a value
// does not depend on which value it is paired with or in which half it sits.
template <class L, class S, class F>
__device__ __forceinline__ void store_node_sr(const float (&d)[L::Q], unsigned salt, F dst)
{
    *dst(0) = S::hi(S::encode_pair(d[0], d[0], salt, salt, 0, 0));
#pragma unroll
    for (int k = 0; k < (L::Q - 1) / 2; ++k) {
        const int i = 2 * k + 1, j = i + 1;
        const unsigned pk = S::encode_pair(d[i], d[j], salt, salt, i, j);
        *dst(i) = S::hi(pk);
        *dst(j) = S::lo(pk);
    }
}

// ---------------------------------------------------------------------------
// Kernel parameters (passed by value).
// ---------------------------------------------------------------------------
enum { MODEL_BGK = 0, MODEL_MRT = 1, MODEL_ELBM = 2, MODEL_REG = 3, MODEL_SMAG = 4 };
// node-type byte of the batched ensemble: bit 0 solid, bit 1 fluid with a
// solid upstream neighbour
enum { FLAG_SOLID = 1, FLAG_NEAR_WALL = 2 };
// node word of a single-domain handle (one 32-bit load per node, issued with
// the population loads): bits 1..26 link mask (bit i: the upstream node
// x - e_i is solid), bit 27 solid, bits 28..31 boundary condition id + 1
constexpr uint32_t NODE_LINKS = 0x07fffffeu, NODE_SOLID = 1u << 27;
// On a solid node (whose link bits are otherwise unused), bit 1 marks a node
// that shares its 32-byte sector of every direction plane with a fluid node
// (AB pattern only): the AB kernels write the rest state (deviation 0) into
// its slots so that the sector is written whole.  A partly written sector
// costs the memory a read of the whole sector first (read-modify-write):
// 0.38 GB per step of the 512x256x256 sphere duct in FP32.  Nothing reads
// those slots.
constexpr uint32_t NODE_FILL = 1u << 1;
constexpr int NODE_BC_SHIFT = 28;
constexpr int kMaxBC = 15;
// ELBM counter replicas: slots 0..5 evals, skipped, clamped, at cap, guarded,
// updated; 6 sum of |g(alpha)|/a2 (double bits), 7 its max (double bits),
// 8 residual samples
constexpr int kCtrReplicas = 64, kCtrStride = 16;

// One velocity or pressure boundary condition (Sec. 2.3's list).
struct BCEntry {
    int kind;          // 1 velocity, 2 pressure
    int method;        // 0 equilibrium, 1 Zou-He, 2 regularized
    int axis, sign;    // inward normal: sign times the unit vector of axis (0 x, 1 y, 2 z)
    double val[3];     // prescribed velocity, or the density in val[0]
    float val_f[3];
    float pad_;
};
enum { STATUS_NAN = 1u, STATUS_NOCONV = 2u, STATUS_TIMEOUT = 4u };
// ELBM per-node outcome, shared meaning with the counters of the ABI
enum { ALPHA_CONV = 0, ALPHA_SKIP = 1, ALPHA_CLAMP = 2, ALPHA_NOCONV = 3, ALPHA_GUARDED = 5 };
enum { MLP_NPARAM = 1394 };

struct StepParams {
    const void* A;             // post-collision distributions at t (read)
    void* B;                   // post-collision distributions at t+1 (written)
    const uint32_t* nodes;     // node words, or nullptr without a geometry
    // plane i of A and B (A + i sq, B + i sq): the kernels address each
    // direction's plane through these, so a load is one 32-bit offset from a
    // parameter-bank pointer instead of a 64-bit plane product per access
    const void* Ap[27];
    void* Bp[27];      // node-type map (FLAG_*) or nullptr
    void* rho;                 // output fields (compute type), padded layout
    void* u;                   // [D][sq]
    double* alpha_out;         // ELBM per-node alpha or nullptr
    unsigned int* status;      // STATUS_* bits
    unsigned long long* elbm_ctr;  // counter replicas (kCtrStride slots each) or nullptr
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
    int row0, nrows;           // rows updated: z layers (3-D lattices) or y rows (D2Q9)
    int zrun;                  // z layers per thread of the masked z-run kernel (set at launch)
    int salt_off;              // node-index offset of the dither salt (subdomains)
    // time-step clock of the stochastic rounding: the launch that takes step
    // t reads t from step_ctr[step_slot] and one of its threads stores t + 1
    // into step_ctr[step_slot ^ 1] (several launches of one step, e.g. the
    // row ranges of a subdomain, store the same value); nullptr for storage
    // types without stochastic rounding
    unsigned* step_ctr;
    int step_slot;
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
    BCEntry bc[kMaxBC];        // boundary conditions by id
    // ELBM
    int alpha_mode, max_iter, guard_steps, feq_variant;
    int elbm_diag;             // 1: accumulate the entropy-condition residual
    double tol, skip_eps, guard_tol;
    const float* mlp;          // MLP_NPARAM floats (BF16-rounded weights)
};

// Salt term of the launch's time step for the stochastic-rounding hash:
// t * kSaltStep + salt_off * kSaltNode, so that node n's salt is
// n * kSaltNode + step_salt(p).  Reads t from the step clock; thread 0 of
// block 0 stores t + 1 into the clock's other slot for the next step (no
// thread of this launch reads that slot).  0 without a clock.
__device__ __forceinline__ unsigned step_salt(const StepParams& p)
{
    if (!p.step_ctr) return (unsigned)p.salt_off * kSaltNode;
    const unsigned t = p.step_ctr[p.step_slot];
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0)
        p.step_ctr[p.step_slot ^ 1] = t + 1;
    return t * kSaltStep + (unsigned)p.salt_off * kSaltNode;
}

// Parameter in the compute type: the FP32 copy for float, FP64 for double.
template <class R>
__host__ __device__ __forceinline__ R sel(float f, double d);
template <>
__host__ __device__ __forceinline__ float sel<float>(float f, double) { return f; }
template <>
__host__ __device__ __forceinline__ double sel<double>(float, double d) { return d; }

}  // namespace lbm
