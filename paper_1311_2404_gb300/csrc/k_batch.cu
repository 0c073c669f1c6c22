// Batched ensemble of independent D2Q9 LBGK domains of uneven sizes, advanced
// by one persistent cooperative launch per lbm_batch_step call.
//
// Layout: every domain d owns, inside one arena, its own AB pair of SoA
// distribution arrays [9][ny][nxp] (x padded to 32), a node-type map and
// output fields rho, ux, uy.  The work list is the set of tiles (domain,
// x0, y0) of tw x th nodes over all domains; persistent CTA g owns the
// contiguous tile range [g T / G, (g+1) T / G).  After each time step all
// CTAs meet at a grid barrier whose spin is bounded: if it gives up, the CTA
// records STATUS_TIMEOUT and returns, so a lost arrival ends the launch with
// an error status instead of a hang.  The per-node update is the same code as
// the single-domain kernel (pull streaming, half-way bounce-back, LBGK with
// Guo forcing), so every domain evolves exactly as it would alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "collide.cuh"
#include "lbm_internal.h"

using namespace lbm;

namespace {

struct DomDev {
    long long offA, offB, offF, offO;   // byte offsets in the arena
    long long sq;                       // elements per direction plane
    int nx, ny, nxp, has_force;
    float omega, gx, gy, pad;
};

struct BatchParams {
    char* base;
    const DomDev* dom;
    const int4* tiles;                  // (domain, x0, y0, 0)
    int ntiles;
    int nsteps;
    int cur;                            // 0: state in A regions
    int th;                             // tile rows
    int tw;                             // tile width (the staged kernel's tiles)
    unsigned* bar;                      // [0] arrivals, [1] generation
    unsigned* status;
    long long wait_limit;               // spins before giving up
    int withhold;                       // test hooks: 1 CTA 0 skips its first grid-barrier
                                        // arrival; 2 (staged kernel) the first stage of
                                        // the launch gets no copies and no arrivals
    int round_nearest;                  // FP16 storage: 1 round to nearest, 0 dither
    // time-step clock of the stochastic rounding (two slots): a launch of
    // nsteps steps starting at step t reads t from clock[clock_slot], and
    // thread 0 of CTA 0 stores t + nsteps into clock[clock_slot ^ 1]
    unsigned* clock;
    int clock_slot;
};

// First step index of this launch from the rounding clock (half-width
// storage); advances the clock by the launch's steps.
template <class S>
__device__ __forceinline__ unsigned batch_clock(const BatchParams& bp)
{
    if constexpr (!S::kHalf) return 0u;
    const unsigned t = bp.clock[bp.clock_slot];
    if ((blockIdx.x | threadIdx.x | threadIdx.y) == 0)
        bp.clock[bp.clock_slot ^ 1] = t + (unsigned)bp.nsteps;
    return t;
}

// Bounded grid barrier (generation counter).  Returns false when this CTA
// must stop (its wait ran out, or it withheld its arrival).
__device__ bool grid_barrier(const BatchParams& bp, bool skip_arrive)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ok = 1;
        volatile unsigned* vgen = bp.bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        if (skip_arrive) {
            ok = 0;
        } else {
            const unsigned prev = atomicAdd(bp.bar, 1u);
            if (prev == gridDim.x - 1) {
                atomicExch(bp.bar, 0u);
                __threadfence();
                atomicAdd(bp.bar + 1, 1u);
            } else {
                long long spins = 0;
                while (*vgen == gen) {
                    if (++spins > bp.wait_limit) {
                        atomicOr(bp.status, STATUS_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(128);
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// A population written during this launch (by any CTA, in an earlier step):
// a coherent load, not the read-only (non-coherent) path.
template <class S>
__device__ __forceinline__ float bload(const typename S::T* p)
{
    if constexpr (S::kHalf) return __half2float(*p);
    else return *p;
}

// Pull loads of one node's incoming populations (periodic wrap).  They do
// not wait for the node's flag byte, which is loaded beside them and
// returned: a solid node's populations are read and dropped, and the
// half-way bounce-back substitution (batch_bounce) follows only where the
// flag says a neighbour is solid.
template <class S>
__device__ __forceinline__ unsigned batch_load(const DomDev& D, const typename S::T* __restrict__ A,
                                               const uint8_t* __restrict__ flags, int x, int y,
                                               float (&d)[9])
{
    using L = D2Q9;
    // element indices in 32 bits (a domain holds at most 9 x 2^20 values):
    // one widening multiply-add per access instead of 64-bit plane products
    const int sq = (int)D.sq;
    const int cx[3] = {x == 0 ? D.nx - 1 : x - 1, x, x == D.nx - 1 ? 0 : x + 1};
    const int ry[3] = {(y == 0 ? D.ny - 1 : y - 1) * D.nxp, y * D.nxp,
                       (y == D.ny - 1 ? 0 : y + 1) * D.nxp};
#pragma unroll
    for (int i = 0; i < 9; ++i)
        d[i] = bload<S>(A + (i * sq + ry[1 - L::ey(i)] + cx[1 - L::ex(i)]));
    return flags[ry[1] + x];
}

// Half-way bounce-back of a node next to a solid one: an incoming
// population whose upstream node is solid is the node's own outgoing
// population in the opposite direction from the previous step.
template <class S>
__device__ __forceinline__ void batch_bounce(const DomDev& D, const typename S::T* __restrict__ A,
                                             const uint8_t* __restrict__ flags, int x, int y,
                                             float (&d)[9])
{
    using L = D2Q9;
    const int sq = (int)D.sq;
    const int n = y * D.nxp + x;
    const int cx[3] = {x == 0 ? D.nx - 1 : x - 1, x, x == D.nx - 1 ? 0 : x + 1};
    const int ry[3] = {(y == 0 ? D.ny - 1 : y - 1) * D.nxp, y * D.nxp,
                       (y == D.ny - 1 ? 0 : y + 1) * D.nxp};
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int src = ry[1 - L::ey(i)] + cx[1 - L::ex(i)];
        if (flags[src] & FLAG_SOLID) d[i] = bload<S>(A + (L::opp(i) * sq + n));
    }
}

// Collision and store of one node (the single-domain kernel's arithmetic).
// tsalt: the time step's term of the stochastic-rounding salt, t * kSaltStep
template <class S>
__device__ __forceinline__ void batch_update(const DomDev& D, const BatchParams& bp,
                                             typename S::T* __restrict__ B,
                                             float* __restrict__ o, int n, bool out,
                                             unsigned tsalt, float (&d)[9])
{
    using L = D2Q9;
    const int sq = (int)D.sq;
    float drho, v[3];   // drho = rho - 1, the form the rho output field holds
    bgk_collide<L, float>(d, D.omega, D.gx, D.gy, 0.f, D.has_force != 0, drho, v);
    if constexpr (S::kHalf) {
        if (!bp.round_nearest) {
            store_node_sr<L, S>(d, (unsigned)n * kSaltNode + tsalt,
                                [&](int i) { return B + (i * sq + n); });
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) S::store(B + (i * sq + n), d[i], L::w(i));
        }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) S::store(B + (i * sq + n), d[i], L::w(i));
    }
    if (out) {
        o[n] = drho;
        o[sq + n] = v[0];
        o[2 * sq + n] = v[1];
        if (!isfinite(drho) || !isfinite(v[0]) || !isfinite(v[1])) atomicOr(bp.status, STATUS_NAN);
    }
}

// One persistent launch for n steps.  CTA g owns the contiguous tile range
// [g T / G, (g+1) T / G) of the list ordered by (domain, y0, x0); it reads
// only its first tile from the list and walks the rest arithmetically,
// loading a domain's record when it enters that domain.  A thread handles
// column x0 + threadIdx.x of a tile and rows threadIdx.y + k blockDim.y; NPT
// of its rows are loaded together before any is updated.
template <class S, int NPT>
__global__ void __launch_bounds__(512) k_batch(const BatchParams bp)
{
    using T = typename S::T;
    const int G = gridDim.x;
    const int t0 = (int)((long long)bp.ntiles * blockIdx.x / G);
    const int t1 = (int)((long long)bp.ntiles * (blockIdx.x + 1) / G);
    const int tw = blockDim.x, by = blockDim.y;
    int4 first = make_int4(0, 0, 0, 0);
    if (t0 < t1) first = bp.tiles[t0];
    int cur = bp.cur;
    const unsigned clk = batch_clock<S>(bp);
    for (int step = 0; step < bp.nsteps; ++step) {
        const bool out = (step == bp.nsteps - 1);
        const unsigned tsalt = (clk + (unsigned)step) * kSaltStep;
        int dom = first.x, x0 = first.y, y0 = first.z;
        DomDev D{};
        if (t0 < t1) D = bp.dom[dom];
        for (int t = t0; t < t1; ++t) {
            const T* __restrict__ A =
                reinterpret_cast<const T*>(bp.base + (cur == 0 ? D.offA : D.offB));
            T* __restrict__ B = reinterpret_cast<T*>(bp.base + (cur == 0 ? D.offB : D.offA));
            const uint8_t* __restrict__ flags = reinterpret_cast<const uint8_t*>(bp.base + D.offF);
            float* __restrict__ o = reinterpret_cast<float*>(bp.base + D.offO);
            const int x = x0 + threadIdx.x;
            const int yend = min(y0 + bp.th, D.ny);
            if (x < D.nx) {
                for (int ya = y0 + threadIdx.y; ya < yend; ya += NPT * by) {
                    float d[NPT][9];
                    unsigned fl[NPT];
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int y = ya + k * by;
                        fl[k] = 0x80u;                       // no node (beyond the tile)
                        if (k == 0 || y < yend) fl[k] = batch_load<S>(D, A, flags, x, y, d[k]);
                    }
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int y = ya + k * by;
                        if (fl[k] & 0x80u) continue;
                        const int n = y * D.nxp + x;
                        if (fl[k] & FLAG_SOLID) {
                            if (out) { o[n] = -1.f; o[D.sq + n] = 0.f; o[2 * D.sq + n] = 0.f; }
                            continue;
                        }
                        if (fl[k] & FLAG_NEAR_WALL) batch_bounce<S>(D, A, flags, x, y, d[k]);
                        batch_update<S>(D, bp, B, o, n, out, tsalt, d[k]);
                    }
                }
            }
            // the next tile in (domain, y0, x0) order
            x0 += tw;
            if (x0 >= D.nx) {
                x0 = 0;
                y0 += bp.th;
                if (y0 >= D.ny) {
                    y0 = 0;
                    ++dom;
                    if (t + 1 < t1) D = bp.dom[dom];
                }
            }
        }
        cur ^= 1;
        if (step + 1 < bp.nsteps) {
            const bool skip = bp.withhold == 1 && blockIdx.x == 0 && step == 0;
            if (!grid_barrier(bp, skip)) return;
        }
    }
}

// ---- register kernel, two x-adjacent nodes per thread ----------------------
//
// Half-width storage makes the one-node kernel instruction-bound (about 317
// instructions per D2Q9 node).  Here a thread updates columns x and x + 1
// (x even; tiles are a multiple of 64 wide): the three directions without an
// x component are one pair load, the two flag bytes one 16-bit load, and an
// active pair is written with one store per direction (one stochastic-rounding
// conversion for both values), with the per-value hashes of the one-node
// kernel, so the fields are bitwise the same.
template <class S>
__device__ __forceinline__ void batch_load_pair(const typename S::T* __restrict__ row, float& a,
                                                float& b)
{
    if constexpr (S::kHalf) {
        const __half2 h = *reinterpret_cast<const __half2*>(row);
        a = __low2float(h);
        b = __high2float(h);
    } else {
        const float2 f = *reinterpret_cast<const float2*>(row);
        a = f.x;
        b = f.y;
    }
}

template <class S, int NPT>
__device__ __forceinline__ void batch2_body(const BatchParams& bp)
{
    using T = typename S::T;
    using L = D2Q9;
    const int G = gridDim.x;
    const int t0 = (int)((long long)bp.ntiles * blockIdx.x / G);
    const int t1 = (int)((long long)bp.ntiles * (blockIdx.x + 1) / G);
    const int tw = 2 * blockDim.x, by = blockDim.y;
    int4 first = make_int4(0, 0, 0, 0);
    if (t0 < t1) first = bp.tiles[t0];
    int cur = bp.cur;
    const unsigned clk = batch_clock<S>(bp);
    for (int step = 0; step < bp.nsteps; ++step) {
        const bool out = (step == bp.nsteps - 1);
        const unsigned tsalt = (clk + (unsigned)step) * kSaltStep;
        int dom = first.x, x0 = first.y, y0 = first.z;
        DomDev D{};
        if (t0 < t1) D = bp.dom[dom];
        for (int t = t0; t < t1; ++t) {
            const T* __restrict__ A =
                reinterpret_cast<const T*>(bp.base + (cur == 0 ? D.offA : D.offB));
            T* __restrict__ B = reinterpret_cast<T*>(bp.base + (cur == 0 ? D.offB : D.offA));
            const uint8_t* __restrict__ flags = reinterpret_cast<const uint8_t*>(bp.base + D.offF);
            float* __restrict__ o = reinterpret_cast<float*>(bp.base + D.offO);
            const int x = x0 + 2 * (int)threadIdx.x;
            const int yend = min(y0 + bp.th, D.ny);
            if (x < D.nx) {
                const int sq = (int)D.sq;
                const bool has1 = x + 1 < D.nx;
                // source columns of node k for e_x = +1, 0, -1 (periodic); a
                // padding node x + 1 reads inside the row and is not written
                const int cx[2][3] = {{x == 0 ? D.nx - 1 : x - 1, x, x + 1 >= D.nx ? 0 : x + 1},
                                      {x, x + 1, x + 2 >= D.nx ? x + 2 - D.nx : x + 2}};
                for (int ya = y0 + threadIdx.y; ya < yend; ya += NPT * by) {
                    float d[NPT][2][9];
                    unsigned fl[NPT];
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int y = ya + k * by;
                        fl[k] = 0x8080u;                     // no node (beyond the tile)
                        if (k == 0 || y < yend) {
                            const int ry[3] = {(y == 0 ? D.ny - 1 : y - 1) * D.nxp, y * D.nxp,
                                               (y == D.ny - 1 ? 0 : y + 1) * D.nxp};
#pragma unroll
                            for (int i = 0; i < 9; ++i) {
                                const int rs = i * sq + ry[1 - L::ey(i)];
                                if (L::ex(i) == 0) {
                                    batch_load_pair<S>(A + (rs + x), d[k][0][i], d[k][1][i]);
                                } else {
                                    d[k][0][i] = bload<S>(A + (rs + cx[0][1 - L::ex(i)]));
                                    d[k][1][i] = bload<S>(A + (rs + cx[1][1 - L::ex(i)]));
                                }
                            }
                            fl[k] = *reinterpret_cast<const unsigned short*>(flags + ry[1] + x);
                            if (!has1) fl[k] |= 0x8000u;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int y = ya + k * by;
                        if (fl[k] & 0x80u) continue;
                        const int n = y * D.nxp + x;
                        bool act[2];
                        float rho[2], v[2][3];
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const unsigned f = (fl[k] >> (8 * c)) & 0xffu;
                            act[c] = !(f & (0x80u | FLAG_SOLID));
                            if (!(f & 0x80u) && (f & FLAG_SOLID) && out) {
                                o[n + c] = -1.f;
                                o[sq + n + c] = 0.f;
                                o[2 * sq + n + c] = 0.f;
                            }
                            if (!act[c]) continue;
                            if (f & FLAG_NEAR_WALL) batch_bounce<S>(D, A, flags, x + c, y, d[k][c]);
                            bgk_collide<L, float>(d[k][c], D.omega, D.gx, D.gy, 0.f,
                                                  D.has_force != 0, rho[c], v[c]);
                        }
                        if (act[0] && act[1]) {
                            if constexpr (S::kHalf) {
                                if (!bp.round_nearest) {
                                    const unsigned s0 = (unsigned)n * kSaltNode + tsalt,
                                                   s1 = s0 + kSaltNode;
#pragma unroll
                                    for (int i = 0; i < 9; ++i)
                                        *reinterpret_cast<unsigned*>(B + (i * sq + n)) =
                                            S::encode_pair(d[k][1][i], d[k][0][i], s1, s0, i, i);
                                } else {
#pragma unroll
                                    for (int i = 0; i < 9; ++i) {
                                        S::store(B + (i * sq + n), d[k][0][i], L::w(i));
                                        S::store(B + (i * sq + n + 1), d[k][1][i], L::w(i));
                                    }
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < 9; ++i)
                                    *reinterpret_cast<float2*>(B + (i * sq + n)) =
                                        make_float2(d[k][0][i], d[k][1][i]);
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < 2; ++c) {
                                if (!act[c]) continue;
                                const int m = n + c;
                                if constexpr (S::kHalf) {
                                    if (!bp.round_nearest) {
                                        store_node_sr<L, S>(d[k][c], (unsigned)m * kSaltNode + tsalt,
                                                            [&](int i) { return B + (i * sq + m); });
                                    } else {
#pragma unroll
                                        for (int i = 0; i < 9; ++i)
                                            S::store(B + (i * sq + m), d[k][c][i], L::w(i));
                                    }
                                } else {
#pragma unroll
                                    for (int i = 0; i < 9; ++i)
                                        S::store(B + (i * sq + m), d[k][c][i], L::w(i));
                                }
                            }
                        }
                        if (out) {
                            bool bad = false;
#pragma unroll
                            for (int c = 0; c < 2; ++c) {
                                if (!act[c]) continue;
                                o[n + c] = rho[c];
                                o[sq + n + c] = v[c][0];
                                o[2 * sq + n + c] = v[c][1];
                                bad |= !isfinite(rho[c]) || !isfinite(v[c][0]) || !isfinite(v[c][1]);
                            }
                            if (bad) atomicOr(bp.status, STATUS_NAN);
                        }
                    }
                }
            }
            // the next tile in (domain, y0, x0) order
            x0 += tw;
            if (x0 >= D.nx) {
                x0 = 0;
                y0 += bp.th;
                if (y0 >= D.ny) {
                    y0 = 0;
                    ++dom;
                    if (t + 1 < t1) D = bp.dom[dom];
                }
            }
        }
        cur ^= 1;
        if (step + 1 < bp.nsteps) {
            const bool skip = bp.withhold == 1 && blockIdx.x == 0 && step == 0;
            if (!grid_barrier(bp, skip)) return;
        }
    }
}

// Register budgets per instance (launches of up to 512 threads would allow
// 128; the compiler then spends them and occupancy drops): the largest
// budget without spills, measured with -Xptxas -v, except the one-row FP16S
// instance: capped at 64 (84 bytes of spill) it runs two 512-thread CTAs per
// SM and the 512-channel ensemble 87.0 -> 89.9 GLUPS; at 72 the autotuner
// takes 128-thread CTAs (88.0), at 56 it falls back to the two-row kernel
// (83.7).
template <class S, int NPT, int MAXR>
__global__ void __maxnreg__(MAXR) k_batch2(const BatchParams bp)
{
    batch2_body<S, NPT>(bp);
}

// ---- staged variant: bulk copies into shared memory ------------------------
//
// The register kernel's bytes in flight are bounded by its registers (one
// node's 9 loads per thread).  Here a producer warp copies tiles' inputs into
// a ring of kStages shared-memory stages with cp.async.bulk, up to kStages
// tiles ahead, while the consumer warps update nodes from the filled stages:
// the bytes in flight are several tiles per CTA, and no CTA-wide barrier is
// taken inside a step (a "full" mbarrier per stage signals landed bytes, an
// "empty" one the consumers' release).  Stage layout (bytes, esize = sizeof(T)):
//   planes  [9][th][tw] x esize: row r of plane i holds global row
//           y0 + r - e_iy (wrapped), columns [x0, x0 + tw)
//   flags   [th][tw]: the tile's own node flags
//   halo    [6][th] 32-bit words: for the planes with e_x = +1 the column
//           left of the tile (x0 - 1, or nx - 1 at x0 = 0), for e_x = -1 the
//           column right of it (x0 + tw, or 0 when the tile reaches nx); the
//           aligned 4-byte word holding that element
// Row copies start at element x0 + (plane, row) offsets, all multiples of 32
// elements from a 256-byte aligned region: 16-byte aligned, and their length
// min(tw, nxp - x0) elements is a multiple of 32.

constexpr int kStages = 4;
constexpr int kStagedMaxThreads = 256;   // consumer threads per CTA

__host__ __device__ constexpr int tile_stage_bytes(int esize, int tw, int th)
{
    return (((9 * th * tw * esize + th * tw + 15) & ~15) + 6 * th * 4 + 127) & ~127;
}
__host__ __device__ constexpr int stage_halo_offset(int esize, int tw, int th)
{
    return (9 * th * tw * esize + th * tw + 15) & ~15;
}

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// arrive (counts one) and raise the expected transaction bytes of the phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// global -> shared bulk copy completing on bar (bytes a multiple of 16, both
// addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 4-byte asynchronous copy (src 4-byte aligned); its completion is signalled
// by the issuing thread's later cp_arrive_noinc
__device__ __forceinline__ void cp4_g2s(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_arrive_noinc(unsigned long long* bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// order this thread's generic-proxy view of global memory with its later
// (or, on the writing side, others' later) bulk-copy reads
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait for a stage's phase: gives up after `cycles` SM clocks.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  long long cycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

// D2Q9 planes with e_x = +1 (their pull reads the left halo) and e_x = -1
// (right halo), in halo-slot order, as 4-bit fields of one constant; e_y + 1
// of every plane as 2-bit fields (no run-time indexed local arrays)
constexpr unsigned kHaloPlanes = 1u | 5u << 4 | 7u << 8 | 2u << 12 | 6u << 16 | 8u << 20;
static_assert(D2Q9::ex(1) == 1 && D2Q9::ex(5) == 1 && D2Q9::ex(7) == 1 && D2Q9::ex(2) == -1 &&
                  D2Q9::ex(6) == -1 && D2Q9::ex(8) == -1,
              "halo planes");
__host__ __device__ constexpr unsigned ey_code()
{
    unsigned c = 0;
    for (int i = 0; i < 9; ++i) c |= (unsigned)(D2Q9::ey(i) + 1) << (2 * i);
    return c;
}
__device__ __forceinline__ int halo_plane(int k) { return (int)((kHaloPlanes >> (4 * k)) & 15u); }
__device__ __forceinline__ int d2q9_ey(int i) { return (int)((ey_code() >> (2 * i)) & 3u) - 1; }
__host__ __device__ constexpr int halo_slot(int i)
{
    return i == 1 ? 0 : i == 5 ? 1 : i == 7 ? 2 : i == 2 ? 3 : i == 6 ? 4 : 5;
}

// Warp-0 side: queue the copies of tile (D, x0, y0) into stage st (all 32
// lanes call it).  The phase completes when the expected bytes have landed
// and all 32 lanes' 4-byte copies are done (count 33 = 1 + 32).
template <class S>
__device__ __forceinline__ void stage_issue(const BatchParams& bp, const DomDev& D, int cur, int x0,
                                            int y0, int tw, int th, unsigned char* st,
                                            unsigned long long* bar)
{
    using T = typename S::T;
    constexpr int es = (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    const int nrows = min(th, D.ny - y0);
    const int ncols = min(tw, D.nxp - x0);
    const unsigned rowb = (unsigned)(ncols * es);
    const int pb = th * tw * es;
    const char* A = bp.base + (cur == 0 ? D.offA : D.offB);
    const char* F = bp.base + D.offF;
    const int sq = (int)D.sq;
    if (lane == 0)
        mbar_arrive_expect_tx(bar, 9u * nrows * rowb + (unsigned)(nrows * ncols));
    for (int c = lane; c < 10 * nrows; c += 32) {
        const int i = c / nrows, r = c - i * nrows;
        if (i < 9) {
            int ys = y0 + r - d2q9_ey(i);
            ys = ys < 0 ? ys + D.ny : (ys >= D.ny ? ys - D.ny : ys);
            bulk_g2s(st + i * pb + r * tw * es, A + (size_t)(i * sq + ys * D.nxp + x0) * es, rowb,
                     bar);
        } else {
            bulk_g2s(st + 9 * pb + r * tw, F + (size_t)((y0 + r) * D.nxp + x0), (unsigned)ncols,
                     bar);
        }
    }
    const int cl = x0 == 0 ? D.nx - 1 : x0 - 1;
    const int cr = x0 + tw < D.nx ? x0 + tw : 0;
    unsigned* halo = reinterpret_cast<unsigned*>(st + stage_halo_offset(es, tw, th));
    for (int c = lane; c < 6 * nrows; c += 32) {
        const int k = c / nrows, r = c - k * nrows;
        const int i = halo_plane(k);
        int ys = y0 + r - d2q9_ey(i);
        ys = ys < 0 ? ys + D.ny : (ys >= D.ny ? ys - D.ny : ys);
        int col = k < 3 ? cl : cr;
        if (es == 2) col &= ~1;                      // the aligned pair holding it
        cp4_g2s(halo + k * th + r, A + (size_t)(i * sq + ys * D.nxp + col) * es);
    }
    cp_arrive_noinc(bar);
}

template <class S>
__device__ __forceinline__ float stage_dec(typename S::T v)
{
    if constexpr (S::kHalf) return __half2float(v);
    else return v;
}

// a halo element from its 4-byte word (half-width: the half at column col)
template <class S>
__device__ __forceinline__ float halo_dec(unsigned w, int col)
{
    if constexpr (S::kHalf) {
        const unsigned short h = (col & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
        return __half2float(__ushort_as_half(h));
    } else {
        return __uint_as_float(w);
    }
}

// next tile in (domain, y0, x0) order; loads the domain record on entering
// a domain when `more`
__device__ __forceinline__ void tile_advance(const BatchParams& bp, DomDev& D, int& dom, int& x0,
                                             int& y0, int tw, bool more)
{
    x0 += tw;
    if (x0 >= D.nx) {
        x0 = 0;
        y0 += bp.th;
        if (y0 >= D.ny) {
            y0 = 0;
            ++dom;
            if (more) D = bp.dom[dom];
        }
    }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up when another thread of the CTA has
// raised *abort.
__device__ __forceinline__ bool mbar_wait_abortable(unsigned long long* bar, unsigned parity,
                                                    long long cycles, volatile int* abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > cycles) return false;
    }
    return true;
}

// rho - 1 and v of an output step, with the non-finite check (the rho field
// holds the deviation, -1 at solid nodes; readback adds 1 in FP64)
__device__ __forceinline__ void batch_out(const DomDev& D, const BatchParams& bp,
                                          float* __restrict__ o, int n, float rho,
                                          const float (&v)[3])
{
    o[n] = rho;
    o[D.sq + n] = v[0];
    o[2 * D.sq + n] = v[1];
    if (!isfinite(rho) || !isfinite(v[0]) || !isfinite(v[1])) atomicOr(bp.status, STATUS_NAN);
}

// store of one node's nine values (the one-node path's rounding)
template <class S>
__device__ __forceinline__ void staged_store1(const BatchParams& bp, typename S::T* __restrict__ B,
                                              int sq, int n, unsigned salt, const float (&d)[9])
{
    using L = D2Q9;
    if constexpr (S::kHalf) {
        if (!bp.round_nearest) {
            store_node_sr<L, S>(d, salt, [&](int i) { return B + (i * sq + n); });
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) S::store(B + (i * sq + n), d[i], L::w(i));
}

// Update of two x-adjacent nodes (tile columns c0 = 2 pp and c0 + 1) on the
// rows ty, ty + cy, ... of one staged tile.  Same per-node arithmetic and the
// same per-value stochastic rounding as the one-node path: a half-width
// direction of the pair is one conversion and one 32-bit store, an FP32
// direction one 64-bit store.
template <class S>
__device__ __forceinline__ void staged_tile2(const BatchParams& bp, const DomDev& D, int cur,
                                             int x0, int y0, int tw, int th, int pp, int ty,
                                             int cy, bool out, unsigned tsalt,
                                             const unsigned char* st)
{
    using T = typename S::T;
    using L = D2Q9;
    constexpr int es = (int)sizeof(T);
    const int pb = th * tw * es;
    const T* __restrict__ A = reinterpret_cast<const T*>(bp.base + (cur == 0 ? D.offA : D.offB));
    T* __restrict__ B = reinterpret_cast<T*>(bp.base + (cur == 0 ? D.offB : D.offA));
    const uint8_t* __restrict__ flags = reinterpret_cast<const uint8_t*>(bp.base + D.offF);
    float* __restrict__ o = reinterpret_cast<float*>(bp.base + D.offO);
    const T* pl = reinterpret_cast<const T*>(st);
    const unsigned* halo = reinterpret_cast<const unsigned*>(st + stage_halo_offset(es, tw, th));
    const int c0 = 2 * pp;
    const int xa = x0 + c0;
    if (xa >= D.nx) return;
    const bool vb = xa + 1 < D.nx;              // node b exists
    const int nrows = min(th, D.ny - y0);
    const int sq = (int)D.sq;
    const int cl = x0 == 0 ? D.nx - 1 : x0 - 1;
    const int cr = x0 + tw < D.nx ? x0 + tw : 0;
    const bool a_left = c0 == 0;                 // node a's e_x = +1 source is the left halo
    const bool a_right = !vb;                    // node a = nx - 1: its e_x = -1 source wraps
    const bool b_right = c0 + 2 == tw || xa + 2 == D.nx;
    for (int r = ty; r < nrows; r += cy) {
        const int y = y0 + r;
        const int n = y * D.nxp + xa;
        const unsigned char* frow = st + 9 * pb + r * tw;
        const unsigned fa = frow[c0];
        const unsigned fb = vb ? frow[c0 + 1] : (unsigned)FLAG_SOLID;
        const bool la = !(fa & FLAG_SOLID), lb = !(fb & FLAG_SOLID);
        if (!la && !lb) {
            if (out) {
                o[n] = -1.f; o[sq + n] = 0.f; o[2 * sq + n] = 0.f;
                if (vb) { o[n + 1] = -1.f; o[sq + n + 1] = 0.f; o[2 * sq + n + 1] = 0.f; }
            }
            continue;
        }
        float da[9], db[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T* row = pl + (i * th + r) * tw;
            if (L::ex(i) == 0) {
                da[i] = stage_dec<S>(row[c0]);
                db[i] = stage_dec<S>(row[c0 + 1]);
            } else if (L::ex(i) == 1) {
                da[i] = a_left ? halo_dec<S>(halo[halo_slot(i) * th + r], cl)
                               : stage_dec<S>(row[c0 - 1]);
                db[i] = stage_dec<S>(row[c0]);
            } else {
                da[i] = a_right ? halo_dec<S>(halo[halo_slot(i) * th + r], cr)
                                : stage_dec<S>(row[c0 + 1]);
                db[i] = b_right ? halo_dec<S>(halo[halo_slot(i) * th + r], cr)
                                : stage_dec<S>(row[c0 + 2]);
            }
        }
        float ra = 0.f, rb = 0.f, va[3] = {0.f, 0.f, 0.f}, vbv[3] = {0.f, 0.f, 0.f};
        if (la) {
            if (fa & FLAG_NEAR_WALL) batch_bounce<S>(D, A, flags, xa, y, da);
            bgk_collide<L, float>(da, D.omega, D.gx, D.gy, 0.f, D.has_force != 0, ra, va);
        }
        if (lb) {
            if (fb & FLAG_NEAR_WALL) batch_bounce<S>(D, A, flags, xa + 1, y, db);
            bgk_collide<L, float>(db, D.omega, D.gx, D.gy, 0.f, D.has_force != 0, rb, vbv);
        }
        const unsigned s0 = (unsigned)n * kSaltNode + tsalt, s1 = s0 + kSaltNode;
        if (la && lb) {
            if constexpr (S::kHalf) {
                if (!bp.round_nearest) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        *reinterpret_cast<unsigned*>(B + (i * sq + n)) =
                            S::encode_pair(db[i], da[i], s1, s0, i, i);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        S::store(B + (i * sq + n), da[i], L::w(i));
                        S::store(B + (i * sq + n + 1), db[i], L::w(i));
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    *reinterpret_cast<float2*>(B + (i * sq + n)) = make_float2(da[i], db[i]);
            }
        } else if (la) {
            staged_store1<S>(bp, B, sq, n, s0, da);
        } else {
            staged_store1<S>(bp, B, sq, n + 1, s1, db);
        }
        if (out) {
            if (la) batch_out(D, bp, o, n, ra, va);
            else { o[n] = -1.f; o[sq + n] = 0.f; o[2 * sq + n] = 0.f; }
            if (vb) {
                if (lb) batch_out(D, bp, o, n + 1, rb, vbv);
                else { o[n + 1] = -1.f; o[sq + n + 1] = 0.f; o[2 * sq + n + 1] = 0.f; }
            }
        }
    }
}

// blockDim.x = 32 + consumer threads: warp 0 produces, the rest consume.
template <class S>
__global__ void __launch_bounds__(kStagedMaxThreads + 32) k_batch_staged(const BatchParams bp)
{
    using T = typename S::T;
    constexpr int es = (int)sizeof(T);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages];
    __shared__ int abort_flag;
    volatile int* abort_v = &abort_flag;
    const int tw = bp.tw, th = bp.th;
    const int ncons = (int)blockDim.x - 32;
    const int sb = tile_stage_bytes(es, tw, th);
    const int G = gridDim.x;
    const int t0 = (int)((long long)bp.ntiles * blockIdx.x / G);
    const int t1 = (int)((long long)bp.ntiles * (blockIdx.x + 1) / G);
    const bool producer = threadIdx.x < 32;
    const int lane = threadIdx.x & 31;
    const long long wait_cycles = bp.wait_limit * 256;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 33);                 // expect_tx arrival + 32 lanes' copies
            mbar_init(&empty[s], ncons / 32);        // one arrival per consumer warp
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int4 first = make_int4(0, 0, 0, 0);
    if (t0 < t1) first = bp.tiles[t0];
    unsigned k = 0;                                  // tiles through the ring so far
    int cur = bp.cur;
    const unsigned clk = batch_clock<S>(bp);
    for (int step = 0; step < bp.nsteps; ++step) {
        const bool out = (step == bp.nsteps - 1);
        const unsigned tsalt = (clk + (unsigned)step) * kSaltStep;
        int dom = first.x, x0 = first.y, y0 = first.z;
        DomDev D{};
        if (t0 < t1) D = bp.dom[dom];
        if (producer) {
            fence_proxy_async_global();
            for (int t = t0; t < t1; ++t, ++k) {
                const int s = (int)(k % kStages);
                const unsigned use = k / kStages;
                if (use > 0 &&
                    !mbar_wait_abortable(&empty[s], (use - 1) & 1u, wait_cycles, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                // test hook 2: the first stage of the launch gets neither copies
                // nor arrivals, so the consumers' wait for it runs out while no
                // copy is in flight for it
                if (!(bp.withhold == 2 && step == 0 && t == t0))
                    stage_issue<S>(bp, D, cur, x0, y0, tw, th, smem + s * sb, &full[s]);
                tile_advance(bp, D, dom, x0, y0, tw, t + 1 < t1);
            }
        } else {
            const int c = (int)threadIdx.x - 32;
            const int hw = tw / 2;                   // threads per tile row (two nodes each)
            const int pp = c % hw, ty = c / hw, cy = ncons / hw;
            for (int t = t0; t < t1; ++t, ++k) {
                const int s = (int)(k % kStages);
                const unsigned use = k / kStages;
                if (!mbar_wait_abortable(&full[s], use & 1u, wait_cycles, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                staged_tile2<S>(bp, D, cur, x0, y0, tw, th, pp, ty, cy, out, tsalt, smem + s * sb);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                tile_advance(bp, D, dom, x0, y0, tw, t + 1 < t1);
            }
        }
        cur ^= 1;
        if (__syncthreads_or(*abort_v)) {
            // the CTA stops together; the producer first lets the copies it
            // issued land (bounded), so no copy targets a finished CTA (a
            // stage whose phase never completes had no copies issued)
            if (producer) {
#pragma unroll 1
                for (int s = 0; s < kStages; ++s) {
                    if (k <= (unsigned)s) continue;
                    const unsigned last = (k - 1 - s) / kStages;       // last use of stage s
                    mbar_wait_bounded(&full[s], last & 1u, wait_cycles);
                }
            }
            if (threadIdx.x == 0) atomicOr(bp.status, STATUS_TIMEOUT);
            return;
        }
        if (step + 1 < bp.nsteps) {
            fence_proxy_async_global();
            const bool skip = bp.withhold == 1 && blockIdx.x == 0 && step == 0;
            if (!grid_barrier(bp, skip)) return;
        }
    }
}

template <class S>
const void* staged_kernel_ptr() { return reinterpret_cast<const void*>(&k_batch_staged<S>); }

template <class S, int NPT>
const void* batch_kernel_ptr() { return reinterpret_cast<const void*>(&k_batch<S, NPT>); }
template <class S, int NPT, int MAXR>
const void* batch2_kernel_ptr() { return reinterpret_cast<const void*>(&k_batch2<S, NPT, MAXR>); }

}  // namespace

struct lbm_batch_ctx {
    int ndom = 0, dtype = 0;
    size_t esize = 4;
    std::vector<DomDev> dom;
    std::vector<char> inited, has_mask;
    char* base = nullptr;
    size_t bytes = 0, off_tables = 0, off_tiles = 0, off_bar = 0, off_stage = 0, stage_bytes = 0;
    std::vector<int4> tiles;
    int ntiles = 0;
    cudaStream_t stream = nullptr;
    int threads = 256, ctas = 0, tw = 128, th = 8, npt = 1;   // launch configuration
    int sms = 0, tiles_tw = 0, tiles_th = 0;          // tiles currently uploaded for (tw, th)
    int cur = 0;
    int lp = 0;                       // launch parity: the rounding clock's slot holding t
    unsigned clk_host[2] = {0, 0};    // source of the clock copy after autotuning
    long long t = 0, launches = 0, wait_limit = 20000000LL;
    int withhold = 0;
    int round_nearest = 0;
    bool use_graph = true;
    std::map<std::tuple<int, int, int, int, int, int>, cudaGraphExec_t> graphs;
    std::string err;
};

static thread_local std::string g_batch_err;

static int bfail(lbm_batch b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_err = buf;
    return code;
}

#define BCK(b, call, what)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return bfail((b), LBM_ECUDA, "%s: %s", (what),            \
                                            cudaGetErrorString(e_));                    \
    } while (0)

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

static bool dev_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void drop_graphs(lbm_batch b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// npt: 0 the staged kernel; 1, 2, 4 the register kernel with that many rows
// per thread and pass; -1, -2 the same with two x-adjacent nodes per thread
static const void* kernel_for(int dtype, int npt)
{
    if (npt < 0) {
        if (dtype == LBM_F16S)
            return npt == -2 ? batch2_kernel_ptr<StoreF16S, 2, 104>()
                             : batch2_kernel_ptr<StoreF16S, 1, 64>();
        return npt == -2 ? batch2_kernel_ptr<StoreF32S, 2, 128>()
                         : batch2_kernel_ptr<StoreF32S, 1, 96>();
    }
    if (dtype == LBM_F16S)
        return npt == 0   ? staged_kernel_ptr<StoreF16S>()
             : npt == 4 ? batch_kernel_ptr<StoreF16S, 4>()
             : npt == 2 ? batch_kernel_ptr<StoreF16S, 2>() : batch_kernel_ptr<StoreF16S, 1>();
    return npt == 0   ? staged_kernel_ptr<StoreF32S>()
         : npt == 4 ? batch_kernel_ptr<StoreF32S, 4>()
         : npt == 2 ? batch_kernel_ptr<StoreF32S, 2>() : batch_kernel_ptr<StoreF32S, 1>();
}

// dynamic shared memory of a launch (the staged kernel's two stages)
static size_t launch_smem(lbm_batch b, int tw, int th, int npt)
{
    return npt == 0 ? kStages * (size_t)tile_stage_bytes((int)b->esize, tw, th) : 0;
}

constexpr size_t kMaxStagedSmem = 200 * 1024;

// Build and upload the tile list for tile shape (tw, th).
static int upload_tiles(lbm_batch b, int tw, int th)
{
    if (b->tiles_tw == tw && b->tiles_th == th) return LBM_OK;
    std::vector<int4> tl;
    for (int d = 0; d < b->ndom; ++d)
        for (int y0 = 0; y0 < b->dom[d].ny; y0 += th)
            for (int x0 = 0; x0 < b->dom[d].nx; x0 += tw) tl.push_back(make_int4(d, x0, y0, 0));
    const size_t cap = b->off_bar - b->off_tiles;
    if (tl.size() * sizeof(int4) > cap)
        return bfail(b, LBM_EINVAL, "tile list of %zu tiles exceeds its reserve", tl.size());
    BCK(b, cudaMemcpy(b->base + b->off_tiles, tl.data(), tl.size() * sizeof(int4),
                      cudaMemcpyHostToDevice),
        "upload tiles");
    b->ntiles = (int)tl.size();
    b->tiles_tw = tw;
    b->tiles_th = th;
    drop_graphs(b);
    return LBM_OK;
}

static int max_ctas(lbm_batch b, int threads, int npt, int tw, int th)
{
    const size_t smem = launch_smem(b, tw, th, npt);
    if (smem > kMaxStagedSmem) return 0;
    const void* k = kernel_for(b->dtype, npt);
    if (npt == 0 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxStagedSmem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, npt == 0 ? threads + 32 : threads,
                                                      smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * b->sms;
}

static cudaError_t launch_batch(lbm_batch b, int nsteps, int from)
{
    BatchParams bp;
    bp.base = b->base;
    bp.dom = reinterpret_cast<const DomDev*>(b->base + b->off_tables);
    bp.tiles = reinterpret_cast<const int4*>(b->base + b->off_tiles);
    bp.ntiles = b->ntiles;
    bp.nsteps = nsteps;
    bp.cur = from;
    bp.th = b->th;
    bp.tw = b->tw;
    bp.bar = reinterpret_cast<unsigned*>(b->base + b->off_bar);
    bp.status = reinterpret_cast<unsigned*>(b->base + b->off_bar + 8);
    bp.wait_limit = b->wait_limit;
    bp.withhold = b->withhold;
    bp.round_nearest = b->round_nearest;
    bp.clock = reinterpret_cast<unsigned*>(b->base + b->off_bar + 16);
    bp.clock_slot = b->lp;
    cudaError_t e = cudaMemsetAsync(bp.bar, 0, 8, b->stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(b->ctas);
    // the staged kernel adds its producer warp to the consumer threads
    cfg.blockDim = b->npt == 0  ? dim3(b->threads + 32)
                 : b->npt < 0 ? dim3(b->tw / 2, b->threads / (b->tw / 2))
                              : dim3(b->tw, b->threads / b->tw);
    cfg.dynamicSmemBytes = launch_smem(b, b->tw, b->th, b->npt);
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {&bp};
    return cudaLaunchKernelExC(&cfg, kernel_for(b->dtype, b->npt), args);
}

extern "C" {

int lbm_batch_create(int ndom, const int* nx, const int* ny, const double* tau, int lattice,
                     int dtype, lbm_batch* out)
{
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (ndom < 1 || !nx || !ny || !tau) return bfail(nullptr, LBM_EINVAL, "bad arguments");
    if (lattice != LBM_D2Q9) return bfail(nullptr, LBM_EINVAL, "batched domains are LBM_D2Q9");
    if (dtype != LBM_F32S && dtype != LBM_F16S)
        return bfail(nullptr, LBM_EINVAL, "batch storage must be LBM_F32S or LBM_F16S");
    lbm_batch b = new lbm_batch_ctx();
    b->ndom = ndom;
    b->dtype = dtype;
    b->esize = dtype == LBM_F16S ? 2 : 4;
    b->dom.resize(ndom);
    b->inited.assign(ndom, 0);
    b->has_mask.assign(ndom, 0);
    size_t o = 0, max_nodes = 0, max_tiles = 0;
    for (int d = 0; d < ndom; ++d) {
        if (nx[d] < 1 || ny[d] < 1 || !(tau[d] > 0.5) || !(tau[d] < 1e6)) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "domain %d: bad size or tau", d);
        }
        DomDev& D = b->dom[d];
        D.nx = nx[d];
        D.ny = ny[d];
        D.nxp = (nx[d] + 31) / 32 * 32;
        D.sq = ((long long)D.nxp * D.ny + 127) / 128 * 128;
        if (D.sq > 0x7fffffffLL / 16) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "domain %d too large", d);
        }
        D.omega = (float)(1.0 / tau[d]);
        D.gx = D.gy = 0.f;
        D.has_force = 0;
        D.pad = 0.f;
        D.offA = (long long)o; o = a256(o + 9 * D.sq * b->esize);
        D.offB = (long long)o; o = a256(o + 9 * D.sq * b->esize);
        D.offF = (long long)o; o = a256(o + D.sq);
        D.offO = (long long)o; o = a256(o + 3 * D.sq * 4);
        max_nodes = std::max(max_nodes, (size_t)nx[d] * ny[d]);
        // smallest tile shape the autotuner tries is 32 x 1
        max_tiles += (size_t)((nx[d] + 31) / 32) * ny[d];
    }
    b->off_tables = o; o = a256(o + sizeof(DomDev) * ndom);
    b->off_tiles = o; o = a256(o + sizeof(int4) * max_tiles);
    // grid barrier (+0, 8 B), status (+8), rounding clock (+16, two slots),
    // mask check (+32)
    b->off_bar = o; o = a256(o + 64);
    b->off_stage = o;
    b->stage_bytes = a256(max_nodes * 3 * 8);
    o = a256(o + b->stage_bytes);
    b->bytes = o;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    void* p = nullptr;
    cudaError_t e = dev_alloc(&p, b->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(nullptr, LBM_ENOMEM, "cudaMalloc(%zu): %s", o, cudaGetErrorString(e));
    }
    b->base = static_cast<char*>(p);
    e = cudaMemset(b->base, 0, b->bytes);   // flags = fluid, f = w (rest), status clear
    if (e == cudaSuccess)
        e = cudaMemcpy(b->base + b->off_tables, b->dom.data(), sizeof(DomDev) * ndom,
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p);
        delete b;
        return bfail(nullptr, LBM_ECUDA, "initialise arena: %s", cudaGetErrorString(e));
    }
    int r = upload_tiles(b, b->tw, b->th);
    if (r) {
        std::string m = b->err;
        cudaFree(p);
        delete b;
        return bfail(nullptr, r, "%s", m.c_str());
    }
    b->ctas = std::min(max_ctas(b, b->threads, b->npt, b->tw, b->th), std::max(1, b->ntiles));
    if (b->ctas < 1) {
        cudaFree(p);
        delete b;
        return bfail(nullptr, LBM_ECUDA, "batched kernel cannot be resident");
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b)
{
    if (!b) return LBM_OK;
    drop_graphs(b);
    if (b->base) cudaFree(b->base);
    delete b;
    return LBM_OK;
}

const char* lbm_batch_last_error(lbm_batch b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

int lbm_batch_set_stream(lbm_batch b, void* stream)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (b->stream != static_cast<cudaStream_t>(stream)) drop_graphs(b);
    b->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

int lbm_batch_set_geometry(lbm_batch b, int d, const uint8_t* mask)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (d < 0 || d >= b->ndom || !mask) return bfail(b, LBM_EINVAL, "bad domain or mask");
    const DomDev& D = b->dom[d];
    const size_t n = (size_t)D.nx * D.ny;
    uint8_t* stage = reinterpret_cast<uint8_t*>(b->base + b->off_stage);
    BCK(b, cudaMemcpyAsync(stage, mask, n, dev_ptr(mask) ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice, b->stream),
        "copy mask");
    int* bad = reinterpret_cast<int*>(b->base + b->off_bar + 32);
    BCK(b, cudaMemsetAsync(bad, 0, sizeof(int), b->stream), "clear mask check");
    BCK(b, launch_flags(0, stage, nullptr, reinterpret_cast<uint8_t*>(b->base + D.offF), D.nx,
                        D.ny, 1, D.nxp, 1, bad, nullptr, 0, b->stream),
        "node-type map kernel");
    b->launches += 1;
    int hbad = 0;
    BCK(b, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
        "read mask check");
    BCK(b, cudaStreamSynchronize(b->stream), "synchronise");
    if (hbad) return bfail(b, LBM_EINVAL, "batch masks take 0 (fluid) and 1 (solid) only");
    b->has_mask[d] = 1;
    return LBM_OK;
}

int lbm_batch_set_force(lbm_batch b, int d, double fx, double fy)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (d < 0 || d >= b->ndom || !std::isfinite(fx) || !std::isfinite(fy))
        return bfail(b, LBM_EINVAL, "bad domain or force");
    DomDev& D = b->dom[d];
    D.gx = (float)fx;
    D.gy = (float)fy;
    D.has_force = (fx != 0.0 || fy != 0.0);
    BCK(b, cudaMemcpy(b->base + b->off_tables + sizeof(DomDev) * d, &D, sizeof(DomDev),
                      cudaMemcpyHostToDevice),
        "upload domain table");
    return LBM_OK;
}

int lbm_batch_init_equilibrium(lbm_batch b, int d, const void* rho, const void* u,
                               int field_dtype)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (d < 0 || d >= b->ndom || !rho || !u) return bfail(b, LBM_EINVAL, "bad arguments");
    if (field_dtype != LBM_FIELD_F32 && field_dtype != LBM_FIELD_F64)
        return bfail(b, LBM_EINVAL, "unknown field dtype");
    const DomDev& D = b->dom[d];
    const size_t fs = field_dtype == LBM_FIELD_F64 ? 8 : 4;
    const size_t nb = (size_t)D.nx * D.ny * fs;
    char* stage = b->base + b->off_stage;
    // device memory and pinned host memory are read in place by the init
    // kernel; pageable host memory is staged
    const void* dr = kernel_view(rho);
    const void* du = kernel_view(u);
    if (!dr) {
        BCK(b, cudaMemcpyAsync(stage, rho, nb, cudaMemcpyHostToDevice, b->stream), "copy rho");
        dr = stage;
    }
    if (!du) {
        BCK(b, cudaMemcpyAsync(stage + nb, u, 2 * nb, cudaMemcpyHostToDevice, b->stream),
            "copy u");
        du = stage + nb;
    }
    // the buffer that holds the current state (A before any step); the other
    // domains and the batch's step parity and time are unchanged
    BCK(b, launch_init(0, b->dtype, dr, du, field_dtype == LBM_FIELD_F32,
                       b->base + (b->cur ? D.offB : D.offA), D.nx, D.ny, 1, D.nxp, D.sq, 0, 0, 0,
                       b->stream),
        "init kernel");
    b->launches += 1;
    BCK(b, cudaStreamSynchronize(b->stream), "synchronise");
    b->inited[d] = 1;
    return LBM_OK;
}

static int check_ready(lbm_batch b)
{
    for (int d = 0; d < b->ndom; ++d)
        if (!b->inited[d]) return bfail(b, LBM_ESTATE, "domain %d not initialised", d);
    return LBM_OK;
}

static int step_impl(lbm_batch b, int n)
{
    const auto key = std::make_tuple(n, b->cur * 2 + b->lp, b->threads, b->ctas, b->tw,
                                     b->th * 8 + b->npt);
    if (b->use_graph && b->stream != nullptr && !b->withhold) {
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t g;
            BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
                "begin capture");
            cudaError_t le = launch_batch(b, n, b->cur);
            cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (le == cudaSuccess && ce == cudaSuccess) {
                cudaGraphExec_t ge;
                cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (ie == cudaSuccess) it = b->graphs.emplace(key, ge).first;
            } else if (ce == cudaSuccess) {
                cudaGraphDestroy(g);
            }
            if (it == b->graphs.end()) {   // capture not possible: launch directly
                cudaGetLastError();
                b->use_graph = false;
            }
        }
        if (it != b->graphs.end()) {
            BCK(b, cudaGraphLaunch(it->second, b->stream), "graph launch");
            b->launches += 1;
            b->lp ^= 1;
            b->cur ^= (n & 1);
            b->t += n;
            return LBM_OK;
        }
    }
    BCK(b, launch_batch(b, n, b->cur), "persistent batched kernel");
    b->launches += 1;
    b->lp ^= 1;
    b->cur ^= (n & 1);
    b->t += n;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int n)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (n < 1) return bfail(b, LBM_EINVAL, "n must be >= 1");
    int r = check_ready(b);
    if (r) return r;
    return step_impl(b, n);
}

int lbm_batch_autotune(lbm_batch b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    int r = check_ready(b);
    if (r) return r;
    // keep the state: copy the per-domain regions aside and restore them
    const size_t span = b->off_tables;     // every per-domain region lies below the tables
    void* save = nullptr;
    {
        const cudaError_t e = dev_alloc(&save, span);
        if (e != cudaSuccess)
            return bfail(b, LBM_ENOMEM, "autotune backup (%zu bytes): %s", span,
                         cudaGetErrorString(e));
    }
    BCK(b, cudaMemcpyAsync(save, b->base, span, cudaMemcpyDeviceToDevice, b->stream), "backup");
    const int saved_cur = b->cur;
    const long long saved_t = b->t;
    const bool saved_graph = b->use_graph;
    b->use_graph = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bt = b->threads, bc = b->ctas, bw = b->tw, bh = b->th, bn = b->npt;
    const int steps = 4;
    // npt 0: the staged kernel; 1, 2, 4: the register kernel's rows per pass
    for (int npt : {0, 1, 2, 4, -1, -2})
        for (int threads : {128, 256, 512})
            for (int tw : {64, 128, 256}) {
                if (tw > threads) continue;
                for (int th : {2, 4, 8, 16, 32, 64}) {
                    // every consumer thread gets a row (staged and paired: two
                    // columns per thread)
                    if (th < (npt == 0 ? 2 * (threads / tw)
                              : npt < 0 ? -npt * (threads / (tw / 2)) : npt * (threads / tw)))
                        continue;
                    if (npt == 0 && (th > 32 || threads > kStagedMaxThreads)) continue;
                    const int mc = max_ctas(b, threads, npt, tw, th);
                    if (mc < 1) continue;
                    if (upload_tiles(b, tw, th)) continue;
                    const int per_sm = std::max(1, mc / b->sms);
                    for (int k = 1; k <= per_sm; k = (k * 2 > per_sm && k < per_sm) ? per_sm : k * 2) {
                        b->threads = threads; b->tw = tw; b->th = th; b->npt = npt;
                        b->ctas = std::min(k * b->sms, b->ntiles);
                        if (launch_batch(b, 1, b->cur) != cudaSuccess) {
                            cudaGetLastError();
                            continue;
                        }
                        cudaEventRecord(e0, b->stream);
                        cudaError_t le = launch_batch(b, steps, b->cur);
                        cudaEventRecord(e1, b->stream);
                        if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                            cudaGetLastError();
                            continue;
                        }
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (ms < best) {
                            best = ms; bt = threads; bc = b->ctas; bw = tw; bh = th; bn = npt;
                        }
                    }
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->threads = bt; b->ctas = bc; b->npt = bn;
    int ur = upload_tiles(b, bw, bh);
    b->tw = bw; b->th = bh;
    BCK(b, cudaMemcpyAsync(b->base, save, span, cudaMemcpyDeviceToDevice, b->stream), "restore");
    BCK(b, cudaMemsetAsync(b->base + b->off_bar, 0, 64, b->stream), "clear status");
    // the rounding clock resumes at the saved step (both slots)
    b->clk_host[0] = b->clk_host[1] = (unsigned)saved_t;
    BCK(b, cudaMemcpyAsync(b->base + b->off_bar + 16, b->clk_host, sizeof b->clk_host,
                           cudaMemcpyHostToDevice, b->stream),
        "restore the rounding clock");
    BCK(b, cudaStreamSynchronize(b->stream), "synchronise");
    cudaFree(save);
    b->cur = saved_cur;
    b->t = saved_t;
    b->use_graph = saved_graph;
    drop_graphs(b);
    return ur;
}

int lbm_batch_get_config(lbm_batch b, int* out5)
{
    if (!b || !out5) return bfail(b, LBM_EINVAL, "NULL argument");
    out5[0] = b->threads;
    out5[1] = b->ctas;
    out5[2] = b->tw;
    out5[3] = b->th;
    out5[4] = b->npt;
    return LBM_OK;
}

int lbm_batch_set_config(lbm_batch b, const int* in5)
{
    if (!b || !in5) return bfail(b, LBM_EINVAL, "NULL argument");
    const int threads = in5[0], ctas = in5[1], tw = in5[2], th = in5[3], npt = in5[4];
    if (tw < 32 || tw % 32 || threads < tw || threads > 512 || threads % tw)
        return bfail(b, LBM_EINVAL, "threads %d / tile width %d: need 32 | tw, tw | threads <= 512",
                     threads, tw);
    if (npt != 0 && npt != 1 && npt != 2 && npt != 4 && npt != -1 && npt != -2)
        return bfail(b, LBM_EINVAL,
                     "variant must be 0 (staged), 1, 2, 4 or (two nodes per thread) -1, -2");
    if (npt < 0 && (tw % 64 || threads % (tw / 2)))
        return bfail(b, LBM_EINVAL, "two nodes per thread: tile width %d must be a multiple of 64"
                     " and threads %d a multiple of half of it", tw, threads);
    if (npt == 0 && threads > kStagedMaxThreads)
        return bfail(b, LBM_EINVAL, "the staged kernel takes at most %d consumer threads",
                     kStagedMaxThreads);
    if (th < 1 || th > 4096) return bfail(b, LBM_EINVAL, "tile rows %d out of range", th);
    if (launch_smem(b, tw, th, npt) > kMaxStagedSmem)
        return bfail(b, LBM_EINVAL, "staged tile %d x %d needs %zu bytes of shared memory", tw, th,
                     launch_smem(b, tw, th, npt));
    const int mc = max_ctas(b, threads, npt, tw, th);
    if (ctas < 1 || ctas > mc)
        return bfail(b, LBM_EINVAL, "%d CTAs: between 1 and %d can be co-resident", ctas, mc);
    int r = upload_tiles(b, tw, th);
    if (r) return r;
    b->threads = threads;
    b->tw = tw;
    b->th = th;
    b->npt = npt;
    b->ctas = std::min(ctas, b->ntiles);
    drop_graphs(b);
    return LBM_OK;
}

int lbm_batch_set_wait_limit(lbm_batch b, long long spins)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (spins < 1) return bfail(b, LBM_EINVAL, "spins must be >= 1");
    b->wait_limit = spins;
    drop_graphs(b);
    return LBM_OK;
}

int lbm_batch_set_rounding(lbm_batch b, int mode)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (mode != LBM_ROUND_DITHER && mode != LBM_ROUND_NEAREST)
        return bfail(b, LBM_EINVAL, "unknown rounding mode %d", mode);
    b->round_nearest = (mode == LBM_ROUND_NEAREST);
    drop_graphs(b);
    return LBM_OK;
}

int lbm_batch_inject_missing_arrival(lbm_batch b, int on)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (on < 0 || on > 2) return bfail(b, LBM_EINVAL, "hook %d: 0, 1 or 2", on);
    b->withhold = on;
    drop_graphs(b);
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    unsigned st = 0;
    BCK(b, cudaMemcpyAsync(&st, b->base + b->off_bar + 8, 4, cudaMemcpyDeviceToHost, b->stream),
        "read status");
    BCK(b, cudaStreamSynchronize(b->stream), "synchronise");
    if (st & STATUS_TIMEOUT) {
        BCK(b, cudaMemset(b->base + b->off_bar + 8, 0, 4), "clear status");
        return bfail(b, LBM_ETIMEOUT, "a grid-barrier wait gave up; the state is incomplete");
    }
    if (st & STATUS_NAN) return bfail(b, LBM_ENAN, "non-finite rho or v on an output step");
    return LBM_OK;
}

int lbm_batch_get_macro(lbm_batch b, int d, void* rho, void* u, int field_dtype)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch");
    if (d < 0 || d >= b->ndom) return bfail(b, LBM_EINVAL, "bad domain");
    if (field_dtype != LBM_FIELD_F32 && field_dtype != LBM_FIELD_F64)
        return bfail(b, LBM_EINVAL, "unknown field dtype");
    if (b->t == 0) return bfail(b, LBM_ESTATE, "no step has produced output yet");
    const DomDev& D = b->dom[d];
    const int f32 = field_dtype == LBM_FIELD_F32;
    const size_t fs = f32 ? 4 : 8;
    const size_t nb = (size_t)D.nx * D.ny * fs;
    char* stage = b->base + b->off_stage;
    // device memory and pinned host memory are written in place by the pack
    // kernel; pageable host memory is staged (rho at the start of the staging
    // area, u after it) and copied out.  One synchronisation, in
    // lbm_batch_sync, covers both fields and the status word.
    struct { void* dst; long long off; int nf; size_t soff; } parts[2] = {
        {rho, 0, 1, 0}, {u, D.sq * 4, 2, nb}};
    for (auto& pt : parts) {
        if (!pt.dst) continue;
        void* view = const_cast<void*>(kernel_view(pt.dst));
        void* outp = view ? view : stage + pt.soff;
        BCK(b, launch_pack(0, b->base + D.offO + pt.off, f32, outp, pt.nf, D.nx, D.ny, 1, D.nxp,
                           D.sq, pt.off == 0 ? 1.0 : 0.0, b->stream),
            "pack kernel");
        b->launches += 1;
        if (!view)
            BCK(b, cudaMemcpyAsync(pt.dst, outp, nb * pt.nf, cudaMemcpyDeviceToHost, b->stream),
                "copy out");
    }
    return lbm_batch_sync(b);
}

long long lbm_batch_launch_count(lbm_batch b) { return b ? b->launches : 0; }

size_t lbm_batch_nodes(lbm_batch b)
{
    if (!b) return 0;
    size_t n = 0;
    for (const DomDev& D : b->dom) n += (size_t)D.nx * D.ny;
    return n;
}

}  // extern "C"
