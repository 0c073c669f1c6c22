// The fused stream-and-collide kernel (Algorithm cnp, Sec. 3.3, re-designed
// for sm_103a as a pull scheme).
//
// One thread per node; a CTA covers BX consecutive x nodes of BY rows.  Each
// thread gathers the q populations that stream into its node from the
// previous step's post-collision array A (f_i(x) = F_i(x - e_i), periodic
// wrap), replaces those whose upstream node is solid by the node's own
// opposite population (half-way bounce-back, Sec. 2.3), collides in registers
// and writes all q post-collision values to B at its own node.  Reads of the
// e_x = 0 directions and all writes are aligned, fully coalesced rows; the
// e_x = +-1 reads are shifted by one element and touch one extra 32-byte
// sector per warp row, which the L2 serves (DRAM moves each byte once).
// On output steps the same pass writes rho and v (Eq. edm_momentum); the rho
// field holds the deviation rho - 1 (solid nodes: -1, i.e. rho = 0), which
// readback turns into rho in FP64.
//
// AA pattern (one array, Sec. 3.3): the post-collision values alternate
// between two placements.  A pull/push step (even t) reads f_i(x) from slot
// opp(i) of node x - e_i and writes f*_i(x) to slot i of node x + e_i; an
// in-place step (odd t) reads slot i of node x and writes f*_i(x) to slot
// opp(i) of node x.  Each location is read and then written by the same
// thread, so the update is race-free.  Half-way bounce-back: on a pull/push
// step the bounced value is node x's own slot i (its previous in-place
// write), on an in-place step it is slot opp(i) of the solid node x - e_i
// (where node x's own push landed).
#pragma once

#include "collide.cuh"

namespace lbm {

constexpr int kStepThreads = 128;

template <class L, class S, int MODEL, bool MASK, bool AA>
__device__ __forceinline__ void stream_collide_body(const StepParams& p)
{
    using R = typename S::R;
    using T = typename S::T;
    constexpr bool ELBM = (MODEL == MODEL_ELBM);
    __shared__ float smlp[ELBM ? MLP_NPARAM : 1];
    __shared__ unsigned long long sctr[ELBM ? (kStepThreads / 32) * 9 : 1];
    if (ELBM && p.alpha_mode == 2) {
        for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < MLP_NPARAM;
             k += blockDim.x * blockDim.y)
            smlp[k] = p.mlp[k];
        __syncthreads();
    }

    // rows row0 .. row0 + nrows - 1 of the slowest axis (z, or y on D2Q9)
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int yb = blockIdx.y * blockDim.y + threadIdx.y;
    const int y = (L::D == 2) ? p.row0 + yb : yb;
    const int z = (L::D == 3) ? p.row0 + (int)blockIdx.z : 0;
    bool active = (x < p.nx) && ((L::D == 2) ? (yb < p.nrows) : (y < p.ny));
    unsigned tsalt = 0;   // the time step's term of the stochastic-rounding salt
    if constexpr (S::kHalf) tsalt = step_salt(p);
    const int plane = p.ny * p.nxp;
    const int n = z * plane + y * p.nxp + x;
    // The node-type byte and the q populations are loaded independently: the
    // loads do not wait for the flag (a solid node's populations are read and
    // dropped), so a masked domain keeps the unmasked kernel's memory-level
    // parallelism.
    uint32_t fl = 0;
    if (MASK && active) fl = __ldg(p.nodes + n);
    auto Ai = [&](int i) { return static_cast<const T*>(p.Ap[i]); };
    auto Bi = [&](int i) { return static_cast<T*>(p.Bp[i]); };
    // neighbour coordinates (periodic)
    const int cx[3] = {x == 0 ? p.nx - 1 : x - 1, x, x == p.nx - 1 ? 0 : x + 1};
    const int ry[3] = {(y == 0 ? p.ny - 1 : y - 1) * p.nxp, y * p.nxp,
                       (y == p.ny - 1 ? 0 : y + 1) * p.nxp};
    const int zm = (L::D == 3) ? (z == 0 ? p.nz - 1 : z - 1) : z;
    const int zp = (L::D == 3) ? (z == p.nz - 1 ? 0 : z + 1) : z;
    const int rz[3] = {zm * plane, z * plane, zp * plane};
    const bool pushpull = AA && p.aa_pushpull;
    R d[L::Q];
    if (active) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int src = rz[1 - L::ez(i)] + ry[1 - L::ey(i)] + cx[1 - L::ex(i)];
            if (!AA)
                d[i] = S::load(Ai(i) + src, L::w(i));
            else if (pushpull)
                d[i] = S::load(Ai(L::opp(i)) + src, L::w(i));
            else
                d[i] = S::load(Ai(i) + n, L::w(i));
        }
    }
    if (active && (fl & NODE_SOLID)) {
        if (p.out) {
            static_cast<R*>(p.rho)[n] = R(-1);
#pragma unroll
            for (int a = 0; a < L::D; ++a) static_cast<R*>(p.u)[a * p.sq + n] = R(0);
            if (ELBM && p.alpha_out) p.alpha_out[n] = 0.0;
        }
        if (MASK && !AA && (fl & NODE_FILL)) {   // rest state: whole-sector writes
#pragma unroll
            for (int i = 0; i < L::Q; ++i) d[i] = R(0);
            if constexpr (S::kHalf) {
                if (!p.round_nearest) {
                    store_node_sr<L, S>(d, (unsigned)n * kSaltNode + tsalt,
                                        [&](int i) { return Bi(i) + n; });
                } else {
#pragma unroll
                    for (int i = 0; i < L::Q; ++i) S::store(Bi(i) + n, d[i], L::w(i));
                }
            } else {
#pragma unroll
                for (int i = 0; i < L::Q; ++i) S::store(Bi(i) + n, d[i], L::w(i));
            }
        }
        active = false;
    }
    int evals = 0, astat = -1;
    double resid = 0.0;
    if (active) {
        if (MASK && (fl & NODE_LINKS)) {
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const int src = rz[1 - L::ez(i)] + ry[1 - L::ey(i)] + cx[1 - L::ex(i)];
                if ((fl >> i) & 1u) {
                    if (!AA)
                        d[i] = S::load(Ai(L::opp(i)) + n, L::w(i));
                    else if (pushpull)
                        d[i] = S::load(Ai(i) + n, L::w(i));
                    else
                        d[i] = S::load(Ai(L::opp(i)) + src, L::w(i));
                }
            }
        }
        if (MASK && (fl >> NODE_BC_SHIFT))
            bc_apply<L, R>(d, p.bc[(fl >> NODE_BC_SHIFT) - 1],
                           sel<R>(p.F_f[0], p.F[0]), sel<R>(p.F_f[1], p.F[1]),
                           sel<R>(p.F_f[2], p.F[2]));
        R drho, v[3];
        float feat[8];
        bool have_feat = false;
        AlphaResult ar{2.0, 0, -1};
        if (MODEL == MODEL_BGK) {
            bgk_collide<L, R>(d, sel<R>(p.omega_f, p.omega), sel<R>(p.F_f[0], p.F[0]),
                              sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]),
                              p.has_force != 0, drho, v);
        } else if (MODEL == MODEL_MRT) {
            if constexpr (L::Q == 19) mrt_collide<R>(d, p, drho, v);
        } else if (MODEL == MODEL_REG || MODEL == MODEL_SMAG) {
            les_collide<L, R, MODEL == MODEL_SMAG>(
                d, sel<R>(p.omega_f, p.omega), sel<R>(p.tau_f, p.tau),
                sel<R>(p.smag_cs2_f, p.smag_cs2), sel<R>(p.F_f[0], p.F[0]),
                sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]), p.has_force != 0, drho, v);
        } else {
            ar = elbm_collide<L, R>(d, p, smlp, drho, v, feat, have_feat);
            evals = ar.evals;
            astat = ar.status;
            resid = ar.resid;
        }
        // destination of population i: own node, slot i (AB); node x + e_i,
        // slot i (AA pull/push); own node, slot opp(i) (AA in place)
        auto dst = [&](int i) -> T* {
            if (!AA) return Bi(i) + n;
            if (pushpull)
                return Bi(i) + (rz[1 + L::ez(i)] + ry[1 + L::ey(i)] + cx[1 + L::ex(i)]);
            return Bi(L::opp(i)) + n;
        };
        if constexpr (S::kHalf) {
            if (!p.round_nearest) {
                store_node_sr<L, S>(d, (unsigned)n * kSaltNode + tsalt, dst);
            } else {
#pragma unroll
                for (int i = 0; i < L::Q; ++i) S::store(dst(i), d[i], L::w(i));
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) S::store(dst(i), d[i], L::w(i));
        }
        if (p.out) {
            static_cast<R*>(p.rho)[n] = drho;
#pragma unroll
            for (int a = 0; a < L::D; ++a) static_cast<R*>(p.u)[a * p.sq + n] = v[a];
            bool bad = !isfinite((float)drho);
#pragma unroll
            for (int a = 0; a < L::D; ++a) bad |= !isfinite((float)v[a]);
            if (bad) atomicOr(p.status, STATUS_NAN);
            if (ELBM && p.alpha_out) p.alpha_out[n] = ar.alpha;
        }
        if (ELBM && p.pairs_X && have_feat && astat == ALPHA_CONV &&
            (n % p.pairs_stride) == 0) {
            const int slot = atomicAdd(p.pairs_count, 1);
            if (slot < p.pairs_cap) {
#pragma unroll
                for (int k = 0; k < 8; ++k) p.pairs_X[(size_t)slot * 8 + k] = feat[k];
                p.pairs_y[slot] = ar.alpha;
            }
        }
    }
    if (ELBM && p.elbm_ctr) {
        // counters: evals, skipped, clamped, at cap, guarded, updated nodes,
        // and in diagnostic mode the residual sum, max and sample count
        const bool hr = p.elbm_diag && (astat == ALPHA_CONV || astat == ALPHA_GUARDED);
        unsigned long long c[7] = {(unsigned long long)evals, astat == ALPHA_SKIP,
                                   astat == ALPHA_CLAMP, astat == ALPHA_NOCONV,
                                   astat == ALPHA_GUARDED, astat >= 0, hr};
        double rs = hr ? resid : 0.0, rm = rs;
        const int lane = threadIdx.x & 31;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int warp = tid >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 7; ++k) c[k] += __shfl_down_sync(0xffffffffu, c[k], o);
            rs += __shfl_down_sync(0xffffffffu, rs, o);
            rm = fmax(rm, __shfl_down_sync(0xffffffffu, rm, o));
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 7; ++k) sctr[warp * 9 + k] = c[k];
            sctr[warp * 9 + 7] = __double_as_longlong(rs);
            sctr[warp * 9 + 8] = __double_as_longlong(rm);
        }
        __syncthreads();
        if (tid < 9) {
            const int nw = (blockDim.x * blockDim.y) >> 5;
            // spread over the replicas to limit contention on one address
            const int rep = (blockIdx.x + blockIdx.y * 7 + blockIdx.z * 13) & (kCtrReplicas - 1);
            unsigned long long* slot = p.elbm_ctr + (size_t)rep * kCtrStride;
            if (tid < 7) {
                unsigned long long s = 0;
                for (int w = 0; w < nw; ++w) s += sctr[w * 9 + tid];
                // slots 0..5, and the sample count in slot 8
                if (s) atomicAdd(&slot[tid < 6 ? tid : 8], s);
                if (tid == 3 && s) atomicOr(p.status, STATUS_NOCONV);
            } else if (tid == 7) {
                double s = 0;
                for (int w = 0; w < nw; ++w) s += __longlong_as_double(sctr[w * 9 + 7]);
                if (s > 0) atomicAdd(reinterpret_cast<double*>(&slot[6]), s);
            } else {
                double m = 0;
                for (int w = 0; w < nw; ++w) m = fmax(m, __longlong_as_double(sctr[w * 9 + 8]));
                // non-negative doubles order like their bit patterns
                if (m > 0) atomicMax(&slot[7], (unsigned long long)__double_as_longlong(m));
            }
        }
    }
}

template <class L, class S, int MODEL, bool MASK, bool AA>
__global__ void __launch_bounds__(kStepThreads) k_stream_collide(const StepParams p)
{
    stream_collide_body<L, S, MODEL, MASK, AA>(p);
}

// The same update with a register budget that keeps MINB CTAs resident per
// SM, for FP32-arithmetic AB instances whose register count would otherwise
// cost warps in flight: the regularized and Smagorinsky operators on unmasked
// domains (10 CTAs, 48 registers; left alone Smagorinsky takes 56 and the
// Kida vortex ran 10% below the LBGK rate) and the masked LBGK / regularized /
// Smagorinsky kernels (9 CTAs, 56 registers instead of 64).
template <class L, class S, int MODEL, bool MASK, bool AA, int MINB>
__global__ void __launch_bounds__(kStepThreads, MINB) k_stream_collide_occ(const StepParams p)
{
    stream_collide_body<L, S, MODEL, MASK, AA>(p);
}

// ---------------------------------------------------------------------------
// Masked domains on 3-D lattices, AB pattern: each thread walks a run of
// p.zrun consecutive z layers at one (x, y) and loads the node word of the
// next layer while it updates the current one.  With its word already in a
// register, a node picks the address of every population before loading it:
// the upstream node x - e_i, or, for a link to a solid node, its own slot
// opp(i) (half-way bounce-back, Sec. 2.3), which lies one plane away in the
// same array.  So each node issues exactly q independent loads, with no
// reload that waits for the word, and solid nodes load nothing.  (Loaded
// together with the populations, the word forces a second round trip on
// every warp holding a near-wall node: 62% of the warps of the 512x256x256
// sphere duct.)
// ---------------------------------------------------------------------------
template <class L>
__host__ __device__ constexpr bool opp_adjacent()
{
    for (int i = 1; i < L::Q; ++i)
        if (L::opp(i) != i + 1 && L::opp(i) != i - 1) return false;
    return true;
}

template <class L, class S, int MODEL>
__device__ __forceinline__ void zrun_body(const StepParams& p)
{
    using R = typename S::R;
    using T = typename S::T;
    static_assert(L::D == 3 && MODEL != MODEL_ELBM, "z runs: 3-D lattices, non-entropic");
    static_assert(opp_adjacent<L>(), "slot opp(i) must be plane i + 1 or i - 1");
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    unsigned tsalt = 0;   // the time step's term of the stochastic-rounding salt
    if constexpr (S::kHalf) tsalt = step_salt(p);
    if (x >= p.nx || y >= p.ny) return;
    const int zb = p.row0 + (int)blockIdx.z * p.zrun;
    const int ze = min(zb + p.zrun, p.row0 + p.nrows);
    if (zb >= ze) return;
    const int plane = p.ny * p.nxp;
    auto Ai = [&](int i) { return static_cast<const T*>(p.Ap[i]); };
    auto Bi = [&](int i) { return static_cast<T*>(p.Bp[i]); };
    const int cx[3] = {x == 0 ? p.nx - 1 : x - 1, x, x == p.nx - 1 ? 0 : x + 1};
    const int ry[3] = {(y == 0 ? p.ny - 1 : y - 1) * p.nxp, y * p.nxp,
                       (y == p.ny - 1 ? 0 : y + 1) * p.nxp};
    int n = zb * plane + y * p.nxp + x;
    uint32_t next = __ldg(p.nodes + n);
    bool bad = false;
    for (int z = zb; z < ze; ++z, n += plane) {
        const uint32_t fl = next;
        if (z + 1 < ze) next = __ldg(p.nodes + n + plane);
        const bool solid = (fl & NODE_SOLID) != 0;
        if (solid && !(fl & NODE_FILL)) {
            if (p.out) {
                static_cast<R*>(p.rho)[n] = R(-1);
#pragma unroll
                for (int a = 0; a < 3; ++a) static_cast<R*>(p.u)[a * p.sq + n] = R(0);
            }
            continue;
        }
        // fluid nodes update; solid nodes that share a sector with one take
        // the same store instructions with the rest state (NODE_FILL)
        R d[L::Q];
        R drho = R(-1), v[3] = {R(0), R(0), R(0)};
        if (!solid) {
            const int zm = z == 0 ? p.nz - 1 : z - 1;
            const int zp = z == p.nz - 1 ? 0 : z + 1;
            const int rz[3] = {zm * plane, z * plane, zp * plane};
            const int own_up = n + p.sq, own_dn = n - p.sq;   // slot opp(i) = i +- 1 of node n
            d[0] = S::load(Ai(0) + n, L::w(0));
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const int src = rz[1 - L::ez(i)] + ry[1 - L::ey(i)] + cx[1 - L::ex(i)];
                const int own = L::opp(i) > i ? own_up : own_dn;
                d[i] = S::load(Ai(i) + (((fl >> i) & 1u) ? own : src), L::w(i));
            }
            if (fl >> NODE_BC_SHIFT)
                bc_apply<L, R>(d, p.bc[(fl >> NODE_BC_SHIFT) - 1], sel<R>(p.F_f[0], p.F[0]),
                               sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]));
            if (MODEL == MODEL_BGK) {
                bgk_collide<L, R>(d, sel<R>(p.omega_f, p.omega), sel<R>(p.F_f[0], p.F[0]),
                                  sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]),
                                  p.has_force != 0, drho, v);
            } else if (MODEL == MODEL_MRT) {
                if constexpr (L::Q == 19) mrt_collide<R>(d, p, drho, v);
            } else {
                les_collide<L, R, MODEL == MODEL_SMAG>(
                    d, sel<R>(p.omega_f, p.omega), sel<R>(p.tau_f, p.tau),
                    sel<R>(p.smag_cs2_f, p.smag_cs2), sel<R>(p.F_f[0], p.F[0]),
                    sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]), p.has_force != 0, drho,
                    v);
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) d[i] = R(0);
        }
        if constexpr (S::kHalf) {
            if (!p.round_nearest) {
                store_node_sr<L, S>(d, (unsigned)n * kSaltNode + tsalt,
                                    [&](int i) { return Bi(i) + n; });
            } else {
#pragma unroll
                for (int i = 0; i < L::Q; ++i) S::store(Bi(i) + n, d[i], L::w(i));
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) S::store(Bi(i) + n, d[i], L::w(i));
        }
        if (p.out) {
            static_cast<R*>(p.rho)[n] = drho;
#pragma unroll
            for (int a = 0; a < 3; ++a) static_cast<R*>(p.u)[a * p.sq + n] = v[a];
            bad |= !isfinite((float)drho);
#pragma unroll
            for (int a = 0; a < 3; ++a) bad |= !isfinite((float)v[a]);
        }
    }
    if (bad) atomicOr(p.status, STATUS_NAN);
}

template <class L, class S, int MODEL>
__global__ void __launch_bounds__(kStepThreads) k_stream_collide_zrun(const StepParams p)
{
    zrun_body<L, S, MODEL>(p);
}

// ---------------------------------------------------------------------------
// Half-width storage, AB pattern: two x-adjacent nodes (x0 even, x0 + 1) per
// thread.  The directions without an x component are read as one 32-bit pair,
// each direction's plane address is formed once for both nodes, and a pair of
// active nodes is narrowed by one stochastic-rounding conversion and written
// with one 32-bit store.  The rounding of every value depends only on the
// value and its (node, direction) salt, so the results are bitwise those of
// the one-node kernel.  A solid node is written only with the rest state and
// only when its sector holds a fluid node (NODE_FILL), as in the one-node
// kernel; padding is never written.
// ---------------------------------------------------------------------------
template <class L, class S, int MODEL, bool MASK>
__device__ __forceinline__ void x2_body(const StepParams& p)
{
    using R = typename S::R;
    using T = typename S::T;
    static_assert(S::kHalf && MODEL != MODEL_ELBM, "two-node kernel: half-width, non-entropic");
    const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int yb = blockIdx.y * blockDim.y + threadIdx.y;
    const int y = (L::D == 2) ? p.row0 + yb : yb;
    const int z = (L::D == 3) ? p.row0 + (int)blockIdx.z : 0;
    const unsigned tsalt = step_salt(p);   // the time step's term of the salt
    if (!(x0 < p.nx && ((L::D == 2) ? (yb < p.nrows) : (y < p.ny)))) return;
    const int nx = p.nx, x1 = x0 + 1;
    const int plane = p.ny * p.nxp;
    const int n0 = z * plane + y * p.nxp + x0;
    bool act[2] = {true, x1 < nx};
    uint32_t fl[2] = {0u, 0u};
    if (MASK) {   // the two node words in one load (padding words are solid)
        const uint2 f2 = __ldg(reinterpret_cast<const uint2*>(p.nodes + n0));
        fl[0] = f2.x;
        fl[1] = f2.y;
    }
    auto Ai = [&](int i) { return static_cast<const T*>(p.Ap[i]); };
    auto Bi = [&](int i) { return static_cast<T*>(p.Bp[i]); };
    // source x of each node for e_x = +1, 0, -1 (index 1 - e_x), periodic;
    // node x0 + 1 may be padding (x1 = nx), whose reads stay inside the row
    const int cx[2][3] = {{x0 == 0 ? nx - 1 : x0 - 1, x0, x1 >= nx ? x1 - nx : x1},
                          {x0, x1, x1 + 1 >= nx ? x1 + 1 - nx : x1 + 1}};
    const int ry[3] = {(y == 0 ? p.ny - 1 : y - 1) * p.nxp, y * p.nxp,
                       (y == p.ny - 1 ? 0 : y + 1) * p.nxp};
    const int zm = (L::D == 3) ? (z == 0 ? p.nz - 1 : z - 1) : z;
    const int zp = (L::D == 3) ? (z == p.nz - 1 ? 0 : z + 1) : z;
    const int rz[3] = {zm * plane, z * plane, zp * plane};
    R d[2][L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int rs = rz[1 - L::ez(i)] + ry[1 - L::ey(i)];
        if (L::ex(i) == 0) {
            S::load2(Ai(i) + rs + x0, d[0][i], d[1][i]);
        } else {
            d[0][i] = S::load(Ai(i) + rs + cx[0][1 - L::ex(i)], L::w(i));
            d[1][i] = S::load(Ai(i) + rs + cx[1][1 - L::ex(i)], L::w(i));
        }
    }
    R drho[2], v[2][3];
    bool bad = false;
    // wr: the node's slots are written (fluid, or a solid node that shares a
    // sector with a fluid one and takes the rest state, NODE_FILL)
    bool wr[2] = {act[0], act[1]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int n = n0 + k;
        if (MASK && (fl[k] & NODE_SOLID)) {
            act[k] = false;
            wr[k] = (fl[k] & NODE_FILL) != 0;
            if (wr[k]) {
#pragma unroll
                for (int i = 0; i < L::Q; ++i) d[k][i] = R(0);
            }
        }
        if (!act[k]) continue;
        if (MASK && (fl[k] & NODE_LINKS)) {
#pragma unroll
            for (int i = 1; i < L::Q; ++i)
                if ((fl[k] >> i) & 1u) d[k][i] = S::load(Ai(L::opp(i)) + n, L::w(i));
        }
        if (MASK && (fl[k] >> NODE_BC_SHIFT))
            bc_apply<L, R>(d[k], p.bc[(fl[k] >> NODE_BC_SHIFT) - 1],
                           p.F_f[0], p.F_f[1], p.F_f[2]);
        if (MODEL == MODEL_BGK) {
            bgk_collide<L, R>(d[k], p.omega_f, p.F_f[0], p.F_f[1], p.F_f[2], p.has_force != 0,
                              drho[k], v[k]);
        } else if (MODEL == MODEL_MRT) {
            if constexpr (L::Q == 19) mrt_collide<R>(d[k], p, drho[k], v[k]);
        } else {
            les_collide<L, R, MODEL == MODEL_SMAG>(d[k], p.omega_f, p.tau_f, p.smag_cs2_f,
                                                   p.F_f[0], p.F_f[1], p.F_f[2],
                                                   p.has_force != 0, drho[k], v[k]);
        }
    }
    const unsigned s0 = (unsigned)n0 * kSaltNode + tsalt, s1 = s0 + kSaltNode;
    if (wr[0] && wr[1]) {
        if (!p.round_nearest) {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const unsigned pk = S::encode_pair(d[1][i], d[0][i], s1, s0, i, i);
                *reinterpret_cast<unsigned*>(Bi(i) + n0) = pk;
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                S::store(Bi(i) + n0, d[0][i], L::w(i));
                S::store(Bi(i) + n0 + 1, d[1][i], L::w(i));
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!wr[k]) continue;
            const int n = n0 + k;
            if (!p.round_nearest)
                store_node_sr<L, S>(d[k], k ? s1 : s0, [&](int i) { return Bi(i) + n; });
            else
#pragma unroll
                for (int i = 0; i < L::Q; ++i) S::store(Bi(i) + n, d[k][i], L::w(i));
        }
    }
    if (p.out) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int n = n0 + k;
            if (k == 1 && x1 >= nx) continue;
            const bool a = act[k];
            static_cast<R*>(p.rho)[n] = a ? drho[k] : R(-1);
#pragma unroll
            for (int c = 0; c < L::D; ++c) static_cast<R*>(p.u)[c * p.sq + n] = a ? v[k][c] : R(0);
            if (a) {
                bad |= !isfinite(drho[k]);
#pragma unroll
                for (int c = 0; c < L::D; ++c) bad |= !isfinite(v[k][c]);
            }
        }
        if (bad) atomicOr(p.status, STATUS_NAN);
    }
}

template <class L, class S, int MODEL, bool MASK>
__global__ void __launch_bounds__(kStepThreads) k_stream_collide_x2(const StepParams p)
{
    x2_body<L, S, MODEL, MASK>(p);
}
// MRT needs ~90 registers for two nodes; capped for 6 CTAs per SM it takes 80
// without spilling and runs 6% faster on the FP16S vortex (61.7 -> 65.2 GLUPS).
// Smagorinsky takes 80 uncapped; capped for 7 CTAs per SM (72 registers, a
// 12-byte spill) the FP16S Kida vortex runs 14% faster (46.9 -> 53.6 GLUPS);
// the regularized operator fits 72 either way.  The masked LBGK pair takes 95
// (5 CTAs); capped for 6 (80 registers, a 16-byte spill in FP16S) the FP16S
// cavity runs 8.5% faster (51.1 -> 55.5 GLUPS).  Both caps hold for up to 19
// directions: D3Q27 pairs need ~95-114 registers and would spill 300-400
// bytes under them.  The unmasked LBGK pair at 69
// registers gains nothing from a cap for 8 CTAs (64 registers: FP16S vortex
// 73.5 -> 72.6, BF16S 67.4 -> 68.8 GLUPS).
template <class L, class S, int MODEL, bool MASK, int MINB>
__global__ void __launch_bounds__(kStepThreads, MINB) k_stream_collide_x2_occ(const StepParams p)
{
    x2_body<L, S, MODEL, MASK>(p);
}

inline dim3 step_block_x2(int nxp)
{
    const int pairs = nxp / 2;   // a multiple of 16
    const int bx = pairs >= kStepThreads ? kStepThreads : (pairs + 31) / 32 * 32;
    return dim3(bx, kStepThreads / bx, 1);
}

// Block shape: BX along x (a multiple of 32, at most kStepThreads), BY rows.
inline dim3 step_block(int nxp)
{
    const int bx = nxp >= kStepThreads ? kStepThreads : nxp;
    return dim3(bx, kStepThreads / bx, 1);
}

template <class L, class S, int MODEL>
cudaError_t launch_step_t(const StepParams& p, bool mask, bool aa, cudaStream_t s)
{
    if constexpr (L::D == 3 && MODEL != MODEL_ELBM) {
        // masked AB step in z runs (the host sets p.zrun from the geometry)
        if (mask && !aa && p.zrun > 0) {
            if (p.nrows <= 0) return cudaSuccess;
            const dim3 block = step_block(p.nxp);
            const dim3 grid((p.nx + block.x - 1) / block.x, (p.ny + block.y - 1) / block.y,
                            (p.nrows + p.zrun - 1) / p.zrun);
            k_stream_collide_zrun<L, S, MODEL><<<grid, block, 0, s>>>(p);
            return cudaGetLastError();
        }
    }
    if constexpr (S::kHalf && MODEL != MODEL_ELBM) {
        // masked MRT keeps the one-node kernel: solid neighbours split the
        // pairs and two MRT nodes need ~94 registers (sphere duct FP16S:
        // 35.7 GLUPS with two nodes per thread, 39.0 with one)
        if (!aa && !(MODEL == MODEL_MRT && mask)) {
            if (p.nrows <= 0) return cudaSuccess;
            const bool d2 = (L::D == 2);
            const dim3 block = step_block_x2(p.nxp);
            const dim3 grid(((p.nx + 1) / 2 + block.x - 1) / block.x,
                            ((d2 ? p.nrows : p.ny) + block.y - 1) / block.y, d2 ? 1 : p.nrows);
            if (mask) {
                if constexpr (MODEL == MODEL_BGK && L::Q <= 19)
                    k_stream_collide_x2_occ<L, S, MODEL, true, 6><<<grid, block, 0, s>>>(p);
                else
                    k_stream_collide_x2<L, S, MODEL, true><<<grid, block, 0, s>>>(p);
            } else if constexpr (MODEL == MODEL_MRT) {
                k_stream_collide_x2_occ<L, S, MODEL, false, 6><<<grid, block, 0, s>>>(p);
            } else if constexpr ((MODEL == MODEL_SMAG || MODEL == MODEL_REG) && L::Q <= 19) {
                k_stream_collide_x2_occ<L, S, MODEL, false, 7><<<grid, block, 0, s>>>(p);
            } else {
                k_stream_collide_x2<L, S, MODEL, false><<<grid, block, 0, s>>>(p);
            }
            return cudaGetLastError();
        }
    }
    const dim3 block = step_block(p.nxp);
    const bool d2 = (L::D == 2);
    const dim3 grid((p.nx + block.x - 1) / block.x,
                    ((d2 ? p.nrows : p.ny) + block.y - 1) / block.y, d2 ? 1 : p.nrows);
    if (p.nrows <= 0) return cudaSuccess;
    if (aa) {
        if (mask)
            k_stream_collide<L, S, MODEL, true, true><<<grid, block, 0, s>>>(p);
        else
            k_stream_collide<L, S, MODEL, false, true><<<grid, block, 0, s>>>(p);
    } else {
        constexpr bool f32 = sizeof(typename S::R) == 4;
        constexpr bool les = MODEL == MODEL_REG || MODEL == MODEL_SMAG;
        if (mask) {
            if constexpr (f32 && (les || MODEL == MODEL_BGK))
                k_stream_collide_occ<L, S, MODEL, true, false, 9><<<grid, block, 0, s>>>(p);
            else
                k_stream_collide<L, S, MODEL, true, false><<<grid, block, 0, s>>>(p);
        } else if constexpr (f32 && les) {
            k_stream_collide_occ<L, S, MODEL, false, false, 10><<<grid, block, 0, s>>>(p);
        } else {
            k_stream_collide<L, S, MODEL, false, false><<<grid, block, 0, s>>>(p);
        }
    }
    return cudaGetLastError();
}

// storage codes 0 F64, 1 F32, 2 F32S, 3 F16S, 4 BF16S; bit k of STORES
// compiles storage k
template <class L, int MODEL, unsigned STORES = 31u>
cudaError_t launch_store(int store, const StepParams& p, bool mask, bool aa, cudaStream_t s)
{
    switch (store) {
    case 0: if constexpr ((STORES & 1u) != 0) return launch_step_t<L, StoreF64, MODEL>(p, mask, aa, s);
            break;
    case 1: if constexpr ((STORES & 2u) != 0) return launch_step_t<L, StoreF32, MODEL>(p, mask, aa, s);
            break;
    case 2: if constexpr ((STORES & 4u) != 0) return launch_step_t<L, StoreF32S, MODEL>(p, mask, aa, s);
            break;
    case 3: if constexpr ((STORES & 8u) != 0) return launch_step_t<L, StoreF16S, MODEL>(p, mask, aa, s);
            break;
    case 4: if constexpr ((STORES & 16u) != 0) return launch_step_t<L, StoreBF16S, MODEL>(p, mask, aa, s);
            break;
    }
    return cudaErrorInvalidValue;
}

// lattice codes: 0 D2Q9, 1 D3Q19, 2 D3Q15, 3 D3Q27.  Bit l of LATS compiles
// lattice l into the calling translation unit (each unit holds a few
// lattices so that the build compiles them in parallel).
template <int MODEL, unsigned LATS, unsigned STORES = 31u>
cudaError_t launch_step_model(int lattice, int store, const StepParams& p, bool mask, bool aa,
                              cudaStream_t s)
{
    if constexpr ((LATS & 1u) != 0 && MODEL != MODEL_MRT)
        if (lattice == 0) return launch_store<D2Q9, MODEL, STORES>(store, p, mask, aa, s);
    if constexpr ((LATS & 2u) != 0)
        if (lattice == 1) return launch_store<D3Q19, MODEL, STORES>(store, p, mask, aa, s);
    if constexpr ((LATS & 4u) != 0 && MODEL != MODEL_MRT)
        if (lattice == 2) return launch_store<D3Q15, MODEL, STORES>(store, p, mask, aa, s);
    if constexpr ((LATS & 8u) != 0 && MODEL != MODEL_MRT)
        if (lattice == 3) return launch_store<D3Q27, MODEL, STORES>(store, p, mask, aa, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
