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
// On output steps the same pass writes rho and v (Eq. edm_momentum).
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
__global__ void __launch_bounds__(kStepThreads) k_stream_collide(const StepParams p)
{
    using R = typename S::R;
    using T = typename S::T;
    constexpr bool ELBM = (MODEL == MODEL_ELBM);
    __shared__ float smlp[ELBM ? MLP_NPARAM : 1];
    __shared__ unsigned long long sctr[ELBM ? (kStepThreads / 32) * 6 : 1];
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
    const int plane = p.ny * p.nxp;
    const int n = z * plane + y * p.nxp + x;
    unsigned fl = 0;
    if (MASK && active) fl = p.flags[n];
    if (active && (fl & FLAG_SOLID)) {
        if (p.out) {
            static_cast<R*>(p.rho)[n] = R(0);
#pragma unroll
            for (int a = 0; a < L::D; ++a) static_cast<R*>(p.u)[a * p.sq + n] = R(0);
            if (ELBM && p.alpha_out) p.alpha_out[n] = 0.0;
        }
        active = false;
    }
    int evals = 0, astat = -1;
    if (active) {
        const T* A = static_cast<const T*>(p.A);
        T* B = static_cast<T*>(p.B);
        // neighbour coordinates (periodic)
        const int cx[3] = {x == 0 ? p.nx - 1 : x - 1, x, x == p.nx - 1 ? 0 : x + 1};
        const int ry[3] = {(y == 0 ? p.ny - 1 : y - 1) * p.nxp, y * p.nxp,
                           (y == p.ny - 1 ? 0 : y + 1) * p.nxp};
        const int zm = (L::D == 3) ? (z == 0 ? p.nz - 1 : z - 1) : z;
        const int zp = (L::D == 3) ? (z == p.nz - 1 ? 0 : z + 1) : z;
        const int rz[3] = {zm * plane, z * plane, zp * plane};
        const bool pushpull = AA && p.aa_pushpull;
        R d[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int src = rz[1 - L::ez(i)] + ry[1 - L::ey(i)] + cx[1 - L::ex(i)];
            if (!AA)
                d[i] = S::load(A + (size_t)i * p.sq + src, L::w(i));
            else if (pushpull)
                d[i] = S::load(A + (size_t)L::opp(i) * p.sq + src, L::w(i));
            else
                d[i] = S::load(A + (size_t)i * p.sq + n, L::w(i));
        }
        if (MASK && (fl & FLAG_NEAR_WALL)) {
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const int src = rz[1 - L::ez(i)] + ry[1 - L::ey(i)] + cx[1 - L::ex(i)];
                if (p.flags[src] & FLAG_SOLID) {
                    if (!AA)
                        d[i] = S::load(A + (size_t)L::opp(i) * p.sq + n, L::w(i));
                    else if (pushpull)
                        d[i] = S::load(A + (size_t)i * p.sq + n, L::w(i));
                    else
                        d[i] = S::load(A + (size_t)L::opp(i) * p.sq + src, L::w(i));
                }
            }
        }
        R rho, v[3];
        double feat[8];
        bool have_feat = false;
        AlphaResult ar{2.0, 0, -1};
        if (MODEL == MODEL_BGK) {
            bgk_collide<L, R>(d, sel<R>(p.omega_f, p.omega), sel<R>(p.F_f[0], p.F[0]),
                              sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]),
                              p.has_force != 0, rho, v);
        } else if (MODEL == MODEL_MRT) {
            if constexpr (L::Q == 19) mrt_collide<R>(d, p, rho, v);
        } else if (MODEL == MODEL_REG || MODEL == MODEL_SMAG) {
            les_collide<L, R, MODEL == MODEL_SMAG>(
                d, sel<R>(p.omega_f, p.omega), sel<R>(p.tau_f, p.tau),
                sel<R>(p.smag_cs2_f, p.smag_cs2), sel<R>(p.F_f[0], p.F[0]),
                sel<R>(p.F_f[1], p.F[1]), sel<R>(p.F_f[2], p.F[2]), p.has_force != 0, rho, v);
        } else {
            ar = elbm_collide<L, R>(d, p, smlp, rho, v, feat, have_feat);
            evals = ar.evals;
            astat = ar.status;
        }
        // destination of population i: own node, slot i (AB); node x + e_i,
        // slot i (AA pull/push); own node, slot opp(i) (AA in place)
        auto dst = [&](int i) -> size_t {
            if (!AA) return (size_t)i * p.sq + n;
            if (pushpull)
                return (size_t)i * p.sq + (rz[1 + L::ez(i)] + ry[1 + L::ey(i)] + cx[1 + L::ex(i)]);
            return (size_t)L::opp(i) * p.sq + n;
        };
        if constexpr (S::kHalf) {
            if (!p.round_nearest) {
                store_node_sr<L, S>(B, d, (unsigned)(n + p.salt_off) * kSaltNode, dst);
            } else {
#pragma unroll
                for (int i = 0; i < L::Q; ++i) S::store(B + dst(i), d[i], L::w(i));
            }
        } else {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) S::store(B + dst(i), d[i], L::w(i));
        }
        if (p.out) {
            static_cast<R*>(p.rho)[n] = rho;
#pragma unroll
            for (int a = 0; a < L::D; ++a) static_cast<R*>(p.u)[a * p.sq + n] = v[a];
            bool bad = !isfinite((float)rho);
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
                for (int k = 0; k < 8; ++k) p.pairs_X[(size_t)slot * 8 + k] = (float)feat[k];
                p.pairs_y[slot] = ar.alpha;
            }
        }
    }
    if (ELBM && p.elbm_ctr) {
        // counters: evals, skipped, clamped, at cap, guarded, updated nodes
        unsigned long long c[6] = {(unsigned long long)evals, astat == ALPHA_SKIP,
                                   astat == ALPHA_CLAMP, astat == ALPHA_NOCONV,
                                   astat == ALPHA_GUARDED, astat >= 0};
        const int lane = threadIdx.x & 31;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int warp = tid >> 5;
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_down_sync(0xffffffffu, c[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 6; ++k) sctr[warp * 6 + k] = c[k];
        __syncthreads();
        if (tid < 6) {
            unsigned long long s = 0;
            const int nw = (blockDim.x * blockDim.y) >> 5;
            for (int w = 0; w < nw; ++w) s += sctr[w * 6 + tid];
            // spread over 64 replicas to limit contention on one address
            const int rep = (blockIdx.x + blockIdx.y * 7 + blockIdx.z * 13) & 63;
            if (s) atomicAdd(&p.elbm_ctr[rep * 8 + tid], s);
            if (tid == 3 && s) atomicOr(p.status, STATUS_NOCONV);
        }
    }
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
        if (mask)
            k_stream_collide<L, S, MODEL, true, false><<<grid, block, 0, s>>>(p);
        else
            k_stream_collide<L, S, MODEL, false, false><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

// lattice: 0 D2Q9, 1 D3Q19; LAT restricts a translation unit to one lattice
// (-1: both).
template <int MODEL, int LAT = -1>
cudaError_t launch_step_model(int lattice, int store, const StepParams& p, bool mask, bool aa,
                              cudaStream_t s)
{
    if (lattice == 0) {
        if constexpr (MODEL != MODEL_MRT && LAT != 1) {
            switch (store) {
            case 0: return launch_step_t<D2Q9, StoreF64, MODEL>(p, mask, aa, s);
            case 1: return launch_step_t<D2Q9, StoreF32, MODEL>(p, mask, aa, s);
            case 2: return launch_step_t<D2Q9, StoreF32S, MODEL>(p, mask, aa, s);
            case 3: return launch_step_t<D2Q9, StoreF16S, MODEL>(p, mask, aa, s);
            case 4: return launch_step_t<D2Q9, StoreBF16S, MODEL>(p, mask, aa, s);
            }
        }
        return cudaErrorInvalidValue;
    }
    if constexpr (LAT != 0) {
        switch (store) {
        case 0: return launch_step_t<D3Q19, StoreF64, MODEL>(p, mask, aa, s);
        case 1: return launch_step_t<D3Q19, StoreF32, MODEL>(p, mask, aa, s);
        case 2: return launch_step_t<D3Q19, StoreF32S, MODEL>(p, mask, aa, s);
        case 3: return launch_step_t<D3Q19, StoreF16S, MODEL>(p, mask, aa, s);
        case 4: return launch_step_t<D3Q19, StoreBF16S, MODEL>(p, mask, aa, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
