// Support kernels around the step: node-type map, equilibrium initialisation,
// field packing to dense caller layout, and deterministic FP64 reductions.
#include "collide.cuh"
#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Node-type map (Sec. 3.4), from the caller's mask (0 fluid, 1 solid, 2 + k a
// boundary node of condition k).  Handles get one 32-bit word per node:
// link mask (bit i set when the upstream node x - e_i is solid), NODE_SOLID,
// condition id + 1 in the top bits.  The batched ensemble gets bytes: bit 0
// solid, bit 1 a fluid node with a solid upstream neighbour.  Exactly one of
// words / flags is non-null.  A mask value above max_code sets *bad.
// dense: [nz][ny][nx]; words and flags: padded rows.
// ---------------------------------------------------------------------------
template <class L>
__global__ void k_flags(const uint8_t* __restrict__ dense, uint32_t* __restrict__ words,
                        uint8_t* __restrict__ flags, int nx, int ny, int nz, int nxp,
                        int max_code, int* __restrict__ bad, unsigned* __restrict__ nearwall_segs,
                        int sector)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= nxp) return;
    const size_t out = ((size_t)z * ny + y) * nxp + x;
    auto put = [&](bool solid, uint32_t lk, int code) {
        if (words)
            words[out] = (solid ? NODE_SOLID : 0u) | lk |
                         (code >= 2 ? (uint32_t)(code - 1) << NODE_BC_SHIFT : 0u);
        else
            flags[out] = (solid ? FLAG_SOLID : 0) | (lk ? FLAG_NEAR_WALL : 0);
    };
    auto at = [&](int xx, int yy, int zz) {
        xx = (xx + nx) % nx;
        yy = (yy + ny) % ny;
        zz = (zz + nz) % nz;
        return dense[((size_t)zz * ny + yy) * nx + xx];
    };
    bool near_wall = false;
    if (x >= nx) {        // padding never updates
        put(true, 0u, 0);
    } else {
        const int code = at(x, y, z);
        if (code > max_code) {
            atomicOr(bad, 1);
            put(true, 0u, 0);
        } else {
            const bool solid = code == 1;
            uint32_t lk = 0;
            if (!solid)
                for (int i = 1; i < L::Q; ++i)
                    if (at(x - L::ex(i), y - L::ey(i), z - L::ez(i)) == 1) lk |= 1u << i;
            if (solid && words && sector > 1) {
                // rest-state fill of a solid node whose sector holds a fluid node
                const int x0 = x & ~(sector - 1), x1 = min(x0 + sector, nx);
                for (int xx = x0; xx < x1; ++xx)
                    if (at(xx, y, z) != 1) { lk = NODE_FILL; break; }
            }
            put(solid, lk, code);
            near_wall = !solid && lk != 0;
        }
    }
    // count the 32-node row segments (one warp of the step kernel) that hold
    // a fluid node with a solid neighbour; nxp is a multiple of 32 when this
    // is requested, so every warp here is complete
    if (nearwall_segs) {
        const unsigned b = __ballot_sync(0xffffffffu, near_wall);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(nearwall_segs, 1u);
    }
}

cudaError_t launch_flags(int lattice, const uint8_t* dense, uint32_t* words, uint8_t* flags,
                         int nx, int ny, int nz, int nxp, int max_code, int* bad,
                         unsigned* nearwall_segs, int sector, cudaStream_t s)
{
    if (sector & (sector - 1)) return cudaErrorInvalidValue;
    if (nearwall_segs && nxp % 32 != 0) return cudaErrorInvalidValue;
    dim3 block(128), grid((nxp + 127) / 128, ny, nz);
    switch (lattice) {
    case 0: k_flags<D2Q9><<<grid, block, 0, s>>>(dense, words, flags, nx, ny, nz, nxp, max_code, bad, nearwall_segs, sector); break;
    case 1: k_flags<D3Q19><<<grid, block, 0, s>>>(dense, words, flags, nx, ny, nz, nxp, max_code, bad, nearwall_segs, sector); break;
    case 2: k_flags<D3Q15><<<grid, block, 0, s>>>(dense, words, flags, nx, ny, nz, nxp, max_code, bad, nearwall_segs, sector); break;
    case 3: k_flags<D3Q27><<<grid, block, 0, s>>>(dense, words, flags, nx, ny, nz, nxp, max_code, bad, nearwall_segs, sector); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// F = f_eq(rho, u) (polynomial, or the entropic form for ELBM) at every node.
// rho [nz][ny][nx], u [D][nz][ny][nx] dense, element type FT.
// ---------------------------------------------------------------------------
// opp != 0 stores f_eq_i in slot opp(i) (the AA pattern's in-place placement,
// which the first AA step, a pull/push step, reads).
template <class L, class S, class FT>
__global__ void k_init(const FT* __restrict__ rho, const FT* __restrict__ u, void* Aout, int nx,
                       int ny, int nz, int nxp, long long sq, int entropic, int feq_variant,
                       int opp)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= nxp) return;
    typename S::T* A = static_cast<typename S::T*>(Aout);
    const size_t n = ((size_t)z * ny + y) * nxp + x;
    double r = 1.0, uu[3] = {0, 0, 0};
    if (x < nx) {
        const size_t nd = ((size_t)z * ny + y) * nx + x;
        const size_t N = (size_t)nx * ny * nz;
        r = (double)rho[nd];
        for (int a = 0; a < L::D; ++a) uu[a] = (double)u[a * N + nd];
    }
    using R = typename S::R;
    if (entropic) {
        double dev[L::Q];   // f_eq - w, FP64 (the entropic form is only used by ELBM)
        elbm_feq<L>(r, uu, feq_variant, dev);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            A[(size_t)(opp ? L::opp(i) : i) * sq + n] = S::encode((R)(dev[i] - L::w(i)), L::w(i));
    } else {
        // Eq. equilibrium in deviation form, w (rho - 1 + rho (3 eu + 9/2 eu^2 - 3/2 u^2)),
        // in the storage's compute type (FP64 arithmetic runs at a small
        // fraction of the FP32 rate on this GPU)
        const R rr = (R)r, dr = (R)(r - 1.0);
        const R u0 = (R)uu[0], u1 = (R)uu[1], u2 = (R)uu[2];
        const R usq = u0 * u0 + u1 * u1 + u2 * u2;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const R eu = L::ex(i) * u0 + L::ey(i) * u1 + L::ez(i) * u2;
            const R dev = (R)L::w(i) * (dr + rr * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq));
            A[(size_t)(opp ? L::opp(i) : i) * sq + n] = S::encode(dev, L::w(i));
        }
    }
}

template <class L, class S>
static cudaError_t init_t(const void* rho, const void* u, int field_f32, void* A, int nx, int ny,
                          int nz, int nxp, long long sq, int entropic, int feq_variant, int opp,
                          cudaStream_t s)
{
    dim3 block(128), grid((nxp + 127) / 128, ny, nz);
    if (field_f32)
        k_init<L, S, float><<<grid, block, 0, s>>>((const float*)rho, (const float*)u, A, nx, ny,
                                                   nz, nxp, sq, entropic, feq_variant, opp);
    else
        k_init<L, S, double><<<grid, block, 0, s>>>((const double*)rho, (const double*)u, A, nx,
                                                    ny, nz, nxp, sq, entropic, feq_variant, opp);
    return cudaGetLastError();
}

template <class L>
static cudaError_t init_l(int store, const void* rho, const void* u, int field_f32, void* A,
                          int nx, int ny, int nz, int nxp, long long sq, int entropic,
                          int feq_variant, int opp, cudaStream_t s)
{
    switch (store) {
    case 0: return init_t<L, StoreF64>(rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic, feq_variant, opp, s);
    case 1: return init_t<L, StoreF32>(rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic, feq_variant, opp, s);
    case 2: return init_t<L, StoreF32S>(rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic, feq_variant, opp, s);
    case 3: return init_t<L, StoreF16S>(rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic, feq_variant, opp, s);
    case 4: return init_t<L, StoreBF16S>(rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic, feq_variant, opp, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init(int lattice, int store, const void* rho, const void* u, int field_f32,
                        void* A, int nx, int ny, int nz, int nxp, long long sq, int entropic,
                        int feq_variant, int opposite_slots, cudaStream_t s)
{
    switch (lattice) {
    case 0: return init_l<D2Q9>(store, rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic,
                                feq_variant, opposite_slots, s);
    case 1: return init_l<D3Q19>(store, rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic,
                                 feq_variant, opposite_slots, s);
    case 2: return init_l<D3Q15>(store, rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic,
                                 feq_variant, opposite_slots, s);
    case 3: return init_l<D3Q27>(store, rho, u, field_f32, A, nx, ny, nz, nxp, sq, entropic,
                                 feq_variant, opposite_slots, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Padded compute-type field -> dense caller field (F32 or F64).
// nfields consecutive planes spaced sq apart in src, N apart in dst; `add`
// is added in FP64 before the conversion (1 for the rho field, which holds
// the deviation rho - 1; 0 otherwise).
// ---------------------------------------------------------------------------
template <class RT, class OT>
__global__ void k_pack(const RT* __restrict__ src, OT* __restrict__ dst, int nfields, int nx,
                       int ny, int nz, int nxp, long long sq, double add)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= nx) return;
    const size_t N = (size_t)nx * ny * nz;
    const size_t nd = ((size_t)z * ny + y) * nx + x;
    const size_t n = ((size_t)z * ny + y) * nxp + x;
    for (int f = 0; f < nfields; ++f) dst[f * N + nd] = (OT)((double)src[f * sq + n] + add);
}

cudaError_t launch_pack(int src_f64, const void* src, int dst_f32, void* dst, int nfields, int nx,
                        int ny, int nz, int nxp, long long sq, double add, cudaStream_t s)
{
    dim3 block(128), grid((nx + 127) / 128, ny, nz);
    if (src_f64) {
        if (dst_f32)
            k_pack<double, float><<<grid, block, 0, s>>>((const double*)src, (float*)dst, nfields,
                                                         nx, ny, nz, nxp, sq, add);
        else
            k_pack<double, double><<<grid, block, 0, s>>>((const double*)src, (double*)dst,
                                                          nfields, nx, ny, nz, nxp, sq, add);
    } else {
        if (dst_f32)
            k_pack<float, float><<<grid, block, 0, s>>>((const float*)src, (float*)dst, nfields,
                                                        nx, ny, nz, nxp, sq, add);
        else
            k_pack<float, double><<<grid, block, 0, s>>>((const float*)src, (double*)dst,
                                                         nfields, nx, ny, nz, nxp, sq, add);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic FP64 sums over fluid nodes: mass, momentum (D), kinetic
// energy.  Pass 1: a fixed grid of kReduceBlocks CTAs, each striding over
// rows in a fixed order and reducing in a fixed tree -> partials.  Pass 2:
// one CTA sums the partials in a fixed tree.  Bitwise reproducible.
// ---------------------------------------------------------------------------
template <class RT>
__global__ void __launch_bounds__(256) k_reduce_partial(const RT* __restrict__ rho,
                                                        const RT* __restrict__ u,
                                                        const uint32_t* __restrict__ nodes, int D,
                                                        int nx, int ny, int nz, int nxp,
                                                        long long sq, double* __restrict__ part)
{
    __shared__ double sh[256][5];
    double acc[5] = {0, 0, 0, 0, 0};
    const long long rows = (long long)ny * nz;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long base = r * nxp;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long n = base + x;
            if (nodes && (nodes[n] & NODE_SOLID)) continue;
            const double rr = 1.0 + (double)rho[n];   // the field holds rho - 1
            double ke = 0;
            acc[0] += rr;
            for (int a = 0; a < D; ++a) {
                const double va = (double)u[a * sq + n];
                acc[1 + a] += rr * va;
                ke += va * va;
            }
            acc[1 + D] += 0.5 * rr * ke;
        }
    }
    for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = sh[0][threadIdx.x];
}

__global__ void __launch_bounds__(256) k_reduce_final(const double* __restrict__ part,
                                                      int nblocks, double* __restrict__ out)
{
    __shared__ double sh[256][5];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 5; ++k) acc[k] += part[b * 5 + k];
    for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[0][threadIdx.x];
}

cudaError_t launch_reduce(int f64, const void* rho, const void* u, const uint32_t* nodes, int D,
                          int nx, int ny, int nz, int nxp, long long sq, double* partials,
                          double* out, cudaStream_t s)
{
    if (f64)
        k_reduce_partial<double><<<kReduceBlocks, 256, 0, s>>>(
            (const double*)rho, (const double*)u, nodes, D, nx, ny, nz, nxp, sq, partials);
    else
        k_reduce_partial<float><<<kReduceBlocks, 256, 0, s>>>(
            (const float*)rho, (const float*)u, nodes, D, nx, ny, nz, nxp, sq, partials);
    k_reduce_final<<<1, 256, 0, s>>>(partials, kReduceBlocks, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Kinetic energy and enstrophy (Sec. 5.2 diagnostics): per-row partial sums
// of |v|^2 and |curl v|^2 (second-order central differences, periodic wrap),
// then one CTA combines the partials in a fixed tree and normalises by 2N.
// ---------------------------------------------------------------------------
template <class RT>
__global__ void __launch_bounds__(256) k_diag_partial(const RT* __restrict__ u, int D, int nx,
                                                     int ny, int nz, int nxp, long long sq,
                                                     double* __restrict__ part)
{
    __shared__ double sh[256][2];
    double e = 0, om = 0;
    const long long rows = (long long)ny * nz;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
        const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
        const long long c = r * nxp;
        const long long cyp = ((long long)z * ny + yp) * nxp, cym = ((long long)z * ny + ym) * nxp;
        const long long czp = ((long long)zp * ny + y) * nxp, czm = ((long long)zm * ny + y) * nxp;
        const RT* ux = u;
        const RT* uy = u + sq;
        const RT* uz = u + 2 * sq;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
            const double vx = ux[c + x], vy = uy[c + x];
            const double vz = D == 3 ? (double)uz[c + x] : 0.0;
            e += vx * vx + vy * vy + vz * vz;
            const double dxvy = 0.5 * ((double)uy[c + xp] - (double)uy[c + xm]);
            const double dyvx = 0.5 * ((double)ux[cyp + x] - (double)ux[cym + x]);
            const double wz = dxvy - dyvx;
            double w2 = wz * wz;
            if (D == 3) {
                const double dyvz = 0.5 * ((double)uz[cyp + x] - (double)uz[cym + x]);
                const double dzvy = 0.5 * ((double)uy[czp + x] - (double)uy[czm + x]);
                const double dzvx = 0.5 * ((double)ux[czp + x] - (double)ux[czm + x]);
                const double dxvz = 0.5 * ((double)uz[c + xp] - (double)uz[c + xm]);
                const double wx = dyvz - dzvy, wy = dzvx - dxvz;
                w2 += wx * wx + wy * wy;
            }
            om += w2;
        }
    }
    sh[threadIdx.x][0] = e;
    sh[threadIdx.x][1] = om;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[threadIdx.x][0] += sh[threadIdx.x + s][0];
            sh[threadIdx.x][1] += sh[threadIdx.x + s][1];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) part[blockIdx.x * 2 + threadIdx.x] = sh[0][threadIdx.x];
}

__global__ void __launch_bounds__(256) k_diag_final(const double* __restrict__ part, int nblocks,
                                                   double inv2n, double* __restrict__ out)
{
    __shared__ double sh[256][2];
    double acc[2] = {0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        acc[0] += part[b * 2];
        acc[1] += part[b * 2 + 1];
    }
    sh[threadIdx.x][0] = acc[0];
    sh[threadIdx.x][1] = acc[1];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[threadIdx.x][0] += sh[threadIdx.x + s][0];
            sh[threadIdx.x][1] += sh[threadIdx.x + s][1];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) out[threadIdx.x] = sh[0][threadIdx.x] * inv2n;
}

cudaError_t launch_diagnostics(int f64, const void* u, int D, int nx, int ny, int nz, int nxp,
                               long long sq, double* partials, double* out, cudaStream_t s)
{
    if (f64)
        k_diag_partial<double><<<kReduceBlocks, 256, 0, s>>>((const double*)u, D, nx, ny, nz, nxp,
                                                             sq, partials);
    else
        k_diag_partial<float><<<kReduceBlocks, 256, 0, s>>>((const float*)u, D, nx, ny, nz, nxp,
                                                            sq, partials);
    k_diag_final<<<1, 256, 0, s>>>(partials, kReduceBlocks,
                                   0.5 / ((double)nx * (double)ny * (double)nz), out);
    return cudaGetLastError();
}

// Sum the 64 replicas of the ELBM counters into 6 values.
// Combine the counter replicas: out[0..5] counts, out[6] residual sum,
// out[7] residual max, out[8] residual samples.
__global__ void k_sum_ctr(const unsigned long long* __restrict__ rep, double* __restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= 9) return;
    if (k == 6) {
        double s = 0;
        for (int r = 0; r < kCtrReplicas; ++r) s += __longlong_as_double(rep[r * kCtrStride + 6]);
        out[6] = s;
    } else if (k == 7) {
        double m = 0;
        for (int r = 0; r < kCtrReplicas; ++r)
            m = fmax(m, __longlong_as_double(rep[r * kCtrStride + 7]));
        out[7] = m;
    } else {
        unsigned long long s = 0;
        for (int r = 0; r < kCtrReplicas; ++r) s += rep[r * kCtrStride + k];
        out[k] = (double)s;
    }
}

cudaError_t launch_sum_ctr(const unsigned long long* rep, double* out, cudaStream_t s)
{
    k_sum_ctr<<<1, 32, 0, s>>>(rep, out);
    return cudaGetLastError();
}

}  // namespace lbm
