// Host runtime and C ABI of the single-domain simulation (include/lbm.h).
//
// A handle owns one device arena (allocated here, or bound by the caller):
//   A, B      two copies of the distributions (AB pattern, Sec. 3.3),
//             [q][z][y][x] structure of arrays, x padded to a multiple of 32
//             elements and direction planes padded to 128 elements
//   flags     node-type map, one byte per (padded) node
//   rho, u    macroscopic output fields in the compute type, padded layout
//             (the rho field holds rho - 1; readback adds 1 in FP64)
//   alpha     ELBM per-node alpha (FP64), ELBM handles only
//   misc      status word, ELBM counters, reduction scratch, MLP parameters
//   stage     dense staging for host transfers and dtype conversion
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "collide.cuh"
#include "lbm_internal.h"

using namespace lbm;

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0, lattice = 0, model = 0, dtype = 0, D = 0, Q = 0;
    double tau = 1.0;
    int nxp = 0;
    long long sq = 0;       // elements per direction plane (padded)
    long long N = 0;        // dense node count
    size_t esize = 0;       // storage element size
    size_t rsize = 0;       // compute (output field) element size
    // arena
    char* base = nullptr;
    size_t bytes = 0;
    bool owned = false;
    size_t off_A = 0, off_B = 0, off_nodes = 0, off_rho = 0, off_u = 0, off_alpha = 0,
           off_misc = 0, off_part = 0, off_mlp = 0, off_stage = 0, stage_bytes = 0;
    int cur = 0;            // 0: state in A, 1: state in B
    bool has_mask = false, inited = false, have_out = false;
    cudaStream_t stream = nullptr;
    double F[3] = {0, 0, 0};
    double s[19];
    int alpha_mode = LBM_ALPHA_NEWTON, max_iter = 20, guard_steps = 2, feq_variant = 0;
    double tol = 1e-12, skip_eps = 1e-3, guard_tol = 1e-6;
    double smag_cs = 0.1;   // Smagorinsky constant C_S
    BCEntry bc[kMaxBC] = {};  // velocity / pressure boundary conditions by id
    bool mlp_loaded = false, alpha_out = false, use_graph = false, round_nearest = false;
    bool aa = false;        // AA access pattern (one distribution array)
    bool elbm_diag = false; // ELBM entropy-condition residual accumulation
    // masked AB steps on 3-D lattices: 0 choose from the geometry, 1 one node
    // per thread, 2 z runs; zrun_pick is the choice for the current geometry
    int masked_kernel = 0;
    bool zrun_pick = false;
    double nearwall_frac = 0.0;  // 32-node row segments with a near-wall fluid node
    long long t = 0, launches = 0;
    unsigned clk_host[2] = {0, 0};   // source of the clock copy in lbm_set_state
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    std::string err;
};

// misc block layout (bytes from off_misc)
enum : size_t {
    MISC_STATUS = 0,        // uint32 status bits
    MISC_PAIRS = 8,         // int pairs counter
    MISC_BAD = 16,          // int: mask value out of range
    MISC_NEARWALL = 20,     // unsigned: near-wall row segments (geometry statistics)
    MISC_STEP = 32,         // 2 unsigned: time-step clock of the stochastic rounding
    MISC_RED = 64,          // 5 doubles reduction result
    MISC_CTR_OUT = 128,     // 9 doubles: combined counters
    MISC_CTR = 256,         // kCtrReplicas x kCtrStride unsigned long long counter replicas
    MISC_BYTES = 256 + kCtrReplicas * kCtrStride * 8
};

static thread_local std::string g_err;

static void drop_graphs(lbm_ctx* h)
{
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

static int fail(lbm_ctx* h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_err = buf;
    return code;
}

static int cuda_fail(lbm_ctx* h, cudaError_t e, const char* what)
{
    return fail(h, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call, what)                                      \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, (what)); \
    } while (0)

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void default_rates(double tau, double* s)
{
    for (int k = 0; k < 19; ++k) s[k] = 0.0;
    const double w = 1.0 / tau;
    s[1] = 1.19;
    s[2] = 1.4;
    s[4] = s[6] = s[8] = 1.2;
    s[9] = s[11] = s[13] = s[14] = s[15] = w;
    s[10] = s[12] = 1.4;
    s[16] = s[17] = s[18] = 1.98;
}

static void layout(lbm_ctx* h)
{
    size_t o = 0;
    const size_t dist = (size_t)h->Q * h->sq * h->esize;
    h->off_A = o; o = align256(o + dist);
    h->off_B = o;
    if (!h->aa) o = align256(o + dist);   // AA: a single array
    h->off_nodes = o; o = align256(o + (size_t)h->sq * 4);
    h->off_rho = o; o = align256(o + (size_t)h->sq * h->rsize);
    h->off_u = o; o = align256(o + (size_t)h->D * h->sq * h->rsize);
    h->off_alpha = o;
    if (h->model == LBM_ELBM) o = align256(o + (size_t)h->sq * 8);
    h->off_misc = o; o = align256(o + MISC_BYTES);
    h->off_part = o; o = align256(o + (size_t)kReduceBlocks * 5 * 8);
    h->off_mlp = o; o = align256(o + MLP_NPARAM * 4);
    h->off_stage = o;
    h->stage_bytes = align256((size_t)h->N * (1 + h->D) * 8);
    o = align256(o + h->stage_bytes);
    h->bytes = o;
}

template <class T>
static T* at(lbm_ctx* h, size_t off) { return reinterpret_cast<T*>(h->base + off); }

static std::atomic<int> g_fail_allocs{0};

namespace lbm {
// An address the kernels can use for p: p itself for device or managed
// memory, the mapped device address of pinned host memory (read or written
// in place over the CPU-GPU link, no staging copy), or nullptr for pageable
// host memory, which goes through a staging area.
const void* kernel_view(const void* p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    return nullptr;
}

cudaError_t dev_alloc(void** p, size_t bytes)
{
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}
}  // namespace lbm

static int ensure_memory(lbm_ctx* h)
{
    if (h->base) return LBM_OK;
    void* p = nullptr;
    cudaError_t e = dev_alloc(&p, h->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LBM_ENOMEM, "cudaMalloc(%zu bytes): %s", h->bytes, cudaGetErrorString(e));
    }
    h->base = static_cast<char*>(p);
    h->owned = true;
    CK(h, cudaMemsetAsync(h->base + h->off_misc, 0, MISC_BYTES, h->stream), "clear status");
    CK(h, cudaMemsetAsync(h->base + h->off_nodes, 0, (size_t)h->sq * 4, h->stream), "clear node words");
    return LBM_OK;
}

static int read_status(lbm_ctx* h, unsigned* st)
{
    CK(h, cudaMemcpyAsync(st, h->base + h->off_misc + MISC_STATUS, 4, cudaMemcpyDeviceToHost,
                          h->stream),
       "read status");
    CK(h, cudaStreamSynchronize(h->stream), "synchronise");
    return LBM_OK;
}

static int sync_status(lbm_ctx* h)
{
    if (!h->base) {
        CK(h, cudaStreamSynchronize(h->stream), "synchronise");
        return LBM_OK;
    }
    unsigned st = 0;
    int r = read_status(h, &st);
    if (r) return r;
    if (st & STATUS_NAN) return fail(h, LBM_ENAN, "non-finite rho or v on an output step");
    return LBM_OK;
}

template <int LAT>
static cudaError_t elbm_dispatch(int store, const StepParams& p, bool mask, bool aa,
                                 cudaStream_t s)
{
    switch (kElbmStoreGroup[store]) {
    case 1u: return launch_step_elbm_part<LAT, 1u>(store, p, mask, aa, s);
    case 6u: return launch_step_elbm_part<LAT, 6u>(store, p, mask, aa, s);
    default: return launch_step_elbm_part<LAT, 24u>(store, p, mask, aa, s);
    }
}

extern "C" {

int lbm_create(int nx, int ny, int nz, int lattice, int model, double tau, int dtype,
               lbm_handle* out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1)
        return fail(nullptr, LBM_EINVAL, "sizes must be >= 1 (got %d x %d x %d)", nx, ny, nz);
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q15 &&
        lattice != LBM_D3Q27)
        return fail(nullptr, LBM_EINVAL, "unknown lattice %d", lattice);
    if (lattice == LBM_D2Q9 && nz != 1)
        return fail(nullptr, LBM_EINVAL, "D2Q9 needs nz = 1 (got %d)", nz);
    if (model != LBM_BGK && model != LBM_MRT && model != LBM_ELBM && model != LBM_REG &&
        model != LBM_SMAG)
        return fail(nullptr, LBM_EINVAL, "unknown model %d", model);
    if (model == LBM_MRT && lattice != LBM_D3Q19)
        return fail(nullptr, LBM_EINVAL, "MRT is implemented for D3Q19 only");
    if (dtype < LBM_F64 || dtype > LBM_BF16S)
        return fail(nullptr, LBM_EINVAL, "unknown dtype %d", dtype);
    if (!(tau > 0.5) || !(tau < 1e6))
        return fail(nullptr, LBM_EINVAL, "tau must be > 1/2 (got %g)", tau);
    const long long nxp = ((long long)nx + 31) / 32 * 32;
    long long sq = nxp * ny * nz;
    sq = (sq + 127) / 128 * 128;
    if (sq > 0x7fffffffLL - 1024)
        return fail(nullptr, LBM_EINVAL, "domain too large: %lld padded nodes > 2^31", sq);
    lbm_ctx* h = new lbm_ctx();
    h->nx = nx; h->ny = ny; h->nz = nz;
    h->lattice = lattice; h->model = model; h->dtype = dtype; h->tau = tau;
    h->D = lattice == LBM_D2Q9 ? 2 : 3;
    h->Q = lattice == LBM_D2Q9 ? 9 : (lattice == LBM_D3Q19 ? 19 : (lattice == LBM_D3Q15 ? 15 : 27));
    h->nxp = (int)nxp;
    h->sq = sq;
    h->N = (long long)nx * ny * nz;
    h->esize = dtype == LBM_F64 ? 8 : (dtype == LBM_F32 || dtype == LBM_F32S) ? 4 : 2;
    h->rsize = dtype == LBM_F64 ? 8 : 4;
    default_rates(tau, h->s);
    layout(h);
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h)
{
    if (!h) return LBM_OK;
    drop_graphs(h);
    if (h->owned && h->base) cudaFree(h->base);
    delete h;
    return LBM_OK;
}

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

size_t lbm_required_bytes(lbm_handle h) { return h ? h->bytes : 0; }

int lbm_bind_memory(lbm_handle h, void* dev_ptr, size_t bytes)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->base) return fail(h, LBM_ESTATE, "memory already in use");
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
        return fail(h, LBM_EINVAL, "bound memory must be non-NULL and 256-byte aligned");
    if (bytes < h->bytes)
        return fail(h, LBM_ENOMEM, "bound memory too small: %zu < %zu bytes", bytes, h->bytes);
    if (!is_device_ptr(dev_ptr)) return fail(h, LBM_EINVAL, "bound memory is not device memory");
    h->base = static_cast<char*>(dev_ptr);
    h->owned = false;
    CK(h, cudaMemsetAsync(h->base + h->off_misc, 0, MISC_BYTES, h->stream), "clear status");
    CK(h, cudaMemsetAsync(h->base + h->off_nodes, 0, (size_t)h->sq * 4, h->stream), "clear node words");
    return LBM_OK;
}

int lbm_debug_fail_allocations(int n)
{
    if (n < 0) return fail(nullptr, LBM_EINVAL, "allocation count %d is negative", n);
    g_fail_allocs.store(n);
    return LBM_OK;
}

int lbm_set_stream(lbm_handle h, void* stream)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->stream != static_cast<cudaStream_t>(stream)) drop_graphs(h);
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

int lbm_set_geometry(lbm_handle h, const uint8_t* mask)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!mask) return fail(h, LBM_EINVAL, "mask is NULL");
    if (h->inited) return fail(h, LBM_ESTATE, "set the geometry before lbm_init_equilibrium");
    int r = ensure_memory(h);
    if (r) return r;
    uint8_t* stage = at<uint8_t>(h, h->off_stage);
    const bool dev = is_device_ptr(mask);
    CK(h, cudaMemcpyAsync(stage, mask, (size_t)h->N,
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream),
       "copy mask");
    int* bad = at<int>(h, h->off_misc + MISC_BAD);
    unsigned* nw = at<unsigned>(h, h->off_misc + MISC_NEARWALL);
    CK(h, cudaMemsetAsync(bad, 0, 2 * sizeof(int), h->stream), "clear mask check");
    CK(h, launch_flags(h->lattice, stage, at<uint32_t>(h, h->off_nodes), nullptr, h->nx, h->ny,
                       h->nz, h->nxp, 1 + kMaxBC, bad, nw,
                       h->aa ? 0 : (int)(32 / h->esize), h->stream),
       "node-type map kernel");
    h->launches += 1;
    int hbad[2] = {0, 0};
    CK(h, cudaMemcpyAsync(hbad, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream),
       "read mask check");
    CK(h, cudaStreamSynchronize(h->stream), "synchronise");
    if (hbad[0]) return fail(h, LBM_EINVAL, "mask values are 0, 1 or 2..%d", 1 + kMaxBC);
    h->has_mask = true;
    const double segs = (double)((h->nx + 31) / 32) * h->ny * h->nz;
    h->nearwall_frac = (unsigned)hbad[1] / segs;
    // Near-wall nodes of the one-node kernel wait for their node word before
    // reloading their bounced populations: a second memory round trip for
    // every warp holding one.  The z-run kernel knows the word beforehand;
    // it pays off where such warps are common (sphere duct: 62% of the
    // segments, FP16S +24%) and loses ~2% where they are not (cavity: 27%).
    h->zrun_pick = h->nearwall_frac > 0.4;
    return LBM_OK;
}

int lbm_set_masked_kernel(lbm_handle h, int mode)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (mode < 0 || mode > 2) return fail(h, LBM_EINVAL, "masked kernel mode is 0, 1 or 2");
    if (h->masked_kernel != mode) drop_graphs(h);
    h->masked_kernel = mode;
    return LBM_OK;
}

int lbm_get_nearwall_fraction(lbm_handle h, double* frac)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!frac) return fail(h, LBM_EINVAL, "frac is NULL");
    if (!h->has_mask) return fail(h, LBM_ESTATE, "no geometry set");
    *frac = h->nearwall_frac;
    return LBM_OK;
}

int lbm_set_force(lbm_handle h, double fx, double fy, double fz)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(fz))
        return fail(h, LBM_EINVAL, "force must be finite");
    if (h->D == 2 && fz != 0.0) return fail(h, LBM_EINVAL, "D2Q9 force has no z component");
    h->F[0] = fx; h->F[1] = fy; h->F[2] = fz;
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_mrt_rates(lbm_handle h, const double* s, int q)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->model != LBM_MRT) return fail(h, LBM_EINVAL, "not an MRT handle");
    if (!s || q != 19) return fail(h, LBM_EINVAL, "need 19 rates");
    for (int k = 0; k < 19; ++k) {
        if (!std::isfinite(s[k])) return fail(h, LBM_EINVAL, "rate %d not finite", k);
        h->s[k] = s[k];
    }
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_boundary(lbm_handle h, int id, int kind, int method, int normal,
                     const double* value)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (id < 0 || id >= kMaxBC) return fail(h, LBM_EINVAL, "condition id must be 0..%d", kMaxBC - 1);
    if (kind != LBM_BC_VELOCITY && kind != LBM_BC_PRESSURE)
        return fail(h, LBM_EINVAL, "unknown condition kind %d", kind);
    if (method != LBM_BC_EQUILIBRIUM && method != LBM_BC_ZOUHE && method != LBM_BC_REGULARIZED)
        return fail(h, LBM_EINVAL, "unknown condition method %d", method);
    const int ax = normal < 0 ? -normal - 1 : normal - 1;
    if (normal == 0 || ax >= h->D)
        return fail(h, LBM_EINVAL, "normal must be +-1..+-%d (got %d)", h->D, normal);
    if (!value) return fail(h, LBM_EINVAL, "value is NULL");
    const int nv = kind == LBM_BC_VELOCITY ? h->D : 1;
    for (int a = 0; a < nv; ++a)
        if (!std::isfinite(value[a])) return fail(h, LBM_EINVAL, "value must be finite");
    if (kind == LBM_BC_PRESSURE && !(value[0] > 0)) return fail(h, LBM_EINVAL, "rho must be > 0");
    BCEntry& b = h->bc[id];
    b.kind = kind;
    b.method = method;
    b.axis = ax;
    b.sign = normal > 0 ? 1 : -1;
    for (int a = 0; a < 3; ++a) {
        b.val[a] = a < nv ? value[a] : 0.0;
        b.val_f[a] = (float)b.val[a];
    }
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_smagorinsky(lbm_handle h, double cs)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->model != LBM_SMAG) return fail(h, LBM_EINVAL, "not a Smagorinsky handle");
    if (!std::isfinite(cs) || cs < 0) return fail(h, LBM_EINVAL, "C_S must be finite and >= 0");
    h->smag_cs = cs;
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_elbm(lbm_handle h, int alpha_mode, double tol, int max_iter, double skip_eps)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->model != LBM_ELBM) return fail(h, LBM_EINVAL, "not an ELBM handle");
    if (alpha_mode < 0 || alpha_mode > 4) return fail(h, LBM_EINVAL, "bad alpha mode");
    if (!(tol > 0) || max_iter < 1 || max_iter > 200 || !(skip_eps >= 0))
        return fail(h, LBM_EINVAL, "bad tolerance / iteration cap / skip threshold");
    h->alpha_mode = alpha_mode; h->tol = tol; h->max_iter = max_iter; h->skip_eps = skip_eps;
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_elbm_guard(lbm_handle h, int guard_steps, double guard_tol)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (guard_steps < 1 || guard_steps > 4 || !(guard_tol > 0))
        return fail(h, LBM_EINVAL, "guard_steps must be 1..4 and guard_tol > 0");
    h->guard_steps = guard_steps; h->guard_tol = guard_tol;
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_elbm_feq(lbm_handle h, int variant)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (variant != 0 && variant != 1) return fail(h, LBM_EINVAL, "variant must be 0 or 1");
    if (h->inited) return fail(h, LBM_ESTATE, "choose the equilibrium before initialising");
    h->feq_variant = variant;
    return LBM_OK;
}

int lbm_load_alpha_mlp(lbm_handle h, const float* params, int n)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!params || n != MLP_NPARAM) return fail(h, LBM_EINVAL, "need %d parameters", MLP_NPARAM);
    int r = ensure_memory(h);
    if (r) return r;
    float host[MLP_NPARAM];
    if (is_device_ptr(params)) {
        CK(h, cudaMemcpy(host, params, sizeof host, cudaMemcpyDeviceToHost), "copy parameters");
    } else {
        std::memcpy(host, params, sizeof host);
    }
    // weight matrices and biases (entries 16 .. 1392) rounded to BF16
    for (int k = 16; k < MLP_NPARAM - 1; ++k)
        host[k] = __bfloat162float(__float2bfloat16_rn(host[k]));
    CK(h, cudaMemcpy(h->base + h->off_mlp, host, sizeof host, cudaMemcpyHostToDevice),
       "upload parameters");
    h->mlp_loaded = true;
    return LBM_OK;
}

int lbm_set_alpha_output(lbm_handle h, int on)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->model != LBM_ELBM) return fail(h, LBM_EINVAL, "alpha output needs an ELBM handle");
    h->alpha_out = on != 0;
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_access_pattern(lbm_handle h, int pattern)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (pattern != LBM_PATTERN_AB && pattern != LBM_PATTERN_AA)
        return fail(h, LBM_EINVAL, "unknown access pattern %d", pattern);
    if (h->base) return fail(h, LBM_ESTATE, "choose the access pattern before memory is in use");
    h->aa = (pattern == LBM_PATTERN_AA);
    layout(h);
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_rounding(lbm_handle h, int mode)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (mode != LBM_ROUND_DITHER && mode != LBM_ROUND_NEAREST)
        return fail(h, LBM_EINVAL, "unknown rounding mode %d", mode);
    h->round_nearest = (mode == LBM_ROUND_NEAREST);
    drop_graphs(h);
    return LBM_OK;
}

int lbm_set_graph(lbm_handle h, int on)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    h->use_graph = on != 0;
    return LBM_OK;
}

int lbm_init_equilibrium(lbm_handle h, const void* rho, const void* u, int field_dtype)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!rho || !u) return fail(h, LBM_EINVAL, "rho and u must be non-NULL");
    if (field_dtype != LBM_FIELD_F64 && field_dtype != LBM_FIELD_F32)
        return fail(h, LBM_EINVAL, "unknown field dtype %d", field_dtype);
    int r = ensure_memory(h);
    if (r) return r;
    const size_t fs = field_dtype == LBM_FIELD_F64 ? 8 : 4;
    const size_t nb = (size_t)h->N * fs;
    const void* drho = lbm::kernel_view(rho);
    const void* du = lbm::kernel_view(u);
    char* stage = at<char>(h, h->off_stage);
    // host memory (pinned: read in place; pageable: staged) is released to the
    // caller only after the init kernel has read it
    const bool host_in = !is_device_ptr(rho) || !is_device_ptr(u);
    if (!drho) {
        CK(h, cudaMemcpyAsync(stage, rho, nb, cudaMemcpyHostToDevice, h->stream), "copy rho");
        drho = stage;
    }
    if (!du) {
        CK(h, cudaMemcpyAsync(stage + nb, u, nb * h->D, cudaMemcpyHostToDevice, h->stream),
           "copy u");
        du = stage + nb;
    }
    CK(h, launch_init(h->lattice, h->dtype, drho, du, field_dtype == LBM_FIELD_F32,
                      h->base + h->off_A, h->nx, h->ny, h->nz, h->nxp, h->sq,
                      h->model == LBM_ELBM, h->feq_variant, h->aa ? 1 : 0, h->stream),
       "init kernel");
    h->launches += 1;
    CK(h, cudaMemsetAsync(h->base + h->off_misc, 0, MISC_BYTES, h->stream), "clear status");
    if (host_in) CK(h, cudaStreamSynchronize(h->stream), "synchronise");
    h->cur = 0;
    h->t = 0;
    h->inited = true;
    h->have_out = false;
    return LBM_OK;
}

static StepParams make_params(lbm_ctx* h)
{
    StepParams p;
    std::memset(&p, 0, sizeof p);
    p.nodes = h->has_mask ? at<uint32_t>(h, h->off_nodes) : nullptr;
    p.rho = h->base + h->off_rho;
    p.u = h->base + h->off_u;
    p.alpha_out = (h->model == LBM_ELBM && h->alpha_out) ? at<double>(h, h->off_alpha) : nullptr;
    p.status = at<unsigned>(h, h->off_misc + MISC_STATUS);
    p.elbm_ctr = h->model == LBM_ELBM ? at<unsigned long long>(h, h->off_misc + MISC_CTR)
                                      : nullptr;
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz; p.nxp = h->nxp;
    p.sq = h->sq;
    p.row0 = 0;
    p.nrows = h->D == 3 ? h->nz : h->ny;
    p.zrun = (h->has_mask && h->D == 3 && !h->aa &&
              (h->masked_kernel == 2 || (h->masked_kernel == 0 && h->zrun_pick))) ? 8 : 0;
    p.salt_off = 0;
    // the clock of the stochastic rounding (half-width storage only)
    p.step_ctr = h->esize == 2 ? at<unsigned>(h, h->off_misc + MISC_STEP) : nullptr;
    p.step_slot = 0;
    p.omega = 1.0 / h->tau;
    p.F[0] = h->F[0]; p.F[1] = h->F[1]; p.F[2] = h->F[2];
    p.has_force = (h->F[0] != 0.0 || h->F[1] != 0.0 || h->F[2] != 0.0);
    p.round_nearest = h->round_nearest ? 1 : 0;
    for (int k = 0; k < 19; ++k) {
        const double n2 = h->lattice == LBM_D3Q19 ? (double)mrt_norm2(k) : 1.0;
        p.mrt_c[k] = h->s[k] / n2;
        p.mrt_cf[k] = (1.0 - 0.5 * h->s[k]) / n2;
        p.mrt_c_f[k] = (float)p.mrt_c[k];
        p.mrt_cf_f[k] = (float)p.mrt_cf[k];
    }
    p.omega_f = (float)p.omega;
    p.tau = h->tau;
    for (int k = 0; k < kMaxBC; ++k) p.bc[k] = h->bc[k];
    p.smag_cs2 = h->smag_cs * h->smag_cs;
    p.tau_f = (float)p.tau;
    p.smag_cs2_f = (float)p.smag_cs2;
    for (int a = 0; a < 3; ++a) p.F_f[a] = (float)p.F[a];
    p.alpha_mode = h->alpha_mode; p.max_iter = h->max_iter;
    p.elbm_diag = h->elbm_diag ? 1 : 0;
    p.guard_steps = h->guard_steps; p.feq_variant = h->feq_variant;
    p.tol = h->tol; p.skip_eps = h->skip_eps; p.guard_tol = h->guard_tol;
    p.mlp = at<float>(h, h->off_mlp);
    p.pairs_stride = 1;
    return p;
}

// One step from buffer `from` (AB) or, for the AA pattern, of parity `from`
// (0: pull/push step at even t, 1: in-place step at odd t).
static cudaError_t launch_one(lbm_ctx* h, StepParams& p, int from, bool out)
{
    if (h->aa) {
        p.A = h->base + h->off_A;
        p.B = h->base + h->off_A;
        p.aa_pushpull = (from == 0) ? 1 : 0;
    } else {
        p.A = h->base + (from == 0 ? h->off_A : h->off_B);
        p.B = h->base + (from == 0 ? h->off_B : h->off_A);
        p.aa_pushpull = 0;
    }
    for (int i = 0; i < h->Q; ++i) {
        p.Ap[i] = static_cast<const char*>(p.A) + (size_t)i * h->sq * h->esize;
        p.Bp[i] = static_cast<char*>(p.B) + (size_t)i * h->sq * h->esize;
    }
    p.out = out ? 1 : 0;
    // the clock slot that holds t: AB alternates buffers and slots together
    // (both slots hold t after lbm_set_state, whose state sits in A), AA
    // steps alternate with the parity of t
    p.step_slot = from;
    const bool mask = h->has_mask;
    const bool aa = h->aa;
    const int lat = h->lattice;
    const bool ext = lat == LBM_D3Q15 || lat == LBM_D3Q27;   // built in separate units
    switch (h->model) {
    case LBM_BGK:
        return ext ? launch_step_bgk_q15q27(lat, h->dtype, p, mask, aa, h->stream)
                   : launch_step_bgk(lat, h->dtype, p, mask, aa, h->stream);
    case LBM_MRT: return launch_step_mrt(lat, h->dtype, p, mask, aa, h->stream);
    case LBM_REG:
        return ext ? launch_step_reg_q15q27(lat, h->dtype, p, mask, aa, h->stream)
                   : launch_step_reg(lat, h->dtype, p, mask, aa, h->stream);
    case LBM_SMAG:
        return ext ? launch_step_smag_q15q27(lat, h->dtype, p, mask, aa, h->stream)
                   : launch_step_smag(lat, h->dtype, p, mask, aa, h->stream);
    }
    switch (lat) {
    case LBM_D2Q9: return elbm_dispatch<0>(h->dtype, p, mask, aa, h->stream);
    case LBM_D3Q19: return elbm_dispatch<1>(h->dtype, p, mask, aa, h->stream);
    case LBM_D3Q15: return elbm_dispatch<2>(h->dtype, p, mask, aa, h->stream);
    default: return elbm_dispatch<3>(h->dtype, p, mask, aa, h->stream);
    }
}

static int check_step_ready(lbm_ctx* h)
{
    if (!h->inited) return fail(h, LBM_ESTATE, "lbm_init_equilibrium must precede lbm_step");
    if (h->model == LBM_ELBM && h->alpha_mode == LBM_ALPHA_MLP_GUARDED && !h->mlp_loaded)
        return fail(h, LBM_ESTATE, "MLP alpha mode needs lbm_load_alpha_mlp");
    return LBM_OK;
}

int lbm_step(lbm_handle h, int n)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (n < 1) return fail(h, LBM_EINVAL, "n must be >= 1 (got %d)", n);
    int r = check_step_ready(h);
    if (r) return r;
    StepParams p = make_params(h);
    if (h->use_graph && h->stream != nullptr) {
        auto key = std::make_pair(n, h->cur);
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            cudaGraph_t g;
            CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal),
               "begin capture");
            int from = h->cur;
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < n && le == cudaSuccess; ++k) {
                le = launch_one(h, p, from, k == n - 1);
                from ^= 1;
            }
            cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
            if (le != cudaSuccess) {
                if (ce == cudaSuccess) cudaGraphDestroy(g);
                return cuda_fail(h, le, "launch during capture");
            }
            CK(h, ce, "end capture");
            cudaGraphExec_t ge;
            cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            CK(h, ie, "instantiate graph");
            it = h->graphs.emplace(key, ge).first;
        }
        CK(h, cudaGraphLaunch(it->second, h->stream), "graph launch");
        h->cur ^= (n & 1);
    } else {
        for (int k = 0; k < n; ++k) {
            CK(h, launch_one(h, p, h->cur, k == n - 1), "stream-collide kernel");
            h->cur ^= 1;
        }
    }
    h->launches += n;
    h->t += n;
    h->have_out = true;
    return LBM_OK;
}

int lbm_get_time(lbm_handle h, long long* t)
{
    if (!h || !t) return fail(h, LBM_EINVAL, "NULL argument");
    *t = h->t;
    return LBM_OK;
}

static int get_field(lbm_ctx* h, size_t src_off, int nfields, void* dst, int field_dtype)
{
    const int dst_f32 = field_dtype == LBM_FIELD_F32;
    const size_t fs = dst_f32 ? 4 : 8;
    const size_t nb = (size_t)h->N * fs * nfields;
    // device or pinned host memory is written in place; pageable memory is staged
    void* view = const_cast<void*>(lbm::kernel_view(dst));
    void* out = view ? view : h->base + h->off_stage;
    CK(h, launch_pack(h->rsize == 8, h->base + src_off, dst_f32, out, nfields, h->nx, h->ny,
                      h->nz, h->nxp, h->sq, src_off == h->off_rho ? 1.0 : 0.0, h->stream),
       "pack kernel");
    h->launches += 1;
    if (!view)
        CK(h, cudaMemcpyAsync(dst, out, nb, cudaMemcpyDeviceToHost, h->stream), "copy out");
    return LBM_OK;
}

int lbm_get_macro(lbm_handle h, void* rho, void* u, int field_dtype)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (field_dtype != LBM_FIELD_F64 && field_dtype != LBM_FIELD_F32)
        return fail(h, LBM_EINVAL, "unknown field dtype %d", field_dtype);
    if (!h->have_out) return fail(h, LBM_ESTATE, "no step has produced output yet");
    int r;
    if (rho && (r = get_field(h, h->off_rho, 1, rho, field_dtype))) return r;
    if (u && (r = get_field(h, h->off_u, h->D, u, field_dtype))) return r;
    return sync_status(h);
}

int lbm_get_alpha(lbm_handle h, double* alpha)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!alpha) return fail(h, LBM_EINVAL, "alpha is NULL");
    if (h->model != LBM_ELBM || !h->alpha_out || !h->have_out)
        return fail(h, LBM_ESTATE, "alpha output needs ELBM, lbm_set_alpha_output and a step");
    const bool dev = is_device_ptr(alpha);
    void* out = dev ? (void*)alpha : h->base + h->off_stage;
    CK(h, launch_pack(1, h->base + h->off_alpha, 0, out, 1, h->nx, h->ny, h->nz, h->nxp, h->sq,
                      0.0, h->stream),
       "pack kernel");
    h->launches += 1;
    if (!dev)
        CK(h, cudaMemcpyAsync(alpha, out, (size_t)h->N * 8, cudaMemcpyDeviceToHost, h->stream),
           "copy alpha");
    return sync_status(h);
}

int lbm_reduce(lbm_handle h, double* out)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (!h->have_out) return fail(h, LBM_ESTATE, "no step has produced output yet");
    double* dres = at<double>(h, h->off_misc + MISC_RED);
    CK(h, launch_reduce(h->rsize == 8, h->base + h->off_rho, h->base + h->off_u,
                        h->has_mask ? at<uint32_t>(h, h->off_nodes) : nullptr, h->D, h->nx, h->ny,
                        h->nz, h->nxp, h->sq, at<double>(h, h->off_part), dres, h->stream),
       "reduce kernels");
    h->launches += 2;
    double tmp[5];
    CK(h, cudaMemcpyAsync(tmp, dres, sizeof tmp, cudaMemcpyDeviceToHost, h->stream), "copy sums");
    int r = sync_status(h);
    for (int k = 0; k < h->D + 2; ++k) out[k] = tmp[k];
    return r;
}

int lbm_set_elbm_diagnostics(lbm_handle h, int on)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->model != LBM_ELBM) return fail(h, LBM_EINVAL, "not an ELBM handle");
    int r = ensure_memory(h);
    if (r) return r;
    CK(h, cudaMemsetAsync(h->base + h->off_misc + MISC_CTR, 0,
                          (size_t)kCtrReplicas * kCtrStride * 8, h->stream),
       "clear counters");
    h->elbm_diag = on != 0;
    drop_graphs(h);
    return LBM_OK;
}

int lbm_get_elbm_entropy_error(lbm_handle h, double* out)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (h->model != LBM_ELBM) return fail(h, LBM_EINVAL, "not an ELBM handle");
    int r = ensure_memory(h);
    if (r) return r;
    double* d = at<double>(h, h->off_misc + MISC_CTR_OUT);
    CK(h, launch_sum_ctr(at<unsigned long long>(h, h->off_misc + MISC_CTR), d, h->stream),
       "counter kernel");
    h->launches += 1;
    double tmp[9];
    CK(h, cudaMemcpyAsync(tmp, d, sizeof tmp, cudaMemcpyDeviceToHost, h->stream), "copy");
    r = sync_status(h);
    out[0] = tmp[8] > 0 ? tmp[6] / tmp[8] : 0.0;
    out[1] = tmp[7];
    out[2] = tmp[8];
    return r;
}

int lbm_kinetic_energy_enstrophy(lbm_handle h, double* out)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (!h->have_out) return fail(h, LBM_ESTATE, "no step has produced output yet");
    if (h->has_mask) return fail(h, LBM_ESTATE, "E/Omega diagnostics need a fully periodic domain");
    double* dres = at<double>(h, h->off_misc + MISC_RED);
    CK(h, launch_diagnostics(h->rsize == 8, h->base + h->off_u, h->D, h->nx, h->ny, h->nz,
                             h->nxp, h->sq, at<double>(h, h->off_part), dres, h->stream),
       "diagnostics kernels");
    h->launches += 2;
    double tmp[2];
    CK(h, cudaMemcpyAsync(tmp, dres, sizeof tmp, cudaMemcpyDeviceToHost, h->stream),
       "copy diagnostics");
    int r = sync_status(h);
    out[0] = tmp[0];
    out[1] = tmp[1];
    return r;
}

int lbm_get_elbm_stats(lbm_handle h, double* out)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (h->model != LBM_ELBM) return fail(h, LBM_EINVAL, "not an ELBM handle");
    int r = ensure_memory(h);
    if (r) return r;
    double* d = at<double>(h, h->off_misc + MISC_CTR_OUT);
    CK(h, launch_sum_ctr(at<unsigned long long>(h, h->off_misc + MISC_CTR), d, h->stream),
       "counter kernel");
    h->launches += 1;
    CK(h, cudaMemcpyAsync(out, d, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
       "copy counters");
    CK(h, cudaStreamSynchronize(h->stream), "synchronise");
    return LBM_OK;
}

size_t lbm_state_bytes(lbm_handle h) { return h ? (size_t)h->Q * h->sq * h->esize : 0; }

int lbm_get_state(lbm_handle h, void* dst, long long* t)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!dst) return fail(h, LBM_EINVAL, "dst is NULL");
    if (!h->inited) return fail(h, LBM_ESTATE, "no state yet");
    const size_t nb = lbm_state_bytes(h);
    CK(h, cudaMemcpyAsync(dst, h->base + ((h->cur == 0 || h->aa) ? h->off_A : h->off_B), nb,
                          cudaMemcpyDefault, h->stream),
       "copy state");
    CK(h, cudaStreamSynchronize(h->stream), "synchronise");
    if (t) *t = h->t;
    return LBM_OK;
}

int lbm_set_state(lbm_handle h, const void* src, long long t)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!src) return fail(h, LBM_EINVAL, "src is NULL");
    int r = ensure_memory(h);
    if (r) return r;
    const size_t nb = lbm_state_bytes(h);
    CK(h, cudaMemcpyAsync(h->base + h->off_A, src, nb, cudaMemcpyDefault, h->stream),
       "copy state");
    // the rounding clock resumes at t (both slots: the next step may read either)
    h->clk_host[0] = h->clk_host[1] = (unsigned)t;
    CK(h, cudaMemcpyAsync(h->base + h->off_misc + MISC_STEP, h->clk_host, sizeof h->clk_host,
                          cudaMemcpyHostToDevice, h->stream),
       "set the rounding clock");
    CK(h, cudaStreamSynchronize(h->stream), "synchronise");
    // AB: the state now sits in A.  AA: one array, whose placement is fixed
    // by the parity of t (the step after an even t is a pull/push step).
    h->cur = h->aa ? (int)(t & 1) : 0;
    h->t = t;
    h->inited = true;
    h->have_out = false;
    return LBM_OK;
}

int lbm_sync(lbm_handle h)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    return sync_status(h);
}

long long lbm_launch_count(lbm_handle h) { return h ? h->launches : 0; }

int lbm_elbm_collect_pairs(lbm_handle h, int stride, float* X_dev, double* y_dev, int cap,
                           int* count)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (h->model != LBM_ELBM) return fail(h, LBM_EINVAL, "not an ELBM handle");
    if (stride < 1 || cap < 1 || !X_dev || !y_dev || !count)
        return fail(h, LBM_EINVAL, "bad pair-capture arguments");
    if (!is_device_ptr(X_dev) || !is_device_ptr(y_dev))
        return fail(h, LBM_EINVAL, "pair buffers must be device memory");
    int r = check_step_ready(h);
    if (r) return r;
    StepParams p = make_params(h);
    int* cnt = at<int>(h, h->off_misc + MISC_PAIRS);
    CK(h, cudaMemsetAsync(cnt, 0, sizeof(int), h->stream), "clear pair count");
    p.pairs_X = X_dev;
    p.pairs_y = y_dev;
    p.pairs_count = cnt;
    p.pairs_cap = cap;
    p.pairs_stride = stride;
    CK(h, launch_one(h, p, h->cur, true), "stream-collide kernel (pair capture)");
    h->cur ^= 1;
    h->launches += 1;
    h->t += 1;
    h->have_out = true;
    int hc = 0;
    CK(h, cudaMemcpyAsync(&hc, cnt, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "count");
    r = sync_status(h);
    *count = hc < cap ? hc : cap;
    return r;
}

}  // extern "C"

// ===========================================================================
// Subdomain decomposition with ghost layers (Sec. 3.6), all subdomains on
// this GPU.  The domain is cut into S slabs of whole rows of its slowest axis
// (z on D3Q19, y on D2Q9); slab s holds rows [lo_s, hi_s) plus one ghost row
// on each side, as an ordinary handle of nrows + 2 rows whose step kernels
// are restricted to the interior rows.  After every step the boundary rows'
// outgoing directions are collected into a linear send buffer, moved to the
// neighbour's receive buffer (the transfer a multi-GPU run would make) and
// distributed into the neighbour's ghost row.  With overlap on, the two
// boundary rows of every slab are updated first, the exchange runs on a
// second stream while the bulk rows update (Sec. 3.6's bulk/boundary split).
// The dither salt of each slab is offset to the global node index, so every
// storage type reproduces the single-domain run bit for bit.
// ===========================================================================
struct lbm_multi_ctx {
    int nx = 0, ny = 0, nz = 0, lattice = 0, D = 0, Q = 0, S = 0, dtype = 0;
    int axis_n = 0;              // rows of the decomposed axis
    long long layer = 0;         // padded elements per row (ny * nxp, or nxp on D2Q9)
    long long layer_dense = 0;   // dense nodes per row (nx * ny, or nx)
    size_t esize = 0;
    std::vector<int> lo, hi;
    std::vector<lbm_ctx*> sub;
    int ndir = 0;
    int dir_up[9], dir_dn[9];    // directions with +1 / -1 along the decomposed axis (<= 9)
    bool overlap = true, use_graph = false, inited = false;
    bool direct = false;         // one kernel stores into the neighbour's ghost row
    cudaStream_t stream = nullptr, comm = nullptr;
    cudaEvent_t ev_bnd = nullptr, ev_halo = nullptr;
    char* mem = nullptr;         // send, recv buffers, segment tables, scratch
    size_t face_bytes = 0;       // one face: ndir runs of one row
    size_t off_send = 0, off_recv = 0, off_tab = 0, off_scr = 0, scr_bytes = 0;
    int nseg = 0;                // segments per table (2 S ndir)
    // one slab of a decomposition across processes (lbm_multi_create_rank):
    // the handle holds slab `rank` of `nsub_global`; its faces go to and come
    // from the neighbouring ranks through the caller, between
    // lbm_multi_step_begin and lbm_multi_step_end
    bool rank_mode = false;
    int rank = 0, nsub_global = 1;
    bool begun = false;          // between lbm_multi_step_begin and _end
    long long t = 0, launches = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    std::string err;
};

static thread_local std::string g_multi_err;

static int mfail(lbm_multi_ctx* m, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (m ? m->err : g_multi_err) = buf;
    return code;
}

#define MCK(m, expr, what)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return mfail((m), LBM_ECUDA, "%s: %s", (what), cudaGetErrorString(e_));         \
    } while (0)

// propagate a sub-handle's error message
static int msub(lbm_multi_ctx* m, lbm_ctx* h, int r)
{
    if (r) m->err = h->err;
    return r;
}

static void mdrop_graphs(lbm_multi_ctx* m)
{
    for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second);
    m->graphs.clear();
}

static void multi_free(lbm_multi_ctx* m)
{
    mdrop_graphs(m);
    for (auto* h : m->sub) lbm_destroy(h);
    if (m->mem) cudaFree(m->mem);
    if (m->ev_bnd) cudaEventDestroy(m->ev_bnd);
    if (m->ev_halo) cudaEventDestroy(m->ev_halo);
    if (m->comm) cudaStreamDestroy(m->comm);
    delete m;
}

// segment tables, per parity (the buffer, 0: A or 1: B, that holds the new
// state after the step): collect, distribute, direct
static HaloSeg* mtable(lbm_multi_ctx* m, int parity, int kind)
{
    return reinterpret_cast<HaloSeg*>(m->mem + m->off_tab) + (size_t)(3 * parity + kind) * m->nseg;
}

static int multi_build_tables(lbm_multi_ctx* m)
{
    const int S = m->S;
    std::vector<HaloSeg> tab((size_t)6 * m->nseg);
    const long long n16 = m->layer * (long long)m->esize / 16;
    for (int parity = 0; parity < 2; ++parity) {
        HaloSeg* pk = &tab[(size_t)(3 * parity) * m->nseg];
        HaloSeg* up = &tab[(size_t)(3 * parity + 1) * m->nseg];
        HaloSeg* dr = &tab[(size_t)(3 * parity + 2) * m->nseg];
        for (int s = 0; s < S; ++s) {
            lbm_ctx* h = m->sub[s];
            char* arr = h->base + (parity == 0 ? h->off_A : h->off_B);
            const int nloc = m->hi[s] - m->lo[s];
            for (int f = 0; f < 2; ++f) {        // 0: upper face (row nloc), 1: lower face (row 1)
                const int row = f == 0 ? nloc : 1;
                const int r = f == 0 ? (s + 1) % S : (s + S - 1) % S;   // receiver
                lbm_ctx* hr = m->sub[r];
                char* arr_r = hr->base + (parity == 0 ? hr->off_A : hr->off_B);
                const int ghost = f == 0 ? 0 : (m->hi[r] - m->lo[r]) + 1;
                for (int k = 0; k < m->ndir; ++k) {
                    const int i = f == 0 ? m->dir_up[k] : m->dir_dn[k];
                    const size_t seg = ((size_t)s * 2 + f) * m->ndir + k;
                    const size_t boff = seg * (size_t)m->layer * m->esize;
                    const char* src = arr + ((size_t)i * h->sq + (size_t)row * m->layer) * m->esize;
                    char* dst = arr_r + ((size_t)i * hr->sq + (size_t)ghost * m->layer) * m->esize;
                    pk[seg] = HaloSeg{reinterpret_cast<const uint4*>(src),
                                      reinterpret_cast<uint4*>(m->mem + m->off_send + boff), n16};
                    up[seg] = HaloSeg{reinterpret_cast<const uint4*>(m->mem + m->off_recv + boff),
                                      reinterpret_cast<uint4*>(dst), n16};
                    dr[seg] = HaloSeg{reinterpret_cast<const uint4*>(src),
                                      reinterpret_cast<uint4*>(dst), n16};
                }
            }
        }
    }
    MCK(m, cudaMemcpy(m->mem + m->off_tab, tab.data(), tab.size() * sizeof(HaloSeg),
                      cudaMemcpyHostToDevice),
        "upload segment tables");
    return LBM_OK;
}

// The exchange after a step whose new state is in buffer `parity`, in three
// parts: collect (boundary rows -> send buffers), transfer (send -> receive
// buffers: the slot of face (s, f) holds, on the receiving side, the face
// that lands in the neighbour's ghost row), distribute (receive buffers ->
// ghost rows).  A rank handle of a decomposition over several processes
// leaves the transfer to its caller.
static cudaError_t multi_collect(lbm_multi_ctx* m, int parity, cudaStream_t s)
{
    return launch_halo_copy(mtable(m, parity, 0), m->nseg, m->layer * (long long)m->esize / 16,
                            s);
}

static cudaError_t multi_distribute(lbm_multi_ctx* m, int parity, cudaStream_t s)
{
    return launch_halo_copy(mtable(m, parity, 1), m->nseg, m->layer * (long long)m->esize / 16,
                            s);
}

static cudaError_t multi_exchange(lbm_multi_ctx* m, int parity, cudaStream_t s)
{
    const long long n16 = m->layer * (long long)m->esize / 16;
    if (m->direct) return launch_halo_copy(mtable(m, parity, 2), m->nseg, n16, s);
    cudaError_t e = multi_collect(m, parity, s);
    if (e != cudaSuccess) return e;
    // transfer: face (s, f) goes to its receiver's buffer slot of the same index
    for (int sd = 0; sd < m->S; ++sd)
        for (int f = 0; f < 2; ++f) {
            const size_t off = ((size_t)sd * 2 + f) * m->face_bytes;
            e = cudaMemcpyAsync(m->mem + m->off_recv + off, m->mem + m->off_send + off,
                                m->face_bytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
    return multi_distribute(m, parity, s);
}

static cudaError_t multi_rows(lbm_multi_ctx* m, int s, int row0, int nrows, bool out, int from)
{
    lbm_ctx* h = m->sub[s];
    StepParams p = make_params(h);
    p.row0 = row0;
    p.nrows = nrows;
    p.salt_off = (int)((long long)(m->lo[s] - 1) * m->layer);
    return launch_one(h, p, from, out);
}

// kernels launched per time step (stream-collide launches + collect + distribute)
static int multi_launches_per_step(const lbm_multi_ctx* m)
{
    int nl = m->direct ? 1 : 2;
    for (int s = 0; s < m->S; ++s) {
        const int nloc = m->hi[s] - m->lo[s];
        nl += m->overlap ? 1 + (nloc > 1) + (nloc > 2) : 1;
    }
    return nl;
}

// one time step of every slab; `from` is the buffer holding the current state
static cudaError_t multi_step_once(lbm_multi_ctx* m, int from, bool out)
{
    cudaError_t e;
    const int to = from ^ 1;
    if (!m->overlap) {
        for (int s = 0; s < m->S; ++s)
            if ((e = multi_rows(m, s, 1, m->hi[s] - m->lo[s], out, from)) != cudaSuccess) return e;
        return multi_exchange(m, to, m->stream);
    }
    for (int s = 0; s < m->S; ++s) {
        const int nloc = m->hi[s] - m->lo[s];
        if ((e = multi_rows(m, s, 1, 1, out, from)) != cudaSuccess) return e;
        if (nloc > 1 && (e = multi_rows(m, s, nloc, 1, out, from)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(m->ev_bnd, m->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(m->comm, m->ev_bnd, 0)) != cudaSuccess) return e;
    if ((e = multi_exchange(m, to, m->comm)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(m->ev_halo, m->comm)) != cudaSuccess) return e;
    for (int s = 0; s < m->S; ++s) {
        const int nloc = m->hi[s] - m->lo[s];
        if (nloc > 2 && (e = multi_rows(m, s, 2, nloc - 2, out, from)) != cudaSuccess) return e;
    }
    return cudaStreamWaitEvent(m->stream, m->ev_halo, 0);
}

// Gather rows lo-1 .. hi (periodic) of a field with `ncomp` components of
// `rowbytes` bytes per row and `nrows_g` rows into dst (device).
static int gather_rows(lbm_multi_ctx* m, const char* src, char* dst, int lo, int hi, int ncomp,
                       size_t rowbytes)
{
    const int n = m->axis_n, nloc = hi - lo;
    for (int c = 0; c < ncomp; ++c) {
        const char* sc = src + (size_t)c * n * rowbytes;
        char* dc = dst + (size_t)c * (nloc + 2) * rowbytes;
        const int below = (lo - 1 + n) % n, above = hi % n;
        MCK(m, cudaMemcpyAsync(dc, sc + (size_t)below * rowbytes, rowbytes, cudaMemcpyDefault,
                               m->stream), "gather row");
        MCK(m, cudaMemcpyAsync(dc + rowbytes, sc + (size_t)lo * rowbytes, (size_t)nloc * rowbytes,
                               cudaMemcpyDefault, m->stream), "gather rows");
        MCK(m, cudaMemcpyAsync(dc + (size_t)(nloc + 1) * rowbytes, sc + (size_t)above * rowbytes,
                               rowbytes, cudaMemcpyDefault, m->stream), "gather row");
    }
    return LBM_OK;
}

// All nsub slabs on this GPU (rank < 0), or only slab `rank` of them (a rank
// handle: S = 1 local slab with its global rows).
static int multi_create_impl(int nx, int ny, int nz, int lattice, int model, double tau,
                             int dtype, int nsub, int rank, lbm_multi* out)
{
    if (!out) return mfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    const int D = lattice == LBM_D2Q9 ? 2 : 3;
    const int axis_n = D == 3 ? nz : ny;
    if (nsub < 1 || nsub > 4096 || axis_n < nsub)
        return mfail(nullptr, LBM_EINVAL,
                     "need 1 <= subdomains <= rows of the decomposed axis (%d), got %d", axis_n,
                     nsub);
    if (rank >= nsub)
        return mfail(nullptr, LBM_EINVAL, "rank %d outside 0..%d", rank, nsub - 1);
    lbm_multi_ctx* m = new lbm_multi_ctx();
    m->nx = nx; m->ny = ny; m->nz = nz; m->lattice = lattice; m->D = D;
    m->S = rank < 0 ? nsub : 1;
    m->dtype = dtype; m->axis_n = axis_n;
    m->rank_mode = rank >= 0;
    m->rank = rank < 0 ? 0 : rank;
    m->nsub_global = nsub;
    for (int s = rank < 0 ? 0 : rank; s < (rank < 0 ? nsub : rank + 1); ++s) {
        m->lo.push_back((int)((long long)axis_n * s / nsub));
        m->hi.push_back((int)((long long)axis_n * (s + 1) / nsub));
    }
    nsub = m->S;   // local slabs from here on
    for (int s = 0; s < nsub; ++s) {
        const int nloc = m->hi[s] - m->lo[s];
        lbm_handle h = nullptr;
        int r = D == 3 ? lbm_create(nx, ny, nloc + 2, lattice, model, tau, dtype, &h)
                       : lbm_create(nx, nloc + 2, 1, lattice, model, tau, dtype, &h);
        if (r) {
            int code = mfail(nullptr, r, "subdomain %d: %s", s, lbm_last_error(nullptr));
            multi_free(m);
            return code;
        }
        m->sub.push_back(h);
    }
    lbm_ctx* h0 = m->sub[0];
    m->Q = h0->Q;
    m->esize = h0->esize;
    m->layer = D == 3 ? (long long)h0->nxp * ny : h0->nxp;
    m->layer_dense = D == 3 ? (long long)nx * ny : nx;
    // directions with a +1 / -1 component along the decomposed axis
    int ndn = 0;
    for (int i = 0; i < m->Q; ++i) {
        const int e = lattice == LBM_D2Q9    ? D2Q9::ey(i)
                      : lattice == LBM_D3Q19 ? D3Q19::ez(i)
                      : lattice == LBM_D3Q15 ? D3Q15::ez(i)
                                             : D3Q27::ez(i);
        if (e == 1) m->dir_up[m->ndir++] = i;
        if (e == -1) m->dir_dn[ndn++] = i;
    }
    m->face_bytes = (size_t)m->ndir * m->layer * m->esize;
    m->nseg = 2 * nsub * m->ndir;
    size_t o = 0;
    m->off_send = o; o = align256(o + m->face_bytes * 2 * nsub);
    m->off_recv = o; o = align256(o + m->face_bytes * 2 * nsub);
    m->off_tab = o; o = align256(o + sizeof(HaloSeg) * 6 * (size_t)m->nseg);
    int maxloc = 0;
    for (int s = 0; s < nsub; ++s) maxloc = std::max(maxloc, m->hi[s] - m->lo[s]);
    m->scr_bytes = (size_t)(maxloc + 2) * m->layer_dense * 8 * (1 + D);
    m->off_scr = o; o = align256(o + m->scr_bytes);
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&m->mem), o);
    if (e != cudaSuccess) {
        int code = mfail(nullptr, LBM_ENOMEM, "multi buffers (%zu bytes): %s", o,
                         cudaGetErrorString(e));
        multi_free(m);
        return code;
    }
    for (auto* h : m->sub) {
        int r = ensure_memory(h);
        if (r) {
            int code = mfail(nullptr, r, "subdomain memory: %s", h->err.c_str());
            multi_free(m);
            return code;
        }
    }
    if ((e = cudaStreamCreateWithFlags(&m->comm, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&m->ev_bnd, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&m->ev_halo, cudaEventDisableTiming)) != cudaSuccess) {
        int code = mfail(nullptr, LBM_ECUDA, "streams/events: %s", cudaGetErrorString(e));
        multi_free(m);
        return code;
    }
    int r = multi_build_tables(m);
    if (r) {
        int code = mfail(nullptr, r, "%s", m->err.c_str());
        multi_free(m);
        return code;
    }
    *out = m;
    return LBM_OK;
}

extern "C" {

int lbm_multi_create(int nx, int ny, int nz, int lattice, int model, double tau, int dtype,
                     int nsub, lbm_multi* out)
{
    return multi_create_impl(nx, ny, nz, lattice, model, tau, dtype, nsub, -1, out);
}

int lbm_multi_create_rank(int nx, int ny, int nz, int lattice, int model, double tau, int dtype,
                          int nsub, int rank, lbm_multi* out)
{
    if (rank < 0) return mfail(nullptr, LBM_EINVAL, "rank must be >= 0 (got %d)", rank);
    return multi_create_impl(nx, ny, nz, lattice, model, tau, dtype, nsub, rank, out);
}

int lbm_multi_destroy(lbm_multi m)
{
    if (!m) return LBM_OK;
    cudaStreamSynchronize(m->stream);
    cudaStreamSynchronize(m->comm);
    multi_free(m);
    return LBM_OK;
}

const char* lbm_multi_last_error(lbm_multi m) { return m ? m->err.c_str() : g_multi_err.c_str(); }

int lbm_multi_set_stream(lbm_multi m, void* stream)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    m->stream = static_cast<cudaStream_t>(stream);
    for (auto* h : m->sub) lbm_set_stream(h, stream);
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_overlap(lbm_multi m, int on)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    m->overlap = on != 0;
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_transfer(lbm_multi m, int mode)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (mode != LBM_TRANSFER_STAGED && mode != LBM_TRANSFER_DIRECT)
        return mfail(m, LBM_EINVAL, "unknown transfer mode %d", mode);
    m->direct = mode == LBM_TRANSFER_DIRECT;
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_graph(lbm_multi m, int on)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    m->use_graph = on != 0;
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_force(lbm_multi m, double fx, double fy, double fz)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    for (auto* h : m->sub) {
        int r = lbm_set_force(h, fx, fy, fz);
        if (r) return msub(m, h, r);
    }
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_rounding(lbm_multi m, int mode)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    for (auto* h : m->sub) {
        int r = lbm_set_rounding(h, mode);
        if (r) return msub(m, h, r);
    }
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_smagorinsky(lbm_multi m, double cs)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    for (auto* h : m->sub) {
        int r = lbm_set_smagorinsky(h, cs);
        if (r) return msub(m, h, r);
    }
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_boundary(lbm_multi m, int id, int kind, int method, int normal,
                           const double* value)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    for (auto* h : m->sub) {
        int r = lbm_set_boundary(h, id, kind, method, normal, value);
        if (r) return msub(m, h, r);
    }
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_elbm(lbm_multi m, int alpha_mode, double tol, int max_iter, double skip_eps)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    for (auto* h : m->sub) {
        int r = lbm_set_elbm(h, alpha_mode, tol, max_iter, skip_eps);
        if (r) return msub(m, h, r);
    }
    mdrop_graphs(m);
    return LBM_OK;
}

int lbm_multi_set_geometry(lbm_multi m, const uint8_t* mask)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (!mask) return mfail(m, LBM_EINVAL, "mask is NULL");
    if (m->inited) return mfail(m, LBM_ESTATE, "set the geometry before the initial state");
    char* scr = m->mem + m->off_scr;
    for (int s = 0; s < m->S; ++s) {
        int r = gather_rows(m, reinterpret_cast<const char*>(mask), scr, m->lo[s], m->hi[s], 1,
                            (size_t)m->layer_dense);
        if (r) return r;
        r = lbm_set_geometry(m->sub[s], reinterpret_cast<const uint8_t*>(scr));
        if (r) return msub(m, m->sub[s], r);
    }
    return LBM_OK;
}

int lbm_multi_init_equilibrium(lbm_multi m, const void* rho, const void* u, int field_dtype)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (!rho || !u) return mfail(m, LBM_EINVAL, "rho and u must be non-NULL");
    if (field_dtype != LBM_FIELD_F64 && field_dtype != LBM_FIELD_F32)
        return mfail(m, LBM_EINVAL, "unknown field dtype %d", field_dtype);
    const size_t fs = field_dtype == LBM_FIELD_F64 ? 8 : 4;
    const size_t rowb = (size_t)m->layer_dense * fs;
    for (int s = 0; s < m->S; ++s) {
        const int nloc = m->hi[s] - m->lo[s];
        char* sr = m->mem + m->off_scr;
        char* su = sr + (size_t)(nloc + 2) * rowb;
        int r = gather_rows(m, static_cast<const char*>(rho), sr, m->lo[s], m->hi[s], 1, rowb);
        if (r) return r;
        r = gather_rows(m, static_cast<const char*>(u), su, m->lo[s], m->hi[s], m->D, rowb);
        if (r) return r;
        r = lbm_init_equilibrium(m->sub[s], sr, su, field_dtype);
        if (r) return msub(m, m->sub[s], r);
    }
    m->t = 0;
    m->inited = true;
    return LBM_OK;
}

int lbm_multi_step(lbm_multi m, int n)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (n < 1) return mfail(m, LBM_EINVAL, "n must be >= 1 (got %d)", n);
    if (!m->inited) return mfail(m, LBM_ESTATE, "the initial state must precede stepping");
    if (m->begun) return mfail(m, LBM_ESTATE, "a step begun with lbm_multi_step_begin is open");
    if (m->rank_mode && m->nsub_global > 1)
        return mfail(m, LBM_ESTATE, "a rank of a decomposition over %d processes steps with "
                                    "lbm_multi_step_begin / lbm_multi_step_end", m->nsub_global);
    for (auto* h : m->sub) {
        int r = check_step_ready(h);
        if (r) return msub(m, h, r);
    }
    const int cur = m->sub[0]->cur;
    if (m->use_graph && m->stream != nullptr) {
        auto key = std::make_pair(n, cur);
        auto it = m->graphs.find(key);
        if (it == m->graphs.end()) {
            cudaGraph_t g;
            MCK(m, cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal),
                "begin capture");
            int from = cur;
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < n && le == cudaSuccess; ++k) {
                le = multi_step_once(m, from, k == n - 1);
                from ^= 1;
            }
            cudaError_t ce = cudaStreamEndCapture(m->stream, &g);
            if (le != cudaSuccess) {
                if (ce == cudaSuccess) cudaGraphDestroy(g);
                return mfail(m, LBM_ECUDA, "launch during capture: %s", cudaGetErrorString(le));
            }
            MCK(m, ce, "end capture");
            cudaGraphExec_t ge;
            cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            MCK(m, ie, "instantiate graph");
            it = m->graphs.emplace(key, ge).first;
        }
        MCK(m, cudaGraphLaunch(it->second, m->stream), "graph launch");
    } else {
        int from = cur;
        for (int k = 0; k < n; ++k) {
            MCK(m, multi_step_once(m, from, k == n - 1), "subdomain step");
            from ^= 1;
        }
    }
    const int nl = n * multi_launches_per_step(m);
    for (auto* h : m->sub) {
        h->cur ^= (n & 1);
        h->t += n;
        h->have_out = true;
    }
    m->t += n;
    m->launches += nl;
    return LBM_OK;
}

int lbm_multi_get_macro(lbm_multi m, void* rho, void* u, int field_dtype)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (field_dtype != LBM_FIELD_F64 && field_dtype != LBM_FIELD_F32)
        return mfail(m, LBM_EINVAL, "unknown field dtype %d", field_dtype);
    if (m->t == 0) return mfail(m, LBM_ESTATE, "no step has produced output yet");
    if (m->begun) return mfail(m, LBM_ESTATE, "a step begun with lbm_multi_step_begin is open");
    const size_t fs = field_dtype == LBM_FIELD_F64 ? 8 : 4;
    const size_t rowb = (size_t)m->layer_dense * fs;
    const size_t ntot = (size_t)m->axis_n * rowb;
    for (int s = 0; s < m->S; ++s) {
        lbm_ctx* h = m->sub[s];
        const int nloc = m->hi[s] - m->lo[s];
        const size_t nb = (size_t)(nloc + 2) * rowb;
        char* scr = m->mem + m->off_scr;
        // dense local fields (ghost rows included), then the interior rows
        for (int fld = 0; fld < 2; ++fld) {
            void* dst = fld == 0 ? rho : u;
            if (!dst) continue;
            const int nc = fld == 0 ? 1 : m->D;
            MCK(m, launch_pack(h->rsize == 8, h->base + (fld == 0 ? h->off_rho : h->off_u),
                               field_dtype == LBM_FIELD_F32, scr, nc, h->nx, h->ny, h->nz, h->nxp,
                               h->sq, fld == 0 ? 1.0 : 0.0, m->stream),
                "pack kernel");
            m->launches += 1;
            for (int c = 0; c < nc; ++c)
                MCK(m, cudaMemcpyAsync(static_cast<char*>(dst) + c * ntot + (size_t)m->lo[s] * rowb,
                                       scr + c * nb + rowb, (size_t)nloc * rowb, cudaMemcpyDefault,
                                       m->stream),
                    "copy rows");
        }
    }
    MCK(m, cudaStreamSynchronize(m->stream), "synchronise");
    for (auto* h : m->sub) {
        int r = sync_status(h);
        if (r) return msub(m, h, r);
    }
    return LBM_OK;
}

int lbm_multi_step_begin(lbm_multi m, int output)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (!m->rank_mode) return mfail(m, LBM_EINVAL, "not a rank handle (lbm_multi_create_rank)");
    if (!m->inited) return mfail(m, LBM_ESTATE, "the initial state must precede stepping");
    if (m->begun) return mfail(m, LBM_ESTATE, "the previous step has not ended");
    lbm_ctx* h = m->sub[0];
    int r = check_step_ready(h);
    if (r) return msub(m, h, r);
    const int from = h->cur, to = from ^ 1;
    const bool out = output != 0;
    const int nloc = m->hi[0] - m->lo[0];
    // the boundary rows, whose faces leave; the collect follows them on the
    // exchange stream while the bulk rows update
    if (m->overlap) {
        MCK(m, multi_rows(m, 0, 1, 1, out, from), "boundary row");
        if (nloc > 1) MCK(m, multi_rows(m, 0, nloc, 1, out, from), "boundary row");
    } else {
        MCK(m, multi_rows(m, 0, 1, nloc, out, from), "slab");
    }
    MCK(m, cudaEventRecord(m->ev_bnd, m->stream), "event");
    MCK(m, cudaStreamWaitEvent(m->comm, m->ev_bnd, 0), "event wait");
    MCK(m, multi_collect(m, to, m->comm), "collect kernel");
    if (m->overlap && nloc > 2) MCK(m, multi_rows(m, 0, 2, nloc - 2, out, from), "bulk rows");
    m->launches += 1 + (m->overlap ? (nloc > 1) + (nloc > 2) : 0);
    m->begun = true;
    return LBM_OK;
}

int lbm_multi_step_end(lbm_multi m)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    if (!m->begun) return mfail(m, LBM_ESTATE, "no step was begun");
    lbm_ctx* h = m->sub[0];
    MCK(m, multi_distribute(m, h->cur ^ 1, m->comm), "distribute kernel");
    MCK(m, cudaEventRecord(m->ev_halo, m->comm), "event");
    MCK(m, cudaStreamWaitEvent(m->stream, m->ev_halo, 0), "event wait");
    m->launches += 1;
    h->cur ^= 1;
    h->t += 1;
    h->have_out = true;
    m->t += 1;
    m->begun = false;
    return LBM_OK;
}

int lbm_multi_face_buffers(lbm_multi m, void** send, void** recv, size_t* face_bytes)
{
    if (!m || !send || !recv || !face_bytes) return mfail(m, LBM_EINVAL, "NULL argument");
    if (!m->rank_mode) return mfail(m, LBM_EINVAL, "not a rank handle (lbm_multi_create_rank)");
    *send = m->mem + m->off_send;
    *recv = m->mem + m->off_recv;
    *face_bytes = m->face_bytes;
    return LBM_OK;
}

int lbm_multi_exchange_stream(lbm_multi m, void** stream)
{
    if (!m || !stream) return mfail(m, LBM_EINVAL, "NULL argument");
    *stream = m->comm;
    return LBM_OK;
}

int lbm_multi_rows(lbm_multi m, int* lo, int* hi)
{
    if (!m || !lo || !hi) return mfail(m, LBM_EINVAL, "NULL argument");
    *lo = m->lo.front();
    *hi = m->hi.back();
    return LBM_OK;
}

int lbm_multi_halo_bytes(lbm_multi m, long long* per_step)
{
    if (!m || !per_step) return mfail(m, LBM_EINVAL, "NULL argument");
    *per_step = (long long)(2 * m->S) * m->ndir * m->layer_dense * (long long)m->esize;
    return LBM_OK;
}

long long lbm_multi_launch_count(lbm_multi m) { return m ? m->launches : 0; }

int lbm_multi_sync(lbm_multi m)
{
    if (!m) return mfail(nullptr, LBM_EINVAL, "NULL handle");
    MCK(m, cudaStreamSynchronize(m->stream), "synchronise");
    MCK(m, cudaStreamSynchronize(m->comm), "synchronise");
    for (auto* h : m->sub) {
        int r = sync_status(h);
        if (r) return msub(m, h, r);
    }
    return LBM_OK;
}

}  // extern "C"
