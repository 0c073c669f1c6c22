/*
 * lbm.h - C ABI of the GB300 (sm_103a) lattice Boltzmann stream-and-collide
 * library.
 *
 * The library advances the particle distributions f_i of a lattice Boltzmann
 * fluid (Januszewski & Kostur, "Sailfish: a flexible multi-GPU implementation
 * of the lattice Boltzmann method", Sec. 2) on one GPU.  One call to
 * lbm_step() performs, per time step and per lattice node, the fused update
 * of Algorithm cnp (Sec. 3.3): pull streaming from the previous step's
 * post-collision array (AB pattern, Sec. 3.3), half-way bounce-back at solid
 * nodes (Sec. 2.3), the macroscopic moments (Eq. lb_macro), the collision
 * (LBGK Eq. lbgk, MRT Eq. mrt_collision or entropic ELBM Eqs. elbm and
 * alpha_cond), the body force (Guo Eq. guo_force or EDM Eq. edm_force) and,
 * on the last step of the call, the output of rho and v (Eq. edm_momentum).
 *
 * Conventions for every entry point:
 *  - Every function returns an int status (LBM_OK = 0 on success).  On error
 *    lbm_last_error(h) returns a message; the handle stays usable unless the
 *    error is LBM_ECUDA from a sticky CUDA fault.
 *  - Arrays crossing the ABI are dense, C-ordered, x fastest: scalar fields
 *    [nz][ny][nx], vector fields [D][nz][ny][nx] (D = 2 for D2Q9, 3 for
 *    D3Q19).  nz = 1 for D2Q9.
 *  - Pointers may be host or device memory unless stated otherwise; the
 *    library detects which with cudaPointerGetAttributes.  Host pointers are
 *    copied synchronously before the call returns.  The library never keeps
 *    a caller pointer beyond the call, except the memory given to
 *    lbm_bind_memory and the stream given to lbm_set_stream.
 *  - Work is enqueued on the handle's stream (lbm_set_stream; default: the
 *    legacy default stream).  Calls that return data to a host pointer or
 *    report device status synchronise that stream.
 *  - The domain is periodic along every axis; walls come only from the mask.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,   /* bad argument: size <= 0, tau <= 1/2, unsupported combination */
    LBM_ESTATE = 2,   /* wrong call order, e.g. lbm_step before lbm_init_equilibrium */
    LBM_ENOMEM = 3,   /* device memory exhausted or bound memory too small */
    LBM_ECUDA = 4,    /* CUDA runtime error (message holds cudaGetErrorString) */
    LBM_ENAN = 5,     /* a non-finite rho or v was produced on an output step */
    LBM_ETIMEOUT = 6, /* a bounded device wait gave up (batched persistent kernel) */
    LBM_ENOCONV = 7   /* ELBM strict mode: some alpha solve hit the iteration cap */
};

/* ---- lattices, collision models, storage types ------------------------ */
/* Velocity sets (Sec. 2, Fig. lattices, Table bgkweights).  MRT is defined
 * on D3Q19 only; every other model runs on all four. */
enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q15 = 2, LBM_D3Q27 = 3 };
/* Collision models: LBGK (Eq. lbgk, Guo forcing), MRT (Eq. mrt_collision,
 * D3Q19), ELBM (Eqs. elbm and alpha_cond, exact-difference forcing),
 * regularized LBGK (Sec. 2.1.1: the non-equilibrium part is replaced by its
 * projection w_i/(2 c_s^4) (e_i e_i - c_s^2 I) : Pi^neq before the LBGK
 * relaxation) and LBGK with the Smagorinsky subgrid model (Sec. 2.1.4,
 * Eqs. smagorinsky and taut: tau = tau0 + tau_t per node). */
enum { LBM_BGK = 0, LBM_MRT = 1, LBM_ELBM = 2, LBM_REG = 3, LBM_SMAG = 4 };
/* Storage of f_i in device memory.  *_S types store f_i - w_i (the
 * round-off-minimising form of Sec. 3.7); arithmetic is FP64 for LBM_F64 and
 * FP32 for all others. */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F32S = 2, LBM_F16S = 3, LBM_BF16S = 4 };
/* Rounding of FP16/BF16 stores.  DITHER (default): add to the dropped bits an
 * offset from a hash of the value's bits, node and direction, then truncate;
 * the rounding error is unbiased like stochastic rounding, without a random
 * number generator (round-to-nearest of a value that barely changes from
 * step to step repeats the same error and drifts).  NEAREST: round to
 * nearest even. */
enum { LBM_ROUND_DITHER = 0, LBM_ROUND_NEAREST = 1 };
/* Access patterns (Sec. 3.3): AB keeps two copies of the distributions and
 * alternates between them; AA keeps one copy, alternating a pull/push step
 * (even t) with an in-place step (odd t).  Same bytes moved per update; AA
 * halves the footprint. */
enum { LBM_PATTERN_AB = 0, LBM_PATTERN_AA = 1 };
/* Element type of macroscopic-field arrays crossing the ABI. */
enum { LBM_FIELD_F64 = 0, LBM_FIELD_F32 = 1 };
/* ELBM alpha modes (Eq. alpha_cond).  NEWTON: safeguarded FP64 Newton from
 * alpha = 2 to the tolerance.  The guarded modes run the same Newton from a
 * guess and accept the first correction of at most guard_tol * alpha within
 * their first guard_steps g evaluations (lbm_set_elbm_guard); otherwise
 * they continue to the tolerance:
 *   SERIES_GUARDED: the second-order small-deviation series guess
 *     s2 = 2 + (a_3 - 2 a_4) / (3 a_2) + 4 a_3^2 / (9 a_2^2), a_k = sum f x^k;
 *   MLP_GUARDED: s2 plus the learned correction (lbm_load_alpha_mlp);
 *   ROOT_GUARDED: the root of g(alpha)/alpha with g's series in alpha
 *     truncated after a_6 and the node's own A = sum Delta ln(f / w) (no
 *     learned part; three Newton steps on that polynomial from s2).
 * FIXED2: alpha = 2 (the LBGK limit; tests only). */
enum { LBM_ALPHA_NEWTON = 0, LBM_ALPHA_SERIES_GUARDED = 1, LBM_ALPHA_MLP_GUARDED = 2,
       LBM_ALPHA_FIXED2 = 3, LBM_ALPHA_ROOT_GUARDED = 4 };

typedef struct lbm_ctx* lbm_handle;

/* ---- creation ---------------------------------------------------------- */

/* Create a simulation of nx x ny x nz nodes (nz = 1 for D2Q9) with the given
 * lattice, collision model and relaxation time tau (nu = (2 tau - 1) / 6,
 * Sec. 2 after Eq. lbgk), storing f_i as dtype.  Supported: every lattice /
 * model / dtype combination except MRT on D2Q9.  ELBM requires tau > 1/2 and
 * is the only model that accepts tau arbitrarily close to 1/2.
 * No device memory is touched until the first call that needs it.
 * Errors: LBM_EINVAL (sizes < 1, nz != 1 with D2Q9, tau <= 1/2, unknown
 * enum, node count beyond 2^31 - 1).  *out is NULL on error; the message is
 * then available from lbm_last_error(NULL). */
LBM_API int lbm_create(int nx, int ny, int nz, int lattice, int model, double tau, int dtype,
               lbm_handle* out);

/* Free the handle and any device memory the library allocated itself
 * (memory given to lbm_bind_memory stays the caller's).  NULL is a no-op. */
LBM_API int lbm_destroy(lbm_handle h);

/* Message of the last error on h (thread-local message for h == NULL). */
LBM_API const char* lbm_last_error(lbm_handle h);

/* Fault injection for testing (no counterpart in the paper): the next n
 * device allocations the library makes (a handle's arena, a batch, the
 * subdomain buffers, the autotuner's backup, the MLP training buffers) fail
 * as if the device were out of memory, without calling cudaMalloc; the call
 * that needed the memory returns LBM_ENOMEM and its object stays valid.
 * n = 0 turns it off.  Process-wide.  LBM_EINVAL for n < 0. */
LBM_API int lbm_debug_fail_allocations(int n);

/* ---- memory and stream ------------------------------------------------- */

/* Bytes of device memory the handle needs: two copies of the distributions
 * (AB pattern), the node-type map, the macroscopic fields, and a staging
 * area for host transfers.  Valid right after lbm_create. */
LBM_API size_t lbm_required_bytes(lbm_handle h);

/* Use caller-owned device memory (at least lbm_required_bytes, 256-byte
 * aligned) instead of allocating.  Must precede lbm_set_geometry and
 * lbm_init_equilibrium.  The caller keeps it alive until lbm_destroy.
 * Errors: LBM_ESTATE (memory already in use), LBM_ENOMEM (too small),
 * LBM_EINVAL (NULL, misaligned or not device memory). */
LBM_API int lbm_bind_memory(lbm_handle h, void* dev_ptr, size_t bytes);

/* Access pattern (LBM_PATTERN_AB default, or LBM_PATTERN_AA).  Must precede
 * any call that puts device memory in use (lbm_bind_memory, lbm_set_geometry,
 * lbm_init_equilibrium, ...); lbm_required_bytes reflects it afterwards.
 * Results are bitwise equal for both patterns.  LBM_ESTATE if memory is
 * already in use. */
LBM_API int lbm_set_access_pattern(lbm_handle h, int pattern);

/* Enqueue all work on this cudaStream_t (NULL = legacy default stream). */
LBM_API int lbm_set_stream(lbm_handle h, void* cuda_stream);

/* ---- geometry and parameters ------------------------------------------ */

/* Node types (Sec. 3.4): mask[n] = 0 fluid, 1 solid, 2 + k a boundary node
 * of condition k (lbm_set_boundary, k = 0..14); nx*ny*nz bytes, dense, host
 * or device.  Solid nodes are walls for half-way bounce-back (Sec. 2.3): a
 * population that would stream out of a solid node is replaced by the
 * opposite population of the receiving node.  Solid nodes are not updated
 * and report rho = 0, v = 0.  The data are copied.  Values above 16 return
 * LBM_EINVAL.  Must precede lbm_init_equilibrium.  Default: all fluid. */
LBM_API int lbm_set_geometry(lbm_handle h, const uint8_t* mask);

/* Kernel for masked AB steps on the 3-D lattices (all models but ELBM):
 *   LBM_MASKED_AUTO (0, default) chooses from the geometry,
 *   LBM_MASKED_NODE (1) one node per thread, node word loaded with the
 *       populations and the bounced populations reloaded after it,
 *   LBM_MASKED_ZRUN (2) each thread walks 8 z layers and loads the next
 *       node's word ahead, so every population load, bounced or streamed
 *       (Sec. 2.3's half-way rule), is issued at once and solid nodes load
 *       nothing.
 * AUTO takes ZRUN when more than 40% of the 32-node row segments hold a fluid
 * node next to a solid one.  Both give bitwise equal results; this is a
 * performance choice only.  LBM_EINVAL for other values. */
#define LBM_MASKED_AUTO 0
#define LBM_MASKED_NODE 1
#define LBM_MASKED_ZRUN 2
LBM_API int lbm_set_masked_kernel(lbm_handle h, int mode);

/* Fraction of the 32-node row segments (x-aligned) that hold a fluid node
 * with a solid upstream neighbour, measured by lbm_set_geometry: the
 * statistic LBM_MASKED_AUTO uses.  LBM_ESTATE before lbm_set_geometry. */
LBM_API int lbm_get_nearwall_fraction(lbm_handle h, double* frac);

/* Uniform body force density F (lattice units), Sec. 2.4.  LBGK and MRT use
 * Guo's term (Eq. guo_force; in moment space with (I - S/2) for MRT), ELBM
 * uses the EDM term (Eq. edm_force).  Default 0. */
LBM_API int lbm_set_force(lbm_handle h, double fx, double fy, double fz);

/* MRT relaxation rates s_k (Eq. mrt_collision) for the 19 moments of the
 * orthogonal D3Q19 basis of d'Humieres et al. (2002), in their order: rho,
 * e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx,
 * my, mz.  q must be 19.  Default: 0 for conserved moments, 1/tau for the
 * five stress moments, 1.19, 1.4, 1.2, 1.4, 1.98 for the others. */
LBM_API int lbm_set_mrt_rates(lbm_handle h, const double* s, int q);

/* Velocity / pressure boundary condition `id` (0..14), used by the nodes
 * whose mask value is 2 + id (Sec. 2.3 lists equilibrium, Zou-He and
 * regularized conditions).  A boundary node is a fluid node; after
 * streaming, its populations with e_i . n > 0 (n the inward normal: +-1 x,
 * +-2 y, +-3 z) came from outside and are replaced before the collision:
 *   rho (1 - v_n) = S_0 + 2 S_out - F_n / 2 gives the missing moment (S_0 and
 *     S_out sum the populations with e.n = 0 and e.n < 0; the momentum is
 *     j = rho v - F/2, so the node reports exactly v);
 *   LBM_BC_VELOCITY: value = v (D components), rho from the relation;
 *   LBM_BC_PRESSURE: value[0] = rho, v = v_n n from the relation;
 *   LBM_BC_EQUILIBRIUM: f_i = f_eq_i(rho, v) - 3/2 w_i e_i . F;
 *   LBM_BC_ZOUHE: unknown f_i = f_opp(i) + f_eq_i - f_eq_opp(i), the
 *     remaining momentum to the normal link and, per tangential axis, evenly
 *     to the shortest unknown links with that component (Zou & He on D2Q9,
 *     its D3Q19 extension; the body diagonals on D3Q15);
 *   LBM_BC_REGULARIZED: the same unknown f_i, then every population rebuilt
 *     as f_eq + w_i 9/2 (e_i e_i - I/3) : Pi^neq - 3/2 w_i e_i . F.
 * Set before lbm_step; LBM_EINVAL for a bad id, kind, method, normal or a
 * non-finite value (rho must be > 0). */
enum { LBM_BC_VELOCITY = 1, LBM_BC_PRESSURE = 2 };
enum { LBM_BC_EQUILIBRIUM = 0, LBM_BC_ZOUHE = 1, LBM_BC_REGULARIZED = 2 };
LBM_API int lbm_set_boundary(lbm_handle h, int id, int kind, int method, int normal,
                             const double* value);

/* Smagorinsky constant C_S of an LBM_SMAG handle (Eq. taut; default 0.1,
 * the value Sec. 2.1.4 gives for LB models).  C_S = 0 is plain LBGK.
 * LBM_EINVAL for another model or C_S < 0 / not finite. */
LBM_API int lbm_set_smagorinsky(lbm_handle h, double cs);

/* ELBM alpha solve (Eq. alpha_cond): mode (LBM_ALPHA_*), Newton relative
 * step tolerance tol (default 1e-12), Newton evaluation cap max_iter
 * (default 20), near-equilibrium skip threshold skip_eps on max_i |x_i| with
 * x_i = (f_eq_i - f_i) / f_i (default 1e-3; alpha = 2 below it).
 * guard_steps / guard_tol are set by lbm_set_elbm_guard. */
LBM_API int lbm_set_elbm(lbm_handle h, int alpha_mode, double tol, int max_iter, double skip_eps);

/* Guarded modes: accept the first Newton correction <= guard_tol * alpha
 * (default 1e-6; the corrected alpha is then off by about its square) within
 * the first guard_steps (1..4, default 2) g evaluations from the guess;
 * otherwise Newton continues from there to the tolerance. */
LBM_API int lbm_set_elbm_guard(lbm_handle h, int guard_steps, double guard_tol);

/* ELBM entropic equilibrium form: 0 = product form with mass/momentum
 * restored (default; exact minimiser on D2Q9), 1 = polynomial Eq. equilibrium. */
LBM_API int lbm_set_elbm_feq(lbm_handle h, int variant);

/* Load the alpha surrogate's parameters (n = 1394 floats, host or device,
 * layout: mean[8], inv_std[8], W1[32][8], b1[32], W2[32][32], b2[32],
 * W3[32], b3, scale).  Weight matrices are rounded to BF16 on load;
 * accumulation is FP32.  Guess: alpha = s2 + scale * out (s2 as for
 * LBM_ALPHA_SERIES_GUARDED). */
LBM_API int lbm_load_alpha_mlp(lbm_handle h, const float* params, int n);

/* Request per-node alpha output (FP64, [nz][ny][nx]) on output steps
 * (ELBM only); read with lbm_get_alpha.  Costs 8 B/node on output steps. */
LBM_API int lbm_set_alpha_output(lbm_handle h, int on);

/* Rounding mode of FP16S / BF16S stores (LBM_ROUND_*); no effect on other
 * storage types. */
LBM_API int lbm_set_rounding(lbm_handle h, int mode);

/* Capture the n launches of lbm_step(h, n) in a CUDA graph and replay it on
 * later calls with the same n (useful for small, launch-bound domains). */
LBM_API int lbm_set_graph(lbm_handle h, int on);

/* ---- initialisation and stepping -------------------------------------- */

/* F = f_eq(rho, u) at every node (polynomial Eq. equilibrium for LBGK/MRT,
 * the model's own equilibrium for ELBM) and t = 0.  rho [nz][ny][nx], u
 * [D][nz][ny][nx], element type field_dtype.  Device memory is read
 * asynchronously on the stream.  Host memory: pinned (page-locked) buffers
 * are read in place by the kernel over the CPU-GPU link, pageable ones
 * through a staging copy; either way the call returns after the data have
 * been read, so the caller may reuse the buffers.  Errors: LBM_EINVAL,
 * LBM_ENOMEM, LBM_ECUDA. */
LBM_API int lbm_init_equilibrium(lbm_handle h, const void* rho, const void* u, int field_dtype);

/* Advance n >= 1 time steps (asynchronous on the stream).  The last step
 * writes rho and v (the force-shifted velocity of Eq. edm_momentum) of every
 * node, computed from the post-streaming distributions of that step.
 * In-kernel errors are reported by the next synchronising call. */
LBM_API int lbm_step(lbm_handle h, int n);

/* Steps taken since lbm_init_equilibrium / lbm_set_state. */
LBM_API int lbm_get_time(lbm_handle h, long long* t);

/* ---- readback ---------------------------------------------------------- */

/* rho [nz][ny][nx] and v [D][nz][ny][nx] of the last step (either pointer
 * may be NULL; device, pinned host or pageable host memory; pinned host
 * memory is written in place by the packing kernel).  Solid nodes give 0.
 * Synchronises the stream; returns LBM_ENAN if a non-finite value was found,
 * LBM_ESTATE before any step. */
LBM_API int lbm_get_macro(lbm_handle h, void* rho, void* u, int field_dtype);

/* Per-node alpha of the last output step (FP64, [nz][ny][nx]); requires
 * lbm_set_alpha_output(h, 1) before the step. */
LBM_API int lbm_get_alpha(lbm_handle h, double* alpha);

/* FP64 sums over fluid nodes of the last step's fields, reduced on the GPU
 * in a fixed order (bitwise reproducible): out[0] = sum rho,
 * out[1..D] = sum rho v_a, out[D+1] = sum rho |v|^2 / 2.  out is host
 * memory of D + 2 doubles.  Synchronises. */
LBM_API int lbm_reduce(lbm_handle h, double* out);

/* ELBM diagnostic mode (on = 1): every node whose alpha converged or was
 * accepted from the guess also evaluates the entropy condition at that alpha
 * by its definition (Eq. alpha_cond with per-direction logarithms, one more
 * g evaluation per node) and accumulates the residual |g(alpha)| / a_2,
 * a_2 = sum_i f_i x_i^2.  Clears all ELBM counters.  Off by default. */
LBM_API int lbm_set_elbm_diagnostics(lbm_handle h, int on);

/* Residual statistics of the steps run in diagnostic mode since it was set:
 * out[0] mean, out[1] max of |g(alpha)| / a_2, out[2] nodes sampled (host
 * memory, 3 doubles).  Synchronises. */
LBM_API int lbm_get_elbm_entropy_error(lbm_handle h, double* out);

/* Kinetic energy and enstrophy of the last step's velocity field (the
 * decaying-turbulence diagnostics of Sec. 5.2): out[0] = E = (1/2N) sum |v|^2,
 * out[1] = Omega = (1/2N) sum |curl v|^2 over all N nodes, the vorticity by
 * second-order central differences with periodic wrap (on D2Q9 only its z
 * component).  Accumulated in FP64 on the GPU in a fixed order (bitwise
 * reproducible).  out is host memory of 2 doubles.  LBM_ESTATE before the
 * first output step or when a geometry is set (the stencil assumes a fully
 * periodic domain).  Synchronises. */
LBM_API int lbm_kinetic_energy_enstrophy(lbm_handle h, double* out);

/* ELBM counters accumulated since init (host, 6 values): g evaluations,
 * skipped nodes, clamped nodes, nodes at the iteration cap, nodes accepted
 * from a guess, node updates.  Synchronises. */
LBM_API int lbm_get_elbm_stats(lbm_handle h, double* out);

/* Size in bytes of the raw state (the current distribution array). */
LBM_API size_t lbm_state_bytes(lbm_handle h);

/* Copy the raw state out / in (host or device pointer, lbm_state_bytes).
 * The layout is internal; a state is only meaningful for a handle created
 * with the same arguments (and access pattern).  set_state also sets the
 * step counter to t.  With the AB pattern the slots of solid nodes carry no
 * information: nothing reads them, and a step may overwrite those next to
 * fluid nodes with the rest state (whole-sector writes). */
LBM_API int lbm_get_state(lbm_handle h, void* dst, long long* t);
LBM_API int lbm_set_state(lbm_handle h, const void* src, long long t);

/* Synchronise the stream and return any pending device status. */
LBM_API int lbm_sync(lbm_handle h);

/* Number of kernels the handle has launched (for launch accounting). */
LBM_API long long lbm_launch_count(lbm_handle h);

/* ---- batched ensemble of independent D2Q9 domains ---------------------- */

typedef struct lbm_batch_ctx* lbm_batch;

/* ndom independent periodic LBGK domains of sizes nx[d] x ny[d] with
 * relaxation times tau[d] on lattice LBM_D2Q9 (the batched kernels are
 * D2Q9; other lattices give LBM_EINVAL), storage dtype LBM_F32S or
 * LBM_F16S.  All domains advance together in one persistent cooperative
 * launch per lbm_batch_step call; that launch is captured in a CUDA graph
 * and replayed. */
LBM_API int lbm_batch_create(int ndom, const int* nx, const int* ny, const double* tau,
                     int lattice, int dtype, lbm_batch* out);
LBM_API int lbm_batch_destroy(lbm_batch b);
LBM_API const char* lbm_batch_last_error(lbm_batch b);
LBM_API int lbm_batch_set_stream(lbm_batch b, void* cuda_stream);
/* Mask of domain d (host or device, ny[d]*nx[d] bytes, 0 fluid). */
LBM_API int lbm_batch_set_geometry(lbm_batch b, int d, const uint8_t* mask);
/* Guo body force of domain d. */
LBM_API int lbm_batch_set_force(lbm_batch b, int d, double fx, double fy);
/* f = f_eq(rho, u) for domain d; rho [ny][nx], u [2][ny][nx].  Every domain
 * must be initialised before the first lbm_batch_step.  Called again later,
 * it replaces domain d's state at the current step (the other domains and
 * the batch's time are unchanged). */
LBM_API int lbm_batch_init_equilibrium(lbm_batch b, int d, const void* rho, const void* u,
                               int field_dtype);
/* Choose the kernel variant, block size, tile shape, rows per thread and
 * CTAs per SM by timing a few steps of each candidate (CUDA events); restores
 * the state afterwards. */
LBM_API int lbm_batch_autotune(lbm_batch b);
/* Current launch configuration (5 ints): threads per CTA, CTAs, tile width,
 * tile rows, and the kernel variant: 1, 2 or 4 = the register kernel with
 * that many rows per thread and pass; -1 or -2 = the same with two
 * x-adjacent nodes per thread (pair loads and pair stores; tile width a
 * multiple of 64); 0 = the staged kernel, which copies each tile's inputs
 * into shared memory with bulk asynchronous copies into a ring of stages
 * while earlier tiles are updated.  Every variant gives the same bits. */
LBM_API int lbm_batch_get_config(lbm_batch b, int* out5);
/* Set the launch configuration (5 ints, as lbm_batch_get_config returns
 * them), e.g. one found by an earlier lbm_batch_autotune.  Threads per CTA
 * at most 512 and a multiple of the tile width, itself a multiple of 32
 * (64 for variants -1, -2); variant 0, 1, 2, 4, -1 or -2 (the
 * staged kernel's stages within 200 KB of
 * shared memory); CTAs between 1 and the number that can be co-resident (the
 * launch is cooperative).  LBM_EINVAL otherwise, with the configuration
 * unchanged. */
LBM_API int lbm_batch_set_config(lbm_batch b, const int* in5);
/* Advance every domain n steps in one persistent launch.  The per-step
 * grid barrier spins a bounded number of times; if it gives up, the kernel
 * exits and the next synchronising call returns LBM_ETIMEOUT. */
LBM_API int lbm_batch_step(lbm_batch b, int n);
LBM_API int lbm_batch_get_macro(lbm_batch b, int d, void* rho, void* u, int field_dtype);
/* Rounding mode of FP16S stores (LBM_ROUND_*; default LBM_ROUND_DITHER). */
LBM_API int lbm_batch_set_rounding(lbm_batch b, int mode);
/* Spin limit of the per-step grid barrier (default 2e7 spins of ~0.1 us,
 * about two seconds).  A wait that exceeds it ends the launch early and the
 * next synchronising call returns LBM_ETIMEOUT. */
LBM_API int lbm_batch_set_wait_limit(lbm_batch b, long long spins);
/* Fault-injection hook for testing the timeout paths.  on = 1: CTA 0 leaves
 * the first grid barrier of the next launch without arriving, so every other
 * CTA's bounded wait runs out.  on = 2 (staged kernel): the producer of each
 * CTA issues no copies for its first stage of the next launch and does not
 * arrive on it, so the consumers' wait for it runs out (the CTA then waits,
 * bounded, for the copies it did issue before it exits).  Either way the
 * next synchronising call returns LBM_ETIMEOUT and the state after that
 * launch is incomplete.  0 turns the hook off. */
LBM_API int lbm_batch_inject_missing_arrival(lbm_batch b, int on);
LBM_API int lbm_batch_sync(lbm_batch b);
LBM_API long long lbm_batch_launch_count(lbm_batch b);
LBM_API size_t lbm_batch_nodes(lbm_batch b);

/* ---- training the alpha surrogate --------------------------------------- */

/* Collect (features, alpha) pairs from the handle's next output step: for
 * every fluid node whose alpha was solved by full Newton (not skipped, not
 * clamped), the 8 invariant features (FP32) and the converged alpha (FP64).
 * Requires an ELBM handle.  Writes at most cap pairs to device buffers X
 * [cap][8] and y [cap]; *count receives the number written.  The sampling is
 * deterministic (every stride-th eligible node). */
LBM_API int lbm_elbm_collect_pairs(lbm_handle h, int stride, float* X_dev, double* y_dev, int cap,
                           int* count);

/* Train the surrogate on n pairs (device X [n][8] FP32, alpha [n] FP64) with
 * minibatch Adam entirely on the GPU (forward, backward and update kernels).
 * params (host, 1394 floats) holds the initial parameters (mean, inv_std and
 * scale are kept fixed) and receives the trained ones.  cfg = {epochs,
 * batch, lr, seed}; loss_out (host, epochs floats) receives the mean loss
 * per epoch.  Synchronises. */
LBM_API int lbm_mlp_train(const float* X_dev, const double* alpha_dev, int n, const double* cfg,
                  float* params, float* loss_out, void* cuda_stream);

/* Forward/backward kernels of the surrogate's training. */
#define LBM_MLP_FP32 0     /* FP32 CUDA-core kernel, one thread per sample */
#define LBM_MLP_BF16_TC 1  /* BF16 tensor-core MMA (FP32 accumulation) on the
                              network with entries 16 .. 1392 rounded to BF16
                              as lbm_load_alpha_mlp rounds them: the gradient
                              of the rounded network's loss updates the FP32
                              master copy.  Activations and back-propagated
                              gradients enter the MMAs as BF16 pairs hi + lo
                              (16 significant bits). */

/* Training configuration: epochs >= 1, batch >= 1 (clamped to n), lr > 0,
 * seed of the per-epoch shuffle, kernel LBM_MLP_*; reserved must be 0. */
typedef struct lbm_mlp_cfg {
    int epochs;
    int batch;
    double lr;
    unsigned long long seed;
    int kernel;
    int reserved;
} lbm_mlp_cfg;

/* Filled by lbm_mlp_train_cfg: Adam steps taken, device time of the
 * training launches (CUDA events around each epoch's forward/backward,
 * reduction and update launches), samples through forward and backward per
 * second of that time, and the last epoch's mean loss. */
typedef struct lbm_train_stats {
    int steps;
    int reserved;
    double gpu_ms;
    double samples_per_s;
    double final_loss;
} lbm_train_stats;

/* lbm_mlp_train with the configuration as a struct and the kernel choice;
 * stats may be NULL.  LBM_EINVAL for a bad configuration, and with
 * LBM_MLP_BF16_TC for an X_dev that is not 8-byte aligned (the kernel reads
 * feature pairs).  Synchronises.
 * lbm_mlp_train is this call with kernel LBM_MLP_FP32. */
LBM_API int lbm_mlp_train_cfg(const float* X_dev, const double* alpha_dev, int n,
                              const lbm_mlp_cfg* cfg, float* params, float* loss_out,
                              lbm_train_stats* stats, void* cuda_stream);

/* One forward+backward pass on a batch (device X [n][8], device targets
 * t [n]), for checking gradients: writes the loss and the gradient of every
 * parameter (host, 1394 floats; zeros for fixed entries).  Synchronises. */
LBM_API int lbm_mlp_grad(const float* X_dev, const float* t_dev, int n, const float* params,
                 float* loss, float* grad, void* cuda_stream);

/* lbm_mlp_grad with the LBM_MLP_BF16_TC kernel: the loss and gradient of the
 * network whose entries 16 .. 1392 are rounded to BF16.  X_dev must be
 * 8-byte aligned (LBM_EINVAL otherwise). */
LBM_API int lbm_mlp_grad_tc(const float* X_dev, const float* t_dev, int n, const float* params,
                            float* loss, float* grad, void* cuda_stream);

/* Same as lbm_mlp_grad, but allocates nothing.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc, such as
 * code running next to another framework's caching allocator that already
 * holds nearly all free device memory, or host code on a real-time path where
 * an allocation (which can synchronise the device) is not allowed.
 *   - All scratch (parameters, gradient, 64 partial rows, loss) lives in one
 *     file-scope static __device__ array of 364 KB, which every GPU that
 *     loads the library holds until the process exits.
 *   - n <= 4096 samples per call; larger n returns LBM_EINVAL (split the
 *     batch).  X_dev [n][8] and t_dev [n] must be device memory; params
 *     (1394 floats) may be host or device; loss and grad (1394 floats) are
 *     written to host or device memory.
 *   - Every call looks up the array's device address on the current device
 *     with cudaGetSymbolAddress (which allocates nothing), so the address is
 *     never stale, also after a device reset.
 *   - Every call shares the array and leaves its contents behind; the call
 *     clears what must start at zero.  Calls that overlap on the GPU (other
 *     streams, other threads) race on the array: serialise them.
 *   - Synchronises the stream and copies the loss to the host before it
 *     returns.  No cudaMalloc, cudaFree or allocating library routine is
 *     called. */
LBM_API int lbm_mlp_grad_static(const float* X_dev, const float* t_dev, int n,
                                const float* params, float* loss, float* grad,
                                void* cuda_stream);

/* Measured rate of the FP64 pipe of the current GPU (no counterpart in the
 * paper; the denominator of the ELBM kernel's roofline, whose FP64 alpha
 * solve of Eq. alpha_cond is bound by that pipe): every thread of a full
 * grid runs independent chains of FP64 fused multiply-adds for tens of
 * milliseconds; the best of three timed runs (CUDA events on cuda_stream)
 * gives FP64 warp instructions per second and FLOP/s (2 per FMA).
 * Synchronises the stream.  LBM_ECUDA on a CUDA error. */
LBM_API int lbm_probe_fp64_rate(void* cuda_stream, double* warp_inst_per_s, double* flops);

/* Message of the last failed lbm_mlp_* call on this thread. */
LBM_API const char* lbm_mlp_last_error(void);

/* Forward pass only: alpha guesses for n feature rows (device in and out). */
LBM_API int lbm_mlp_forward(const float* X_dev, int n, const float* params, float* alpha_dev,
                    void* cuda_stream);

/* ------------------------------------------------------------------------
 * Subdomain decomposition with ghost layers (Sec. 3.6), all subdomains on
 * this GPU.
 *
 * The domain is cut into nsub slabs of whole rows of its slowest axis (z on
 * D3Q19, y on D2Q9; slab s holds rows [floor(n s / nsub), floor(n (s+1) /
 * nsub))).  Each slab is stored with one ghost row on each side.  After every
 * step the populations that cross a slab face, the directions with a
 * component toward the neighbour (5 of 19 on D3Q19, 3 of 9 on D2Q9, Sec.
 * 3.6's direction-limited exchange), are collected from the slab's boundary
 * row into a linear send buffer, moved to the neighbour's receive buffer and
 * distributed into the neighbour's ghost row (periodic: the last slab's
 * neighbour is the first).  With overlap on (default) each step updates the
 * two boundary rows of every slab first and runs the exchange on a second
 * stream while the bulk rows update.  Results equal the single-domain
 * handle's bit for bit, for every model and storage type.  AB pattern only.
 * Arguments as lbm_create; nsub in [1, rows of the decomposed axis].
 * ------------------------------------------------------------------------ */
typedef struct lbm_multi_ctx* lbm_multi;

LBM_API int lbm_multi_create(int nx, int ny, int nz, int lattice, int model, double tau,
                             int dtype, int nsub, lbm_multi* out);
LBM_API int lbm_multi_destroy(lbm_multi m);
LBM_API const char* lbm_multi_last_error(lbm_multi m);
/* Stream of the updates (the exchange runs on an internal stream that
 * joins it every step). */
LBM_API int lbm_multi_set_stream(lbm_multi m, void* cuda_stream);
/* 1: boundary rows first, exchange overlapped with the bulk (default);
 * 0: whole slabs, then the exchange, on one stream. */
LBM_API int lbm_multi_set_overlap(lbm_multi m, int on);
/* Transfer of the face buffers: LBM_TRANSFER_STAGED (default) collects the
 * outgoing runs into a send buffer, copies it to the receiver's buffer and
 * distributes from there, as a run with one GPU per slab would;
 * LBM_TRANSFER_DIRECT stores the runs straight into the neighbour's ghost row
 * in one kernel (the form of a peer-to-peer store). */
enum { LBM_TRANSFER_STAGED = 0, LBM_TRANSFER_DIRECT = 1 };
LBM_API int lbm_multi_set_transfer(lbm_multi m, int mode);
/* Capture lbm_multi_step(n) as one CUDA graph (both streams) and replay it. */
LBM_API int lbm_multi_set_graph(lbm_multi m, int on);
/* As lbm_set_force / lbm_set_rounding / lbm_set_smagorinsky / lbm_set_elbm /
 * lbm_set_boundary, applied to every slab. */
LBM_API int lbm_multi_set_force(lbm_multi m, double fx, double fy, double fz);
LBM_API int lbm_multi_set_rounding(lbm_multi m, int mode);
LBM_API int lbm_multi_set_smagorinsky(lbm_multi m, double cs);
LBM_API int lbm_multi_set_elbm(lbm_multi m, int alpha_mode, double tol, int max_iter,
                               double skip_eps);
LBM_API int lbm_multi_set_boundary(lbm_multi m, int id, int kind, int method, int normal,
                                   const double* value);
/* Whole-domain mask and initial fields, laid out as for lbm_set_geometry and
 * lbm_init_equilibrium (host or device); each slab takes its rows plus the
 * neighbouring row on each side. */
LBM_API int lbm_multi_set_geometry(lbm_multi m, const uint8_t* mask);
LBM_API int lbm_multi_init_equilibrium(lbm_multi m, const void* rho, const void* u,
                                       int field_dtype);
/* n time steps, each followed by the ghost-row exchange.  Asynchronous. */
LBM_API int lbm_multi_step(lbm_multi m, int n);
/* Whole-domain rho and v of the last step (as lbm_get_macro).  Synchronises. */
LBM_API int lbm_multi_get_macro(lbm_multi m, void* rho, void* u, int field_dtype);
/* Bytes that cross slab faces per step: 2 nsub faces x directions x nodes
 * per row x storage element size (what a multi-GPU run would send); for a
 * rank handle, the bytes that rank sends per step (2 faces). */
LBM_API int lbm_multi_halo_bytes(lbm_multi m, long long* per_step);

/* ---- one slab per process (Sec. 3.6's multi-GPU decomposition) ----------
 * A rank handle holds only slab `rank` (0 <= rank < nsub) of the nsub-slab
 * decomposition above, for runs with one process (and GPU) per slab.  Each
 * step moves two face buffers of face_bytes each between neighbouring ranks
 * (periodic: rank nsub - 1's upper neighbour is rank 0), which the caller
 * does between lbm_multi_step_begin and lbm_multi_step_end:
 *   send + 0          the populations leaving through the upper face, to
 *                     rank + 1's recv + 0;
 *   send + face_bytes the populations leaving through the lower face, to
 *                     rank - 1's recv + face_bytes;
 *   recv + 0          from rank - 1 (lands in the lower ghost row);
 *   recv + face_bytes from rank + 1 (lands in the upper ghost row).
 * With nsub = 1 the rank is its own neighbour (copy send to recv).  Each
 * buffer is a list of (directions with a component along the decomposed
 * axis) runs of one padded row, in the handle's storage type.  The setters,
 * lbm_multi_set_geometry and lbm_multi_init_equilibrium work as for
 * lbm_multi_create (whole-domain arrays; the rank takes its rows), and
 * lbm_multi_get_macro writes only the rank's rows of whole-domain arrays.
 * Results equal the single-domain run bit for bit.  lbm_multi_step is
 * refused for nsub > 1 (LBM_ESTATE).  Errors: LBM_EINVAL for rank outside
 * 0..nsub-1, as lbm_multi_create otherwise. */
LBM_API int lbm_multi_create_rank(int nx, int ny, int nz, int lattice, int model, double tau,
                                  int dtype, int nsub, int rank, lbm_multi* out);
/* Device addresses of the rank handle's send and receive buffers (2 faces of
 * face_bytes each, laid out as above; owned by the handle).  LBM_EINVAL for a
 * handle from lbm_multi_create. */
LBM_API int lbm_multi_face_buffers(lbm_multi m, void** send, void** recv, size_t* face_bytes);
/* First half of one time step of a rank handle: updates the slab's two
 * boundary rows, collects their outgoing populations into the send buffers
 * on the exchange stream (lbm_multi_exchange_stream) and, with overlap on,
 * starts the bulk rows on the handle's stream.  output = 1 writes rho and v
 * of this step.  The send buffers are complete when the exchange stream
 * reaches this point; enqueue the transfer there (or synchronise that stream
 * first).  LBM_ESTATE if a begun step has not ended or before the initial
 * state. */
LBM_API int lbm_multi_step_begin(lbm_multi m, int output);
/* Second half: distributes the receive buffers into the ghost rows on the
 * exchange stream (after whatever the caller enqueued there) and makes the
 * handle's stream wait for it.  LBM_ESTATE without a begun step. */
LBM_API int lbm_multi_step_end(lbm_multi m);
/* The internal stream the exchange runs on (a cudaStream_t). */
LBM_API int lbm_multi_exchange_stream(lbm_multi m, void** stream);
/* Rows [lo, hi) of the decomposed axis that the handle updates. */
LBM_API int lbm_multi_rows(lbm_multi m, int* lo, int* hi);
/* Kernels this handle has launched (stream-collide, collect, distribute, pack). */
LBM_API long long lbm_multi_launch_count(lbm_multi m);
LBM_API int lbm_multi_sync(lbm_multi m);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
