/*
 * lbf.h - C ABI of a single-GPU (GB300, sm_103a) moment-represented lattice Boltzmann solver.
 *
 * The method (arXiv 2609.09160, Sec. 2): each lattice site stores only the Hermite coefficients
 * of the populations up to second order - the rescaled pressure p*, the velocity u and the
 * symmetric second-order tensor a2 (10 numbers) - and one time step is the fused pull update of
 * Eq. (pullLLB): every site rebuilds the regularized post-collision populations of its Q
 * neighbours (Eqs. reqtfeq, hermite_teq) including the Guo source (Eq. guoforce), streams them
 * in and takes their moments, followed by the half-force correction of Eq. (corr). D3Q19 and
 * D3Q27 with second-order truncation are supported, and D3Q27h: the D3Q27 velocities with the
 * complete Hermite basis, whose third- to sixth-order coefficients are rebuilt from the stored
 * moments by the recursive closure (Sec. 2; the state is the same 10 fields). The conservative
 * Allen-Cahn phase field of Eq. (ACeq) with the force split of Sec. 2 (capillary, body, pressure
 * and viscous-gradient forces) provides the two-component coupling, with density and viscosity
 * contrast.
 *
 * Conventions shared by every call
 *  - Sites are indexed (z, y, x) with x fastest; a field is nz*ny*nx contiguous values.
 *  - Public moment layout ("public state"): 10 fields [p*, ux, uy, uz, Axx, Ayy, Azz, Axy, Axz,
 *    Ayz] of nz*ny*nx values each, A = a2 the total second coefficient of Eq. (corr). This is the
 *    layout of lbf_set_moments / lbf_moments and of the adjoint cotangents.
 *  - Internal state ("state buffer"): the same 10 fields in the storage dtype, with the tensor
 *    stored as N = A - u u and, for 16-bit storage, every group multiplied by a power of two.
 *    Callers treat it as opaque bytes of size lbf_state_bytes().
 *  - 16-bit storage: by default a time step rounds the p* and u values it stores
 *    stochastically (unbiased), with random bits from a counter-based generator keyed by the site
 *    and the context's count of steps taken, so results are bitwise reproducible for the same
 *    sequence of calls; lbf_params.rounding selects round-to-nearest instead. The N fields, which
 *    a step recomputes rather than accumulates, and every value loaded by lbf_set_moments round
 *    to nearest.
 *  - Every call is ordered on the context's CUDA stream (lbf_params.stream) and returns without
 *    waiting for the GPU, except lbf_reduce and lbf_synchronize, which wait for the stream.
 *  - The library allocates no device memory: the caller provides one workspace of
 *    lbf_workspace_bytes() bytes (256-byte aligned) that the context uses until lbf_destroy.
 *  - Errors are returned as lbf_status codes; nothing aborts and no kernel traps. The message of
 *    the last error on the calling thread is available from lbf_last_error().
 *  - Boundaries: every axis is periodic; sites flagged solid in the mask are walls with halfway
 *    bounce-back (the paper only states "no-slip walls"). Solid sites keep their moments.
 */
#ifndef LBF_H
#define LBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbf_ctx lbf_ctx; /* opaque, host-side; owns no device memory */

/* lattices: D3Q19 and D3Q27 truncated at second order; D3Q27H = D3Q27 velocities with the complete
   Hermite basis (post-collision coefficient of every supported multi-index m: u^m + (1 - omega)
   times the closure of N + half the Guo source, Sec. 2). D3Q27H has no adjoint and no population
   representation (LBF_ENOTSUP). */
enum { LBF_D3Q19 = 19, LBF_D3Q27 = 27, LBF_D3Q27H = 127 };

/* storage / transfer dtypes; F64 storage computes in FP64, every other storage in FP32 */
enum { LBF_F64 = 0, LBF_F32 = 1, LBF_F16 = 2, LBF_BF16 = 3 };

/* rounding of the values a time step stores in 16-bit storage (not in the paper, which has no
   16-bit storage). Round-to-nearest discards every update smaller than half a unit in the last
   place, so a slowly evolving flow freezes in place on large lattices; stochastic rounding keeps
   the expected stored value exact. */
enum { LBF_ROUND_STOCHASTIC = 0, LBF_ROUND_NEAREST = 1 };

typedef enum {
  LBF_OK = 0,
  LBF_EINVAL = 1,      /* bad argument: sizes, tau <= 0.5, null pointer, unsupported combination */
  LBF_ENOMEM = 2,      /* workspace too small or misaligned */
  LBF_ECUDA = 3,       /* a CUDA runtime call failed; see lbf_last_error() */
  LBF_EUNSTABLE = 4,   /* a step produced a non-finite value or |u| > 0.4 */
  LBF_EINTERNAL = 5,   /* broken internal invariant */
  LBF_ENOTSUP = 6      /* a feature the library does not build (see lbf_last_error()) */
} lbf_status;

typedef struct {
  int lattice;          /* LBF_D3Q19, LBF_D3Q27 or LBF_D3Q27H */
  int nx, ny, nz;       /* >= 1 each */
  int storage;          /* LBF_F64, LBF_F32, LBF_F16 or LBF_BF16 */
  double tau;           /* single-component relaxation time, > 0.5; nu = (tau - 1/2)/3
                           (text under Eq. pullLB). Ignored when two_component != 0. */
  double force[3];      /* uniform body force per unit volume, F^b of Sec. 2 */
  const void* force_field; /* optional DEVICE pointer, [3][nz][ny][nx], FP64 when storage is
                           LBF_F64 else FP32; added to force[]; borrowed: must stay valid and may
                           be rewritten by the caller between steps; NULL = none. */
  const uint8_t* mask;  /* optional HOST pointer, nz*ny*nx bytes, nonzero = solid; copied by
                           lbf_create; NULL = all fluid. */
  int two_component;    /* nonzero: conservative Allen-Cahn phase field (Eq. ACeq) coupled through the
                           force split of Sec. 2, F = F^s + F^b + F^p + F^nu: the capillary force
                           F^s = mu grad phi, F^b = force + rho(phi) body_accel, and with
                           rho_l != rho_h the pressure force F^p = -p* cs2 grad rho and the
                           viscous-gradient force F^nu = -(nu omega / cs2) a*_neq . grad rho (a*
                           the raw streamed moments). Walls (mask) keep phi frozen and u = 0 at
                           solid sites (no wetting model). A density contrast or walls need
                           LBF_F32 or LBF_F64 storage; force_field is not supported. */
  double rho_l, rho_h;  /* densities of the light (phi = 0) and heavy (phi = 1) phase */
  double tau_l, tau_h;  /* relaxation times; nu(phi) = nu_l + phi (nu_h - nu_l) */
  double sigma, width;  /* surface tension and interface width W: beta = 12 sigma/W,
                           kappa = 3 sigma W / 2, lambda = 4 D / W */
  double diffusivity;   /* interface diffusivity D of Eq. (ACeq) */
  double scale_hint[3]; /* 16-bit storage: expected max |p*|, |u|, |A - u u|; 0 = take each from
                           the state given to lbf_set_moments */
  void* stream;         /* cudaStream_t used for every call; NULL = legacy default stream */
  int rounding;         /* LBF_ROUND_STOCHASTIC (0, default) or LBF_ROUND_NEAREST: 16-bit stores of
                           a time step; ignored for FP32/FP64 storage */
  int populations;      /* nonzero: population-form reference representation - the context stores
                           the Q populations f(x, t) of Eq. (pullLB) after streaming instead of
                           the 10 moments (the memory layout the paper compares against, Sec. 3)
                           and steps them with the same regularized collision (collide, then push
                           with halfway bounce-back). Every call keeps its meaning (moments in,
                           moments out); state buffers hold Q fields; the sums of lbf_reduce are
                           computed from the state when asked. FP32/FP64 storage, single
                           component, no adjoint (LBF_ENOTSUP). */
  double body_accel[3]; /* two_component only: uniform body acceleration a; F^b gains rho(phi) a
                           (the layered Poiseuille flow of Sec. 4 is driven this way). Must be 0
                           for a single component (use force). */
} lbf_params;

/* Workspace bytes the context needs for these parameters, 0 if the parameters are invalid.
   Host-only: makes no CUDA call. The moment buffers take 2 * 10 * nx*ny*nz * sizeof(storage).
   Paper: Sec. 3 memory model (10 moment fields per site, flip/flop buffers). */
size_t lbf_workspace_bytes(const lbf_params* params);

/* Checks parameters on the host without touching the GPU.
   Paper: Sec. 2 (the lattices; tau > 1/2 from nu = cs2 (tau - 1/2) under Eq. pullLB). */
lbf_status lbf_validate(const lbf_params* params);

/* Creates a context on the current CUDA device. workspace: DEVICE pointer, 256-byte aligned, at
   least lbf_workspace_bytes(params) bytes, owned by the caller and kept alive until lbf_destroy.
   The state is zero (fluid at rest) until lbf_set_moments.
   Paper: Sec. 2 statement of the problem (lattice, domain, tau, walls, body force F^b, phase-field
   parameters of Eq. ACeq) and Sec. 3 (flip/flop moment buffers). */
lbf_status lbf_create(lbf_ctx** out, const lbf_params* params, void* workspace, size_t bytes);

/* Loads the public state. src: 10 fields (public layout) of dtype LBF_F64 or LBF_F32, HOST or
   DEVICE memory (detected); phi: nz*ny*nx phase-field values of the same dtype and memory kind,
   required when two_component, else ignored. Host sources are copied through a staging area of
   the workspace; pinned host memory makes the copies asynchronous. For 16-bit storage the
   power-of-two scales are chosen here (unless scale_hint is set). Also computes the initial
   phase-field force when two_component.
   Paper: Sec. 2, the velocity-pressure Hermite coefficients a(0) = p*, a(1) = u, a(2) of
   Eqs. reqtfeq, hermite_teq; the capillary force F^s = mu grad phi of the force split. */
lbf_status lbf_set_moments(lbf_ctx* ctx, const void* src, int src_dtype, const void* phi);

/* Advances n >= 0 time steps (one fused kernel per step; two more phase-field kernels per step
   when two_component). The conservation sums of the final state are computed on the last step.
   Returns LBF_EUNSTABLE if an earlier lbf_reduce/lbf_synchronize saw the instability flag.
   Paper: Eq. (pullLLB) followed by Eq. (corr), Sec. 2; with two_component also Eq. (ACeq) by FTCS
   and the force split F = F^s + F^b (Sec. 2). */
lbf_status lbf_step(lbf_ctx* ctx, int n);

/* Writes the public state (dst, 10 fields) and, when two_component and phi_dst != NULL, the phase
   field, in dtype LBF_F64 or LBF_F32, to HOST or DEVICE memory (detected). Asynchronous for device
   or pinned host destinations.
   Paper: Sec. 2, the velocity-pressure Hermite coefficients (p*, u, a(2)) after Eq. (corr). */
lbf_status lbf_moments(lbf_ctx* ctx, void* dst, int dst_dtype, void* phi_dst);

/* Waits for the stream and returns FP64 [sum p*, sum ux, sum uy, sum uz, sum phi, sum u.u] over
   fluid sites of the current state (out: HOST, 6 doubles). LBF_EUNSTABLE if any step so far saw a
   non-finite value or |u|^2 > 0.16 (out is still filled).
   Paper: Sec. 4, the kinetic-energy diagnostic E(t) of the Taylor-Green test (sum u.u), and the
   totals that Eq. (pullLLB) conserves (sum p*, sum u without force, sum phi of Eq. ACeq). */
lbf_status lbf_reduce(lbf_ctx* ctx, double* out);

/* The sums of lbf_reduce without waiting: enqueues a copy of the 6 FP64 sums of the current state
   into dst (6 doubles, DEVICE or pinned HOST memory) on the stream and returns. dst holds them once
   the stream has passed the copy (after lbf_synchronize, or an event the caller records). A step
   that follows overwrites the library's copy, not dst, so one dst per step collects a time series
   without stalling the stream. Pageable host memory also works, but the copy then waits (CUDA's
   rule for such copies). Errors of the steps (LBF_EUNSTABLE, LBF_EINTERNAL) are reported by the
   next lbf_synchronize or lbf_reduce, not here.
   Paper: as lbf_reduce (Sec. 4 energy diagnostic E(t); the totals Eq. (pullLLB) conserves). */
lbf_status lbf_reduce_async(lbf_ctx* ctx, double* dst);

/* Waits for the stream; LBF_EUNSTABLE as for lbf_reduce; LBF_EINTERNAL if a step was abandoned
   (a bounded TMA wait gave up, or an index check of the LBF_DEBUG build failed). Such an error is
   reported once and then cleared, so the context stays usable; the state it left is incomplete.
   Paper: no counterpart (stream completion and the library's instability check). */
lbf_status lbf_synchronize(lbf_ctx* ctx);

/* Kernel launches one time step of lbf_step issues with this context's configuration, the FP64
   sums included: 1 for the fused step, 2 when walls in a band of rows split it (the rows near the
   walls on a side stream, the other rows on the context's stream), plus 2 with two components
   (phase-field advance and forces). 0 for a NULL context.
   Paper: no counterpart (launch structure of the implementation). */
int lbf_kernels_per_step(const lbf_ctx* ctx);

/* Bytes of one internal state buffer (10 * nx*ny*nz * sizeof(storage)).
   Paper: Sec. 3 memory model (10 fields per site). */
size_t lbf_state_bytes(const lbf_ctx* ctx);

/* Copies the current internal state to a caller DEVICE buffer of lbf_state_bytes()
   (checkpointing; stream-ordered).
   Paper: no counterpart (checkpoints of the Sec. 3 moment buffers). */
lbf_status lbf_copy_state(lbf_ctx* ctx, void* dst);

/* Loads the current internal state from a caller DEVICE buffer of lbf_state_bytes() (restart;
   stream-ordered).
   Paper: no counterpart (checkpoints of the Sec. 3 moment buffers). */
lbf_status lbf_load_state(lbf_ctx* ctx, const void* src);

/* One single-component step from internal state src to internal state dst (caller DEVICE
   buffers of lbf_state_bytes(); src != dst). The context's own state is not touched. Solid
   sites of dst are not written. A src that is not 16-byte aligned is read without TMA.
   Paper: Eq. (pullLLB) followed by Eq. (corr), Sec. 2. */
lbf_status lbf_step_state(lbf_ctx* ctx, const void* src, void* dst);

/* Adjoint of one single-component step (not in the paper; the discrete adjoint of the step
   above). Given the internal states at t and t+1 (state_t, state_t1), and lambda_in = dL/dM(t+1)
   in the public layout (10 fields, FP64 when storage is LBF_F64 else FP32, DEVICE), writes
   lambda_out = dL/dM(t) (same layout and dtype, DEVICE, distinct from lambda_in) and adds
   dL/dF contributed by this step to grad_force (DEVICE, FP64, [3][nz][ny][nx]) for the total
   per-site force (uniform force + force_field). Solid sites pass lambda through unchanged and
   get no force gradient. Not available for 16-bit storage or two_component (LBF_ENOTSUP).
   Paper: no counterpart (the exact transpose of the linearised Eq. (pullLLB) + Eq. (corr)). */
lbf_status lbf_adjoint_step(lbf_ctx* ctx, const void* state_t, const void* state_t1, const void* lambda_in,
                            void* lambda_out, double* grad_force);

/* One fused single-component step without any device allocation, for callers that cannot
   allocate device memory: code running under another framework's memory pool or a fixed memory
   plan, or an embedder that only receives device buffers from elsewhere, cannot call cudaMalloc
   and so cannot provide the workspace lbf_create needs. (The paper has no counterpart; this is a
   deployment entry point.)
   params: lattice, nx/ny/nz, storage (LBF_F32 or LBF_F64 only), tau, force, force_field and stream
   as for lbf_create; params->mask and the two-component fields are not used.
   src, dst: caller DEVICE buffers of 10*nx*ny*nz values in the internal state layout (the bytes
   lbf_copy_state produces; for FP32/FP64 storage the tensor fields hold a2 - u u), src != dst.
   A src that is 16-byte aligned (and whose rows are a multiple of 16 bytes) is staged with TMA;
   any other src is read by the kernel variant that loads every site directly.
   mask_device: optional DEVICE mask, nx*ny*nz bytes, nonzero = solid (solid sites of dst are not
   written). sums_device: optional DEVICE output of 6 doubles, the sums of lbf_reduce for dst.
   flags_device: optional DEVICE output of one unsigned word, written after the step: 0 = the step
   completed; bit 0 = a non-finite value or |u|^2 > 0.16 was stored (unstable); bit 1 = a TMA plane
   load did not complete in time and bit 2 = a TMA stage was misaligned (in both cases the step was
   abandoned and dst is incomplete); bit 3 = an index check of the LBF_DEBUG build failed.
   The library keeps the per-block partial sums, a block counter and the error flags in one static
   device array of 1 MiB + 256 bytes per GPU that loads it (held until the process exits), enough
   for 16384 CTAs: ceil(nx/30) * ceil(ny/R) must not exceed 16384, else LBF_EINVAL, where R is the
   number of output rows per CTA of the kernel the parameters select (FP32: 8 for D3Q19 and for
   D3Q27/D3Q27H with a mask, 6 for D3Q27/D3Q27H without one; FP64: 4); the error message names R.
   The first call on a device looks up that array's device address (cudaGetSymbolAddress) and
   keeps it for later calls. Every call clears the counter and flags it needs (cudaMemsetAsync, which does not
   allocate). All calls share the array: calls that can overlap on the GPU (other streams, other
   host threads) race on it; calls ordered on one stream are safe. Asynchronous on params->stream.
   Paper: no counterpart; it runs the step of Eq. (pullLLB) + Eq. (corr), Sec. 2. */
lbf_status lbf_step_static(const lbf_params* params, const void* src, void* dst, const uint8_t* mask_device,
                           double* sums_device, unsigned* flags_device);

/* Releases the host-side context. The workspace stays owned by the caller.
   Paper: no counterpart. */
lbf_status lbf_destroy(lbf_ctx* ctx);

/* Name of a status code ("LBF_OK", ...), a static string.
   Paper: no counterpart. */
const char* lbf_status_string(int status);

/* Message of the last error on the calling thread (empty if none), valid until the next call.
   Paper: no counterpart. */
const char* lbf_last_error(void);

/* ABI version of this library.
   Paper: no counterpart. */
int lbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBF_H */
