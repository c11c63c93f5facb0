/*
 * adg.h -- C ABI of the GB300 asynchronous discontinuous Galerkin (ADG / ADG-AT) solver.
 *
 * The library advances 1D nodal DG discretisations of u_t + f(u)_x = 0 on a periodic
 * interval with the fully discrete strong-stability-preserving RK3 step (or the paper's
 * low-storage schemes), on one GPU, in FP64 (the composed step of upwind advection in 58-bit
 * block fixed point: adg_config.variant). Elements are split into P contiguous "processing elements" (PEs); at PE faces the
 * numerical flux uses data of a delayed time level taken from a seeded delay table and a
 * device ring buffer, combined by the standard flux or the asynchrony-tolerant (AT) flux.
 *
 * Paper: "Asynchronous discontinuous Galerkin method" (arXiv 2404.03399):
 *   - problem and discretisation: Section 2, Eqs. wave, DGsolution, DGweakform, DGscheme;
 *   - PE decomposition and delays k in {0..L-1}: Section 3, Eq. asyncEulerDG;
 *   - conservative common delayed level: Section 4.1, Eq. asyncEulerDGconserved;
 *   - AT flux: Section 5, Eqs. at-flux-gen, at-flux-constraints, Table 1;
 *   - delay emulation by binned uniform draws: Section 6.1.
 *
 * Conventions (all entry points):
 *   - Every function returns an adg_status; no C++ exception crosses the ABI. After a
 *     failure adg_last_error(ctx) holds a message (for a NULL ctx: the thread's last one).
 *   - Nodal fields passed across the ABI are FP64, contiguous, shape (K, p+1), row-major
 *     (element-major: u[e*(p+1) + i] is node i of element e). Buffers marked "_dev" are
 *     device pointers on the current CUDA device; "_host" are host pointers.
 *   - The caller owns every buffer it passes; the library copies what it keeps and never
 *     frees caller memory. The library owns its context (state, ring, tables, graphs),
 *     released by adg_destroy.
 *   - Work is ordered on the CUDA stream given at init (NULL = legacy default stream).
 *     Functions that return host values synchronise that stream before returning.
 *   - There is no CPU fallback: without a usable CUDA device adg_init returns ADG_ECUDA.
 */
#ifndef ADG_H
#define ADG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adg_ctx adg_ctx;

typedef enum {
  ADG_OK = 0,
  ADG_EINVAL = -1,     /* invalid argument or configuration */
  ADG_ENOMEM = -2,     /* device or host allocation failed */
  ADG_ECUDA = -3,      /* CUDA runtime error (or no device) */
  ADG_ENONFINITE = -4, /* a NaN or Inf was found in the state */
  ADG_ETIMEOUT = -5,   /* a bounded device wait ran out */
  ADG_ESTATE = -6      /* call not valid in the context's current state */
} adg_status;

enum { ADG_ADVECTION = 0, ADG_BURGERS = 1, ADG_EULER = 2 }; /* a u | u^2/2 | 1D Euler */
enum { ADG_UPWIND = 0, ADG_LLF = 1 };                 /* Section 6.1 fluxes */
enum {                                                  /* time integrator */
  ADG_RK1 = 1,      /* forward Euler, Eq. EulerDG */
  ADG_RK2 = 2,      /* the two-stage RK of Eq. dg2-rk2 */
  ADG_SSPRK3 = 3,   /* three-stage SSP-RK3 (Shu and Osher) */
  ADG_LSRK3 = 4,    /* Williamson's three-stage third-order 2N low-storage scheme */
  ADG_LSRK4 = 5     /* Carpenter and Kennedy's five-stage fourth-order 2N scheme */
};
enum { ADG_SYNC = 0, ADG_ASYNC = 1, ADG_ASYNC_AT = 2 };/* DG | ADG | ADG-AT */
enum {
  ADG_VARIANT_AUTO = 0,
  ADG_VARIANT_STAGED = 1,
  ADG_VARIANT_COMPOSED = 2,
  ADG_VARIANT_COMPOSED_FIXED = 3
};

#define ADG_MAX_P 4        /* polynomial degree 1..4 (2..5 LGL nodes) */
#define ADG_MAX_L 16       /* delays 0..L-1 with L <= 16 */
#define ADG_MAX_Q 5        /* AT order 1..5 */

/*
 * Run configuration (Section 2: mesh, degree, flux, RK; Section 3: P and L; Section 5:
 * AT order; Section 6.1: probability set and seeded draws).
 *   pde, flux : ADG_ADVECTION with ADG_UPWIND, or ADG_BURGERS with ADG_LLF.
 *   rk        : ADG_SSPRK3 (default; every variant, adg_grad and batches), or one of the
 *               low-storage schemes of the kind Section 6 integrates with, run in Williamson's
 *               2N form (dU_s = A_s dU_{s-1} + dt L(U_{s-1}), U_s = U_{s-1} + B_s dU_s) by the
 *               staged kernels: ADG_RK1, ADG_RK2 (Eq. dg2-rk2 as A = (0, -1),
 *               B = (1, 1/2)), ADG_LSRK3, ADG_LSRK4. At PE faces stage s of a step reads the
 *               stage-s inputs of the delayed step. A low-storage scheme is a single-instance
 *               option: adg_batch_init and adg_grad reject it (ADG_EINVAL), and so does a
 *               composed variant (ADG_VARIANT_COMPOSED, ADG_VARIANT_COMPOSED_FIXED).
 *   K, p, P   : elements, polynomial degree (1..ADG_MAX_P), PEs; K % P == 0, P >= 1.
 *   x0, x1    : periodic domain [x0, x1], x1 > x0.
 *   a         : advection speed (advection only).
 *   cfl, dt   : if dt > 0 it is the fixed time step; else dt = (cfl * dx) / speed, with
 *               dx = (x1 - x0) / K and speed = |a| (advection) or max|u0| (Burgers).
 *   mode      : ADG_SYNC, ADG_ASYNC (standard flux at the delayed level) or ADG_ASYNC_AT.
 *   L         : delays are in {0..L-1} (1 <= L <= ADG_MAX_L).
 *   at_order  : AT order q (1..ADG_MAX_Q) for ADG_ASYNC_AT; 0 selects p+1 capped at
 *               ADG_MAX_Q. ADG_ASYNC uses q = 1.
 *   seed, probs: delays drawn from SplitMix64(seed) output n*P + j for step n, PE face j,
 *               binned by probs[0..L-1] (NULL = uniform 1/L), Section 6.1.
 *   delay_table, table_steps: optional caller table, uint8 [table_steps][P], host memory,
 *               used periodically (row n mod table_steps at step n); overrides the seed.
 *               Every entry must be < L.
 *   caa_sync  : 0 (default), or the communication-avoiding cycle of Section 6.3 as the
 *               delay source: every period of caa_sync + L steps has caa_sync synchronised
 *               steps (delay 0), then L steps without communication with delays 0, 1, ..,
 *               L-1 at every PE face (caa_sync = 2, L = 3: the 2D experiment's cycle).
 *               Overrides seed and probs; 0 <= caa_sync <= 64; ADG_EINVAL together with a
 *               caller table.
 *   nu        : 0 (default), or the viscosity of viscous Burgers u_t + u u_x = nu u_xx
 *               (Eq. burgers; pde ADG_BURGERS, nu > 0, finite) by the local DG method of
 *               Section 6: q = u_x with the alternating flux uhat = u^-, the viscous flux
 *               qhat = q^+, Lax-Friedrichs for u u_x; at PE faces uhat, the Lax-Friedrichs
 *               flux and qhat all take the AT sum over the common delayed level. Staged
 *               kernels, any rk; dt from cfl uses max|u0| only (the diffusive limit
 *               nu dt / dx^2 is the caller's: give dt or a small cfl). Single instances only
 *               (adg_batch_init, adg_grad: ADG_EINVAL).
 *   pde ADG_EULER (flux ADG_LLF): the one-dimensional Euler equations of Section 6's Sod
 *               experiment, U = (rho, m, E), E = rho u^2 / 2 + p / 0.4 (gamma = 1.4), local
 *               Lax-Friedrichs flux, SSP Runge-Kutta in Shu and Osher's form (rk ADG_RK1,
 *               ADG_RK2 = SSP-RK2 as in the paper, ADG_SSPRK3), AT sums of the delayed flux
 *               at PE faces. Fields are (3, K, p+1) row-major (u0_dev, adg_get_state; the
 *               components one after another). limiter = 1 applies the TVB-minmod (MUSCL)
 *               slope limiter to every stage output, keeping slopes |a1| <= tvb_m dx^2 / 2
 *               (tvb_m = 0: minmod); its stencil ends at PE faces. dt must be given (> 0).
 *               adg_integral reports the integral of rho. Single instances, staged kernels;
 *               batches, adg_grad and the composed variants reject it (ADG_EINVAL).
 *   variant   : ADG_VARIANT_AUTO (0), ADG_VARIANT_STAGED (1): one kernel per RK stage, or
 *               ADG_VARIANT_COMPOSED (2): the stages of one step of upwind advection with a > 0
 *               (SSP-RK3, or a low-storage scheme of up to three stages) composed into one
 *               stencil per step in FP64, with the delayed / AT flux at PE faces added as a
 *               correction to the elements around each face (needs K/P >= 8 when there are PE
 *               faces), or
 *               ADG_VARIANT_COMPOSED_FIXED (3): the composed step (also for the five-stage
 *               ADG_LSRK4, which then needs K/P >= 10) evaluated in 58-bit block fixed point:
 *               int64 values at one scale per field and step (from the largest magnitude in
 *               u^n), coefficients rounded to 2^-58, 32 x 32 -> 64-bit integer products. A sum
 *               of n terms is off by less than n/2 + 1/2 units of 2^-57 max|u^n|, so the error is
 *               bounded relative to the field's maximum (as FP64's is relative to a sum's
 *               largest term), not per value: values below about 2^-55 max|u^n| keep no
 *               digits. The int64 state holds each element's coordinates in the block basis
 *               of the element operator where that basis is well conditioned (p = 1 .. 4; see
 *               adg_get_fixed_basis), which multiplies that bound by the basis's condition
 *               number (at most 64; 15.1 at p = 3). The state stays in int64 from step to step
 *               and across adg_step calls;
 *               the FP64 state is formed (rounded once) when it is read (adg_get_state,
 *               adg_integral, adg_misfit, adg_check_finite, adg_grad), so every splitting of a
 *               run into calls gives the same result. It needs every composed coefficient below
 *               2 in magnitude (small Courant numbers; ADG_EINVAL otherwise). Results below
 *               2^-1022 are flushed to zero, and a NaN or infinity anywhere in u^n makes all of
 *               u^{n+1} NaN. AUTO picks COMPOSED_FIXED, else COMPOSED, where they apply; a
 *               batch with AUTO times every kind of step that all its instances admit (fixed
 *               point, FP64 composed, staged) at init and keeps the fastest (adg_get_variant
 *               reports it). All give the same scheme up to rounding.
 *   ept       : elements per thread of the composed-step kernels (not a paper quantity):
 *               0 (default) lets init choose: the FP64 step times 1, 2 and 4 and keeps the
 *               fastest; a single instance's fixed-point step takes 2 consecutive elements for
 *               even K (measured faster throughout) and 1 for odd K or K < 2048; a batch's
 *               fixed-point step times 1, 2 and 4 (work items of 256, 512 or 1024 elements);
 *               1, 2 or 4 forces one (ADG_EINVAL where that kernel has no such form). Results
 *               do not depend on it.
 */
typedef struct {
  int32_t pde;
  int32_t flux;
  int32_t rk;
  int32_t K, p, P;
  double x0, x1;
  double a;
  double cfl, dt;
  int32_t mode;
  int32_t L;
  int32_t at_order;
  uint64_t seed;
  const double *probs;
  const uint8_t *delay_table;
  int64_t table_steps;
  int32_t variant;
  int32_t caa_sync;
  double nu;
  int32_t limiter;
  double tvb_m;
  int32_t ept;
} adg_config;

/* Fill cfg with defaults: advection, upwind, SSP-RK3, [0, 2 pi], a = 1, cfl = 0.1, sync. */
void adg_config_default(adg_config *cfg);

/*
 * Create a solver context for one instance and load the initial nodal field.
 *   cfg     : configuration (copied; probs and delay_table are copied too).
 *   u0_dev  : initial nodal values, device FP64 (K, p+1) row-major.
 *   stream  : cudaStream_t (as void*), NULL for the default stream.
 *   out     : receives the context; *out is NULL on failure.
 * Errors: ADG_EINVAL (bad config, or a non-finite u0), ADG_ENOMEM, ADG_ECUDA.
 */
int adg_init(const adg_config *cfg, const double *u0_dev, void *stream, adg_ctx **out);

/*
 * adg_init with the initial field in host memory (the same (K, p+1) row-major FP64 layout,
 * three fields for ADG_EULER). Pinned memory (cudaHostAlloc, cudaMallocHost, cudaHostRegister)
 * and managed memory are read in place by the kernel that lays the field out in node planes,
 * so the transfer over the host link and the layout are one pass; pageable memory is first
 * copied into the instance's scratch field. The call synchronises, so u0_host may be reused or
 * freed when it returns. Errors as adg_init, and ADG_EINVAL when u0_host is device memory.
 */
int adg_init_host(const adg_config *cfg, const double *u0_host, void *stream, adg_ctx **out);

/*
 * Create one context that advances n independent instances together (batched runs):
 * every stage launch covers all instances; chunks of steps replay one CUDA graph.
 * cfgs[i], u0_devs[i] as in adg_init. Only ADG_ADVECTION / ADG_UPWIND instances.
 */
int adg_batch_init(const adg_config *cfgs, const double *const *u0_devs, int32_t n,
                   void *stream, adg_ctx **out);

/* Advance every instance by nsteps >= 0 steps of its Runge-Kutta scheme (SSP-RK3 unless rk
 * says otherwise; Section 4.2.1 structure, Eq. EulerDG-style explicit updates; Eq.
 * asyncEulerDGconserved at PE faces). Asynchronous: returns once the work is queued. */
int adg_step(adg_ctx *c, int64_t nsteps);

/* Advance to time t_end: ceil(t_end/dt - 1e-9) - (current step) steps (none if <= 0). */
int adg_run(adg_ctx *c, double t_end);

/* Copy instance `index` (0 for a single-instance context) to u_dev, device (K, p+1)
 * row-major FP64, and its step counter to *step_out (may be NULL). Synchronises. */
int adg_get_state(adg_ctx *c, int32_t index, double *u_dev, int64_t *step_out);

/* adg_get_state into host memory u_host ((K, p+1) row-major FP64, three fields for
 * ADG_EULER): pinned or managed memory is written in place by the layout kernel over the host
 * link; pageable memory through a device field that holds no state and one copy. Synchronises.
 * ADG_EINVAL when u_host is device memory. */
int adg_get_state_host(adg_ctx *c, int32_t index, double *u_host, int64_t *step_out);

/* The fixed time step of instance `index`. */
int adg_get_dt(adg_ctx *c, int32_t index, double *dt_out);

/* How instance `index` steps (not a paper quantity): *variant_out = the ADG_VARIANT_* in use
 * (STAGED, COMPOSED or COMPOSED_FIXED; AUTO resolved), *ept_out = elements per thread of the
 * composed-step kernel chosen at init (1 for the staged kernels). Either pointer may be NULL. */
int adg_get_variant(adg_ctx *c, int32_t index, int32_t *variant_out, int32_t *ept_out);

/* The coordinates of instance `index`'s fixed-point state (not a paper quantity): *basis_out =
 * 1 when the int64 state holds each element's coordinates w = T^-1 u in a basis of invariant
 * subspaces of the element operator, in which the step matrix G is block diagonal (2 x 2
 * blocks, the first row of each an exact shift-add). COMPOSED_FIXED uses it, for single
 * instances and batched ones, where the basis is well conditioned (cond_inf(T) <= 64: p = 1,
 * 2, 3); 0 for nodal values or another variant. The FP64 state read through the API is nodal
 * either way. basis_out must not be NULL. */
int adg_get_fixed_basis(adg_ctx *c, int32_t index, int32_t *basis_out);

/*
 * Discrete gradient of the final-time L2 misfit
 *     J = 1/2 sum_e (dx/2) (u_N^e - g^e)^T M (u_N^e - g^e)
 * with respect to the initial nodal field, for a single-instance context, over nsteps
 * steps starting from the current state (the state itself is left unchanged). The adjoint
 * is hand-written: transposed stage operators, flux partial derivatives, and a reverse
 * ring buffer over the delay table. Checkpoints every ckpt_every steps, recomputation in
 * between. target_dev and grad_u0_dev are device (K, p+1) row-major FP64; J_out is host.
 * The paper has no adjoint; this follows the discrete forward scheme exactly.
 */
int adg_grad(adg_ctx *c, const double *target_dev, int64_t nsteps, int32_t ckpt_every,
             double *grad_u0_dev, double *J_out);

/* Discrete integral sum_e (dx/2) w^T u^e of instance `index` (Section 4.1 conservation
 * check), into *out (host). Synchronises. */
int adg_integral(adg_ctx *c, int32_t index, double *out);

/* Misfit J = 1/2 sum_e (dx/2) (u^e - g^e)^T M (u^e - g^e) of instance `index` against a
 * target g (device (K, p+1) row-major FP64), into *J_out (host). Synchronises. */
int adg_misfit(adg_ctx *c, int32_t index, const double *target_dev, double *J_out);

/* ADG_ENONFINITE if any instance holds a NaN or Inf, else ADG_OK. Synchronises. */
int adg_check_finite(adg_ctx *c);

/*
 * Same value as adg_integral, sum_e (dx/2) w^T u^e, but for a caller's own field and
 * without allocating anything. The paper has no counterpart; this entry point exists for
 * callers that must not allocate device memory where they call it: code inside a framework
 * that hands out all device memory from its own pool, processes running under a fixed
 * device-memory cap, and latency-critical loops that cannot afford cudaMalloc, which may
 * synchronise the device.
 *   p, K    : degree (1..ADG_MAX_P) and element count (1..2^30).
 *   dx      : element width (finite, > 0).
 *   u_dev   : device (K, p+1) row-major FP64 field (read only, caller-owned).
 *   out_dev : device pointer to one double that receives the integral (caller-owned).
 *   stream  : cudaStream_t (as void*), NULL for the default stream; the call is queued on
 *             it and returns without synchronising.
 * Scratch: a fixed 8 KiB array of 1024 partial sums compiled into the library; each GPU
 * that loads the library holds it until the process exits. Its device address is looked
 * up on the first call made on each device, so make that first call outside any stream
 * capture. Every call shares the array and it keeps the last call's contents (each call
 * overwrites every partial it reads), so calls whose work overlaps on the GPU (other
 * streams, other host threads) race; order them on one stream. Nothing is allocated or
 * freed. Errors: ADG_EINVAL for sizes outside the limits above or NULL pointers,
 * ADG_ECUDA for CUDA failures (message in adg_last_error(NULL)).
 */
int adg_integral_noalloc(int32_t p, int32_t K, double dx, const double *u_dev, double *out_dev,
                         void *stream);

/*
 * Exchanges of PE-face data that a distributed run of the instance `index` over the steps run
 * so far would make (Section 6.3's accounting), against synchronous DG: one exchange is the
 * pair of traces of one PE face for one stage of one step. Synchronous DG exchanges at every
 * step (sync_out = steps * stages * P); under the seeded or caller delays every level is still
 * sent, only late (exchanges_out = sync_out); under the communication-avoiding cycle only its
 * synchronised steps exchange. The emulation itself stores every level in its ring either
 * way. steps_out: steps run since adg_init. Host only (no GPU work); NULL outputs are skipped.
 * Errors: ADG_EINVAL (NULL ctx, bad index).
 */
int adg_comm_stats(const adg_ctx *c, int32_t index, int64_t *steps_out, int64_t *exchanges_out,
                   int64_t *sync_out);

/*
 * Write the delay table the library uses for cfg (seeded, cycle or caller table) for steps
 * first_step .. first_step+steps-1 into out_host (uint8 [steps][P]). Host only; needs no
 * GPU. Errors: ADG_EINVAL.
 */
int adg_delay_table(const adg_config *cfg, int64_t first_step, int64_t steps,
                    uint8_t *out_host);

/*
 * Nodal values of u0(x) = offset + sum_m amp[m] sin(kappa[m] x + phase[m]) (Eq.
 * initialcond) at the library's LGL nodes for cfg's mesh, written to u_dev (device,
 * (K, p+1) row-major FP64), ordered on `stream`.
 */
int adg_eval_modes(const adg_config *cfg, int32_t nmodes, const double *amp,
                   const double *kappa, const double *phase, double offset, double *u_dev,
                   void *stream);

/* LGL nodes (p+1 values, host) of degree p, as the library rounds them to FP64. */
int adg_lgl_nodes(int32_t p, double *nodes_host, double *weights_host);

/* Message of the last failure on c (NULL: the calling thread's last failure). */
const char *adg_last_error(const adg_ctx *c);

/* Release the context and everything it owns. NULL is ignored. */
void adg_destroy(adg_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* ADG_H */
