// Internal types shared by the host library (adg_api.cu) and the kernels (adg_kernels.cu).
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace adg {

constexpr int kMaxNp = 5;
constexpr int kMaxL = 16;
constexpr int kMaxQ = 5;
constexpr int kStages = 3;      // SSP-RK3 (the composed and fixed-point steps, the adjoint)
constexpr int kMaxStages = 5;   // the 2N low-storage schemes (up to five stages)
constexpr int kTile = 256;      // elements (threads) per block

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, read once
// per device and cached; 1 if the query fails).
int sm_count();

// Block size of the stage kernels: 256, or one warp when the mesh gives fewer than two
// 256-blocks per SM. Small meshes are latency-bound and make a single wave, whose length is
// set by the SMs holding the most warps: one-warp blocks spread them evenly (K = 65536, 2185
// warps of the halo-lane kernels: forward 78.1 -> 77.2 ms and gradient 209 -> 205 ms over
// 2000 steps, against 128-thread blocks; 64-thread blocks gave no gain).
inline int stage_block(int K) { return K < 2 * sm_count() * 256 ? 32 : 256; }

// Folded constants of one SSP-RK3 stage in Shu-Osher form, v_out = alpha u + beta (v + dt L(v)),
// with the strong form of Eq. DGscheme
//   dt L(v) = c2 [ D f(v) + LIFT_L (f(v_0) - F_L) - LIFT_R (f(v_p) - F_R) ],  c2 = -2 dt/dx.
// Advection (f = a v; every face flux is a G with G the upwind trace, or at a PE face the
// AT combination of delayed upwind traces):
//   out_i = alpha u_i + sum_j A_ij v_j + lL_i (v_0 - G_L) + lR_i (v_p - G_R),
//   A = beta (I + c2 a D),  lL = beta c2 a LIFT_L,  lR = -beta c2 a LIFT_R.
// Burgers (f = v^2/2, local Lax-Friedrichs face fluxes F):
//   out_i = alpha u_i + beta v_i + sum_j A_ij v_j^2 + lL_i (f(v_0) - F_L) + lR_i (f(v_p) - F_R),
//   A = beta c2 D / 2,  lL = beta c2 LIFT_L,  lR = -beta c2 LIFT_R.
struct StageConsts {
  double A[kMaxNp * kMaxNp];
  double lL[kMaxNp];
  double lR[kMaxNp];
  double alpha, beta;
};

// The S stages (S = 3 for SSP-RK3, up to kMaxCS for the low-storage schemes) of one step of
// upwind advection (a > 0) composed into one stencil. With Y_s the stage inputs (Y_0 = u^e;
// for SSP-RK3 Y_1 = v1, Y_2 = v2 of the Shu-Osher stages) and P_s = Y_s^{e-1}_p the right
// traces of the left neighbour's stage inputs (the channel scalars):
//   u'^e = G u^e + sum_{s<S} h_s P_s,
// and every element forms its own channel scalars from its neighbour's:
//   Y_s^e_p = r_s . u^e + sum_{t<s} k_{s,t} P_t   (s >= 1; Y_0^e_p = u^e_p).
// For SSP-RK3 (M_s = A_s + lL_s e_0^T, c_s = -lL_s of the folded stage form above):
//   G = alpha_2 I + M_2 (alpha_1 I + M_1 M_0), h_0 = M_2 M_1 c_0, h_1 = M_2 c_1, h_2 = c_2,
//   r_1 = M_0^T e_p, r_2 = (alpha_1 I + M_1 M_0)^T e_p, k_10 = c_0[p], k_20 = (M_1 c_0)[p],
//   k_21 = c_1[p];
// for the other schemes from their Butcher form (k_s = W Y_s + w P_s, W = c2 a (D + M^-1
// e_0 e_0^T), w = -c2 a M^-1 e_0). Cost: Np^2 + (2S - 1) Np + S(S-1)/2 multiply-adds per
// element and step (39 at Np = 4, S = 3; 62 at S = 5).
//
// PE-face correction of the composed step (upwind advection is linear): at PE face j
// (e = j Kpe) stage s replaces the synchronous face value by the delayed / AT one, which
// adds lL_s d_s to stage s's output on element e and lR_s d_s on element e-1, with
// d_s = T_s - V_s (T_s the stage-s input's right trace of element e-1, V_s the delayed / AT
// value). The step's result is the synchronous composed step plus
//   sum_s R_s d_s  on elements e-1 .. e+S-1  (R[s][m + 1], m = -1 .. S-1),
// R_s the response of the remaining stages to that injection, and
//   T_s = Y_s^{e-1}_p + sum_{t<s} rho_{s,t} d_t
// (Y_s^{e-1}_p the synchronous channel scalars of element e-1).
constexpr int kMaxCS = 5;   // stages of a composed step
struct StepConsts {
  double G[kMaxNp * kMaxNp];
  double r[kMaxCS][kMaxNp];        // r[s], s >= 1
  double h[kMaxCS][kMaxNp];
  double k[kMaxCS][kMaxCS];        // k[s][t], t < s
  double R[kMaxCS][kMaxCS + 1][kMaxNp];
  double rho[kMaxCS][kMaxCS];      // rho[s][t], t < s
};

// The StepConsts in fixed point for the integer composed step: each coefficient c
// (|c| < 2) is C = round(c 2^58), split into limbs C = ch 2^29 + cl with balanced
// -2^28 <= cl < 2^28 (int2 {ch, cl}).
// In the block basis (Inst.basis) the first row of each 2 x 2 block of G is (1, 2^-k_m),
// exactly: gs[m] = 29 - k_m, and that row is formed by shifts and adds (no multiplies); at
// Np = 5 gs[1] != 0 marks the 3 x 3 block's first row as (1, 2^-k, 0) likewise.
struct StepFixed {
  int2 G[kMaxNp * kMaxNp];
  int2 r[kMaxCS][kMaxNp];
  int2 h[kMaxCS][kMaxNp];
  int2 k[kMaxCS][kMaxCS];
  int gs[kMaxNp / 2];
};

// Formats of a fixed-point composed step (launch_fused_step's fmt): bit 0 the input, bit 1
// the output is int64 fixed point; FP64 otherwise. Bit 2 (set by launch_fixed_step from
// Inst.basis): the int64 state holds block-basis coordinates (below).
constexpr int kFmtInFixed = 1;
constexpr int kFmtOutFixed = 2;
constexpr int kFmtBasis = 4;

// Scale of a field at one step for the fixed-point composed step (adg_fixed.cuh): E is the
// largest biased FP64 exponent (2047: a NaN or infinity is present), sigma and mag the scale
// and the OR of |X| of an int64 field.
struct FxSlot {
  unsigned long long mag;
  int E;
  int sigma;
};

// One DG instance as the kernels see it. Nodal fields are node-major: field[i*K + e].
struct alignas(16) Inst {
  double *u;            // u^n, updated in place by stage 3
  double *v1, *v2;      // stage outputs 1 and 2
  double *unext;        // where stage 3 writes u^{n+1}: u itself, except in recorded sweeps
  double2 *ring;        // [R][3][P] traces (u^-, u^+) of stage inputs at PE faces
  const uint8_t *table; // [table_rows][P] delays
  const int64_t *meta;  // meta[0] = step index of rel 0; meta[1] = first table row's step
  const double *coef;   // AT coefficients [L][q][q]: coef[(k*q + (q'-1))*q + i]
  double a;
  int K, Np, P, Kpe, R, L, q, pde, async, table_rows;
  int fused;            // 0: staged; composed stencil + PE-face fix-up in 1: FP64 (StepConsts),
                        // 2: fixed-point integer arithmetic (StepFixed)
  int ept;              // elements per thread of the composed-step kernel (1, 2 or 4, autotuned)
  FxSlot *fx;           // fused == 2: [3] scale of u^n in slot n % 3
  double *fd;           // fused == 2 with PE faces: [2][P][ns] stage differences d_s of each
                        // face, buffer n & 1 for step n
  StageConsts sc[kStages];
  StepConsts st;
  StepFixed sf;
  // fused == 2: the PE-face responses st.R in fixed point (limbs as in StepFixed), used when
  // face_fx is set (every |R| < 2)
  int2 Rf[kMaxCS][kMaxCS + 1][kMaxNp];
  int face_fx;
  // fused == 2 (where the basis is accepted): the int64 state holds w = Tbi u, the coordinates of u in a
  // basis (columns of Tb) in which every composed-step matrix G is block diagonal (2 x 2
  // blocks (2m, 2m+1), a 1 x 1 block last for odd Np) with block rows 2m equal to
  // (1, 2^-k_m), and whose even columns have right trace 1, odd columns 0 (so u_p = sum of
  // the even w_j); sf and Rf then hold the coefficients in these coordinates (G Tb-similar,
  // h and R multiplied by Tbi, r by Tb). int64 inputs are
  // kept below 2^(57 - fxh); an FP64 input at step n is converted at scale
  // 2^(E - 1079 + fxe) (fxe >= fxh + log2 of the row sums of Tbi).
  int basis, fxh, fxe, pad0_;
  double Tb[kMaxNp * kMaxNp], Tbi[kMaxNp * kMaxNp];
  int ns;               // stages per step: the ring holds [R][ns][P] stage-input traces; the
                        // composed steps' S (3, or 5 for the five-stage scheme)
  int ls;               // 1: a 2N low-storage scheme (k_lsrk_stage, coefficients lsA, lsB)
  int visc;             // 1: viscous Burgers by the local DG method (k_ldg_q, then the stage)
  double lsA[kMaxStages], lsB[kMaxStages];
  // viscous Burgers: nu, q = u_x of the stage input (node-major like the fields), the PE
  // faces' q^+ traces [R][ns][P], and q = QD v + qlL (uhat_L - v_0) + qlR (uhat_R - v_p)
  double nu;
  double *qbuf;
  double *ringq;
  double dt;            // the step (viscous Burgers and Euler kernels)
  double QD[kMaxNp * kMaxNp], qlL[kMaxNp], qlR[kMaxNp];
  // Euler (pde 2): three components per field (component c at field + c K Np), the raw stage
  // output w when the limiter is on, and the limiter's weights: cell average a0 = avg_w . v,
  // P_1 coefficient a1 = p1_w . v, nodes xi; TVB constant tvb_m, element width dx
  int euler, limiter;
  double tvb_m, dx;
  double *w;
  double avg_w[kMaxNp], p1_w[kMaxNp], xi[kMaxNp];
  double pad3_;
};

static_assert(sizeof(Inst) % 16 == 0, "Inst is copied to shared memory as int4");
// Kernel parameters may take up to 32764 bytes (CUDA 12.1 and later); the batched kernels also
// stage an Inst in shared memory.
static_assert(sizeof(Inst) <= 8192, "Inst is passed by value as a kernel parameter");

// Adjoint of one stage (adg_adjoint.cu): w is the adjoint of the stage output, v the stage
// input (Burgers), lv receives the adjoint of the stage input (stages 1, 2); lacc collects
// the adjoint of u^n (stage 2 starts it with alpha w, stage 1 adds alpha w, stage 0 adds the
// adjoint of its input u^n).
struct AdjStage {
  const double *w;
  const double *v;
  double *lv;
  double *lacc;
  int K, Np;
  StageConsts C;
  // PE faces handled inside the stage kernel (K/P >= 8): the delay lookup fields (names
  // shared with Inst), the adjoint ring, and the stage index of this kernel.
  double *lring;
  const uint8_t *table;
  const int64_t *meta;
  const double *coef;
  int rel, stage, P, Kpe, R, q;
  int faces;            // 1: this kernel applies the PE-face adjoint (no separate face pass)
};

// Adjoint of the PE-face pass of one stage. The field names shared with Inst (table, meta,
// coef, P, q, R) let the delay lookup serve both.
struct AdjFace {
  const double *w;
  const double *v;
  double *target;       // adjoint of the stage input (lacc for stage 0)
  double *lring;        // [R][3][P] adjoint of the face values of each stored level
  const uint8_t *table;
  const int64_t *meta;
  const double *coef;
  int rel;              // step index = meta[0] + rel (one graph replays for every segment)
  int K, Np, P, Kpe, R, q, stage;
  double lL[kMaxNp], lR[kMaxNp];
};

// Launchers (adg_kernels.cu). All return cudaGetLastError() after the launch.
// One stage over all elements; for an asynchronous instance the same kernel applies the
// PE-face correction (delayed / AT flux) and writes the ring (step meta[0] + rel).
cudaError_t launch_stage(const Inst &I, int stage, int rel, cudaStream_t s, bool pdl = false);
// Stage s of a 2N low-storage step (I.ls): dU_s = A_s dU_{s-1} + dt L(U_{s-1}) in place in
// I.v1 (A_1 = 0: dU_0 is not read) and U_s = U_{s-1} + B_s dU_s from uin (U_{s-1}) into uout,
// with the delayed / AT flux and the ring write of the stage-input traces at PE faces.
cudaError_t launch_lsrk_stage(const Inst &I, int s, int rel, const double *uin, double *uout,
                              cudaStream_t st);
// Viscous Burgers (I.visc): q = u_x of stage `stage`'s input vin by the local DG method into
// I.qbuf, with the AT value of uhat at PE faces and the owners' ring writes ((u^-, u^+) into
// I.ring, q^+ into I.ringq); launched before that stage's kernel.
cudaError_t launch_ldg_q(const Inst &I, const double *vin, int stage, int rel, cudaStream_t s);
// Euler (I.euler, adg_euler.cu): stage `stage` of SSP-RK in Shu and Osher's form from its input
// (u, v1, v2 by stage) into dst, and the slope limiter src -> dst (src != dst).
cudaError_t launch_euler_stage(const Inst &I, int stage, int rel, double *dst, cudaStream_t s);
cudaError_t launch_euler_limit(const Inst &I, const double *src, double *dst, cudaStream_t s);
cudaError_t launch_batch_stage(const Inst *insts_dev, const int2 *work_dev, int nwork,
                               int stage, int rel, int tile, cudaStream_t s);
// Batched PE-face pass after each batched stage: ring write of the stage-input traces and
// replacement of the synchronous flux by the delayed / AT flux in the elements next to each
// PE face.
cudaError_t launch_batch_faces(const Inst *insts_dev, const int2 *work_dev, int nwork, int stage,
                               int rel, cudaStream_t s);
cudaError_t launch_advance(int64_t *meta, int nmeta_stride, int ninst, int64_t by,
                           cudaStream_t s);
// PE-face work of the fixed-point composed step (fused == 2, with PE faces) on the field u
// between steps rel-1 and rel: mode bit 0 adds step rel-1's correction (differences in I.fd)
// to u, bit 1 then forms step rel's differences from u and the ring (ring write, I.fd). fu: u
// is int64, else FP64; fin_prev: step rel-1 read int64.
constexpr int kFaceApply = 1, kFaceDiff = 2;
// pdl (this and launch_fixed_step): launched as a programmatic dependent of the kernel before
// it in the stream (that kernel must be a k_step_fixed or k_face_step of the same chunk): its
// blocks may start while that kernel drains, and wait (griddepcontrol.wait) for its completion
// before they touch anything it writes.
cudaError_t launch_face_step(const Inst &I, void *u, int rel, int fu, int fin_prev, int mode,
                             cudaStream_t s, bool pdl = false);
// Composed step uin -> uout (rel: step offset from meta[0]) and, with PE faces, the fix-up
// of the elements next to each PE face with the delayed / AT flux. fmt (fixed-point step,
// fused == 2, only): bit 0 the input, bit 1 the output is int64 fixed point (adg_fixed.cuh);
// otherwise both are FP64.
cudaError_t launch_fused_step(const Inst &I, const void *uin, void *uout, int rel,
                              cudaStream_t s, bool with_fixup = true, int fmt = 0);
// The fixed-point composed step alone (adg_fixed.cu).
cudaError_t launch_fixed_step(const Inst &I, const void *uin, void *uout, int rel, int fmt,
                              cudaStream_t s, bool pdl = false);
// A launch with the programmatic-stream-serialization attribute when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                             bool pdl, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
// The same with a scheduling priority for the launch's blocks (lower numbers first, within
// cudaDeviceGetStreamPriorityRange): blocks of a short kernel on the critical path get SM
// resources ahead of queued blocks of kernels on other streams.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_priority(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                                bool pdl, int priority, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
// What the batched fixed-point step reads of an instance when the coefficients are shared
// (below): its fields u, v1, v2, step counter, scale slots, K and Np.
struct BatchLite {
  void *f[3];
  const int64_t *meta;
  FxSlot *fx;
  int K, Np;
  int e0, pad;   // as a work item: the first element of the block's tile
};
// One fixed-point coefficient set per degree (sf[Np - 2]), for batches in which every instance
// of a degree has the same composed coefficients (the same Courant number with a > 0 and the
// step from the Courant number: the folded constants depend on p and sigma only). Passed as a
// kernel parameter, so the coefficients are constant-bank operands as in the single-instance
// step instead of shared-memory loads.
struct UniformFixed {
  StepFixed sf[kMaxNp - 1];
  // per degree: the block basis as in Inst (basis, fxh, fxe, Tbi)
  int basis[kMaxNp - 1], fxh[kMaxNp - 1], fxe[kMaxNp - 1], pad_[kMaxNp - 1];
  double Tbi[kMaxNp - 1][kMaxNp * kMaxNp];
};
struct BatchUniform {
  const BatchLite *items_dev;   // one record per work item (the instance's fields and e0) of
  int nitems, ept;              // ept kTile elements each
  UniformFixed uf;
};

// Batched composed steps over all instances: src / dst select u (0), v1 (1) or v2 (2) of
// every instance. FP64 (fixed false): u -> v1 or v1 -> u. Fixed point (fixed true): fmt as in
// launch_fused_step, with the shared coefficients of bu when bu is not null. Then the PE-face
// correction of every instance: fwork_dev lists (instance, face) for every PE face of every
// instance (nfwork entries).
cudaError_t launch_batch_fused_step(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                    const int2 *fwork_dev, int nfwork, int src, int dst, int fmt,
                                    bool fixed, int rel, cudaStream_t s,
                                    const BatchUniform *bu = nullptr, bool pdl = false);
cudaError_t launch_batch_fixed_uniform(const BatchUniform &bu, const int2 *work_dev, int nwork,
                                       int src, int dst, int fmt, int rel, cudaStream_t s,
                                       bool pdl = false);
// The batched fixed-point step alone (adg_fixed.cu).
cudaError_t launch_batch_fixed_step(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                    int src, int dst, int fmt, int rel, cudaStream_t s,
                                    bool pdl = false);
// Seeded delay-table rows on the device, identical to the host generator: entry (row r,
// face j) is the bin of output (first + r) P + j of SplitMix64(seed), u = (z >> 11) 2^-53,
// bin = the first b with u < edges[b] (else L - 1), compared in integers as
// (z >> 11) < T[b] with T[b] = ceil(edges[b] 2^53) formed exactly on the host.
struct DelayGen {
  uint64_t seed;
  uint64_t T[kMaxL];
  int L, P;
  int caa;   // > 0: the communication-avoiding cycle instead (the same delay at every face)
  int pad;
};
cudaError_t launch_fill_delays(uint8_t *table, int64_t first, int rows, const DelayGen &g,
                               cudaStream_t s);
// Scale slots of the fixed-point composed step for an FP64 field f of n values at step
// index `step`: all three slots cleared, then E of slot step % 3 = largest biased exponent.
cudaError_t launch_fixed_reset(const double *f, size_t n, FxSlot *fx, int64_t step,
                               cudaStream_t s);
// Instance I's field as element-major FP64 rows (K, Np) in dst (device, pinned or managed
// memory): src is FP64 node planes (fixed false) or the int64 state of step `step` (fixed
// true, converted as launch_fixed_to_fp64 converts it).
cudaError_t launch_state_rows(const Inst &I, const void *src, bool fixed, int64_t step,
                              double *dst, cudaStream_t s);
// The FP64 field I.u of the int64 fixed-point field X of step `step`, from the scale slot
// step % 3 of I.fx (NaN everywhere when it marks a NaN or infinity); u = Tb w element by
// element when I.basis is set.
cudaError_t launch_fixed_to_fp64(const Inst &I, const long long *X, int64_t step,
                                 cudaStream_t s);
// Copies v1 into u for every instance (after an odd number of FP64 batched composed steps, or
// a single fixed-point step).
cudaError_t launch_batch_copy_back(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                   cudaStream_t s);
// Row-major (K, Np) values into node planes; src may be pinned host memory (read over the
// host link). emax, when given, is raised to the largest biased FP64 exponent of the values.
cudaError_t launch_to_internal(const double *src_rowmajor, double *dst_nodemajor, int K,
                               int Np, cudaStream_t s, int *emax = nullptr);
cudaError_t launch_to_external(const double *src_nodemajor, double *dst_rowmajor, int K,
                               int Np, cudaStream_t s);
cudaError_t launch_eval_modes(double *u_rowmajor, int K, int Np, double x0, double dx,
                              const double *xi, int nmodes, const double *amp,
                              const double *kappa, const double *phase, double offset,
                              cudaStream_t s);
// Reductions: partial sums per block then one block sums the partials in a fixed order.
// kind 0: sum_e w^T u^e * scale; 1: max |u|; 2: count of non-finite values;
// 3: misfit sum_e (u-g)^T M (u-g) * scale (M given row-major Np x Np in w_or_M).
cudaError_t launch_reduce(int kind, const double *u, const double *g, int K, int Np,
                          const double *w_or_M, double scale, double *partials,
                          int nblocks, double *out, cudaStream_t s);
int reduce_blocks(int K);

// Adjoint launchers (adg_adjoint.cu); dir is the sign of the advection speed.
cudaError_t launch_adj_stage(const AdjStage &A, int pde, int stage, int dir, cudaStream_t s);
cudaError_t launch_adj_faces(const AdjFace &F, int pde, int dir, cudaStream_t s);
cudaError_t launch_adj_init(const double *u, const double *g, int K, int Np, const double *M,
                            double scale, double *lam, cudaStream_t s);

// Host helpers shared by the library's translation units (adg_api.cu).
void set_last_error(const char *msg);
// LGL quadrature weights of degree p (p+1 values), rounded to FP64.
void lgl_weights(int p, double *w);

}  // namespace adg
