// FP64 CUDA kernels of the ADG / ADG-AT SSP-RK3 step for sm_103a.
//
// One thread per element, node-major layout (field[i*K + e]) so that every load and
// store of a nodal plane is a coalesced 256-byte warp access. Face traces of the
// neighbours come from warp shuffles (one global load per warp edge). The element
// right-hand side (strong form of Eq. DGscheme), the Shu-Osher SSP-RK3 stage combine and,
// at PE faces, the delayed / AT flux (Eqs. asyncEulerDGconserved, at-flux-gen) with the
// ring-buffer write of the stage-input traces are fused into one kernel per stage.
#include "adg_device.cuh"
#include "adg_fixed.cuh"

#include <cstdio>

namespace adg {

namespace {

// Vs - V at PE face j, stage `stage`, step n, from the face's traces (tl, tr): the
// synchronous face value minus the delayed / AT value; the owner writes the traces into the
// ring slot of step n.
template <int PDE, int DIR, class I>
__device__ __forceinline__ double pe_face_delta(const I &inst, int j, int64_t n, int stage,
                                                double tl, double tr, bool owner) {
  const double Vs = face_value<PDE, DIR>(inst, tl, tr);
  const double V = pe_value<PDE, DIR>(inst, j, n, stage, tl, tr, owner);
  return __dsub_rn(Vs, V);
}

// A stage of a 2N low-storage step (LS): its input U_{s-1}, output U_s, stage index (for the
// ring), coefficients, and whether it is the first (A_1 = 0: dU_0 is not read).
struct LsArgs {
  const double *uin;
  double *uout;
  int s, first;
  double As, Bs;
};

// One SSP-RK3 stage for element e (all 32 lanes of the warp take part; lanes past the
// end duplicate element K-1 and store nothing). With LS, stage ls.s of a 2N low-storage step
// instead: the same right-hand side dt L(U) from the constants sc[0] (no identity and no
// factor beta), dU_s = A_s dU_{s-1} + dt L(U_{s-1}) in place in v1 and U_s = U_{s-1} + B_s dU_s. DIR is the upwind side for advection
// (+1: a > 0, -1: a < 0) and 0 for Burgers. With FACES, the PE-face correction of the
// delayed / AT flux is applied here too (step n): the element right of PE face j
// (e = j Kpe) owns the face, writes its ring entry and adds lL (Vs - V); the element left
// of it (e = j Kpe - 1) forms the same value with the same arithmetic and adds lR (Vs - V).
// The synchronous output is rounded first, so the result is bit-identical to a stage
// followed by a separate face pass.
template <int NP, int PDE, int STAGE, int DIR, bool FACES, bool LS = false, bool VISC = false,
          class I>
__device__ __forceinline__ void stage_body(const I &inst, int e, int64_t n = 0,
                                           const LsArgs &ls = LsArgs{}) {
  const int K = inst.K;
  const int lane = threadIdx.x & 31;
  const int ec = e < K ? e : K - 1;
  const double *vin = LS ? ls.uin : (STAGE == 0 ? inst.u : (STAGE == 1 ? inst.v1 : inst.v2));
  double *vout = LS ? inst.v1 : (STAGE == 0 ? inst.v1 : (STAGE == 1 ? inst.v2 : inst.unext));
  const StageConsts &C = inst.sc[LS ? 0 : STAGE];
  const double alpha = LS ? ls.As : C.alpha;
  const int rstage = LS ? ls.s : STAGE;

  double v[NP];
  {
    const double *q = vin + ec;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      v[i] = __ldg(q);
      q += K;
    }
  }
  double u[NP];   // the alpha operand: u^n, or dU_{s-1} of a 2N stage
  if (STAGE > 0) {
    if (LS && ls.first) {
#pragma unroll
      for (int i = 0; i < NP; ++i) u[i] = 0.0;
    } else {
      const double *q = (LS ? inst.v1 : inst.u) + ec;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        u[i] = *q;
        q += K;
      }
    }
  }

  const unsigned full = 0xffffffffu;
  const bool edge = (lane == 31) || (ec + 1 >= K);
  const int fR = ec + 1 >= K ? 0 : ec + 1;
  double vLm = 0.0, vRp = 0.0;
  if (PDE == 1 || DIR > 0) {
    vLm = __shfl_up_sync(full, v[NP - 1], 1);
    if (lane == 0) vLm = __ldg(vin + (NP - 1) * K + (ec == 0 ? K - 1 : ec - 1));
  }
  if (PDE == 1 || DIR < 0) {
    vRp = __shfl_down_sync(full, v[0], 1);
    if (edge) vRp = __ldg(vin + fR);
  }
  // Every face takes its synchronous flux here; at PE faces the face pass that follows
  // the stage replaces it by the delayed / AT flux (a correction of the two elements).
  double jL = 0.0, jR = 0.0;
  if (PDE == 0) {
    // Face values in trace units (the flux is a times the value).
    if (DIR > 0) jL = __dsub_rn(v[0], vLm);
    else jR = __dsub_rn(v[NP - 1], vRp);
  } else {
    const double FL = num_flux<1>(0.0, vLm, v[0]);
    double FR = __shfl_down_sync(full, FL, 1);
    if (edge) FR = num_flux<1>(0.0, v[NP - 1], vRp);
    jL = __dsub_rn(phys_flux<1>(0.0, v[0]), FL);
    jR = __dsub_rn(phys_flux<1>(0.0, v[NP - 1]), FR);
  }

  double g[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = PDE == 0 ? v[i] : v[i] * v[i];

  double out[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    double acc;
    if (PDE == 0) {
      acc = STAGE == 0 ? C.A[i * NP] * g[0] : fma(C.A[i * NP], g[0], alpha * u[i]);
    } else {
      if (LS) acc = alpha * u[i];   // no v term: dt L(U) has none
      else acc = STAGE == 0 ? v[i] : fma(C.beta, v[i], C.alpha * u[i]);
      acc = fma(C.A[i * NP], g[0], acc);
    }
#pragma unroll
    for (int jj = 1; jj < NP; ++jj) acc = fma(C.A[i * NP + jj], g[jj], acc);
    out[i] = acc;
  }
  if (PDE == 1 || DIR > 0) {
#pragma unroll
    for (int i = 0; i < NP; ++i) out[i] = fma(C.lL[i], jL, out[i]);
  }
  if (PDE == 1 || DIR < 0) {
#pragma unroll
    for (int i = 0; i < NP; ++i) out[i] = fma(C.lR[i], jR, out[i]);
  }
  if (FACES && e < K) {
    const int Kpe = inst.Kpe;
    const int jq = e / Kpe;
    const int r = e - jq * Kpe;
    if (r == 0) {   // left face is PE face jq; this element owns it
      const double tl = (PDE == 1 || DIR > 0) ? vLm
                        : __ldg(vin + (NP - 1) * K + (e == 0 ? K - 1 : e - 1));
      const double d = pe_face_delta<PDE, DIR>(inst, jq, n, rstage, tl, v[0], true);
      if (nonzero(d)) {
#pragma unroll
        for (int i = 0; i < NP; ++i) out[i] = fma(C.lL[i], d, out[i]);
      }
    }
    if (r == Kpe - 1) {   // right face is PE face jq + 1 (face 0 for the last element)
      const double tr = (PDE == 1 || DIR < 0) ? vRp : __ldg(vin + (e + 1 == K ? 0 : e + 1));
      const int jr = jq + 1 == inst.P ? 0 : jq + 1;
      const double d = pe_face_delta<PDE, DIR>(inst, jr, n, rstage, v[NP - 1], tr, false);
      if (nonzero(d)) {
#pragma unroll
        for (int i = 0; i < NP; ++i) out[i] = fma(C.lR[i], d, out[i]);
      }
    }
  }
  if (VISC && PDE == 1) {
    // Viscous term nu q_x of the local DG method, alternating flux qhat = q^+ (q from the q
    // pass, k_ldg_q), in the stage's folded constants (C.A = b c2 D / 2, C.lL, C.lR):
    //   nu ( -2 C.A q + C.lR (qhat_R - q_p) + C.lL (qhat_L - q_0) ),
    // with qhat_L = q_0 and qhat_R = q^{e+1}_0 at interior faces and the AT value of the stored
    // q^+ traces at PE faces (both elements of the face alike).
    double q[NP];
    {
      const double *qq = inst.qbuf + ec;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        q[i] = *qq;
        qq += K;
      }
    }
    double qRp = __shfl_down_sync(full, q[0], 1);
    if (edge) qRp = inst.qbuf[fR];
    double jqL = 0.0, jqR = __dsub_rn(qRp, q[NP - 1]);
    if (FACES && e < K) {
      const int Kpe = inst.Kpe;
      const int jq = e / Kpe;
      const int r = e - jq * Kpe;
      if (r == 0) jqL = __dsub_rn(pe_value_q(inst, jq, n, rstage, q[0]), q[0]);
      if (r == Kpe - 1) {
        const int jr = jq + 1 == inst.P ? 0 : jq + 1;
        jqR = __dsub_rn(pe_value_q(inst, jr, n, rstage, qRp), q[NP - 1]);
      }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double vq = C.A[i * NP] * q[0];
#pragma unroll
      for (int jj = 1; jj < NP; ++jj) vq = fma(C.A[i * NP + jj], q[jj], vq);
      out[i] = fma(inst.nu, fma(C.lL[i], jqL, fma(C.lR[i], jqR, -2.0 * vq)), out[i]);
    }
  }
  if (e < K) {
    double *q = vout + e;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      *q = out[i];
      q += K;
    }
    if (LS) {
      double *w = ls.uout + e;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        *w = fma(ls.Bs, out[i], v[i]);
        w += K;
      }
    }
  }
}

// One SSP-RK3 stage with halo lanes: warp w takes elements 30w .. 30w+29 in lanes 1 .. 30,
// and lanes 0 and 31 hold the elements on either side (periodic), so every face flux is formed
// by one full-warp instruction sequence (lane l forms the flux of its left face; lane l-1
// reads it as its right face) instead of an extra flux on the warp's last lane. At a PE face
// the delayed / AT value is formed once, by the lane of the element right of the face (which,
// owned, also writes the ring), and the element left of it reads the difference from the next
// lane. Per element the arithmetic is that of stage_body, so the results are bit-identical to
// it (the halo lanes' 2/32 redundant work replaces the single-lane flux and the second
// evaluation of every PE-face value, which a warp's FP64 instruction pays in full whatever its
// active lanes).
template <int NP, int PDE, int STAGE, int DIR, bool FACES, class I>
__device__ __forceinline__ void stage_body_halo(const I &inst, int warp, int64_t n) {
  const int K = inst.K;
  const int lane = threadIdx.x & 31;
  const int e = 30 * warp + lane - 1;
  const bool own = lane >= 1 && lane <= 30 && e < K;
  // the element's periodic image (halo lanes at the ends wrap; lanes past the halo reuse 0)
  const int ec = e < 0 ? e + K : (e < K ? e : (e == K ? 0 : 0));
  const double *vin = STAGE == 0 ? inst.u : (STAGE == 1 ? inst.v1 : inst.v2);
  double *vout = STAGE == 0 ? inst.v1 : (STAGE == 1 ? inst.v2 : inst.unext);
  const StageConsts &C = inst.sc[STAGE];

  double v[NP];
  {
    const double *q = vin + ec;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      v[i] = __ldg(q);
      q += K;
    }
  }
  double u[NP];   // the alpha operand u^n (owned lanes)
  if (STAGE > 0) {
    const double *q = inst.u + (own ? ec : 0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      u[i] = own ? *q : 0.0;
      q += K;
    }
  }
  const unsigned full = 0xffffffffu;
  const double vLm = __shfl_up_sync(full, v[NP - 1], 1);   // lanes >= 1
  const double vRp = __shfl_down_sync(full, v[0], 1);      // lanes <= 30
  double jL = 0.0, jR = 0.0;
  if (PDE == 0) {
    if (DIR > 0) jL = __dsub_rn(v[0], vLm);
    else jR = __dsub_rn(v[NP - 1], vRp);
  } else {
    const double FL = num_flux<1>(0.0, vLm, v[0]);
    const double FR = __shfl_down_sync(full, FL, 1);
    jL = __dsub_rn(phys_flux<1>(0.0, v[0]), FL);
    jR = __dsub_rn(phys_flux<1>(0.0, v[NP - 1]), FR);
  }

  double g[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = PDE == 0 ? v[i] : v[i] * v[i];

  double out[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    double acc;
    if (PDE == 0) {
      acc = STAGE == 0 ? C.A[i * NP] * g[0] : fma(C.A[i * NP], g[0], C.alpha * u[i]);
    } else {
      acc = STAGE == 0 ? v[i] : fma(C.beta, v[i], C.alpha * u[i]);
      acc = fma(C.A[i * NP], g[0], acc);
    }
#pragma unroll
    for (int jj = 1; jj < NP; ++jj) acc = fma(C.A[i * NP + jj], g[jj], acc);
    out[i] = acc;
  }
  if (PDE == 1 || DIR > 0) {
#pragma unroll
    for (int i = 0; i < NP; ++i) out[i] = fma(C.lL[i], jL, out[i]);
  }
  if (PDE == 1 || DIR < 0) {
#pragma unroll
    for (int i = 0; i < NP; ++i) out[i] = fma(C.lR[i], jR, out[i]);
  }
  if (FACES) {
    // lane l (1 .. 31) forms the PE-face difference of its left face when its element owns
    // one (e = j Kpe, or e = K: face 0 seen from element K-1); owned lanes write the ring
    const int Kpe = inst.Kpe;
    const int eo = e < K ? e : e - K;
    const int jq = eo / Kpe;
    const bool face = lane >= 1 && e <= K && eo - jq * Kpe == 0;
    double d = 0.0;
    if (face) d = pe_face_delta<PDE, DIR>(inst, jq, n, STAGE, vLm, v[0], own);
    const double dR = __shfl_down_sync(full, d, 1);
    const bool faceR = __shfl_down_sync(full, face ? 1 : 0, 1) != 0;
    if (own && face && nonzero(d)) {
#pragma unroll
      for (int i = 0; i < NP; ++i) out[i] = fma(C.lL[i], d, out[i]);
    }
    if (own && faceR && nonzero(dR)) {
#pragma unroll
      for (int i = 0; i < NP; ++i) out[i] = fma(C.lR[i], dR, out[i]);
    }
  }
  if (own) {
    double *q = vout + e;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      *q = out[i];
      q += K;
    }
  }
}

template <int NP, int PDE, int STAGE, int DIR, bool FACES>
__global__ void __launch_bounds__(kTile) k_stage_halo(const Inst inst, int rel) {
  pdl_wait();   // the stage before (programmatic launch) has written this one's input
  pdl_trigger();
  const int64_t n = FACES ? inst.meta[0] + rel : 0;
  stage_body_halo<NP, PDE, STAGE, DIR, FACES>(inst, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, n);
}

template <int NP, int PDE, int STAGE, int DIR, bool FACES, bool VISC = false>
__global__ void __launch_bounds__(kTile) k_stage(const Inst inst, int rel) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = FACES ? inst.meta[0] + rel : 0;
  stage_body<NP, PDE, STAGE, DIR, FACES, false, VISC>(inst, blockIdx.x * blockDim.x + threadIdx.x,
                                                      n);
}

// Stage ls.s of a 2N low-storage step (Williamson's form; I.ls).
template <int NP, int PDE, int DIR, bool FACES, bool VISC = false>
__global__ void __launch_bounds__(kTile) k_lsrk_stage(const Inst inst, int rel, const LsArgs ls) {
  const int64_t n = FACES ? inst.meta[0] + rel : 0;
  stage_body<NP, PDE, 1, DIR, FACES, true, VISC>(inst, blockIdx.x * blockDim.x + threadIdx.x, n,
                                                 ls);
}

// The q pass of viscous Burgers by the local DG method (Eq. burgers, Section 6): q = u_x of
// the stage input v with the alternating flux uhat = u^- (the left element's right trace),
//   q^e = (2/dx) [ D v^e + M^{-1} e_p (uhat_R - v^e_p) - M^{-1} e_0 (uhat_L - v^e_0) ]
//       = QD v^e + qlR (uhat_R - v^e_p) + qlL (uhat_L - v^e_0),
// uhat_L = v^{e-1}_p and uhat_R = v^e_p at interior faces (the right term vanishes). At a PE
// face both elements take uhat as the AT sum of the stored u^- traces (pe_value of the upwind
// kind); its owner stores the stage input's traces (u^-, u^+) and its q^+ = q^e_0 for the
// later steps.
template <int NP, bool FACES>
__global__ void __launch_bounds__(kTile) k_ldg_q(const Inst inst, const double *__restrict__ vin,
                                                 int stage, int rel) {
  const int K = inst.K;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int ec = e < K ? e : K - 1;
  double v[NP];
  {
    const double *q = vin + ec;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      v[i] = __ldg(q);
      q += K;
    }
  }
  double vLm = __shfl_up_sync(0xffffffffu, v[NP - 1], 1);
  if (lane == 0) vLm = __ldg(vin + (NP - 1) * K + (ec == 0 ? K - 1 : ec - 1));
  double dL = __dsub_rn(vLm, v[0]), dR = 0.0;
  int jown = -1;
  if (FACES && e < K) {
    const int64_t n = inst.meta[0] + rel;
    const int Kpe = inst.Kpe;
    const int jq = e / Kpe;
    const int r = e - jq * Kpe;
    if (r == 0) {
      dL = __dsub_rn(pe_value<0, 1>(inst, jq, n, stage, vLm, v[0], true), v[0]);
      jown = jq;
    }
    if (r == Kpe - 1) {
      const double tr = __ldg(vin + (e + 1 == K ? 0 : e + 1));
      const int jr = jq + 1 == inst.P ? 0 : jq + 1;
      dR = __dsub_rn(pe_value<0, 1>(inst, jr, n, stage, v[NP - 1], tr, false), v[NP - 1]);
    }
  }
  if (e >= K) return;
  double q[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    double acc = inst.QD[i * NP] * v[0];
#pragma unroll
    for (int j = 1; j < NP; ++j) acc = fma(inst.QD[i * NP + j], v[j], acc);
    acc = fma(inst.qlL[i], dL, acc);
    q[i] = fma(inst.qlR[i], dR, acc);
  }
  double *o = inst.qbuf + e;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    *o = q[i];
    o += K;
  }
  if (FACES && jown >= 0) {
    const int64_t n = inst.meta[0] + rel;
    inst.ringq[((size_t)(n % inst.R) * inst.ns + stage) * inst.P + jown] = q[0];
  }
}

// Composed SSP-RK3 step of upwind advection (a > 0), all faces synchronous (StepConsts):
// one thread per element forms its right trace p = u_p and the own parts r1 . u, r2 . u of
// its channel scalars, then, in two rounds through shared memory, v1_p and v2_p from its
// left neighbour's, and finally u'^e = G u^e + h_0 P0 + h_1 P1 + h_2 P2 from the left
// neighbour's three channel scalars. The first three threads of a block form the scalars of
// the three elements before the block themselves, with the same arithmetic.
template <int NP>
__device__ __forceinline__ void own_scalars(const StepConsts &S, const double *u, double &sp,
                                            double &s1, double &s2) {
  sp = u[NP - 1];
  s1 = S.r[1][0] * u[0];
  s2 = S.r[2][0] * u[0];
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    s1 = fma(S.r[1][j], u[j], s1);
    s2 = fma(S.r[2][j], u[j], s2);
  }
}

// Channel scalars of the elements of one block: slots 0..2 hold the three elements before
// the block, slot 3+m the block's element m (EPT kTile elements per block).
template <int EPT>
struct FusedShared {
  double p[EPT * kTile + 3], q1[EPT * kTile + 3], q2[EPT * kTile + 3];
};

// Composed step for EPT elements per thread: thread t owns elements e0 + t + h kTile,
// h < EPT, so the loads and FMA chains of EPT elements are in flight together.
template <int NP, int EPT, class I>
__device__ __forceinline__ void fused_body(const I &inst, const double *__restrict__ uin,
                                           double *__restrict__ uout, int e0,
                                           FusedShared<EPT> &sh) {
  const int K = inst.K;
  const int t = threadIdx.x;
  const StepConsts &S = inst.st;
  double hs1 = 0.0, hs2 = 0.0;   // own parts of the halo element's channel scalars
  if (t < 3) {
    int m = e0 - 3 + t;
    if (m < 0) m += K;     // K >= 8 on this path
    double w[NP], a;
    load_elem<NP>(uin, K, m, w);
    own_scalars<NP>(S, w, a, hs1, hs2);
    sh.p[t] = a;
  }
  double u[EPT][NP], s1[EPT], s2[EPT];
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int e = e0 + t + h * kTile;
    load_elem<NP>(uin, K, e < K ? e : K - 1, u[h]);
  }
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    double sp;
    own_scalars<NP>(S, u[h], sp, s1[h], s2[h]);
    sh.p[t + h * kTile + 3] = sp;
  }
  __syncthreads();
  // v1_p = r1 . u + k_0 P0 (the halo's first element needs none)
  if (t == 1 || t == 2) sh.q1[t] = fma(S.k[1][0], sh.p[t - 1], hs1);
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int sl = t + h * kTile + 3;
    sh.q1[sl] = fma(S.k[1][0], sh.p[sl - 1], s1[h]);
  }
  __syncthreads();
  // v2_p = r2 . u + k_1 P0 + k_2 P1 (of the halo, only the element just before the block)
  if (t == 2) sh.q2[2] = fma(S.k[2][1], sh.q1[1], fma(S.k[2][0], sh.p[1], hs2));
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int sl = t + h * kTile + 3;
    sh.q2[sl] = fma(S.k[2][1], sh.q1[sl - 1], fma(S.k[2][0], sh.p[sl - 1], s2[h]));
  }
  __syncthreads();
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int b = t + h * kTile;   // left neighbour's slot is b + 2
    const int e = e0 + b;
    const double P0 = sh.p[b + 2], P1 = sh.q1[b + 2], P2 = sh.q2[b + 2];
    double *o = uout + e;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double acc = S.G[i * NP] * u[h][0];
#pragma unroll
      for (int j = 1; j < NP; ++j) acc = fma(S.G[i * NP + j], u[h][j], acc);
      acc = fma(S.h[0][i], P0, acc);
      acc = fma(S.h[1][i], P1, acc);
      acc = fma(S.h[2][i], P2, acc);
      if (e < K) *o = acc;
      o += K;
    }
  }
}

template <int NP, int EPT>
__global__ void __launch_bounds__(kTile) k_step_fused(const Inst inst, const double *__restrict__ uin,
                                                      double *__restrict__ uout) {
  __shared__ FusedShared<EPT> sh;
  fused_body<NP, EPT>(inst, uin, uout, blockIdx.x * (kTile * EPT), sh);
}

// What the PE-face correction of face j at step n reads besides the field: its delay k and
// order q' (delay_at), the AT coefficients, and the upwind traces of levels n-k-i (i < q')
// for the S stages from the ring [slot][stage][P] (zero when k = 0).
template <int S>
struct FaceLoads {
  double Rv[S][kMaxQ];
  double c[kMaxQ];
  int k, qe, nm;   // nm: the ring slot of step n
};

// n mod m for n >= 0, m > 0 (a 32-bit remainder while n fits in 31 bits).
__device__ __forceinline__ int mod_step(int64_t n, int m) {
  return n <= 0x7fffffff ? (int)((unsigned)n % (unsigned)m) : (int)(n % m);
}

template <int S>
__device__ __forceinline__ void face_loads(const Inst &I, int j, int64_t n, FaceLoads<S> &f) {
  const DelayAt dl = delay_at(I, j, n);
  const int P = I.P, R = I.R;
  const int nm = mod_step(n, R);
  f.nm = nm;
  const double2 *col = I.ring + j;
  f.k = dl.k;
  f.qe = dl.qe;
#pragma unroll
  for (int i = 0; i < kMaxQ; ++i) {
    int sl = nm - (dl.k + i);
    if (sl < 0) sl += R;
    const bool use = dl.k > 0 && i < dl.qe;
    f.c[i] = i < dl.qe ? dl.c[i] : 0.0;
    const double2 *lv = col + (size_t)sl * (S * P);
#pragma unroll
    for (int st = 0; st < S; ++st) f.Rv[st][i] = use ? lv[st * P].x : 0.0;
  }
}

// The synchronous traces of element e-1's stage inputs at a PE face (e the face's element):
// T[0] = p^{e-1}, the right trace of u^{e-1}, and the channel scalars T[s] = Y_s^{e-1}_p =
// r_s . u^{e-1} + sum_{t<s} k_st Y_t^{e-2}_p, from elements e-S .. e-1 (w = 0 .. S-1).
template <int S>
struct FaceTraces {
  double T[S];
};

// The channel scalars Y_s^m_p of elements m = e-S+1 .. e-1 in FP64, from the elements
// e-S .. e-1 (U[w], w = 0 .. S-1): element e-S+w forms Y_1 .. Y_w from its values and the
// scalars of the element before it.
template <int NP, int S>
__device__ __forceinline__ FaceTraces<S> face_traces(const Inst &I, const double (*U)[NP]) {
  const StepConsts &C = I.st;
  double Yp[S];   // the channel scalars of the element one to the left (Yp[0] = its trace)
  Yp[0] = U[0][NP - 1];
#pragma unroll
  for (int w = 1; w < S; ++w) {
    const int ns = w;   // channels 1 .. w of element e-S+w
    double Y[S];
    Y[0] = U[w][NP - 1];
#pragma unroll
    for (int s = 1; s <= ns; ++s) {
      double a = C.r[s][0] * U[w][0];
#pragma unroll
      for (int i = 1; i < NP; ++i) a = fma(C.r[s][i], U[w][i], a);
#pragma unroll
      for (int t = 0; t < s; ++t) a = fma(C.k[s][t], Yp[t], a);
      Y[s] = a;
    }
#pragma unroll
    for (int s = 0; s <= ns; ++s) Yp[s] = Y[s];
  }
  FaceTraces<S> t;
#pragma unroll
  for (int s = 0; s < S; ++s) t.T[s] = Yp[s];
  return t;
}

// The right trace of an int64 element: its last value, or for block-basis coordinates the
// sum of the first coordinate of each block, w_0 + w_2 (exact).
template <int NP>
__device__ __forceinline__ long long fx_trace(const Inst &I, const long long *X) {
  if (!I.basis) return X[NP - 1];
  return NP > 2 ? X[0] + X[2] : X[0];
}

// From int64 values X at scale 2^sig: the same sums in the composed step's two-limb integer
// arithmetic (StepFixed coefficients) at a scale chosen from these S elements alone
// (|X'| < 2^(56 - fxh), so the result does not depend on any other face), then rounded to
// FP64. Off the FP64 pipe but for S conversions.
template <int NP, int S>
__device__ __forceinline__ FaceTraces<S> face_traces_fixed(const Inst &I, const long long (*X)[NP],
                                                           int sig) {
  const StepFixed &F = I.sf;
  unsigned long long m = 0;
#pragma unroll
  for (int w = 0; w < S; ++w)
#pragma unroll
    for (int i = 0; i < NP; ++i) m |= fx_mag(X[w][i]);
  const int L = m ? 64 - __clzll((long long)m) : 0;   // |X| < 2^(L+1)
  const int top = 55 - I.fxh;
  const int sh = L > top ? L - top : 0;
  long long Yp[S];
  {
    long long Xs[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) Xs[i] = fx_rescale(X[0][i], sh);
    Yp[0] = fx_trace<NP>(I, Xs);
  }
#pragma unroll
  for (int w = 1; w < S; ++w) {
    const int ns = w;   // channels 1 .. w of element e-S+w
    int xh[NP], xl[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) fx_split(fx_rescale(X[w][i], sh), xh[i], xl[i]);
    int ph[S], pl[S];
#pragma unroll
    for (int t = 0; t < S - 1; ++t)
      if (t < ns) fx_split(Yp[t], ph[t], pl[t]);
    long long Y[S];
    {
      long long Xs[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) Xs[i] = fx_rescale(X[w][i], sh);
      Y[0] = fx_trace<NP>(I, Xs);
    }
#pragma unroll
    for (int s = 1; s <= ns; ++s) {
      FxAcc acc;
#pragma unroll
      for (int i = 0; i < NP; ++i) fx_mac(acc, F.r[s][i], xh[i], xl[i]);
#pragma unroll
      for (int t = 0; t < s; ++t) fx_mac(acc, F.k[s][t], ph[t], pl[t]);
      Y[s] = fx_round(acc);
    }
#pragma unroll
    for (int s = 0; s <= ns; ++s) Yp[s] = Y[s];
  }
  FaceTraces<S> t;
  t.T[0] = pow2_scale((double)fx_trace<NP>(I, X[S - 1]), sig);
#pragma unroll
  for (int s = 1; s < S; ++s) t.T[s] = pow2_scale((double)Yp[s], sig + sh);
  return t;
}

// The stage differences d_s = T_s - V_s at PE face j, step n, from the synchronous traces and
// the face's loads, and the ring write of T_s (the PE-face correction below).
template <int S>
__device__ __forceinline__ void face_diffs(const Inst &I, int j, const FaceLoads<S> &f,
                                           const FaceTraces<S> &tr, double *d) {
  const int P = I.P;
  const StepConsts &C = I.st;
  double2 *col = I.ring + j;
  const int k = f.k, qe = f.qe;
  double V[S];
#pragma unroll
  for (int st = 0; st < S; ++st) {
    double v = __dmul_rn(f.c[0], f.Rv[st][0]);
#pragma unroll
    for (int i = 1; i < kMaxQ; ++i) {
      if (i < qe) {
        const double ci = f.c[i];
        if (ci != 0.0) v = __dadd_rn(v, __dmul_rn(ci, f.Rv[st][i]));
      }
    }
    V[st] = v;
  }
  // T_s: the traces plus the responses to the earlier stages' corrections; with zero delay
  // V_s = T_s (the current traces), so d_s = 0
  double2 *lv = col + (size_t)f.nm * (S * P);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    double T = tr.T[s];
#pragma unroll
    for (int t = 0; t < s; ++t) T = fma(C.rho[s][t], d[t], T);
    d[s] = k > 0 ? __dsub_rn(T, V[s]) : 0.0;
    lv[s * P] = make_double2(T, 0.0);
  }
}

// PE-face correction of a three-stage composed step (upwind advection, a > 0; StepConsts):
// thread j forms, for PE face j (e = j Kpe), the synchronous right traces of element e-1's
// stage inputs (p, q1 = v1_p, q2 = v2_p, from elements e-3 .. e-1 with the composed step's
// coefficients), then stage by stage T_s (those traces plus the responses to the earlier
// corrections), the delayed / AT value V_s (Eq. at-flux-gen over the upwind traces of levels
// n-k-i in the ring; the face's delay k is one per step, so V_s does not depend on T), and
// d_s = T_s - V_s, writes T_s into the ring slot of step n (only the upwind trace is read back
// for a > 0; the other slot holds 0), and adds sum_s R_s d_s to the composed (synchronous)
// result of elements e-1 .. e+2. Every load (delay, ring levels of all three stages, inputs,
// outputs) is issued before any of them is used. A zero delay gives d_s = 0 exactly and leaves
// the composed result as it is. Windows of different faces are disjoint when Kpe >= 8. fmt:
// the fixed-point step's formats (bit 0: uin, bit 1: uout int64 at the step's scale). The
// AT sums and the stage-by-stage traces are FP64; with an int64 input the synchronous traces,
// and with an int64 output the correction itself, are formed in the step's integer limbs (as in
// k_face_step, so batched and single runs agree bit for bit).
template <int NP, bool FOUT>
__device__ __forceinline__ void fixup_body(const Inst &I, int j, const void *__restrict__ uin,
                                           void *__restrict__ uout, int rel, bool fin) {
  const int K = I.K;
  const int e = j * I.Kpe;
  const int64_t n = I.meta[0] + rel;
  const bool fout = FOUT;
  const StepConsts &S = I.st;
  // Loads that do not depend on the step kernel before this one (its input u^n, the delay, AT
  // coefficients and earlier ring levels) come before waiting for it (programmatic launch).
  long long Xr[3][NP];   // raw 64-bit values of e-3 .. e-1: int64, or the bits of FP64
  for (int w = 0; w < 3; ++w) {
    int m = e - 3 + w;
    if (m < 0) m += K;
    const long long *q = static_cast<const long long *>(uin) + m;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      Xr[w][i] = *q;
      q += K;
    }
  }
  FaceLoads<3> fl;
  face_loads<3>(I, j, n, fl);
  pdl_wait();
  pdl_trigger();
  FxScale sc{0, 0, 0, false};
  int sig_in = 0;
  if (I.fused == 2) {
    sc = fx_scale(I.fx, n, fin, I.fxh, I.fxe);
    sig_in = I.fx[sc.slot].sigma;
  }
  // the composed result of e-1 .. e+2 (w = 0 .. 3)
  int mw[4];
  for (int w = 0; w < 4; ++w) {
    int m = e - 1 + w;
    if (m < 0) m += K;
    if (m >= K) m -= K;
    mw[w] = m;
  }
  long long Xq[4][NP];
  double Yd[4][NP];
  for (int w = 0; w < 4; ++w) {
    if (fout) {
      const long long *q = static_cast<const long long *>(uout) + mw[w];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        Xq[w][i] = *q;
        q += K;
      }
    } else {
      const double *q = static_cast<const double *>(uout) + mw[w];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        Yd[w][i] = *q;
        q += K;
      }
    }
  }
  FaceTraces<3> tr;
  if (fin) {
    tr = face_traces_fixed<NP, 3>(I, Xr, sig_in);
  } else {
    double U[3][NP];
#pragma unroll
    for (int w = 0; w < 3; ++w)
#pragma unroll
      for (int i = 0; i < NP; ++i) U[w][i] = __longlong_as_double(Xr[w][i]);
    tr = face_traces<NP, 3>(I, U);
  }
  double dd[3];
  face_diffs<3>(I, j, fl, tr, dd);
  const double d0 = dd[0], d1 = dd[1], d2 = dd[2];
  // with a NaN or infinity in u^n the fixed-point step has already written NaN (or carries
  // the mark); nothing is added
  if (!(nonzero(d0) || nonzero(d1) || nonzero(d2)) || sc.bad) return;
  int emax = 0;
  unsigned long long mag = 0;
  if (fout && I.face_fx) {
    // the fixed-point step's int64 output: the integer correction of k_face_step
    const double sf = pow2_scale(1.0, -sc.sigma);
    const long long D0 = llrint(d0 * sf), D1 = llrint(d1 * sf), D2 = llrint(d2 * sf);
    const long long lim = 1ll << 57;
    if (D0 > -lim && D0 < lim && D1 > -lim && D1 < lim && D2 > -lim && D2 < lim) {
      int h0, l0, h1, l1, h2, l2;
      fx_split(D0, h0, l0);
      fx_split(D1, h1, l1);
      fx_split(D2, h2, l2);
      for (int w = 0; w < 4; ++w) {
        long long *q = static_cast<long long *>(uout) + mw[w];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          FxAcc acc;
          fx_mac(acc, I.Rf[0][w][i], h0, l0);
          fx_mac(acc, I.Rf[1][w][i], h1, l1);
          fx_mac(acc, I.Rf[2][w][i], h2, l2);
          const long long X = Xq[w][i] + fx_round(acc);
          *q = X;
          q += K;
          mag |= fx_mag(X);
        }
      }
      or_slot(&I.fx[fx_next(sc.slot)].mag, mag);
      return;
    }
  }
  for (int w = 0; w < 4; ++w) {   // elements e-1 .. e+2
    if (fout) {
      // FP64 sum (block-basis coordinates: the nodal correction times Tbi)
      double c[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i)
        c[i] = fma(S.R[2][w][i], d2, fma(S.R[1][w][i], d1, S.R[0][w][i] * d0));
      if (I.basis) {
        double cb[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          cb[i] = I.Tbi[i * NP] * c[0];
#pragma unroll
          for (int k = 1; k < NP; ++k) cb[i] = fma(I.Tbi[i * NP + k], c[k], cb[i]);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) c[i] = cb[i];
      }
      long long *q = static_cast<long long *>(uout) + mw[w];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const long long X = Xq[w][i] + llrint(pow2_scale(c[i], -sc.sigma));
        *q = X;
        q += K;
        mag |= fx_mag(X);
      }
    } else {
      double *q = static_cast<double *>(uout) + mw[w];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const double c = fma(S.R[2][w][i], d2, fma(S.R[1][w][i], d1, S.R[0][w][i] * d0));
        const double y = __dadd_rn(Yd[w][i], c);
        *q = y;
        q += K;
        const int be = biased_exponent(y);
        emax = be > emax ? be : emax;
      }
    }
  }
  // the fixed-point composed step takes the scale of u^{n+1} from every value written
  if (I.fused == 2) {
    FxSlot &nx = I.fx[fx_next(sc.slot)];
    if (fout) or_slot(&nx.mag, mag);
    else raise_slot(&nx.E, emax);
  }
}

// PE-face work of the fixed-point step between two steps, on the field u that is the output
// of step n-1 and the input of step n (n = meta[0] + rel), for PE face j (e = j Kpe), with S
// the composed step's stages. A block of (S+1) warps takes 32 faces, warp w element e-1+w of
// their correction windows (so the FP64 work of the differences runs in full warps):
//   kFaceApply: adds step n-1's correction sum_s R_s[w] d_s (its differences in I.fd, buffer
//               (n-1) & 1) to element e-1+w of u at step n-1's working scale, with the scale
//               bookkeeping of the values written (slot n % 3);
//   kFaceDiff:  warp 0 then forms step n's differences d_s from elements e-S .. e-1 of u
//               (e-1 as corrected) and the ring (face_diffs), writes the ring slot of step n
//               and I.fd buffer n & 1.
// fu: u is int64 (at the scale of slot n % 3), else FP64; fin_prev: step n-1 read int64. Every
// load is issued before any value is used; the windows of different faces (e-S .. e+S-1) are
// disjoint when Kpe >= 2S.
template <int NP, int S>
__global__ void __launch_bounds__(32 * (S + 1)) k_face_step(const Inst I, void *__restrict__ u,
                                                          int rel, int fu, int fin_prev,
                                                          int mode) {
  const int j = blockIdx.x * 32 + (threadIdx.x & 31), w = threadIdx.x >> 5;
  if (j >= I.P) return;
  const int K = I.K, P = I.P;
  const int e = j * I.Kpe;
  const int64_t n = I.meta[0] + rel;
  const bool diff = (mode & kFaceDiff) && w == 0;
  long long *uq = static_cast<long long *>(u);
  int m = e - 1 + w;   // this thread's element; warp 0 also reads e-S .. e-2
  if (m < 0) m += K;
  if (m >= K) m -= K;
  // The delay, AT coefficients and ring levels of steps before n do not depend on the step
  // kernel before this one: loaded before waiting for it (programmatic launch).
  FaceLoads<S> fl;
  if (diff) face_loads<S>(I, j, n, fl);
  pdl_wait();
  pdl_trigger();
  long long V[S][NP];   // raw 64-bit values (int64, or the bits of FP64): e-S .. e-2, own
  {
    const long long *q = uq + m;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      V[S - 1][i] = *q;
      q += K;
    }
  }
  if (diff) {
#pragma unroll
    for (int b = 0; b < S - 1; ++b) {
      int mb = e - S + b;
      if (mb < 0) mb += K;
      const long long *q = uq + mb;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        V[b][i] = *q;
        q += K;
      }
    }
  }
  if (mode & kFaceApply) {
    const double *dd = I.fd + (size_t)((n - 1) & 1) * S * P + S * (size_t)j;
    double d[S];
    bool any = false;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      d[s] = dd[s];
      any = any || nonzero(d[s]);
    }
    const FxScale sc = fx_scale(I.fx, n - 1, fin_prev != 0, I.fxh, I.fxe);
    if (any && !sc.bad) {
      bool done = false;
      if (fu && I.face_fx) {
        // D_s = round(d_s 2^-sigma) and sum_s R_s D_s in the step's two-limb arithmetic
        const double sf = pow2_scale(1.0, -sc.sigma);
        const long long lim = 1ll << 57;
        long long D[S];
        bool inr = true;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          D[s] = llrint(d[s] * sf);
          inr = inr && D[s] > -lim && D[s] < lim;
        }
        if (inr) {
          int hh[S], ll[S];
#pragma unroll
          for (int s = 0; s < S; ++s) fx_split(D[s], hh[s], ll[s]);
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            FxAcc acc;
#pragma unroll
            for (int s = 0; s < S; ++s) fx_mac(acc, I.Rf[s][w][i], hh[s], ll[s]);
            V[S - 1][i] += fx_round(acc);
          }
          done = true;
        }
      }
      if (!done) {
        // FP64: an FP64 output, or a difference beyond the integer range (block-basis
        // coordinates: the nodal correction times Tbi)
        const StepConsts &C = I.st;
        double c[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          c[i] = C.R[0][w][i] * d[0];
#pragma unroll
          for (int s = 1; s < S; ++s) c[i] = fma(C.R[s][w][i], d[s], c[i]);
        }
        if (fu && I.basis) {
          double cb[NP];
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            cb[i] = I.Tbi[i * NP] * c[0];
#pragma unroll
            for (int k = 1; k < NP; ++k) cb[i] = fma(I.Tbi[i * NP + k], c[k], cb[i]);
          }
#pragma unroll
          for (int i = 0; i < NP; ++i) c[i] = cb[i];
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          if (fu) V[S - 1][i] += llrint(pow2_scale(c[i], -sc.sigma));
          else V[S - 1][i] = __double_as_longlong(__dadd_rn(__longlong_as_double(V[S - 1][i]), c[i]));
        }
      }
      int emax = 0;
      unsigned long long mag = 0;
      long long *q = uq + m;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const long long X = V[S - 1][i];
        *q = X;
        q += K;
        if (fu) {
          mag |= fx_mag(X);
        } else {
          const int be = biased_exponent(__longlong_as_double(X));
          emax = be > emax ? be : emax;
        }
      }
      FxSlot &nx = I.fx[fx_next(sc.slot)];
      if (fu) or_slot(&nx.mag, mag);
      else raise_slot(&nx.E, emax);
    }
  }
  if (diff) {
    FaceTraces<S> tr;
    if (fu) {
      tr = face_traces_fixed<NP, S>(I, V, I.fx[(int)(n % 3)].sigma);
    } else {
      double U[S][NP];
#pragma unroll
      for (int b = 0; b < S; ++b)
#pragma unroll
        for (int i = 0; i < NP; ++i) U[b][i] = __longlong_as_double(V[b][i]);
      tr = face_traces<NP, S>(I, U);
    }
    double d[S];
    face_diffs<S>(I, j, fl, tr, d);
    double *o = I.fd + (size_t)(n & 1) * S * P + S * (size_t)j;
#pragma unroll
    for (int s = 0; s < S; ++s) o[s] = d[s];
  }
}

template <int NP>
__global__ void __launch_bounds__(64) k_step_fixup(const Inst I, const void *__restrict__ uin,
                                                   void *__restrict__ uout, int rel, int fmt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= I.P) return;
  if (fmt & kFmtOutFixed) fixup_body<NP, true>(I, j, uin, uout, rel, (fmt & kFmtInFixed) != 0);
  else fixup_body<NP, false>(I, j, uin, uout, rel, (fmt & kFmtInFixed) != 0);
}

// Batched composed steps: block b takes work item (instance, first element); `parity`
// selects the ping-pong direction (0: u -> v1, 1: v1 -> u) shared by every instance.
__global__ void __launch_bounds__(kTile) k_batch_fused(const Inst *__restrict__ insts,
                                                       const int2 *__restrict__ work, int parity) {
  __shared__ __align__(16) unsigned char smem[sizeof(Inst)];
  __shared__ FusedShared<1> sh;
  const int2 w = work[blockIdx.x];
  {
    const int4 *src = reinterpret_cast<const int4 *>(insts + w.x);
    int4 *dst = reinterpret_cast<int4 *>(smem);
    for (int t = threadIdx.x; t < (int)(sizeof(Inst) / sizeof(int4)); t += blockDim.x)
      dst[t] = __ldg(src + t);
  }
  __syncthreads();
  const Inst &I = *reinterpret_cast<const Inst *>(smem);
  const double *uin = parity ? I.v1 : I.u;
  double *uout = parity ? I.u : I.v1;
  switch (I.Np) {
    case 2: fused_body<2, 1>(I, uin, uout, w.y, sh); break;
    case 3: fused_body<3, 1>(I, uin, uout, w.y, sh); break;
    case 4: fused_body<4, 1>(I, uin, uout, w.y, sh); break;
    default: fused_body<5, 1>(I, uin, uout, w.y, sh); break;
  }
}

// The PE-face corrections of a batched composed step, one thread per PE face of any instance:
// fflat lists (instance, face) for every PE face of every instance, so the threads of a block
// are all busy however few faces an instance has.
// FOUT: the step wrote int64 (fixed point), else FP64 (the FP64 composed step).
template <bool FOUT>
__global__ void __launch_bounds__(64) k_batch_fixup(const Inst *__restrict__ insts,
                                                    const int2 *__restrict__ fflat, int nflat,
                                                    int src, int dst, bool fin, int rel) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nflat) return;
  const int2 w = fflat[t];
  const Inst &I = insts[w.x];
  const int j = w.y;
  const void *uin = src == 0 ? (const void *)I.u : (src == 1 ? (const void *)I.v1 : (const void *)I.v2);
  void *uout = dst == 0 ? (void *)I.u : (dst == 1 ? (void *)I.v1 : (void *)I.v2);
  switch (I.Np) {
    case 2: fixup_body<2, FOUT>(I, j, uin, uout, rel, fin); break;
    case 3: fixup_body<3, FOUT>(I, j, uin, uout, rel, fin); break;
    case 4: fixup_body<4, FOUT>(I, j, uin, uout, rel, fin); break;
    default: fixup_body<5, FOUT>(I, j, uin, uout, rel, fin); break;
  }
}

// Copies v1 into u for every instance (after an odd number of batched composed steps).
__global__ void k_batch_copy_back(const Inst *__restrict__ insts, const int2 *__restrict__ work) {
  const int2 w = work[blockIdx.x];
  const Inst &I = insts[w.x];
  const int e = w.y + threadIdx.x;
  if (e >= I.K) return;
  for (int i = 0; i < I.Np; ++i) I.u[(size_t)i * I.K + e] = I.v1[(size_t)i * I.K + e];
}

// Face pass of one batched stage, run after the stage kernel. For PE face j (between elements
// e-1 = j Kpe - 1 and e = j Kpe) it reads the stage-input traces, forms the synchronous
// face value Vs and the delayed / AT value V from the ring, writes the traces into the ring
// slot of step n, and replaces the synchronous flux by the delayed one in both elements:
// out^e += lL (Vs - V), out^{e-1} += lR (Vs - V) (the flux enters the stage linearly through
// the lift terms). With Kpe == 1 an element borders two PE faces; then thread j owns
// element j and applies the corrections of both its faces.
template <int PDE, int DIR, class I>
__device__ __forceinline__ double face_delta(const I &inst, const double *vin, int j, int64_t n,
                                             int stage, bool owner) {
  const int K = inst.K;
  const int e = j * inst.Kpe;
  const double tl = vin[(size_t)(inst.Np - 1) * K + (e == 0 ? K - 1 : e - 1)];
  const double tr = vin[e];
  return pe_face_delta<PDE, DIR>(inst, j, n, stage, tl, tr, owner);
}

template <class I>
__device__ __forceinline__ void apply_delta(const I &inst, double *out, int e, const double *lift,
                                            double d) {
  if (!nonzero(d)) return;
  const int K = inst.K;
  for (int i = 0; i < inst.Np; ++i) out[(size_t)i * K + e] = fma(lift[i], d, out[(size_t)i * K + e]);
}

template <int PDE, int DIR, class I>
__device__ __forceinline__ void face_body(const I &inst, int stage, int j, int64_t n) {
  const double *vin = stage == 0 ? inst.u : (stage == 1 ? inst.v1 : inst.v2);
  double *out = stage == 0 ? inst.v1 : (stage == 1 ? inst.v2 : inst.unext);
  const StageConsts &C = inst.sc[stage];
  const int K = inst.K;
  if (inst.Kpe > 1) {
    // The two elements' outputs are loaded before the ring work so the loads overlap it.
    const int e = j * inst.Kpe;
    const int eL = e == 0 ? K - 1 : e - 1;
    double oe[kMaxNp], ol[kMaxNp];
#pragma unroll
    for (int i = 0; i < kMaxNp; ++i) {
      if (i < inst.Np) {
        oe[i] = out[(size_t)i * K + e];
        ol[i] = out[(size_t)i * K + eL];
      }
    }
    const double d = face_delta<PDE, DIR>(inst, vin, j, n, stage, true);
    if (nonzero(d)) {
#pragma unroll
      for (int i = 0; i < kMaxNp; ++i) {
        if (i < inst.Np) {
          out[(size_t)i * K + e] = fma(C.lL[i], d, oe[i]);
          out[(size_t)i * K + eL] = fma(C.lR[i], d, ol[i]);
        }
      }
    }
  } else {
    // element j borders faces j (left) and j+1 (right); the right face's value is formed
    // again here with the same arithmetic as by its owner, so both agree bit for bit.
    const double dL = face_delta<PDE, DIR>(inst, vin, j, n, stage, true);
    const double dR = face_delta<PDE, DIR>(inst, vin, j + 1 == inst.P ? 0 : j + 1, n, stage, false);
    double *o = out;
    if (nonzero(dL) || nonzero(dR)) {
      for (int i = 0; i < inst.Np; ++i) {
        double x = o[(size_t)i * K + j];
        if (nonzero(dL)) x = fma(C.lL[i], dL, x);
        if (nonzero(dR)) x = fma(C.lR[i], dR, x);
        o[(size_t)i * K + j] = x;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_batch_faces(const Inst *__restrict__ insts,
                                                     const int2 *__restrict__ work, int stage,
                                                     int rel) {
  const int2 w = work[blockIdx.x];
  const Inst &I = insts[w.x];
  const int j = w.y + threadIdx.x;
  if (j >= I.P) return;
  const int64_t n = I.meta[0] + rel;
  if (I.pde == 1) face_body<1, 0>(I, stage, j, n);
  else if (I.a >= 0.0) face_body<0, 1>(I, stage, j, n);
  else face_body<0, -1>(I, stage, j, n);
}

template <int STAGE, int NP>
__device__ __forceinline__ void batch_dispatch_pde(const Inst &I, int e) {
  if (I.pde == 0) {
    if (I.a >= 0.0) stage_body<NP, 0, STAGE, 1, false>(I, e);
    else stage_body<NP, 0, STAGE, -1, false>(I, e);
  } else {
    stage_body<NP, 1, STAGE, 0, false>(I, e);
  }
}

// Batched stage: block b handles work item (instance, first element); the instance's
// descriptor is staged in shared memory, then the element code runs as above.
template <int STAGE>
__global__ void __launch_bounds__(kTile) k_batch_stage(const Inst *__restrict__ insts,
                                                       const int2 *__restrict__ work) {
  __shared__ __align__(16) unsigned char smem[sizeof(Inst)];
  const int2 w = work[blockIdx.x];
  {
    const int4 *src = reinterpret_cast<const int4 *>(insts + w.x);
    int4 *dst = reinterpret_cast<int4 *>(smem);
    for (int t = threadIdx.x; t < (int)(sizeof(Inst) / sizeof(int4)); t += blockDim.x)
      dst[t] = __ldg(src + t);
  }
  __syncthreads();
  const Inst &I = *reinterpret_cast<const Inst *>(smem);
  const int e = w.y + threadIdx.x;
  switch (I.Np) {
    case 2: batch_dispatch_pde<STAGE, 2>(I, e); break;
    case 3: batch_dispatch_pde<STAGE, 3>(I, e); break;
    case 4: batch_dispatch_pde<STAGE, 4>(I, e); break;
    default: batch_dispatch_pde<STAGE, 5>(I, e); break;
  }
}

__global__ void k_advance(int64_t *meta, int stride, int ninst, int64_t by) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ninst) meta[(size_t)i * stride] += by;
}

// Element-major rows into node planes (dst[i K + e] = src[e Np + i]); with emax, the
// largest biased FP64 exponent of the values is raised into *emax (one atomic per block;
// 2047 marks a NaN or an infinity among them), so that loading a field also yields its
// finiteness and the exponent the fixed-point step scales it by.
__global__ void __launch_bounds__(256) k_to_internal(const double *__restrict__ src,
                                                     double *__restrict__ dst, int K, int Np,
                                                     int *__restrict__ emax) {
  const size_t n = (size_t)K * Np;
  int m = 0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const double x = src[idx];
    const size_t e = idx / Np, i = idx % Np;
    dst[i * K + e] = x;
    const int be = biased_exponent(x);
    m = be > m ? be : m;
  }
  if (!emax) return;
  __shared__ int wm[8];
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wm[w] > m ? wm[w] : m;
    raise_slot(emax, m);
  }
}

__global__ void k_to_external(const double *__restrict__ src, double *__restrict__ dst, int K,
                              int Np) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)K * Np) return;
  const size_t e = idx / Np, i = idx % Np;
  dst[idx] = src[i * K + e];
}

struct ModeArgs {
  double xi[kMaxNp];
  double amp[16], kappa[16], phase[16];
};

__global__ void k_eval_modes(double *u, int K, int Np, double x0, double dx, ModeArgs m,
                             int nmodes, double offset) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)K * Np) return;
  const size_t e = idx / Np;
  const int i = (int)(idx % Np);
  // x = x0 + e dx + (1 + xi_i) dx/2, evaluated in this order without contraction.
  const double x = __dadd_rn(__dadd_rn(x0, __dmul_rn((double)e, dx)),
                             __dmul_rn(__dadd_rn(1.0, m.xi[i]), __dmul_rn(dx, 0.5)));
  double val = offset;
  for (int t = 0; t < nmodes; ++t)
    val = __dadd_rn(val, __dmul_rn(m.amp[t], sin(__dadd_rn(__dmul_rn(m.kappa[t], x), m.phase[t]))));
  u[idx] = val;
}

constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads)
    k_reduce(int kind, const double *__restrict__ u, const double *__restrict__ g, int K, int Np,
             const double *__restrict__ wm, double *partials) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
    if (kind == 0) {
      double s = 0.0;
      for (int i = 0; i < Np; ++i) s = fma(wm[i], u[(size_t)i * K + e], s);
      acc += s;
    } else if (kind == 1) {
      for (int i = 0; i < Np; ++i) acc = fmax(acc, fabs(u[(size_t)i * K + e]));
    } else if (kind == 2) {
      for (int i = 0; i < Np; ++i) acc += isfinite(u[(size_t)i * K + e]) ? 0.0 : 1.0;
    } else {
      double d[kMaxNp];
      for (int i = 0; i < Np; ++i) d[i] = u[(size_t)i * K + e] - g[(size_t)i * K + e];
      double s = 0.0;
      for (int i = 0; i < Np; ++i) {
        double r = 0.0;
        for (int j = 0; j < Np; ++j) r = fma(wm[i * Np + j], d[j], r);
        s = fma(d[i], r, s);
      }
      acc += s;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      sh[threadIdx.x] = kind == 1 ? fmax(sh[threadIdx.x], sh[threadIdx.x + h])
                                  : sh[threadIdx.x] + sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedThreads)
    k_reduce_final(int kind, const double *partials, int n, double scale, double *out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x)
    acc = kind == 1 ? fmax(acc, partials[t]) : acc + partials[t];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      sh[threadIdx.x] = kind == 1 ? fmax(sh[threadIdx.x], sh[threadIdx.x + h])
                                  : sh[threadIdx.x] + sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (kind == 0 || kind == 3) ? sh[0] * scale : sh[0];
}

template <int NP, int PDE, int STAGE, int DIR>
cudaError_t launch_np_pde_stage(const Inst &I, int rel, cudaStream_t s, bool pdl) {
  const int bs = stage_block(I.K);
  const unsigned grid = (unsigned)((I.K + bs - 1) / bs);
  if (PDE == 1 && I.visc) {
    if (I.async)
      return launch_maybe_pdl(k_stage<NP, PDE, STAGE, DIR, true, true>, dim3(grid), dim3(bs), s,
                              pdl, I, rel);
    return launch_maybe_pdl(k_stage<NP, PDE, STAGE, DIR, false, true>, dim3(grid), dim3(bs), s,
                            pdl, I, rel);
  }
  // 30 elements per warp (halo lanes); one-thread-per-element stage_body is kept for the 2N
  // low-storage, viscous and batched stages
  const int64_t warps = (I.K + 29) / 30;
  const dim3 g((unsigned)((warps * 32 + bs - 1) / bs));
  if (I.async)
    return launch_maybe_pdl(k_stage_halo<NP, PDE, STAGE, DIR, true>, g, dim3(bs), s, pdl, I, rel);
  return launch_maybe_pdl(k_stage_halo<NP, PDE, STAGE, DIR, false>, g, dim3(bs), s, pdl, I, rel);
}

template <int NP, int PDE, int DIR>
cudaError_t launch_np_pde(const Inst &I, int stage, int rel, cudaStream_t s, bool pdl) {
  switch (stage) {
    case 0: return launch_np_pde_stage<NP, PDE, 0, DIR>(I, rel, s, pdl);
    case 1: return launch_np_pde_stage<NP, PDE, 1, DIR>(I, rel, s, pdl);
    default: return launch_np_pde_stage<NP, PDE, 2, DIR>(I, rel, s, pdl);
  }
}

template <int NP>
cudaError_t launch_np(const Inst &I, int stage, int rel, cudaStream_t s, bool pdl) {
  if (I.pde == 1) return launch_np_pde<NP, 1, 0>(I, stage, rel, s, pdl);
  return I.a >= 0.0 ? launch_np_pde<NP, 0, 1>(I, stage, rel, s, pdl)
                    : launch_np_pde<NP, 0, -1>(I, stage, rel, s, pdl);
}

}  // namespace

cudaError_t launch_stage(const Inst &I, int stage, int rel, cudaStream_t s, bool pdl) {
  switch (I.Np) {
    case 2: return launch_np<2>(I, stage, rel, s, pdl);
    case 3: return launch_np<3>(I, stage, rel, s, pdl);
    case 4: return launch_np<4>(I, stage, rel, s, pdl);
    case 5: return launch_np<5>(I, stage, rel, s, pdl);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

template <int NP, int PDE, int DIR>
cudaError_t lsrk_np_pde(const Inst &I, int rel, const LsArgs &ls, cudaStream_t s) {
  const int bs = stage_block(I.K);
  const unsigned grid = (unsigned)((I.K + bs - 1) / bs);
  if (PDE == 1 && I.visc) {
    if (I.async) k_lsrk_stage<NP, PDE, DIR, true, true><<<grid, bs, 0, s>>>(I, rel, ls);
    else k_lsrk_stage<NP, PDE, DIR, false, true><<<grid, bs, 0, s>>>(I, rel, ls);
  } else if (I.async) {
    k_lsrk_stage<NP, PDE, DIR, true><<<grid, bs, 0, s>>>(I, rel, ls);
  } else {
    k_lsrk_stage<NP, PDE, DIR, false><<<grid, bs, 0, s>>>(I, rel, ls);
  }
  return cudaGetLastError();
}

template <int NP>
cudaError_t ldg_q_np(const Inst &I, const double *vin, int stage, int rel, cudaStream_t s) {
  const int bs = stage_block(I.K);
  const unsigned grid = (unsigned)((I.K + bs - 1) / bs);
  if (I.async) k_ldg_q<NP, true><<<grid, bs, 0, s>>>(I, vin, stage, rel);
  else k_ldg_q<NP, false><<<grid, bs, 0, s>>>(I, vin, stage, rel);
  return cudaGetLastError();
}

template <int NP>
cudaError_t lsrk_np(const Inst &I, int rel, const LsArgs &ls, cudaStream_t s) {
  if (I.pde == 1) return lsrk_np_pde<NP, 1, 0>(I, rel, ls, s);
  return I.a >= 0.0 ? lsrk_np_pde<NP, 0, 1>(I, rel, ls, s) : lsrk_np_pde<NP, 0, -1>(I, rel, ls, s);
}

}  // namespace

cudaError_t launch_ldg_q(const Inst &I, const double *vin, int stage, int rel, cudaStream_t s) {
  if (!I.visc || !I.qbuf || stage < 0 || stage >= I.ns) return cudaErrorInvalidValue;
  switch (I.Np) {
    case 2: return ldg_q_np<2>(I, vin, stage, rel, s);
    case 3: return ldg_q_np<3>(I, vin, stage, rel, s);
    case 4: return ldg_q_np<4>(I, vin, stage, rel, s);
    case 5: return ldg_q_np<5>(I, vin, stage, rel, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_lsrk_stage(const Inst &I, int s, int rel, const double *uin, double *uout,
                              cudaStream_t st) {
  if (!I.ls || s < 0 || s >= I.ns || uin == uout) return cudaErrorInvalidValue;
  LsArgs ls;
  ls.uin = uin;
  ls.uout = uout;
  ls.s = s;
  ls.first = s == 0;
  ls.As = I.lsA[s];
  ls.Bs = I.lsB[s];
  switch (I.Np) {
    case 2: return lsrk_np<2>(I, rel, ls, st);
    case 3: return lsrk_np<3>(I, rel, ls, st);
    case 4: return lsrk_np<4>(I, rel, ls, st);
    case 5: return lsrk_np<5>(I, rel, ls, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_stage(const Inst *insts_dev, const int2 *work_dev, int nwork, int stage,
                               int rel, int tile, cudaStream_t s) {
  (void)tile;
  switch (stage) {
    case 0: k_batch_stage<0><<<nwork, kTile, 0, s>>>(insts_dev, work_dev); break;
    case 1: k_batch_stage<1><<<nwork, kTile, 0, s>>>(insts_dev, work_dev); break;
    default: k_batch_stage<2><<<nwork, kTile, 0, s>>>(insts_dev, work_dev); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_faces(const Inst *insts_dev, const int2 *work_dev, int nwork, int stage,
                               int rel, cudaStream_t s) {
  if (nwork > 0) k_batch_faces<<<nwork, 256, 0, s>>>(insts_dev, work_dev, stage, rel);
  return cudaGetLastError();
}

namespace {
template <int NP>
cudaError_t fused_np(const Inst &I, const void *uin, void *uout, int rel, cudaStream_t s,
                     bool with_fixup, int fmt) {
  if (I.fused == 2) {
    cudaError_t e = launch_fixed_step(I, uin, uout, rel, fmt, s);
    if (e != cudaSuccess) return e;
  } else {
    const double *ui = static_cast<const double *>(uin);
    double *uo = static_cast<double *>(uout);
    fmt = 0;
    if (I.ept == 4)
      k_step_fused<NP, 4><<<(unsigned)((I.K + 4 * kTile - 1) / (4 * kTile)), kTile, 0, s>>>(I, ui, uo);
    else if (I.ept == 2)
      k_step_fused<NP, 2><<<(unsigned)((I.K + 2 * kTile - 1) / (2 * kTile)), kTile, 0, s>>>(I, ui, uo);
    else
      k_step_fused<NP, 1><<<(unsigned)((I.K + kTile - 1) / kTile), kTile, 0, s>>>(I, ui, uo);
  }
  if (I.async && with_fixup)
    k_step_fixup<NP><<<(unsigned)((I.P + 63) / 64), 64, 0, s>>>(I, uin, uout, rel, fmt);
  return cudaGetLastError();
}
}  // namespace

template <int S>
cudaError_t face_step_s(const Inst &I, void *u, int rel, int fu, int fin_prev, int mode,
                        cudaStream_t s, bool pdl) {
  const dim3 g((unsigned)((I.P + 31) / 32)), b(32 * (S + 1));   // 32 faces per block
  switch (I.Np) {
    case 2: return launch_maybe_pdl(k_face_step<2, S>, g, b, s, pdl, I, u, rel, fu, fin_prev, mode);
    case 3: return launch_maybe_pdl(k_face_step<3, S>, g, b, s, pdl, I, u, rel, fu, fin_prev, mode);
    case 4: return launch_maybe_pdl(k_face_step<4, S>, g, b, s, pdl, I, u, rel, fu, fin_prev, mode);
    case 5: return launch_maybe_pdl(k_face_step<5, S>, g, b, s, pdl, I, u, rel, fu, fin_prev, mode);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_face_step(const Inst &I, void *u, int rel, int fu, int fin_prev, int mode,
                             cudaStream_t s, bool pdl) {
  if (I.ns == 3) return face_step_s<3>(I, u, rel, fu, fin_prev, mode, s, pdl);
  if (I.ns == kMaxCS) return face_step_s<kMaxCS>(I, u, rel, fu, fin_prev, mode, s, pdl);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_step(const Inst &I, const void *uin, void *uout, int rel,
                              cudaStream_t s, bool with_fixup, int fmt) {
  if (I.fused == 2 && I.async && with_fixup && I.fd) {
    // fixed point with PE faces: the step's differences, the step, its correction
    const int fin = (fmt & kFmtInFixed) ? 1 : 0, fout = (fmt & kFmtOutFixed) ? 1 : 0;
    cudaError_t e = launch_face_step(I, const_cast<void *>(uin), rel, fin, 0, kFaceDiff, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_fixed_step(I, uin, uout, rel, fmt, s)) != cudaSuccess) return e;
    return launch_face_step(I, uout, rel + 1, fout, fin, kFaceApply, s);
  }
  switch (I.Np) {
    case 2: return fused_np<2>(I, uin, uout, rel, s, with_fixup, fmt);
    case 3: return fused_np<3>(I, uin, uout, rel, s, with_fixup, fmt);
    case 4: return fused_np<4>(I, uin, uout, rel, s, with_fixup, fmt);
    case 5: return fused_np<5>(I, uin, uout, rel, s, with_fixup, fmt);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
__global__ void k_fill_delays(uint8_t *__restrict__ table, int64_t first, int64_t total,
                              const DelayGen g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (g.caa > 0) {   // step first + i / P of the cycle
      const int m = (int)((first + i / g.P) % (g.caa + g.L));
      table[i] = (uint8_t)(m < g.caa ? 0 : m - g.caa);
      continue;
    }
    const uint64_t idx = (uint64_t)first * (uint64_t)g.P + (uint64_t)i;   // (first + r) P + j
    uint64_t z = g.seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const uint64_t m = z >> 11;
    int k = g.L - 1;
    for (int b = g.L - 1; b >= 0; --b)
      if (m < g.T[b]) k = b;
    table[i] = (uint8_t)k;
  }
}
}  // namespace

cudaError_t launch_fill_delays(uint8_t *table, int64_t first, int rows, const DelayGen &g,
                               cudaStream_t s) {
  const int64_t total = (int64_t)rows * g.P;
  const int64_t want = (total + 255) / 256;
  const int64_t cap = 8 * (int64_t)sm_count();
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  k_fill_delays<<<grid, 256, 0, s>>>(table, first, total, g);
  return cudaGetLastError();
}

cudaError_t launch_batch_fused_step(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                    const int2 *fwork_dev, int nfwork, int src, int dst, int fmt,
                                    bool fixed, int rel, cudaStream_t s, const BatchUniform *bu,
                                    bool pdl) {
  cudaError_t e;
  if (fixed) {
    e = bu ? launch_batch_fixed_uniform(*bu, work_dev, nwork, src, dst, fmt, rel, s, pdl)
           : launch_batch_fixed_step(insts_dev, work_dev, nwork, src, dst, fmt, rel, s, pdl);
    if (e != cudaSuccess) return e;
  } else {
    fmt = 0;
    k_batch_fused<<<nwork, kTile, 0, s>>>(insts_dev, work_dev, src == 1 ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (nfwork > 0) {
    // a programmatic dependent of the step kernel: its input, delay and ring loads overlap it
    const dim3 g((unsigned)((nfwork + 63) / 64)), b(64);
    const bool fin = (fmt & kFmtInFixed) != 0;
    // the fix-up is the short, latency-bound link between a part's steps: its blocks take
    // SM resources ahead of the other parts' queued step blocks (64 threads a block: 32
    // measured 0.3329 against 0.3324 ms per batched step)
    static int prio = [] {
      int least = 0, greatest = 0;
      if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
      }
      return greatest;
    }();
    if (fmt & kFmtOutFixed)
      e = launch_pdl_priority(k_batch_fixup<true>, g, b, s, true, prio, insts_dev, fwork_dev,
                              nfwork, src, dst, fin, rel);
    else
      e = launch_pdl_priority(k_batch_fixup<false>, g, b, s, true, prio, insts_dev, fwork_dev,
                              nfwork, src, dst, fin, rel);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_copy_back(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                   cudaStream_t s) {
  k_batch_copy_back<<<nwork, kTile, 0, s>>>(insts_dev, work_dev);
  return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *meta, int stride, int ninst, int64_t by, cudaStream_t s) {
  k_advance<<<(ninst + 255) / 256, 256, 0, s>>>(meta, stride, ninst, by);
  return cudaGetLastError();
}

cudaError_t launch_to_internal(const double *src, double *dst, int K, int Np, cudaStream_t s,
                               int *emax) {
  const size_t n = (size_t)K * Np;
  const size_t want = (n + 255) / 256;
  const size_t cap = 16 * (size_t)sm_count();
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  k_to_internal<<<grid, 256, 0, s>>>(src, dst, K, Np, emax);
  return cudaGetLastError();
}

cudaError_t launch_to_external(const double *src, double *dst, int K, int Np, cudaStream_t s) {
  const size_t n = (size_t)K * Np;
  k_to_external<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, K, Np);
  return cudaGetLastError();
}

cudaError_t launch_eval_modes(double *u, int K, int Np, double x0, double dx, const double *xi,
                              int nmodes, const double *amp, const double *kappa,
                              const double *phase, double offset, cudaStream_t s) {
  if (nmodes < 0 || nmodes > 16 || Np > kMaxNp) return cudaErrorInvalidValue;
  ModeArgs m{};
  for (int i = 0; i < Np; ++i) m.xi[i] = xi[i];
  for (int t = 0; t < nmodes; ++t) {
    m.amp[t] = amp[t];
    m.kappa[t] = kappa[t];
    m.phase[t] = phase[t];
  }
  const size_t n = (size_t)K * Np;
  k_eval_modes<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(u, K, Np, x0, dx, m, nmodes, offset);
  return cudaGetLastError();
}

int sm_count() {
  constexpr int kMaxDev = 64;
  static int cached[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < kMaxDev && cached[dev] > 0) return cached[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  if (dev < kMaxDev) cached[dev] = n;
  return n;
}

int reduce_blocks(int K) {
  int b = (K + kRedThreads - 1) / kRedThreads;
  return b < 1024 ? (b < 1 ? 1 : b) : 1024;
}

cudaError_t launch_reduce(int kind, const double *u, const double *g, int K, int Np,
                          const double *wm, double scale, double *partials, int nblocks,
                          double *out, cudaStream_t s) {
  k_reduce<<<nblocks, kRedThreads, 0, s>>>(kind, u, g, K, Np, wm, partials);
  k_reduce_final<<<1, kRedThreads, 0, s>>>(kind, partials, nblocks, scale, out);
  return cudaGetLastError();
}

}  // namespace adg
