// Discrete adjoint of the ADG / ADG-AT SSP-RK3 step (used by adg_grad).
//
// The forward stage, per element, is (see adg_internal.h)
//   out = alpha u + A v + lL (f(v_0) - F_L) + lR (f(v_p) - F_R)      (Burgers adds beta v,
// with A applied to v^2), followed at PE faces by out^e += lL d, out^{e-1} += lR d with
// d = F_sync - F_delayed. Its transpose, for the adjoint w of the stage output, is
//   lambda_u += alpha w,
//   lambda_v  = A^T w (advection) or beta w + 2 v (A^T w) (Burgers),
//   face adjoint mu_f = -(lL . w^f) - (lR . w^{f-1}) applied through the flux partial
//   derivatives to the traces of the stage input,
// and at PE faces the delayed flux F = sum_i c_i fhat(T_{n-k-i}) sends c_i mu_f to an
// adjoint ring indexed like the forward one; the entry of level m, stage s is turned into
// trace adjoints when the reverse sweep reaches step m, stage s.
#include "adg_device.cuh"

namespace adg {
namespace {

// Partial derivatives of the local Lax-Friedrichs flux
//   F = 1/2 (uL^2/2 + uR^2/2) - 1/2 lam (uR - uL),  lam = max(|uL|, |uR|),
// with lam taken from uL when |uL| >= |uR| and d|u|/du = +1 for u >= 0, -1 otherwise.
__device__ __forceinline__ void llf_partials(double uL, double uR, double &dL, double &dR) {
  const bool fromL = abs_bits(uL) >= abs_bits(uR);
  const double lam = fromL ? fabs(uL) : fabs(uR);
  const double jump = uR - uL;
  double gL = 0.0, gR = 0.0;
  if (fromL) gL = nonneg(uL) ? 1.0 : -1.0;
  else gR = nonneg(uR) ? 1.0 : -1.0;
  dL = 0.5 * uL + 0.5 * lam - 0.5 * gL * jump;
  dR = 0.5 * uR - 0.5 * lam - 0.5 * gR * jump;
}

// Partials of the face value (trace units for advection, flux for Burgers).
template <int PDE, int DIR>
__device__ __forceinline__ void value_partials(double tl, double tr, double &dL, double &dR) {
  if (PDE == 0) {
    dL = DIR > 0 ? 1.0 : 0.0;
    dR = DIR > 0 ? 0.0 : 1.0;
  } else {
    llf_partials(tl, tr, dL, dR);
  }
}

// Adjoint of one stage with halo lanes (the layout of the forward k_stage_halo): warp w takes
// elements 30w .. 30w+29 in lanes 1 .. 30 and lanes 0 and 31 hold the elements on either side
// (periodic), so every face adjoint is formed by full-warp instructions (lane l forms the
// adjoint of its left face and hands the left element its part through a shuffle) and a PE
// face's adjoint g = nu + r (or r) is formed once, by the lane of the element right of the face
// (which, owned, also posts the delayed levels and clears the ring entry). A warp's FP64
// instruction costs the same pipe time whatever its active lanes, so the halo lanes' 2/32
// redundant work is cheaper than single-lane edge and face work.
template <int NP, int PDE, int STAGE, int DIR, bool FACES>
__global__ void __launch_bounds__(kTile) k_adj_stage_halo(const AdjStage A) {
  const int K = A.K;
  const int lane = threadIdx.x & 31;
  const int e = 30 * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) + lane - 1;
  const bool own = lane >= 1 && lane <= 30 && e < K;
  const int ec = e < 0 ? e + K : (e < K ? e : 0);
  const StageConsts &C = A.C;
  const unsigned full = 0xffffffffu;

  double w[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) w[i] = __ldg(A.w + (size_t)i * K + ec);
  double sL = 0.0, sR = 0.0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    sL = fma(C.lL[i], w[i], sL);
    sR = fma(C.lR[i], w[i], sR);
  }
  double v[NP];
  if (PDE == 1) {
#pragma unroll
    for (int i = 0; i < NP; ++i) v[i] = __ldg(A.v + (size_t)i * K + ec);
  }
  double lv[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    double acc = C.A[j] * w[0];
#pragma unroll
    for (int i = 1; i < NP; ++i) acc = fma(C.A[i * NP + j], w[i], acc);
    lv[j] = PDE == 0 ? acc : fma(C.beta, w[j], 2.0 * v[j] * acc);
  }
  const double sRp = __shfl_up_sync(full, sR, 1);     // sR of the element to the left
  if (PDE == 0) {
    if (DIR > 0) {
      lv[0] += sL;
      lv[NP - 1] -= __shfl_down_sync(full, sL, 1);
    } else {
      lv[NP - 1] += sR;
      lv[0] -= sRp;
    }
  } else {
    lv[0] = fma(v[0], sL, lv[0]);
    lv[NP - 1] = fma(v[NP - 1], sR, lv[NP - 1]);
    // left face of e: adjoint mu = -sL^e - sR^{e-1}, traces (v_p^{e-1}, v_0^e)
    const double vLm = __shfl_up_sync(full, v[NP - 1], 1);
    const double muL = -sL - sRp;
    double dL, dR;
    llf_partials(vLm, v[0], dL, dR);
    lv[0] = fma(muL, dR, lv[0]);
    lv[NP - 1] += __shfl_down_sync(full, muL * dL, 1);
  }

  if (FACES) {
    // lane l (1 .. 31) forms the adjoint of its left face when its element owns a PE face
    // (e = j Kpe, or e = K: face 0 seen from element K-1):
    //   nu = sL^e + sR^{e-1}, g = nu + r - [k == 0] nu, r = ring entry of (n, s, j),
    // and both elements add g times the value's partial derivative to their trace node (the
    // left one through a shuffle); an owned lane also posts c_i (-nu) to the delayed levels
    // (never to level n) and clears the ring entry the previous adjoint kernel read.
    const double tl = PDE == 1 ? __shfl_up_sync(full, v[NP - 1], 1) : 0.0;
    const int eo = e < K ? e : e - K;
    const int jq = eo / A.Kpe;
    const bool face = lane >= 1 && e <= K && eo - jq * A.Kpe == 0;
    double g = 0.0, pL = 0.0, pR = 0.0;
    if (face) {
      const int64_t n = A.meta[0] + A.rel;
      const int nm = (int)(n % A.R);
      auto slot_of = [&](int m) {   // ring slot of level n - m
        int sl = nm - m;
        if (sl < 0) sl += A.R;
        return sl;
      };
      const double nu = sL + sRp;
      const DelayAt d = delay_at(A, jq, n);
      const double r = A.lring[((size_t)nm * kStages + STAGE) * A.P + jq];
      g = d.k == 0 ? r : nu + r;
      value_partials<PDE, DIR>(tl, PDE == 1 ? v[0] : 0.0, pL, pR);
      if (own) {
        for (int i = 0; i < d.qe; ++i) {
          const double ci = d.c[i];
          if (ci != 0.0 && d.k + i >= 1)
            A.lring[((size_t)slot_of(d.k + i) * kStages + STAGE) * A.P + jq] += ci * (-nu);
        }
        const int pst = STAGE == 2 ? 0 : STAGE + 1;
        const int psl = STAGE == 2 ? (nm + 1 == A.R ? 0 : nm + 1) : nm;
        A.lring[((size_t)psl * kStages + pst) * A.P + jq] = 0.0;
      }
    }
    if (own && face) lv[0] = fma(g, pR, lv[0]);
    const double gR = __shfl_down_sync(full, g, 1);
    const double pLR = __shfl_down_sync(full, pL, 1);
    const bool faceR = __shfl_down_sync(full, face ? 1 : 0, 1) != 0;
    if (own && faceR) lv[NP - 1] = fma(gR, pLR, lv[NP - 1]);
  }

  if (own) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const size_t o = (size_t)i * K + e;
      if (STAGE == 0) {
        A.lacc[o] += lv[i];
      } else {
        A.lv[o] = lv[i];
        A.lacc[o] = STAGE == 2 ? C.alpha * w[i] : fma(C.alpha, w[i], A.lacc[o]);
      }
    }
  }
}

// Adjoint of the PE-face pass of one stage, face j = blockIdx.x*256 + threadIdx.x:
//   nu = lL . w^e + lR . w^{e-1}  (the delayed flux has adjoint -nu);
//   the synchronous flux the stage kernel assumed is undone (+nu on its partials);
//   the delayed levels receive c_i (-nu) in the adjoint ring;
//   the ring entry of this step and stage becomes trace adjoints, then is cleared.
template <int PDE, int DIR>
__global__ void __launch_bounds__(256) k_adj_faces(const AdjFace F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= F.P) return;
  const int K = F.K, Np = F.Np;
  const int e = j * F.Kpe;
  const int eL = e == 0 ? K - 1 : e - 1;
  double nu = 0.0;
  for (int i = 0; i < Np; ++i) {
    nu = fma(F.lL[i], F.w[(size_t)i * K + e], nu);
    nu = fma(F.lR[i], F.w[(size_t)i * K + eL], nu);
  }
  const int64_t n = F.meta[0] + F.rel;
  const DelayAt d = delay_at(F, j, n);
  const int s = F.stage;
  for (int i = 0; i < d.qe; ++i) {
    const double ci = d.c[i];
    if (ci != 0.0) F.lring[(ring_slot(n - d.k - i, F.R) * kStages + s) * F.P + j] += ci * (-nu);
  }
  double *slot = F.lring + (ring_slot(n, F.R) * kStages + s) * F.P + j;
  const double r = *slot;
  *slot = 0.0;
  double tl = 0.0, tr = 0.0;
  if (PDE == 1) {
    tl = F.v[(size_t)(Np - 1) * K + eL];
    tr = F.v[e];
  }
  double dL, dR;
  value_partials<PDE, DIR>(tl, tr, dL, dR);
  const double g = nu + r;
  F.target[(size_t)(Np - 1) * K + eL] += g * dL;
  F.target[e] += g * dR;
}

__global__ void k_adj_init(const double *__restrict__ u, const double *__restrict__ g, int K,
                           int Np, const double *__restrict__ M, double scale, double *lam) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  double d[kMaxNp];
  for (int i = 0; i < Np; ++i) d[i] = u[(size_t)i * K + e] - g[(size_t)i * K + e];
  for (int i = 0; i < Np; ++i) {
    double r = 0.0;
    for (int jj = 0; jj < Np; ++jj) r = fma(M[i * Np + jj], d[jj], r);
    lam[(size_t)i * K + e] = scale * r;
  }
}

template <int NP, int PDE, int STAGE, bool FACES>
cudaError_t adj_launch(const AdjStage &A, int dir, cudaStream_t s) {
  const int bs = stage_block(A.K);
  const unsigned grid = (unsigned)((A.K + bs - 1) / bs);
  (void)grid;
  // 30 elements per warp (halo lanes)
  const int64_t warps = (A.K + 29) / 30;
  const unsigned g = (unsigned)((warps * 32 + bs - 1) / bs);
  if (PDE == 1) k_adj_stage_halo<NP, 1, STAGE, 0, FACES><<<g, bs, 0, s>>>(A);
  else if (dir > 0) k_adj_stage_halo<NP, 0, STAGE, 1, FACES><<<g, bs, 0, s>>>(A);
  else k_adj_stage_halo<NP, 0, STAGE, -1, FACES><<<g, bs, 0, s>>>(A);
  return cudaGetLastError();
}

template <int NP, int PDE, int STAGE>
cudaError_t adj_np_pde_stage(const AdjStage &A, int dir, cudaStream_t s) {
  return A.faces ? adj_launch<NP, PDE, STAGE, true>(A, dir, s) : adj_launch<NP, PDE, STAGE, false>(A, dir, s);
}

template <int NP, int PDE>
cudaError_t adj_np_pde(const AdjStage &A, int stage, int dir, cudaStream_t s) {
  switch (stage) {
    case 0: return adj_np_pde_stage<NP, PDE, 0>(A, dir, s);
    case 1: return adj_np_pde_stage<NP, PDE, 1>(A, dir, s);
    default: return adj_np_pde_stage<NP, PDE, 2>(A, dir, s);
  }
}

template <int NP>
cudaError_t adj_np(const AdjStage &A, int pde, int stage, int dir, cudaStream_t s) {
  return pde == 1 ? adj_np_pde<NP, 1>(A, stage, dir, s) : adj_np_pde<NP, 0>(A, stage, dir, s);
}

}  // namespace

cudaError_t launch_adj_stage(const AdjStage &A, int pde, int stage, int dir, cudaStream_t s) {
  switch (A.Np) {
    case 2: return adj_np<2>(A, pde, stage, dir, s);
    case 3: return adj_np<3>(A, pde, stage, dir, s);
    case 4: return adj_np<4>(A, pde, stage, dir, s);
    case 5: return adj_np<5>(A, pde, stage, dir, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adj_faces(const AdjFace &F, int pde, int dir, cudaStream_t s) {
  const unsigned grid = (unsigned)((F.P + 255) / 256);
  if (pde == 1) k_adj_faces<1, 0><<<grid, 256, 0, s>>>(F);
  else if (dir > 0) k_adj_faces<0, 1><<<grid, 256, 0, s>>>(F);
  else k_adj_faces<0, -1><<<grid, 256, 0, s>>>(F);
  return cudaGetLastError();
}

cudaError_t launch_adj_init(const double *u, const double *g, int K, int Np, const double *M,
                            double scale, double *lam, cudaStream_t s) {
  k_adj_init<<<(K + 255) / 256, 256, 0, s>>>(u, g, K, Np, M, scale, lam);
  return cudaGetLastError();
}

}  // namespace adg
