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

template <int NP, int PDE, int STAGE, int DIR, bool FACES>
__global__ void __launch_bounds__(kTile) k_adj_stage(const AdjStage A) {
  const int K = A.K;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int ec = e < K ? e : K - 1;
  const bool edge = (lane == 31) || (ec + 1 >= K);
  const int eR = ec + 1 >= K ? 0 : ec + 1;
  const int eL = ec == 0 ? K - 1 : ec - 1;
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

  if (PDE == 0) {
    if (DIR > 0) {
      // jL^e = v_0^e - v_p^{e-1}: own node 0 gets sL^e, node p gets -sL^{e+1}.
      lv[0] += sL;
      double sLn = __shfl_down_sync(full, sL, 1);
      if (edge) {
        sLn = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) sLn = fma(C.lL[i], __ldg(A.w + (size_t)i * K + eR), sLn);
      }
      lv[NP - 1] -= sLn;
    } else {
      // jR^e = v_p^e - v_0^{e+1}: own node p gets sR^e, node 0 gets -sR^{e-1}.
      lv[NP - 1] += sR;
      double sRp = __shfl_up_sync(full, sR, 1);
      if (lane == 0) {
        sRp = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) sRp = fma(C.lR[i], __ldg(A.w + (size_t)i * K + eL), sRp);
      }
      lv[0] -= sRp;
    }
  } else {
    lv[0] = fma(v[0], sL, lv[0]);
    lv[NP - 1] = fma(v[NP - 1], sR, lv[NP - 1]);
    // Left face of e: adjoint mu = -sL^e - sR^{e-1}, traces (v_p^{e-1}, v_0^e).
    double sRp = __shfl_up_sync(full, sR, 1);
    double vLm = __shfl_up_sync(full, v[NP - 1], 1);
    if (lane == 0) {
      sRp = 0.0;
#pragma unroll
      for (int i = 0; i < NP; ++i) sRp = fma(C.lR[i], __ldg(A.w + (size_t)i * K + eL), sRp);
      vLm = __ldg(A.v + (size_t)(NP - 1) * K + eL);
    }
    const double muL = -sL - sRp;
    double dL, dR;
    llf_partials(vLm, v[0], dL, dR);
    lv[0] = fma(muL, dR, lv[0]);
    double fromRight = __shfl_down_sync(full, muL * dL, 1);
    if (edge) {
      double sLn = 0.0;
#pragma unroll
      for (int i = 0; i < NP; ++i) sLn = fma(C.lL[i], __ldg(A.w + (size_t)i * K + eR), sLn);
      const double vRp = __ldg(A.v + eR);
      double dL2, dR2;
      llf_partials(v[NP - 1], vRp, dL2, dR2);
      fromRight = (-sLn - sR) * dL2;
    }
    lv[NP - 1] += fromRight;
  }

  if (FACES) {
    // PE faces among this block's faces (K/P >= 8). Element e is right of PE face j (peL)
    // or left of PE face jr (peR); both elements form the face's adjoint g themselves:
    //   nu = sL^e + sR^{e-1}, g = nu + r - [k == 0] nu, r = ring entry of (n, s, j),
    // and add g times the value's partial derivative to their trace node. The owner (right
    // element) posts c_i (-nu) to the delayed levels (never to level n) and clears the ring
    // entry the previous adjoint kernel read (it is read no more).
    __shared__ int s_first, s_jfirst;
    const int e0 = blockIdx.x * blockDim.x;
    if (threadIdx.x == 0) {
      const int jf = (e0 + A.Kpe - 1) / A.Kpe;
      s_jfirst = jf;
      s_first = jf * A.Kpe;
    }
    __syncthreads();
    int jL = -1, jR = -1;
    {
      int f = s_first, jf = s_jfirst;
      for (; f <= e0 + (int)blockDim.x && f < K; f += A.Kpe, ++jf) {
        if (f == ec) jL = jf;
        if (f == ec + 1) jR = jf;
      }
      if (ec + 1 == K) jR = 0;
    }
    if ((jL >= 0 || jR >= 0) && e < K) {
      const int64_t n = A.meta[0] + A.rel;
      const int nm = (int)(n % A.R);
      auto slot_of = [&](int m) {   // ring slot of level n - m
        int sl = nm - m;
        if (sl < 0) sl += A.R;
        return sl;
      };
      // neighbour adjoint scalars and traces (direct loads: this branch is rare)
      double sRm = 0.0, sLp = 0.0;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        sRm = fma(C.lR[i], __ldg(A.w + (size_t)i * K + eL), sRm);
        sLp = fma(C.lL[i], __ldg(A.w + (size_t)i * K + eR), sLp);
      }
      if (jL >= 0) {
        const double nu = sL + sRm;
        const DelayAt d = delay_at(A, jL, n);
        const double r = A.lring[((size_t)nm * kStages + STAGE) * A.P + jL];
        const double g = d.k == 0 ? r : nu + r;
        double tl = 0.0, tr = 0.0;
        if (PDE == 1) {
          tl = __ldg(A.v + (size_t)(NP - 1) * K + eL);
          tr = v[0];
        }
        double dL, dR;
        value_partials<PDE, DIR>(tl, tr, dL, dR);
        lv[0] = fma(g, dR, lv[0]);
        for (int i = 0; i < d.qe; ++i) {
          const double ci = d.c[i];
          if (ci != 0.0 && d.k + i >= 1)
            A.lring[((size_t)slot_of(d.k + i) * kStages + STAGE) * A.P + jL] += ci * (-nu);
        }
        // clear the entry the previous adjoint kernel read: (n, s+1), or (n+1, 0) for s = 2
        const int pst = STAGE == 2 ? 0 : STAGE + 1;
        const int psl = STAGE == 2 ? (nm + 1 == A.R ? 0 : nm + 1) : nm;
        A.lring[((size_t)psl * kStages + pst) * A.P + jL] = 0.0;
      }
      if (jR >= 0) {
        const double nu = sLp + sR;
        const DelayAt d = delay_at(A, jR, n);
        const double r = A.lring[((size_t)nm * kStages + STAGE) * A.P + jR];
        const double g = d.k == 0 ? r : nu + r;
        double tl = 0.0, tr = 0.0;
        if (PDE == 1) {
          tl = v[NP - 1];
          tr = __ldg(A.v + eR);
        }
        double dL, dR;
        value_partials<PDE, DIR>(tl, tr, dL, dR);
        lv[NP - 1] = fma(g, dL, lv[NP - 1]);
      }
    }
  }

  if (e < K) {
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
  if (PDE == 1) k_adj_stage<NP, 1, STAGE, 0, FACES><<<grid, bs, 0, s>>>(A);
  else if (dir > 0) k_adj_stage<NP, 0, STAGE, 1, FACES><<<grid, bs, 0, s>>>(A);
  else k_adj_stage<NP, 0, STAGE, -1, FACES><<<grid, bs, 0, s>>>(A);
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
