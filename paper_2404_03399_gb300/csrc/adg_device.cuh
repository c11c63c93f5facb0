// Device helpers shared by the forward (adg_kernels.cu) and adjoint (adg_adjoint.cu) kernels.
#pragma once

#include "adg_internal.h"

namespace adg {
namespace {

// Physical flux f(u): a u (advection) or u^2/2 (Burgers). Explicit round-to-nearest
// intrinsics keep every evaluation of a face flux bit-identical wherever it is computed.
template <int PDE>
__device__ __forceinline__ double phys_flux(double a, double u) {
  if (PDE == 0) return __dmul_rn(a, u);
  return __dmul_rn(0.5, __dmul_rn(u, u));
}

// Numerical flux (Section 6.1): upwind a u^- (a >= 0) or a u^+ (a < 0); local
// Lax-Friedrichs 1/2 (f(u^-) + f(u^+)) - 1/2 max(|u^-|, |u^+|) (u^+ - u^-) for Burgers.
template <int PDE>
__device__ __forceinline__ double num_flux(double a, double uL, double uR) {
  if (PDE == 0) return __dmul_rn(a, a >= 0.0 ? uL : uR);
  const double lam = fmax(fabs(uL), fabs(uR));
  const double avg = __dmul_rn(0.5, __dadd_rn(phys_flux<1>(a, uL), phys_flux<1>(a, uR)));
  return __dsub_rn(avg, __dmul_rn(__dmul_rn(0.5, lam), __dsub_rn(uR, uL)));
}

__device__ __forceinline__ int64_t ring_slot(int64_t level, int R) { return level % R; }

__device__ __forceinline__ bool nonzero(double x) {
  return (__double_as_longlong(x) << 1) != 0;   // integer test: not +0 or -0
}

// Delay of PE face j at step n, clamped to k <= n, the order in use q' = min(q, n-k+1) and
// the AT coefficients c_i(k; q') (row of the [L][q][q] table).
struct DelayAt {
  int k;
  int qe;
  const double *c;
};

template <class I>
__device__ __forceinline__ DelayAt delay_at(const I &inst, int j, int64_t n) {
  const int q = inst.q;
  const int64_t row = n - inst.meta[1];
  int64_t k = inst.table[row * inst.P + j];
  if (k > n) k = n;
  const int64_t qe = n - k + 1 < q ? n - k + 1 : q;
  DelayAt d;
  d.k = (int)k;
  d.qe = (int)qe;
  d.c = inst.coef + ((size_t)k * q + (qe - 1)) * q;
  return d;
}

// Value at PE face j for step n, stage s (Eqs. asyncEulerDGconserved and at-flux-gen):
// delay k = min(D[n][j], n), order q' = min(q, n-k+1),
//   V = sum_{i<q'} c_i(k; q') v(T_{n-k-i, s, j}),
// where T are the traces (u^-, u^+) of the stage-s input of step n-k-i and v is the
// numerical flux (Burgers) or, for linear advection, the upwind trace (the flux is a V,
// the same AT flux with the factor a taken out of the sum). Level n (k = 0) uses the
// current traces (tl, tr); the owner (the element right of the face) stores T_{n,s,j}.
template <int PDE, int DIR, class I>
__device__ __forceinline__ double face_value(const I &inst, double uL, double uR) {
  if (PDE == 0) return DIR > 0 ? uL : uR;
  return num_flux<1>(0.0, uL, uR);
}

template <int PDE, int DIR, class I>
__device__ __forceinline__ double pe_value(const I &inst, int j, int64_t n, int s, double tl,
                                        double tr, bool owner) {
  const int P = inst.P;
  const int R = inst.R;
  const DelayAt d = delay_at(inst, j, n);
  const int64_t k = d.k;
  const int qe = d.qe;
  const double *c = d.c;
  double V;
  if (k == 0) {
    V = __dmul_rn(c[0], face_value<PDE, DIR>(inst, tl, tr));
  } else {
    const double2 T = inst.ring[(ring_slot(n - k, R) * kStages + s) * P + j];
    V = __dmul_rn(c[0], face_value<PDE, DIR>(inst, T.x, T.y));
  }
  for (int i = 1; i < qe; ++i) {
    const double ci = c[i];
    if (ci != 0.0) {
      const double2 T = inst.ring[(ring_slot(n - k - i, R) * kStages + s) * P + j];
      V = __dadd_rn(V, __dmul_rn(ci, face_value<PDE, DIR>(inst, T.x, T.y)));
    }
  }
  if (owner) inst.ring[(ring_slot(n, R) * kStages + s) * P + j] = make_double2(tl, tr);
  return V;
}

}  // namespace
}  // namespace adg
