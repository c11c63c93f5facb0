// Device helpers shared by the forward (adg_kernels.cu) and adjoint (adg_adjoint.cu) kernels.
#pragma once

#include "adg_internal.h"

namespace adg {
namespace {

// Waits until the kernel this one was launched as a programmatic dependent of (launch_maybe_pdl)
// has completed and its writes are visible; returns at once for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel of the chain (launched with the attribute) start launching its blocks
// once every block of this one has passed this point. Called after pdl_wait, so the kernel
// before this one has completed when the next one starts.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Physical flux f(u): a u (advection) or u^2/2 (Burgers). Explicit round-to-nearest
// intrinsics keep every evaluation of a face flux bit-identical wherever it is computed.
template <int PDE>
__device__ __forceinline__ double phys_flux(double a, double u) {
  if (PDE == 0) return __dmul_rn(a, u);
  return __dmul_rn(0.5, __dmul_rn(u, u));
}

// Numerical flux (Section 6.1): upwind a u^- (a >= 0) or a u^+ (a < 0); local
// Lax-Friedrichs 1/2 (f(u^-) + f(u^+)) - 1/2 max(|u^-|, |u^+|) (u^+ - u^-) for Burgers.
// Comparisons and max/abs on FP64 values done on their IEEE bit patterns with integer
// instructions (exact for finite values; on this part FP64 compares and min/max occupy the
// FP64 pipe). |x| as bits, max(|a|, |b|), and "x >= 0" (true for +0 and -0).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ double abs_max(double a, double b) {
  const unsigned long long ia = abs_bits(a), ib = abs_bits(b);
  return __longlong_as_double((long long)(ia >= ib ? ia : ib));
}
__device__ __forceinline__ bool nonneg(double x) {
  return __double_as_longlong(x) >= 0 || abs_bits(x) == 0;
}

template <int PDE>
__device__ __forceinline__ double num_flux(double a, double uL, double uR) {
  if (PDE == 0) return __dmul_rn(a, a >= 0.0 ? uL : uR);
  const double lam = abs_max(uL, uR);
  const double avg = __dmul_rn(0.5, __dadd_rn(phys_flux<1>(a, uL), phys_flux<1>(a, uR)));
  return __dsub_rn(avg, __dmul_rn(__dmul_rn(0.5, lam), __dsub_rn(uR, uL)));
}

__device__ __forceinline__ int64_t ring_slot(int64_t level, int R) { return level % R; }

// Loads the Np nodal values of element e from a node-major field by pointer steps of K
// (no per-node 64-bit index products).
template <int NP, class T>
__device__ __forceinline__ void load_elem(const T *__restrict__ f, int K, int e, T *u) {
  const T *q = f + e;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    u[i] = __ldg(q);
    q += K;
  }
}

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

// Ring levels prefetched by pe_value (rings with more levels fall back to dependent loads).
constexpr int kPrefetchR = 12;

template <int PDE, int DIR, class I>
__device__ __forceinline__ double pe_value(const I &inst, int j, int64_t n, int s, double tl,
                                        double tr, bool owner) {
  const int P = inst.P;
  const int R = inst.R;
  // Every slot of this face and stage is loaded up front, in parallel with the delay-table
  // lookup that decides which of them the sum uses.
  double2 *col = inst.ring + (size_t)s * P + j;
  const bool pre = R <= kPrefetchR;
  double2 T[kPrefetchR];
  if (pre) {
    const double2 *q = col;
#pragma unroll
    for (int r = 0; r < kPrefetchR; ++r) {
      if (r < R) T[r] = *q;
      q += (size_t)inst.ns * P;
    }
  }
  const int nm = (int)(n % R);
  auto fetch = [&](int m) -> double2 {   // traces of level n - m, 1 <= m < R
    int slot = nm - m;
    if (slot < 0) slot += R;
    if (pre) {
      double2 x = T[0];
#pragma unroll
      for (int r = 1; r < kPrefetchR; ++r)
        if (r == slot) x = T[r];
      return x;
    }
    return col[(size_t)slot * inst.ns * P];
  };
  const DelayAt d = delay_at(inst, j, n);
  const int k = d.k;
  const int qe = d.qe;
  const double *c = d.c;
  double V;
  if (k == 0) {
    V = __dmul_rn(c[0], face_value<PDE, DIR>(inst, tl, tr));
  } else {
    const double2 t0 = fetch(k);
    V = __dmul_rn(c[0], face_value<PDE, DIR>(inst, t0.x, t0.y));
  }
  for (int i = 1; i < qe; ++i) {
    const double ci = c[i];
    if (ci != 0.0) {
      const double2 ti = fetch(k + i);
      V = __dadd_rn(V, __dmul_rn(ci, face_value<PDE, DIR>(inst, ti.x, ti.y)));
    }
  }
  if (owner) col[(size_t)nm * inst.ns * P] = make_double2(tl, tr);
  return V;
}

// The AT value of q^+ at PE face j for step n, stage s (viscous Burgers, alternating flux
// qhat = q^+): the same sum as pe_value over the stored q^+ traces of levels n-k-i; level n
// (k = 0) uses the current q^+ (qcur). The ring write happens in the q pass (k_ldg_q).
template <class I>
__device__ __forceinline__ double pe_value_q(const I &inst, int j, int64_t n, int s, double qcur) {
  const int P = inst.P;
  const int R = inst.R;
  const double *col = inst.ringq + (size_t)s * P + j;
  const int nm = (int)(n % R);
  const DelayAt d = delay_at(inst, j, n);
  const int k = d.k;
  auto fetch = [&](int m) -> double {   // q^+ of level n - m, 1 <= m < R
    int slot = nm - m;
    if (slot < 0) slot += R;
    return col[(size_t)slot * inst.ns * P];
  };
  double V = __dmul_rn(d.c[0], k == 0 ? qcur : fetch(k));
  for (int i = 1; i < d.qe; ++i) {
    const double ci = d.c[i];
    if (ci != 0.0) V = __dadd_rn(V, __dmul_rn(ci, fetch(k + i)));
  }
  return V;
}

}  // namespace
}  // namespace adg
