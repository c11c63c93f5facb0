// One-dimensional Euler equations (Section 6, Sod's shock tube): FP64 stage and limiter
// kernels for sm_103a.
//
// State U = (rho, m, E), E = rho u^2 / 2 + p / (gamma - 1), gamma = 1.4, three node-major
// planes per component (component c of a field at field + c K Np). One thread per element;
// in the stage kernel a warp takes 30 elements with their two neighbours in its edge lanes.
//   * k_euler_stage: one stage of SSP-RK in Shu and Osher's form,
//       out = alpha u + beta (v + dt L(v)),   dt L(v) = dt [ -QD f + qlL (f_0 - F_L) + qlR (f_p - F_R) ]
//     (the strong form of the nodal DG operator, QD = (2/dx) D, qlL = -(2/dx) M^{-1} e_0,
//     qlR = (2/dx) M^{-1} e_p), with the local Lax-Friedrichs flux at faces; at PE faces the
//     flux is the AT sum (Eq. at-flux-gen) of the Lax-Friedrichs flux of the stored traces of
//     the common delayed level, and the face owner stores the stage input's traces.
//   * k_euler_limit: the TVB-minmod slope limiter on every component (cell average a0 and
//     P_1 coefficient a1; a1' = minmod(2 a1, d+, d-) / 2 unless |a1| <= M dx^2 / 2; an
//     element whose a1 changes becomes a0 + a1' xi). Its stencil ends at PE faces (one-sided
//     there), so it needs no exchange.
#include "adg_device.cuh"

namespace adg {

namespace {

constexpr double kGamma = 1.4;

// Flux f(U) of a state (u = m / rho through one division 1/rho, as below).
__device__ __forceinline__ void euler_flux(const double U[3], double f[3]) {
  const double u = U[1] * (1.0 / U[0]);
  const double p = (kGamma - 1.0) * (U[2] - 0.5 * U[1] * u);
  f[0] = U[1];
  f[1] = fma(U[1], u, p);
  f[2] = (U[2] + p) * u;
}

// Flux f(U) and wave speed |u| + c of a state, with one division (1/rho) and one square root.
__device__ __forceinline__ void euler_flux_speed(const double U[3], double f[3], double &speed) {
  const double r = 1.0 / U[0];
  const double u = U[1] * r;
  const double p = (kGamma - 1.0) * (U[2] - 0.5 * U[1] * u);
  f[0] = U[1];
  f[1] = fma(U[1], u, p);
  f[2] = (U[2] + p) * u;
  speed = fabs(u) + sqrt(kGamma * p * r);
}

// Local Lax-Friedrichs flux from the traces' states, fluxes and wave speeds.
__device__ __forceinline__ void euler_llf_from(const double UL[3], const double UR[3],
                                               const double fl[3], const double fr[3], double sl,
                                               double sr, double F[3]) {
  const double lam = fmax(sl, sr);
#pragma unroll
  for (int c = 0; c < 3; ++c) F[c] = 0.5 * (fl[c] + fr[c]) - 0.5 * lam * (UR[c] - UL[c]);
}

// Local Lax-Friedrichs flux of traces UL = U^-, UR = U^+ (the same arithmetic as the
// interior faces, so a zero delay reproduces the synchronous flux bit for bit).
__device__ __forceinline__ void euler_llf(const double UL[3], const double UR[3], double F[3]) {
  double fl[3], fr[3], sl, sr;
  euler_flux_speed(UL, fl, sl);
  euler_flux_speed(UR, fr, sr);
  euler_llf_from(UL, UR, fl, fr, sl, sr, F);
}

// AT value of the flux at PE face j, step n, stage s from the ring [R][ns][3][P] of (U^-, U^+)
// traces; level n (k = 0) from the current traces (TL, TR), which the owner also stores.
__device__ void euler_pe_flux(const Inst &I, int j, int64_t n, int s, const double TL[3],
                              const double TR[3], bool owner, double F[3]) {
  const int P = I.P, R = I.R;
  const int nm = (int)(n % R);
  const DelayAt d = delay_at(I, j, n);
  auto level = [&](int m, double *out) {   // flux of level n - m from the ring, m >= 1
    int slot = nm - m;
    if (slot < 0) slot += R;
    const double2 *col = I.ring + ((size_t)slot * I.ns + s) * 3 * P + j;
    double a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 t = col[(size_t)c * P];
      a[c] = t.x;
      b[c] = t.y;
    }
    euler_llf(a, b, out);
  };
  double G[3];
  if (d.k == 0) euler_llf(TL, TR, G);
  else level(d.k, G);
#pragma unroll
  for (int c = 0; c < 3; ++c) F[c] = __dmul_rn(d.c[0], G[c]);
  for (int i = 1; i < d.qe; ++i) {
    const double ci = d.c[i];
    if (ci != 0.0) {
      level(d.k + i, G);
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] = __dadd_rn(F[c], __dmul_rn(ci, G[c]));
    }
  }
  if (owner) {
    double2 *col = I.ring + ((size_t)nm * I.ns + s) * 3 * P + j;
#pragma unroll
    for (int c = 0; c < 3; ++c) col[(size_t)c * P] = make_double2(TL[c], TR[c]);
  }
}

// Elements per warp of k_euler_stage: lanes 1 .. 30 own elements, lanes 0 and 31 hold their
// left and right neighbours, so every face flux of the warp is formed by the lanes together.
constexpr int kEulerLanes = 30;

template <int NP, int STAGE, bool FACES>
__global__ void __launch_bounds__(kTile) k_euler_stage(const Inst I, int rel, double *__restrict__ dst) {
  const int K = I.K;
  const size_t nd = (size_t)K * NP;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int eraw = gw * kEulerLanes - 1 + lane;   // -1 .. K + 30
  const int ec = (int)(((long long)eraw + K) % K);
  const bool own = lane >= 1 && lane <= kEulerLanes && eraw < K;
  const int e = own ? eraw : K;   // K: not this lane's to write
  const double *vin = STAGE == 0 ? I.u : (STAGE == 1 ? I.v1 : I.v2);
  const StageConsts &C = I.sc[STAGE];
  double V[3][NP];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double *q = vin + c * nd + ec;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      V[c][i] = __ldg(q);
      q += K;
    }
  }
  const unsigned full = 0xffffffffu;
  // node fluxes, and the wave speeds of the two end nodes
  double f[3][NP], s0 = 0.0, sp = 0.0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const double Ui[3] = {V[0][i], V[1][i], V[2][i]};
    double fi[3];
    if (i == 0 || i == NP - 1) {
      double si;
      euler_flux_speed(Ui, fi, si);
      if (i == 0) s0 = si;
      if (i == NP - 1) sp = si;
    } else {
      euler_flux(Ui, fi);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c][i] = fi[c];
  }
  // left face: U^- with its flux and speed from the left neighbour's last node (the lane
  // below), U^+ this element's first node; the right face's flux from the lane above
  double VLm[3], VRp[3], V0[3], Vp[3], fLm[3], f0[3], fp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V0[c] = V[c][0];
    Vp[c] = V[c][NP - 1];
    f0[c] = f[c][0];
    fp[c] = f[c][NP - 1];
    VLm[c] = __shfl_up_sync(full, Vp[c], 1);
    fLm[c] = __shfl_up_sync(full, fp[c], 1);
    VRp[c] = __shfl_down_sync(full, V0[c], 1);
  }
  const double sLm = __shfl_up_sync(full, sp, 1);
  double FL[3], FR[3];
  euler_llf_from(VLm, V0, fLm, f0, sLm, s0, FL);
#pragma unroll
  for (int c = 0; c < 3; ++c) FR[c] = __shfl_down_sync(full, FL[c], 1);
  if (FACES && e < K) {
    const int64_t n = I.meta[0] + rel;
    const int Kpe = I.Kpe;
    const int jq = e / Kpe;
    const int r = e - jq * Kpe;
    if (r == 0) euler_pe_flux(I, jq, n, STAGE, VLm, V0, true, FL);
    if (r == Kpe - 1) euler_pe_flux(I, jq + 1 == I.P ? 0 : jq + 1, n, STAGE, Vp, VRp, false, FR);
  }
  if (e >= K) return;
  const double dt = I.dt;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double jl = __dsub_rn(f[c][0], FL[c]);
    const double jr = __dsub_rn(f[c][NP - 1], FR[c]);
    double u[NP];
    if (STAGE > 0) {
      const double *q = I.u + c * nd + e;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        u[i] = *q;
        q += K;
      }
    }
    double *o = dst + c * nd + e;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double r = -I.QD[i * NP] * f[c][0];
#pragma unroll
      for (int j = 1; j < NP; ++j) r = fma(-I.QD[i * NP + j], f[c][j], r);
      r = fma(I.qlL[i], jl, r);
      r = fma(I.qlR[i], jr, r);
      double out = C.beta * fma(dt, r, V[c][i]);
      if (STAGE > 0) out = fma(C.alpha, u[i], out);
      *o = out;
      o += K;
    }
  }
}

// Sign of a non-NaN double from its bit pattern (-0 and +0 give 0).
__device__ __forceinline__ int bit_sign(long long b) { return b > 0 ? 1 : ((b << 1) != 0 ? -1 : 0); }

// minmod of 2 a1 and the used differences, halved (0 where the signs disagree). Signs,
// magnitudes and minima are taken on the IEEE bit patterns (integer pipe): for non-negative
// doubles the patterns order like the values.
__device__ __forceinline__ double limited_slope(double a1, double dp, double dm, bool use_p,
                                                bool use_m) {
  const long long mask = 0x7fffffffffffffffLL;
  const long long bt = __double_as_longlong(2.0 * a1);
  const int st = bit_sign(bt);
  long long mag = bt & mask;
  bool ok = st != 0;
  if (use_p) {
    const long long b = __double_as_longlong(dp);
    ok = ok && bit_sign(b) == st;
    const long long m = b & mask;
    mag = m < mag ? m : mag;
  }
  if (use_m) {
    const long long b = __double_as_longlong(dm);
    ok = ok && bit_sign(b) == st;
    const long long m = b & mask;
    mag = m < mag ? m : mag;
  }
  const double r = 0.5 * __longlong_as_double(mag);
  return ok ? (st > 0 ? r : -r) : 0.0;
}

template <int NP>
__device__ __forceinline__ double cell_average(const Inst &I, const double *v) {
  double a = I.avg_w[0] * v[0];
#pragma unroll
  for (int j = 1; j < NP; ++j) a = fma(I.avg_w[j], v[j], a);
  return a;
}

template <int NP, bool PES>
__global__ void __launch_bounds__(kTile) k_euler_limit(const Inst I, const double *__restrict__ src,
                                                       double *__restrict__ dst) {
  const int K = I.K;
  const size_t nd = (size_t)K * NP;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int ec = e < K ? e : K - 1;
  const bool edge = (lane == 31) || (ec + 1 >= K);
  const int fR = ec + 1 >= K ? 0 : ec + 1;
  const int fL = ec == 0 ? K - 1 : ec - 1;
  const bool use_m = !(PES && ec % I.Kpe == 0);
  const bool use_p = !(PES && (ec + 1) % I.Kpe == 0);
  const double keep = I.tvb_m * (I.dx * I.dx) * 0.5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double v[NP], w[NP];
    const double *q = src + c * nd + ec;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      v[i] = __ldg(q);
      q += K;
    }
    const double a0 = cell_average<NP>(I, v);
    double a1 = I.p1_w[0] * v[0];
#pragma unroll
    for (int j = 1; j < NP; ++j) a1 = fma(I.p1_w[j], v[j], a1);
    double aL = __shfl_up_sync(0xffffffffu, a0, 1);
    double aR = __shfl_down_sync(0xffffffffu, a0, 1);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NP; ++i) w[i] = __ldg(src + c * nd + (size_t)i * K + fL);
      aL = cell_average<NP>(I, w);
    }
    if (edge) {
#pragma unroll
      for (int i = 0; i < NP; ++i) w[i] = __ldg(src + c * nd + (size_t)i * K + fR);
      aR = cell_average<NP>(I, w);
    }
    if (e >= K) continue;
    double a1n = limited_slope(a1, aR - a0, a0 - aL, use_p, use_m);
    if ((__double_as_longlong(a1) & 0x7fffffffffffffffLL) <= __double_as_longlong(keep)) a1n = a1;
    double *o = dst + c * nd + e;
    const bool change = a1n != a1;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      *o = change ? fma(a1n, I.xi[i], a0) : v[i];
      o += K;
    }
  }
}

template <int NP, int STAGE>
cudaError_t euler_stage_np(const Inst &I, int rel, double *dst, cudaStream_t s) {
  const int bs = stage_block(I.K);
  const long long threads = (long long)((I.K + kEulerLanes - 1) / kEulerLanes) * 32;
  const unsigned grid = (unsigned)((threads + bs - 1) / bs);
  if (I.async) k_euler_stage<NP, STAGE, true><<<grid, bs, 0, s>>>(I, rel, dst);
  else k_euler_stage<NP, STAGE, false><<<grid, bs, 0, s>>>(I, rel, dst);
  return cudaGetLastError();
}

template <int NP>
cudaError_t euler_stage(const Inst &I, int stage, int rel, double *dst, cudaStream_t s) {
  switch (stage) {
    case 0: return euler_stage_np<NP, 0>(I, rel, dst, s);
    case 1: return euler_stage_np<NP, 1>(I, rel, dst, s);
    default: return euler_stage_np<NP, 2>(I, rel, dst, s);
  }
}

template <int NP>
cudaError_t euler_limit(const Inst &I, const double *src, double *dst, cudaStream_t s) {
  const int bs = stage_block(I.K);
  const unsigned grid = (unsigned)((I.K + bs - 1) / bs);
  if (I.P > 1) k_euler_limit<NP, true><<<grid, bs, 0, s>>>(I, src, dst);
  else k_euler_limit<NP, false><<<grid, bs, 0, s>>>(I, src, dst);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_euler_stage(const Inst &I, int stage, int rel, double *dst, cudaStream_t s) {
  if (stage < 0 || stage >= I.ns || stage > 2) return cudaErrorInvalidValue;
  switch (I.Np) {
    case 2: return euler_stage<2>(I, stage, rel, dst, s);
    case 3: return euler_stage<3>(I, stage, rel, dst, s);
    case 4: return euler_stage<4>(I, stage, rel, dst, s);
    case 5: return euler_stage<5>(I, stage, rel, dst, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_euler_limit(const Inst &I, const double *src, double *dst, cudaStream_t s) {
  if (src == dst) return cudaErrorInvalidValue;
  switch (I.Np) {
    case 2: return euler_limit<2>(I, src, dst, s);
    case 3: return euler_limit<3>(I, src, dst, s);
    case 4: return euler_limit<4>(I, src, dst, s);
    case 5: return euler_limit<5>(I, src, dst, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace adg
