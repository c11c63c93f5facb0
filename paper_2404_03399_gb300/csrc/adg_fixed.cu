// Composed step of upwind advection (a > 0; SSP-RK3, or a low-storage scheme of up to five
// stages) in fixed-point integer arithmetic: the StepConsts stencil (adg_internal.h) evaluated
// with 32 x 32 -> 64-bit integer multiply-adds on two-limb values (adg_fixed.cuh). The field
// stays int64 from step to step; only a run's first step reads FP64. A single instance keeps
// the coordinates of each element in the block basis of the element operator (Inst.basis,
// FMT bit kFmtBasis): G is then block diagonal with 2 x 2 blocks whose first rows are shifts
// and adds, and the right trace is the sum of the even coordinates.
#include <type_traits>

#include "adg_device.cuh"
#include "adg_fixed.cuh"

namespace adg {
namespace {

// Per element slot (S slots before the block's tile for the elements e0-S .. e0-1): the right
// trace p and the unrounded own parts (a, b) of its channel scalars r_s . u, s = 1 .. S-1.
template <int EPT, int S>
struct FixedShared {
  long long p[EPT * kTile + S];
  long long sa[S - 1][EPT * kTile + S], sb[S - 1][EPT * kTile + S];
  FxScale sc;
};

// Working-scale value of node j of an element (FP64 input, or int64 input already brought
// to the working scale).
template <bool FIN>
__device__ __forceinline__ long long fx_in(double x, long long X, const FxScale &sc) {
  if (FIN) return X;
  return fx_from_double(x, sc.sigma + 1079);
}

// p = the element's right trace, own[s-1] = the own parts r_s . u of its channel scalars
// (unrounded sums, s = 1 .. S-1), and the limbs of its values for the output rows. BLK: the
// values are block-basis coordinates w (an FP64 input is transformed, w = Tbi u, in FP64
// before its conversion) and the right trace is the exact sum w_0 + w_2 (the first
// coordinate of each block).
template <int NP, bool FIN, int S, bool BLK>
__device__ __forceinline__ void fx_own(const StepFixed &F, const double *Tbi, const double *ud,
                                       const long long *uq, const FxScale &sc, long long &p,
                                       FxAcc *own, int *xh, int *xl) {
  double wd[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if (BLK && !FIN) {
      double a = Tbi[i * NP] * ud[0];
#pragma unroll
      for (int k = 1; k < NP; ++k) a = fma(Tbi[i * NP + k], ud[k], a);
      wd[i] = a;
    } else {
      wd[i] = FIN ? 0.0 : ud[i];
    }
  }
  p = 0;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const long long X = fx_in<FIN>(wd[j], FIN ? uq[j] : 0ll, sc);
    fx_split(X, xh[j], xl[j]);
#pragma unroll
    for (int s = 1; s < S; ++s) fx_mac(own[s - 1], F.r[s][j], xh[j], xl[j]);
    if (BLK ? (j == 0 || j == 2) : (j == NP - 1)) p += X;
  }
}

template <int EPT, int S>
__device__ __forceinline__ void fx_publish(FixedShared<EPT, S> &sh, int sl, long long p,
                                           const FxAcc *own) {
  sh.p[sl] = p;
#pragma unroll
  for (int s = 0; s < S - 1; ++s) {
    sh.sa[s][sl] = own[s].a;
    sh.sb[s][sl] = own[s].b;
  }
}

// The channel scalars of element e-1 (P[s], split into limbs) from the published slots
// b .. b+S-1 of elements e-S .. e-1: element e-S+w forms Y_1 .. Y_w from its own parts and the
// scalars of the element before it, Y_s = r_s . u + sum_{t<s} k_st Y_t (each rounded once; every
// thread that needs one of them forms it from the same values, so all agree bit for bit).
template <int EPT, int S>
__device__ __forceinline__ void fx_left_channels(const StepFixed &F, const FixedShared<EPT, S> &sh,
                                                 int b, int (*P)[2]) {
  long long Yp[S];
  Yp[0] = sh.p[b];
#pragma unroll
  for (int w = 1; w < S; ++w) {
    int ph[S], pl[S];
#pragma unroll
    for (int t = 0; t < w; ++t) fx_split(Yp[t], ph[t], pl[t]);
    long long Y[S];
    Y[0] = sh.p[b + w];
#pragma unroll
    for (int s = 1; s <= w; ++s) {
      FxAcc c{sh.sa[s - 1][b + w], sh.sb[s - 1][b + w]};
#pragma unroll
      for (int t = 0; t < s; ++t) fx_mac(c, F.k[s][t], ph[t], pl[t]);
      Y[s] = fx_round(c);
    }
#pragma unroll
    for (int s = 0; s <= w; ++s) Yp[s] = Y[s];
  }
#pragma unroll
  for (int s = 0; s < S; ++s) fx_split(Yp[s], P[s][0], P[s][1]);
}

// u'^e = G u^e + sum_s h_s P_s for output row i. BLK: G's entries of row i's block only
// (blocks {0, 1} and {2, .., NP-1}); the first row of a 2 x 2 block (and of the 3 x 3 block
// where it was sheared) is (1, 2^-k), whose
// products, X_i and xh_{i+1} 2^(29-k) + xl_{i+1} 2^(29-k) 2^-29, are shifts (the same sums
// as the multiply-adds with the limbs {2^29, 0} and {2^(29-k), 0}).
template <int NP, int S, bool BLK>
__device__ __forceinline__ long long fx_row(const StepFixed &F, int i, const int *xh, const int *xl,
                                            const int (*P)[2]) {
  FxAcc acc;
  if (BLK) {
    const int j0 = i < 2 ? 0 : 2, j1 = i < 2 ? 2 : NP;   // the block [j0, j1)
    // a pair's first row, or the triple's (NP = 5) when its basis was sheared (gs[1] != 0):
    // (1, 2^-k) or (1, 2^-k, 0)
    if (i == j0 && (j1 - j0 == 2 || (j1 - j0 == 3 && F.gs[1] != 0))) {
      // 64-bit values from 32-bit funnel shifts of the limbs (sign words s0, s1)
      const unsigned sh = (unsigned)F.gs[i >> 1];
      const unsigned h0 = (unsigned)xh[i], s0 = (unsigned)(xh[i] >> 31);
      const unsigned h1 = (unsigned)xh[i + 1], s1 = (unsigned)(xh[i + 1] >> 31);
      const unsigned l1 = (unsigned)xl[i + 1];
      const long long x0 = fx_join(__funnelshift_l(0u, h0, 29) | (unsigned)xl[i],
                                   __funnelshift_l(h0, s0, 29));   // X_i
      const long long t1 = fx_join(__funnelshift_l(0u, h1, sh), __funnelshift_l(h1, s1, sh));
      const long long b1 = fx_join(__funnelshift_l(0u, l1, sh), __funnelshift_l(l1, 0u, sh));
      acc.a += x0 + t1;
      acc.b += b1;
    } else {
#pragma unroll
      for (int j = j0; j < j1; ++j) fx_mac(acc, F.G[i * NP + j], xh[j], xl[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NP; ++j) fx_mac(acc, F.G[i * NP + j], xh[j], xl[j]);
  }
#pragma unroll
  for (int s = 0; s < S; ++s) fx_mac(acc, F.h[s][i], P[s][0], P[s][1]);
  return fx_round(acc);
}

// The block's scale read (thread 0, one barrier; every warp reading it itself measured 4%
// slower) and the slot bookkeeping of the block holding element 0: it clears the slot of
// u^{n+2} and, for an int64 output, sets u^{n+1}'s scale and NaN mark.
template <bool FIN, bool FOUT, bool BLK, class I, class SH>
__device__ __forceinline__ FxScale fx_block_scale(const I &inst, int e0, int rel, SH &sh) {
  if (threadIdx.x == 0) {
    int hb = 0, he = 0;
    if constexpr (BLK) {
      hb = inst.fxh;
      he = inst.fxe;
    }
    const FxScale sc = fx_scale(inst.fx, inst.meta[0] + rel, FIN, hb, he);
    sh.sc = sc;
    if (e0 == 0) {
      FxSlot &c = inst.fx[fx_clear(sc.slot)];
      c.mag = 0;
      c.E = 0;
      c.sigma = 0;
      if (FOUT) {
        inst.fx[fx_next(sc.slot)].sigma = sc.sigma;
        if (sc.bad) inst.fx[fx_next(sc.slot)].E = 2047;
      }
    }
  }
  __syncthreads();
  return sh.sc;
}

// The scale of u^{n+1}: OR of |y| (int64 output) or largest exponent (FP64 output), one slot
// update per warp.
template <bool FOUT, class I>
__device__ __forceinline__ void fx_block_next(const I &inst, const FxScale &sc,
                                              unsigned long long mag, int emax) {
  FxSlot &nx = inst.fx[fx_next(sc.slot)];
  if (FOUT) {
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)mag);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(mag >> 32));
    if ((threadIdx.x & 31) == 0) or_slot(&nx.mag, ((unsigned long long)hi << 32) | lo);
  } else {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((threadIdx.x & 31) == 0) raise_slot(&nx.E, emax);
  }
}

// One thread per element (EPT elements per thread, e = e0 + t + h kTile): the right trace and
// the unrounded own parts of the channel scalars go to shared memory (one barrier); each
// thread then forms its left neighbour's channel scalars from those of elements e-S .. e-1
// and u'^e = G u^e + sum_s h_s P_s. The first S threads publish the S elements before the
// block with the same arithmetic (the working scale is one per field, so every element
// converts the same way).
template <int NP, int EPT, int FMT, int S, class I>
__device__ __forceinline__ void fixed_body(const I &inst, const void *__restrict__ uin_,
                                           void *__restrict__ uout_, int e0, int rel,
                                           FixedShared<EPT, S> &sh) {
  constexpr bool FIN = (FMT & kFmtInFixed) != 0;
  constexpr bool FOUT = (FMT & kFmtOutFixed) != 0;
  constexpr bool BLK = (FMT & kFmtBasis) != 0;
  static_assert(FOUT || !BLK, "a block-basis state is written as int64");
  const double *uin_d = static_cast<const double *>(uin_);
  const long long *uin_q = static_cast<const long long *>(uin_);
  const int K = inst.K;
  const int t = threadIdx.x;
  const StepFixed &F = inst.sf;
  const double *Tbi = nullptr;
  if constexpr (BLK) Tbi = inst.Tbi;

  // loads first: they do not depend on the scale
  double hd[NP];
  long long hq[NP];
  if (t < S) {
    int m = e0 - S + t;
    if (m < 0) m += K;   // K >= 8 on this path
    if (FIN) load_elem<NP>(uin_q, K, m, hq);
    else load_elem<NP>(uin_d, K, m, hd);
  }
  double ud[EPT][NP];
  long long uq[EPT][NP];
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int e = e0 + t + h * kTile;
    if (FIN) load_elem<NP>(uin_q, K, e < K ? e : K - 1, uq[h]);
    else load_elem<NP>(uin_d, K, e < K ? e : K - 1, ud[h]);
  }
  const FxScale sc = fx_block_scale<FIN, FOUT, BLK>(inst, e0, rel, sh);
  if (FIN && sc.shift != 0) {   // block-uniform: the field grew past 2^57 or shrank
#pragma unroll
    for (int j = 0; j < NP; ++j) hq[j] = fx_rescale(hq[j], sc.shift);
#pragma unroll
    for (int h = 0; h < EPT; ++h)
#pragma unroll
      for (int j = 0; j < NP; ++j) uq[h][j] = fx_rescale(uq[h][j], sc.shift);
  }
  // publish p and the unrounded own parts of every element's channel scalars (the halo's too)
  if (t < S) {
    int xh[NP], xl[NP];
    long long p;
    FxAcc own[S - 1];
    fx_own<NP, FIN, S, BLK>(F, Tbi, hd, hq, sc, p, own, xh, xl);
    fx_publish(sh, t, p, own);
  }
  int xh[EPT][NP], xl[EPT][NP];
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    long long p;
    FxAcc own[S - 1];
    fx_own<NP, FIN, S, BLK>(F, Tbi, ud[h], uq[h], sc, p, own, xh[h], xl[h]);
    fx_publish(sh, t + h * kTile + S, p, own);
  }
  __syncthreads();
  unsigned long long mag = 0;   // FOUT: OR of |y|
  int emax = 0;                 // FP64 output: largest biased exponent
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int b = t + h * kTile;   // slots of the elements e-S .. e-1: b .. b+S-1
    const int e = e0 + b;
    int P[S][2];
    fx_left_channels(F, sh, b, P);
    double *od = static_cast<double *>(uout_) + (size_t)e;
    long long *oq = static_cast<long long *>(uout_) + (size_t)e;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const long long y = fx_row<NP, S, BLK>(F, i, xh[h], xl[h], P);
      if (FOUT) {
        if (e < K) {
          *oq = y;
          mag |= fx_mag(y);
        }
      } else {
        const double v = sc.bad ? __longlong_as_double(0x7ff8000000000000ll) : fx_to_double(y, sc.sigma);
        if (e < K) {
          *od = v;
          const int be = biased_exponent(v);
          emax = be > emax ? be : emax;
        }
      }
      od += K;
      oq += K;
    }
  }
  fx_block_next<FOUT>(inst, sc, mag, emax);
}

// Two consecutive elements per thread (e = e0 + 2t and e + 1, the block's 512-element tile; K
// even): each node plane is read and written as one 128-bit access per thread (a fallback to
// two 64-bit accesses for odd K cost 5% in this kernel, so odd meshes take one element per
// thread), the elements e-S .. e-1 come from the published slots (one barrier),
// and the odd element takes its left neighbour's channel scalars from the even element's
// registers (S(S-1)/2 multiply-adds instead of the recursion over S-1 elements, half the
// shared-memory reads). The arithmetic of every sum is that of fixed_body, so the results are
// bit-identical to it.
template <int NP, int FMT, int S, class I>
__device__ __forceinline__ void fixed_body_pair(const I &inst, const void *__restrict__ uin_,
                                                void *__restrict__ uout_, int e0, int rel,
                                                FixedShared<2, S> &sh) {
  constexpr bool FIN = (FMT & kFmtInFixed) != 0;
  constexpr bool FOUT = (FMT & kFmtOutFixed) != 0;
  constexpr bool BLK = (FMT & kFmtBasis) != 0;
  static_assert(FOUT || !BLK, "a block-basis state is written as int64");
  const double *uin_d = static_cast<const double *>(uin_);
  const long long *uin_q = static_cast<const long long *>(uin_);
  const int K = inst.K;
  const int t = threadIdx.x;
  const StepFixed &F = inst.sf;
  const double *Tbi = nullptr;
  if constexpr (BLK) Tbi = inst.Tbi;
  double hd[NP];
  long long hq[NP];
  if (t < S) {
    int m = e0 - S + t;
    if (m < 0) m += K;
    if (FIN) load_elem<NP>(uin_q, K, m, hq);
    else load_elem<NP>(uin_d, K, m, hd);
  }
  const int e = e0 + 2 * t;
  // K even: both elements in range or both out, every pair 16-byte aligned in every plane
  const int el = e < K ? e : K - 2;
  double ud[2][NP];
  long long uq[2][NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    if (FIN) {
      const longlong2 v = __ldg(reinterpret_cast<const longlong2 *>(uin_q + (size_t)j * K + el));
      uq[0][j] = v.x;
      uq[1][j] = v.y;
    } else {
      const double2 v = __ldg(reinterpret_cast<const double2 *>(uin_d + (size_t)j * K + el));
      ud[0][j] = v.x;
      ud[1][j] = v.y;
    }
  }
  const FxScale sc = fx_block_scale<FIN, FOUT, BLK>(inst, e0, rel, sh);
  if (FIN && sc.shift != 0) {
#pragma unroll
    for (int j = 0; j < NP; ++j) hq[j] = fx_rescale(hq[j], sc.shift);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < NP; ++j) uq[h][j] = fx_rescale(uq[h][j], sc.shift);
  }
  if (t < S) {
    int xh[NP], xl[NP];
    long long p;
    FxAcc own[S - 1];
    fx_own<NP, FIN, S, BLK>(F, Tbi, hd, hq, sc, p, own, xh, xl);
    fx_publish(sh, t, p, own);
  }
  int xh[2][NP], xl[2][NP];
  long long pE;
  FxAcc ownE[S - 1];
  {
    long long pO;
    FxAcc ownO[S - 1];
    fx_own<NP, FIN, S, BLK>(F, Tbi, ud[0], uq[0], sc, pE, ownE, xh[0], xl[0]);
    fx_own<NP, FIN, S, BLK>(F, Tbi, ud[1], uq[1], sc, pO, ownO, xh[1], xl[1]);
    fx_publish(sh, 2 * t + S, pE, ownE);
    fx_publish(sh, 2 * t + S + 1, pO, ownO);
  }
  __syncthreads();
  // the even element's left channels from slots 2t .. 2t+S-1 (elements E-S .. E-1)
  int P[2][S][2];
  fx_left_channels(F, sh, 2 * t, P[0]);
  // the odd element's left neighbour is E: Y_s^E = r_s . u^E + sum_{t<s} k_st P_t(E)
  fx_split(pE, P[1][0][0], P[1][0][1]);
#pragma unroll
  for (int s = 1; s < S; ++s) {
    FxAcc c = ownE[s - 1];
#pragma unroll
    for (int q = 0; q < s; ++q) fx_mac(c, F.k[s][q], P[0][q][0], P[0][q][1]);
    fx_split(fx_round(c), P[1][s][0], P[1][s][1]);
  }
  unsigned long long mag = 0;
  int emax = 0;
  const bool ok = e < K;
  double *od = static_cast<double *>(uout_) + (size_t)el;
  long long *oq = static_cast<long long *>(uout_) + (size_t)el;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    long long y[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) y[h] = fx_row<NP, S, BLK>(F, i, xh[h], xl[h], P[h]);
    if (FOUT) {
      if (ok) {
        *reinterpret_cast<longlong2 *>(oq) = make_longlong2(y[0], y[1]);
        mag |= fx_mag(y[0]) | fx_mag(y[1]);
      }
    } else {
      const double v0 = sc.bad ? __longlong_as_double(0x7ff8000000000000ll) : fx_to_double(y[0], sc.sigma);
      const double v1 = sc.bad ? __longlong_as_double(0x7ff8000000000000ll) : fx_to_double(y[1], sc.sigma);
      if (ok) {
        *reinterpret_cast<double2 *>(od) = make_double2(v0, v1);
        emax = max(emax, max(biased_exponent(v0), biased_exponent(v1)));
      }
    }
    od += K;
    oq += K;
  }
  fx_block_next<FOUT>(inst, sc, mag, emax);
}

// One element per thread runs at full occupancy (8 blocks of 256 threads per SM, at most 32
// registers); two per thread keep 48 registers for the second element's values (five
// blocks per SM: 2% faster than four with 64 registers on the large mesh). The five-stage
// step keeps more channel scalars live and takes one block fewer per SM.
template <int NP, int EPT, int FMT, int S>
__global__ void __launch_bounds__(kTile, EPT == 1 ? (S == 3 ? 8 : 6) : (S == 3 ? 5 : 4))
    k_step_fixed(const Inst inst, const void *__restrict__ uin, void *__restrict__ uout, int rel) {
  __shared__ FixedShared<EPT, S> sh;
  pdl_wait();   // the face kernel before it corrects u^n near the PE faces
  pdl_trigger();
  if constexpr (EPT == 2)
    fixed_body_pair<NP, FMT, S>(inst, uin, uout, blockIdx.x * (kTile * 2), rel, sh);
  else
    fixed_body<NP, EPT, FMT, S>(inst, uin, uout, blockIdx.x * (kTile * EPT), rel, sh);
}

__device__ __forceinline__ void *inst_field(const Inst &I, int sel) {
  return sel == 0 ? (void *)I.u : (sel == 1 ? (void *)I.v1 : (void *)I.v2);
}

// Batched fixed-point steps: block b takes work item (instance, first element); the
// instance's descriptor is staged in shared memory; src / dst select u (0), v1 (1) or v2 (2)
// of every instance, FMT their formats (int64 output), the instance's own flag the block
// basis.
template <int FMT>
__global__ void __launch_bounds__(kTile)
    k_batch_fixed(const Inst *__restrict__ insts, const int2 *__restrict__ work, int src, int dst,
                  int rel) {
  __shared__ __align__(16) unsigned char smem[sizeof(Inst)];
  __shared__ FixedShared<1, 3> sh;
  pdl_wait();   // the fix-up before it corrects u^n near the PE faces
  pdl_trigger();
  const int2 w = work[blockIdx.x];
  {
    const int4 *from = reinterpret_cast<const int4 *>(insts + w.x);
    int4 *to = reinterpret_cast<int4 *>(smem);
    for (int t = threadIdx.x; t < (int)(sizeof(Inst) / sizeof(int4)); t += blockDim.x)
      to[t] = __ldg(from + t);
  }
  __syncthreads();
  const Inst &I = *reinterpret_cast<const Inst *>(smem);
  const void *uin = inst_field(I, src);
  void *uout = inst_field(I, dst);
  constexpr int FB = FMT | kFmtBasis;
  switch (I.Np) {
    case 2:
      if (I.basis) fixed_body<2, 1, FB, 3>(I, uin, uout, w.y, rel, sh);
      else fixed_body<2, 1, FMT, 3>(I, uin, uout, w.y, rel, sh);
      break;
    case 3:
      if (I.basis) fixed_body<3, 1, FB, 3>(I, uin, uout, w.y, rel, sh);
      else fixed_body<3, 1, FMT, 3>(I, uin, uout, w.y, rel, sh);
      break;
    case 4:
      if (I.basis) fixed_body<4, 1, FB, 3>(I, uin, uout, w.y, rel, sh);
      else fixed_body<4, 1, FMT, 3>(I, uin, uout, w.y, rel, sh);
      break;
    default:
      if (I.basis) fixed_body<5, 1, FB, 3>(I, uin, uout, w.y, rel, sh);
      else fixed_body<5, 1, FMT, 3>(I, uin, uout, w.y, rel, sh);
      break;
  }
}

// The fields fixed_body reads, with the coefficients (and the block basis of the degree)
// taken from a kernel parameter.
struct LiteView {
  int K;
  const int64_t *meta;
  FxSlot *fx;
  const StepFixed &sf;
  int fxh, fxe;
  const double *Tbi;
};

// Batched fixed-point steps with the coefficients shared per degree (BatchUniform): block b
// reads its work item's record (the instance's fields and the tile's first element; one load
// ahead of the data instead of a work-list entry and then the instance) and takes EPT kTile
// elements.
template <int FMT, int EPT>
__global__ void __launch_bounds__(kTile, EPT == 1 ? 6 : (EPT == 2 ? 5 : 2))
    k_batch_fixed_uniform(const BatchLite *__restrict__ items, int src, int dst, int rel,
                          const UniformFixed uf) {
  __shared__ FixedShared<EPT, 3> sh;
  const BatchLite L = items[blockIdx.x];
  pdl_wait();   // the fix-up before it corrects u^n near the PE faces
  pdl_trigger();
  const int2 w = make_int2(0, L.e0);
  const void *uin = src == 0 ? L.f[0] : (src == 1 ? L.f[1] : L.f[2]);
  void *uout = dst == 0 ? L.f[0] : (dst == 1 ? L.f[1] : L.f[2]);
  // one body per degree, in the block basis where the degree has one
  auto body = [&](auto np) {
    constexpr int NP = decltype(np)::value;
    const int d = NP - 2;
    const LiteView V{L.K, L.meta, L.fx, uf.sf[d], uf.fxh[d], uf.fxe[d], uf.Tbi[d]};
    if constexpr (EPT == 2) {
      if (uf.basis[d]) fixed_body_pair<NP, FMT | kFmtBasis, 3>(V, uin, uout, w.y, rel, sh);
      else fixed_body_pair<NP, FMT, 3>(V, uin, uout, w.y, rel, sh);
    } else {
      if (uf.basis[d]) fixed_body<NP, EPT, FMT | kFmtBasis, 3>(V, uin, uout, w.y, rel, sh);
      else fixed_body<NP, EPT, FMT, 3>(V, uin, uout, w.y, rel, sh);
    }
  };
  switch (L.Np) {
    case 2: body(std::integral_constant<int, 2>()); break;
    case 3: body(std::integral_constant<int, 3>()); break;
    case 4: body(std::integral_constant<int, 4>()); break;
    default: body(std::integral_constant<int, 5>()); break;
  }
}

__global__ void k_fixed_reset(const double *__restrict__ f, size_t n, int *E) {
  int m = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int be = biased_exponent(f[i]);
    m = be > m ? be : m;
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) raise_slot(E, m);
}

// The FP64 values of an int64 field at step `step`: X 2^sigma from the field's scale slot,
// rounded to nearest even, or NaN everywhere when the slot marks a NaN or infinity.
__global__ void k_fixed_to_fp64(const long long *__restrict__ X, double *__restrict__ u, size_t n,
                                const FxSlot *__restrict__ fx, int slot) {
  const int sigma = fx[slot].sigma;
  const bool bad = fx[slot].E >= 2047;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    u[i] = bad ? __longlong_as_double(0x7ff8000000000000ll) : fx_to_double(X[i], sigma);
}

// The same for a block-basis state, element by element: u = Tb w with the coordinates w_j =
// X_j 2^sigma rounded to FP64 first.
template <int NP>
__global__ void __launch_bounds__(256) k_fixed_to_fp64_basis(const Inst I, const long long *__restrict__ X,
                                                             int slot) {
  const int sigma = I.fx[slot].sigma;
  const bool bad = I.fx[slot].E >= 2047;
  const int K = I.K;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
    double w[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) w[j] = fx_to_double(X[(size_t)j * K + e], sigma);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double a = I.Tb[i * NP] * w[0];
#pragma unroll
      for (int j = 1; j < NP; ++j) a = fma(I.Tb[i * NP + j], w[j], a);
      I.u[(size_t)i * K + e] = bad ? __longlong_as_double(0x7ff8000000000000ll) : a;
    }
  }
}

// The state as element-major FP64 rows (K, NP), for adg_get_state(_host): a block forms the
// values of 256 consecutive elements, stages them in shared memory and writes them as one
// contiguous run of 16-byte stores, so that into pinned host memory every warp store fills
// whole lines of the host link. MODE 0 copies FP64 node planes; 1 and 2 convert an int64
// state (nodal values, block-basis coordinates) as k_fixed_to_fp64 and k_fixed_to_fp64_basis
// do, giving the values of the FP64 field the state reads as.
template <int NP, int MODE>
__global__ void __launch_bounds__(256) k_state_rows(const Inst I, const void *__restrict__ src,
                                                    int slot, double *__restrict__ dst) {
  __shared__ __align__(16) double buf[256 * NP];
  const int K = I.K;
  int sigma = 0;
  bool bad = false;
  if (MODE != 0) {
    sigma = I.fx[slot].sigma;
    bad = I.fx[slot].E >= 2047;
  }
  const bool vec = (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
  for (int e0 = blockIdx.x * 256; e0 < K; e0 += gridDim.x * 256) {
    const int e = e0 + threadIdx.x;
    if (e < K) {
      double v[NP];
      if (MODE == 0) {
        const double *u = static_cast<const double *>(src);
#pragma unroll
        for (int j = 0; j < NP; ++j) v[j] = u[(size_t)j * K + e];
      } else {
        const long long *X = static_cast<const long long *>(src);
        double w[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) w[j] = fx_to_double(X[(size_t)j * K + e], sigma);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          double a = w[i];
          if (MODE == 2) {
            a = I.Tb[i * NP] * w[0];
#pragma unroll
            for (int j = 1; j < NP; ++j) a = fma(I.Tb[i * NP + j], w[j], a);
          }
          v[i] = bad ? __longlong_as_double(0x7ff8000000000000ll) : a;
        }
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) buf[threadIdx.x * NP + i] = v[i];
    }
    __syncthreads();
    const int cnt = min(256, K - e0) * NP;
    double *out = dst + (size_t)e0 * NP;
    if (vec) {   // e0 NP doubles from a 16-byte aligned dst: 16-byte aligned
      const double2 *b2 = reinterpret_cast<const double2 *>(buf);
      double2 *o2 = reinterpret_cast<double2 *>(out);
      for (int k = threadIdx.x; k < cnt / 2; k += 256) o2[k] = b2[k];
      if ((cnt & 1) && threadIdx.x == 0) out[cnt - 1] = buf[cnt - 1];
    } else {
      for (int k = threadIdx.x; k < cnt; k += 256) out[k] = buf[k];
    }
    __syncthreads();
  }
}

template <int NP, int FMT, int S>
cudaError_t fixed_np_fmt_s(const Inst &I, const void *uin, void *uout, int rel, cudaStream_t s,
                           bool pdl) {
  if (I.ept == 2)
    return launch_maybe_pdl(k_step_fixed<NP, 2, FMT, S>,
                            dim3((unsigned)((I.K + 2 * kTile - 1) / (2 * kTile))), dim3(kTile), s,
                            pdl, I, uin, uout, rel);
  return launch_maybe_pdl(k_step_fixed<NP, 1, FMT, S>, dim3((unsigned)((I.K + kTile - 1) / kTile)),
                          dim3(kTile), s, pdl, I, uin, uout, rel);
}

template <int NP, int FMT>
cudaError_t fixed_np_fmt(const Inst &I, const void *uin, void *uout, int rel, cudaStream_t s,
                         bool pdl) {
  if (I.ns == kMaxCS) return fixed_np_fmt_s<NP, FMT, kMaxCS>(I, uin, uout, rel, s, pdl);
  return fixed_np_fmt_s<NP, FMT, 3>(I, uin, uout, rel, s, pdl);
}

// Single-instance steps write int64 (the state stays in fixed point until it is read).
template <int NP>
cudaError_t fixed_np(const Inst &I, const void *uin, void *uout, int rel, int fmt,
                     cudaStream_t s, bool pdl) {
  switch (fmt) {
    case kFmtOutFixed: return fixed_np_fmt<NP, kFmtOutFixed>(I, uin, uout, rel, s, pdl);
    case kFmtInFixed | kFmtOutFixed:
      return fixed_np_fmt<NP, kFmtInFixed | kFmtOutFixed>(I, uin, uout, rel, s, pdl);
    case kFmtBasis | kFmtOutFixed:
      return fixed_np_fmt<NP, kFmtBasis | kFmtOutFixed>(I, uin, uout, rel, s, pdl);
    default:
      return fixed_np_fmt<NP, kFmtBasis | kFmtInFixed | kFmtOutFixed>(I, uin, uout, rel, s, pdl);
  }
}

}  // namespace

cudaError_t launch_fixed_step(const Inst &I, const void *uin, void *uout, int rel, int fmt,
                              cudaStream_t s, bool pdl) {
  if (!(fmt & kFmtOutFixed)) return cudaErrorInvalidValue;
  fmt = (fmt & (kFmtInFixed | kFmtOutFixed)) | (I.basis ? kFmtBasis : 0);
  switch (I.Np) {
    case 2: return fixed_np<2>(I, uin, uout, rel, fmt, s, pdl);
    case 3: return fixed_np<3>(I, uin, uout, rel, fmt, s, pdl);
    case 4: return fixed_np<4>(I, uin, uout, rel, fmt, s, pdl);
    case 5: return fixed_np<5>(I, uin, uout, rel, fmt, s, pdl);
    default: return cudaErrorInvalidValue;
  }
}

// Batched steps write int64 (fmt has kFmtOutFixed; the state stays in fixed point).
cudaError_t launch_batch_fixed_step(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                    int src, int dst, int fmt, int rel, cudaStream_t s, bool pdl) {
  if (nwork <= 0) return cudaSuccess;
  if (!(fmt & kFmtOutFixed)) return cudaErrorInvalidValue;
  if (fmt & kFmtInFixed)
    return launch_maybe_pdl(k_batch_fixed<kFmtInFixed | kFmtOutFixed>, dim3(nwork), dim3(kTile), s,
                            pdl, insts_dev, work_dev, src, dst, rel);
  return launch_maybe_pdl(k_batch_fixed<kFmtOutFixed>, dim3(nwork), dim3(kTile), s, pdl, insts_dev,
                          work_dev, src, dst, rel);
}

namespace {
template <int EPT>
cudaError_t batch_uniform_ept(const BatchUniform &bu, int src, int dst, int fmt, int rel,
                              cudaStream_t s, bool pdl) {
  const dim3 g(bu.nitems), b(kTile);
  if (fmt & kFmtInFixed)
    return launch_maybe_pdl(k_batch_fixed_uniform<kFmtInFixed | kFmtOutFixed, EPT>, g, b, s, pdl,
                            bu.items_dev, src, dst, rel, bu.uf);
  return launch_maybe_pdl(k_batch_fixed_uniform<kFmtOutFixed, EPT>, g, b, s, pdl, bu.items_dev, src,
                          dst, rel, bu.uf);
}
}  // namespace

cudaError_t launch_batch_fixed_uniform(const BatchUniform &bu, const int2 *work_dev, int nwork,
                                       int src, int dst, int fmt, int rel, cudaStream_t s,
                                       bool pdl) {
  (void)work_dev;
  (void)nwork;
  if (bu.nitems <= 0) return cudaSuccess;
  if (!(fmt & kFmtOutFixed)) return cudaErrorInvalidValue;
  if (bu.ept == 4) return batch_uniform_ept<4>(bu, src, dst, fmt, rel, s, pdl);
  if (bu.ept == 2) return batch_uniform_ept<2>(bu, src, dst, fmt, rel, s, pdl);
  return batch_uniform_ept<1>(bu, src, dst, fmt, rel, s, pdl);
}

cudaError_t launch_state_rows(const Inst &I, const void *src, bool fixed, int64_t step,
                              double *dst, cudaStream_t s) {
  const int slot = (int)(step % 3);
  const size_t want = ((size_t)I.K + 255) / 256;
  const size_t cap = 8 * (size_t)sm_count();
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  const int mode = fixed ? (I.basis ? 2 : 1) : 0;
  auto go = [&](auto np) -> cudaError_t {
    constexpr int NP = decltype(np)::value;
    if (mode == 0) k_state_rows<NP, 0><<<grid, 256, 0, s>>>(I, src, slot, dst);
    else if (mode == 1) k_state_rows<NP, 1><<<grid, 256, 0, s>>>(I, src, slot, dst);
    else k_state_rows<NP, 2><<<grid, 256, 0, s>>>(I, src, slot, dst);
    return cudaGetLastError();
  };
  switch (I.Np) {
    case 2: return go(std::integral_constant<int, 2>());
    case 3: return go(std::integral_constant<int, 3>());
    case 4: return go(std::integral_constant<int, 4>());
    case 5: return go(std::integral_constant<int, 5>());
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fixed_to_fp64(const Inst &I, const long long *X, int64_t step,
                                 cudaStream_t s) {
  const int slot = (int)(step % 3);
  const size_t n = I.basis ? (size_t)I.K : (size_t)I.K * I.Np;
  const size_t want = (n + 255) / 256;
  const size_t cap = 8 * (size_t)sm_count();
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  if (!I.basis) {
    k_fixed_to_fp64<<<grid, 256, 0, s>>>(X, I.u, n, I.fx, slot);
  } else {
    switch (I.Np) {
      case 2: k_fixed_to_fp64_basis<2><<<grid, 256, 0, s>>>(I, X, slot); break;
      case 3: k_fixed_to_fp64_basis<3><<<grid, 256, 0, s>>>(I, X, slot); break;
      case 4: k_fixed_to_fp64_basis<4><<<grid, 256, 0, s>>>(I, X, slot); break;
      case 5: k_fixed_to_fp64_basis<5><<<grid, 256, 0, s>>>(I, X, slot); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_fixed_reset(const double *f, size_t n, FxSlot *fx, int64_t step,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(fx, 0, 3 * sizeof(FxSlot), s);
  if (e != cudaSuccess) return e;
  const size_t want = (n + 255) / 256;
  const size_t cap = 4 * (size_t)sm_count();
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  k_fixed_reset<<<grid, 256, 0, s>>>(f, n, &fx[(int)(step % 3)].E);
  return cudaGetLastError();
}

}  // namespace adg
