// Composed SSP-RK3 step of upwind advection (a > 0) in fixed-point integer arithmetic:
// the StepConsts stencil (adg_internal.h) evaluated with 32 x 32 -> 64-bit integer
// multiply-adds on two-limb values (adg_fixed.cuh). Within a chunk of steps the field stays
// int64 between steps; only the chunk's first step reads FP64 and its last writes FP64.
#include "adg_device.cuh"
#include "adg_fixed.cuh"

namespace adg {
namespace {

template <int EPT>
struct FixedShared {
  // per element slot: the right trace p and the unrounded own parts (a, b) of its channel
  // scalars r1 . u, r2 . u
  long long p[EPT * kTile + 3];
  long long s1a[EPT * kTile + 3], s1b[EPT * kTile + 3];
  long long s2a[EPT * kTile + 3], s2b[EPT * kTile + 3];
  FxScale sc;
};

// Working-scale value of node j of an element (FP64 input, or int64 input already brought
// to the working scale).
template <bool FIN>
__device__ __forceinline__ long long fx_in(double x, long long X, const FxScale &sc) {
  if (FIN) return X;
  return fx_from_double(x, sc.sigma + 1079);
}

// p = the element's right trace, s1 / s2 = the own parts r1 . u, r2 . u of its channel
// scalars (unrounded sums), and the limbs of its values for the output rows.
template <int NP, bool FIN>
__device__ __forceinline__ void fx_own(const StepFixed &F, const double *ud, const long long *uq,
                                       const FxScale &sc, long long &p, FxAcc &s1, FxAcc &s2,
                                       int *xh, int *xl) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const long long X = fx_in<FIN>(FIN ? 0.0 : ud[j], FIN ? uq[j] : 0ll, sc);
    fx_split(X, xh[j], xl[j]);
    fx_mac(s1, F.r1[j], xh[j], xl[j]);
    fx_mac(s2, F.r2[j], xh[j], xl[j]);
    if (j == NP - 1) p = X;
  }
}

// One thread per element (EPT elements per thread, e = e0 + t + h kTile): the right trace and
// the unrounded own parts of the channel scalars go to shared memory (one barrier); each
// thread then forms its left neighbour's v1_p and v2_p from those of elements e-3 .. e-1 and
// u'^e = G u^e + h_0 P0 + h_1 P1 + h_2 P2. The first three threads publish the three elements
// before the block with the same arithmetic (the working scale is one per field, so every
// element converts the same way).
// The block holding element 0 clears the scale slot of u^{n+2}.
template <int NP, int EPT, int FMT, class I>
__device__ __forceinline__ void fixed_body(const I &inst, const void *__restrict__ uin_,
                                           void *__restrict__ uout_, int e0, int rel,
                                           FixedShared<EPT> &sh) {
  constexpr bool FIN = (FMT & kFmtInFixed) != 0;
  constexpr bool FOUT = (FMT & kFmtOutFixed) != 0;
  const double *uin_d = static_cast<const double *>(uin_);
  const long long *uin_q = static_cast<const long long *>(uin_);
  const int K = inst.K;
  const int t = threadIdx.x;
  const StepFixed &F = inst.sf;

  // loads first: they do not depend on the scale
  double hd[NP];
  long long hq[NP];
  if (t < 3) {
    int m = e0 - 3 + t;
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
  // thread 0 reads the scale of u^n for the block (every warp reading it itself, without
  // this barrier, measured 4% slower)
  if (t == 0) {
    const FxScale sc = fx_scale(inst.fx, inst.meta[0] + rel, FIN);
    sh.sc = sc;
    if (e0 == 0) {
      FxSlot &c = inst.fx[fx_clear(sc.slot)];   // the slot of u^{n+2}
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
  const FxScale sc = sh.sc;
  if (FIN && sc.shift != 0) {   // block-uniform: the field grew past 2^57 or shrank
#pragma unroll
    for (int j = 0; j < NP; ++j) hq[j] = fx_rescale(hq[j], sc.shift);
#pragma unroll
    for (int h = 0; h < EPT; ++h)
#pragma unroll
      for (int j = 0; j < NP; ++j) uq[h][j] = fx_rescale(uq[h][j], sc.shift);
  }
  // publish p and the unrounded own parts of every element's channel scalars (the halo's too)
  if (t < 3) {
    int xh[NP], xl[NP];
    long long p;
    FxAcc hs1, hs2;
    fx_own<NP, FIN>(F, hd, hq, sc, p, hs1, hs2, xh, xl);
    sh.p[t] = p;
    sh.s1a[t] = hs1.a;
    sh.s1b[t] = hs1.b;
    sh.s2a[t] = hs2.a;
    sh.s2b[t] = hs2.b;
  }
  int xh[EPT][NP], xl[EPT][NP];
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    long long p;
    FxAcc s1, s2;
    fx_own<NP, FIN>(F, ud[h], uq[h], sc, p, s1, s2, xh[h], xl[h]);
    const int sl = t + h * kTile + 3;
    sh.p[sl] = p;
    sh.s1a[sl] = s1.a;
    sh.s1b[sl] = s1.b;
    sh.s2a[sl] = s2.a;
    sh.s2b[sl] = s2.b;
  }
  __syncthreads();
  unsigned long long mag = 0;   // FOUT: OR of |y|
  int emax = 0;                 // FP64 output: largest biased exponent
#pragma unroll
  for (int h = 0; h < EPT; ++h) {
    const int b = t + h * kTile;   // slots of the elements e-3, e-2, e-1: b, b+1, b+2
    const int e = e0 + b;
    // the left neighbour's channel scalars, each rounded once from the published parts:
    // v1_p^{e-2} = r1 . u^{e-2} + k_0 p^{e-3}, v1_p^{e-1} = r1 . u^{e-1} + k_0 p^{e-2},
    // v2_p^{e-1} = r2 . u^{e-1} + k_1 p^{e-2} + k_2 v1_p^{e-2} (every thread that needs one of
    // them forms it from the same values, so all agree bit for bit)
    int p3h, p3l, p2h, p2l;
    fx_split(sh.p[b], p3h, p3l);
    fx_split(sh.p[b + 1], p2h, p2l);
    FxAcc c1m2{sh.s1a[b + 1], sh.s1b[b + 1]};
    fx_mac(c1m2, F.k[0], p3h, p3l);
    const long long q1m2 = fx_round(c1m2);
    FxAcc c1m1{sh.s1a[b + 2], sh.s1b[b + 2]};
    fx_mac(c1m1, F.k[0], p2h, p2l);
    const long long q1m1 = fx_round(c1m1);
    int qh, ql;
    fx_split(q1m2, qh, ql);
    FxAcc c2m1{sh.s2a[b + 2], sh.s2b[b + 2]};
    fx_mac(c2m1, F.k[1], p2h, p2l);
    fx_mac(c2m1, F.k[2], qh, ql);
    const long long q2m1 = fx_round(c2m1);
    int P0h, P0l, P1h, P1l, P2h, P2l;
    fx_split(sh.p[b + 2], P0h, P0l);
    fx_split(q1m1, P1h, P1l);
    fx_split(q2m1, P2h, P2l);
    const size_t base = (size_t)e;
    double *od = static_cast<double *>(uout_) + base;
    long long *oq = static_cast<long long *>(uout_) + base;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      FxAcc acc;
#pragma unroll
      for (int j = 0; j < NP; ++j) fx_mac(acc, F.G[i * NP + j], xh[h][j], xl[h][j]);
      fx_mac(acc, F.h[0][i], P0h, P0l);
      fx_mac(acc, F.h[1][i], P1h, P1l);
      fx_mac(acc, F.h[2][i], P2h, P2l);
      const long long y = fx_round(acc);
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
  // the scale of u^{n+1}: OR of |y| (int64 output) or largest exponent (FP64 output), one
  // slot update per warp
  FxSlot &nx = inst.fx[fx_next(sc.slot)];
  if (FOUT) {
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)mag);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(mag >> 32));
    if ((t & 31) == 0) or_slot(&nx.mag, ((unsigned long long)hi << 32) | lo);
  } else {
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((t & 31) == 0) raise_slot(&nx.E, emax);
  }
}

// One element per thread runs at full occupancy (8 blocks of 256 threads per SM, at most 32
// registers); two per thread keep 64 registers for the second element's values.
template <int NP, int EPT, int FMT>
__global__ void __launch_bounds__(kTile, EPT == 1 ? 8 : 4)
    k_step_fixed(const Inst inst, const void *__restrict__ uin, void *__restrict__ uout, int rel) {
  __shared__ FixedShared<EPT> sh;
  fixed_body<NP, EPT, FMT>(inst, uin, uout, blockIdx.x * (kTile * EPT), rel, sh);
}

__device__ __forceinline__ void *inst_field(const Inst &I, int sel) {
  return sel == 0 ? (void *)I.u : (sel == 1 ? (void *)I.v1 : (void *)I.v2);
}

// Batched fixed-point steps: block b takes work item (instance, first element); the
// instance's descriptor is staged in shared memory; src / dst select u (0), v1 (1) or v2 (2)
// of every instance, FMT their formats.
template <int FMT>
__global__ void __launch_bounds__(kTile)
    k_batch_fixed(const Inst *__restrict__ insts, const int2 *__restrict__ work, int src, int dst,
                  int rel) {
  __shared__ __align__(16) unsigned char smem[sizeof(Inst)];
  __shared__ FixedShared<1> sh;
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
  switch (I.Np) {
    case 2: fixed_body<2, 1, FMT>(I, uin, uout, w.y, rel, sh); break;
    case 3: fixed_body<3, 1, FMT>(I, uin, uout, w.y, rel, sh); break;
    case 4: fixed_body<4, 1, FMT>(I, uin, uout, w.y, rel, sh); break;
    default: fixed_body<5, 1, FMT>(I, uin, uout, w.y, rel, sh); break;
  }
}

// The fields fixed_body reads, with the coefficients taken from a kernel parameter.
struct LiteView {
  int K;
  const int64_t *meta;
  FxSlot *fx;
  const StepFixed &sf;
};

// Batched fixed-point steps with the coefficients shared per degree (BatchUniform): block b
// reads its work item's record (the instance's fields and the tile's first element; one load
// ahead of the data instead of a work-list entry and then the instance) and takes EPT kTile
// elements.
template <int FMT, int EPT>
__global__ void __launch_bounds__(kTile, EPT == 1 ? 6 : (EPT == 2 ? 4 : 2))
    k_batch_fixed_uniform(const BatchLite *__restrict__ items, int src, int dst, int rel,
                          const UniformFixed uf) {
  __shared__ FixedShared<EPT> sh;
  const BatchLite L = items[blockIdx.x];
  const int2 w = make_int2(0, L.e0);
  const void *uin = src == 0 ? L.f[0] : (src == 1 ? L.f[1] : L.f[2]);
  void *uout = dst == 0 ? L.f[0] : (dst == 1 ? L.f[1] : L.f[2]);
  switch (L.Np) {
    case 2: fixed_body<2, EPT, FMT>(LiteView{L.K, L.meta, L.fx, uf.sf[0]}, uin, uout, w.y, rel, sh); break;
    case 3: fixed_body<3, EPT, FMT>(LiteView{L.K, L.meta, L.fx, uf.sf[1]}, uin, uout, w.y, rel, sh); break;
    case 4: fixed_body<4, EPT, FMT>(LiteView{L.K, L.meta, L.fx, uf.sf[2]}, uin, uout, w.y, rel, sh); break;
    default: fixed_body<5, EPT, FMT>(LiteView{L.K, L.meta, L.fx, uf.sf[3]}, uin, uout, w.y, rel, sh); break;
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

template <int NP, int FMT>
void fixed_np_fmt(const Inst &I, const void *uin, void *uout, int rel, cudaStream_t s) {
  if (I.ept == 2)
    k_step_fixed<NP, 2, FMT><<<(unsigned)((I.K + 2 * kTile - 1) / (2 * kTile)), kTile, 0, s>>>(I, uin, uout, rel);
  else
    k_step_fixed<NP, 1, FMT><<<(unsigned)((I.K + kTile - 1) / kTile), kTile, 0, s>>>(I, uin, uout, rel);
}

template <int NP>
void fixed_np(const Inst &I, const void *uin, void *uout, int rel, int fmt, cudaStream_t s) {
  switch (fmt & 3) {
    case 0: fixed_np_fmt<NP, 0>(I, uin, uout, rel, s); break;
    case 1: fixed_np_fmt<NP, 1>(I, uin, uout, rel, s); break;
    case 2: fixed_np_fmt<NP, 2>(I, uin, uout, rel, s); break;
    default: fixed_np_fmt<NP, 3>(I, uin, uout, rel, s); break;
  }
}

}  // namespace

cudaError_t launch_fixed_step(const Inst &I, const void *uin, void *uout, int rel, int fmt,
                              cudaStream_t s) {
  switch (I.Np) {
    case 2: fixed_np<2>(I, uin, uout, rel, fmt, s); break;
    case 3: fixed_np<3>(I, uin, uout, rel, fmt, s); break;
    case 4: fixed_np<4>(I, uin, uout, rel, fmt, s); break;
    case 5: fixed_np<5>(I, uin, uout, rel, fmt, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_fixed_step(const Inst *insts_dev, const int2 *work_dev, int nwork,
                                    int src, int dst, int fmt, int rel, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  switch (fmt & 3) {
    case 0: k_batch_fixed<0><<<nwork, kTile, 0, s>>>(insts_dev, work_dev, src, dst, rel); break;
    case 1: k_batch_fixed<1><<<nwork, kTile, 0, s>>>(insts_dev, work_dev, src, dst, rel); break;
    case 2: k_batch_fixed<2><<<nwork, kTile, 0, s>>>(insts_dev, work_dev, src, dst, rel); break;
    default: k_batch_fixed<3><<<nwork, kTile, 0, s>>>(insts_dev, work_dev, src, dst, rel); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_fixed_uniform(const BatchUniform &bu, const int2 *work_dev, int nwork,
                                       int src, int dst, int fmt, int rel, cudaStream_t s) {
  (void)work_dev;
  (void)nwork;
  const int n = bu.nitems;
  if (n <= 0) return cudaSuccess;
  const BatchLite *l = bu.items_dev;
  if (bu.ept == 4) {
    switch (fmt & 3) {
      case 0: k_batch_fixed_uniform<0, 4><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      case 1: k_batch_fixed_uniform<1, 4><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      case 2: k_batch_fixed_uniform<2, 4><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      default: k_batch_fixed_uniform<3, 4><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
    }
  } else if (bu.ept == 2) {
    switch (fmt & 3) {
      case 0: k_batch_fixed_uniform<0, 2><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      case 1: k_batch_fixed_uniform<1, 2><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      case 2: k_batch_fixed_uniform<2, 2><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      default: k_batch_fixed_uniform<3, 2><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
    }
  } else {
    switch (fmt & 3) {
      case 0: k_batch_fixed_uniform<0, 1><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      case 1: k_batch_fixed_uniform<1, 1><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      case 2: k_batch_fixed_uniform<2, 1><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
      default: k_batch_fixed_uniform<3, 1><<<n, kTile, 0, s>>>(l, src, dst, rel, bu.uf); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_fixed_to_fp64(const long long *X, double *u, size_t n, const FxSlot *fx,
                                int64_t step, cudaStream_t s) {
  const size_t want = (n + 255) / 256;
  const size_t cap = 8 * (size_t)sm_count();
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  k_fixed_to_fp64<<<grid, 256, 0, s>>>(X, u, n, fx, (int)(step % 3));
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
