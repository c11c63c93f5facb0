// Host side of the C ABI declared in include/adg.h: configuration checks, reference-element
// operators (built in long double, rounded once to FP64), delay and AT tables, device
// buffers, the step driver (CUDA-graph replay of fixed chunks of steps) and reductions.
#include "adg.h"
#include "adg_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

using adg::Inst;
using adg::kMaxNp;
using adg::kStages;

namespace {

thread_local std::string g_last_error;

// ---------------------------------------------------------------------------------------
// Reference-element operators (Section 2, Eq. matrices-reference), long double.
// ---------------------------------------------------------------------------------------
using ld = long double;

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, ld x, ld &P, ld &dP) {
  ld p0 = 1, p1 = x;
  if (n == 0) { P = 1; dP = 0; return; }
  for (int k = 2; k <= n; ++k) {
    ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = (x * x == 1) ? 0.5L * n * (n + 1) * (x > 0 ? 1 : ((n % 2) ? 1 : -1))
                    : n * (x * p1 - p0) / (x * x - 1);
}

// LGL nodes: +-1 and the roots of P_p'; Newton on q(x) = (1 - x^2) P_p'(x), whose
// derivative is -p(p+1) P_p(x). Weights 2 / (p (p+1) P_p(x)^2).
void lgl(int p, std::vector<ld> &x, std::vector<ld> &w) {
  const int Np = p + 1;
  x.assign(Np, 0);
  w.assign(Np, 0);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < Np; ++i) {
    ld xi = -std::cos(pi * i / p);
    if (i > 0 && i < p) {
      for (int it = 0; it < 100; ++it) {
        ld P, dP;
        legendre(p, xi, P, dP);
        const ld qv = (1 - xi * xi) * dP;
        const ld dq = -(ld)p * (p + 1) * P;
        const ld dx = qv / dq;
        xi -= dx;
        if (std::fabs(dx) < 1e-30L) break;
      }
    }
    x[i] = xi;
  }
  for (int i = 0; i < Np; ++i) {  // symmetric set
    const ld s = 0.5L * (x[i] - x[p - i]);
    x[i] = s;
  }
  x[0] = -1;
  x[p] = 1;
  if (p % 2 == 0) x[p / 2] = 0;
  for (int i = 0; i < Np; ++i) {
    ld P, dP;
    legendre(p, x[i], P, dP);
    w[i] = 2.0L / ((ld)p * (p + 1) * P * P);
  }
}

// Gauss-Legendre nodes/weights with n points (roots of P_n), for exact mass integrals.
void gauss(int n, std::vector<ld> &x, std::vector<ld> &w) {
  x.assign(n, 0);
  w.assign(n, 0);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    ld xi = -std::cos(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(n, xi, P, dP);
      const ld dx = P / dP;
      xi -= dx;
      if (std::fabs(dx) < 1e-30L) break;
    }
    ld P, dP;
    legendre(n, xi, P, dP);
    x[i] = xi;
    w[i] = 2.0L / ((1 - xi * xi) * dP * dP);
  }
}

struct Ops {
  int p = 0, Np = 0;
  std::vector<ld> x, w, D, Minv;  // D[i*Np+j] = l_j'(x_i); Minv row-major
  std::vector<ld> M;
};

// Lagrange basis value l_j(t) on nodes x.
ld lagr(const std::vector<ld> &x, int j, ld t) {
  ld v = 1;
  for (size_t m = 0; m < x.size(); ++m)
    if ((int)m != j) v *= (t - x[m]) / (x[j] - x[m]);
  return v;
}

bool invert(std::vector<ld> A, int n, std::vector<ld> &inv) {
  inv.assign(n * n, 0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(inv[c * n + k], inv[piv * n + k]);
    }
    const ld d = A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] /= d;
      inv[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const ld f = A[r * n + c];
      if (f == 0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  return true;
}

Ops make_ops(int p) {
  Ops o;
  o.p = p;
  o.Np = p + 1;
  const int Np = o.Np;
  lgl(p, o.x, o.w);
  // Barycentric differentiation: D_ij = (b_j / b_i) / (x_i - x_j), D_ii = -sum_{j!=i} D_ij.
  std::vector<ld> b(Np, 1);
  for (int j = 0; j < Np; ++j)
    for (int m = 0; m < Np; ++m)
      if (m != j) b[j] /= (o.x[j] - o.x[m]);
  o.D.assign(Np * Np, 0);
  for (int i = 0; i < Np; ++i) {
    ld s = 0;
    for (int j = 0; j < Np; ++j) {
      if (i == j) continue;
      o.D[i * Np + j] = (b[j] / b[i]) / (o.x[i] - o.x[j]);
      s += o.D[i * Np + j];
    }
    o.D[i * Np + i] = -s;
  }
  std::vector<ld> gx, gw;
  gauss(p + 2, gx, gw);
  o.M.assign(Np * Np, 0);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      ld s = 0;
      for (size_t q = 0; q < gx.size(); ++q) s += gw[q] * lagr(o.x, i, gx[q]) * lagr(o.x, j, gx[q]);
      o.M[i * Np + j] = s;
    }
  invert(o.M, Np, o.Minv);
  return o;
}

// AT coefficients c_i(k; q) = prod_{m != i, 0 <= m < q} (k + m) / (m - i): Lagrange
// extrapolation to level n from levels n-k, ..., n-k-q+1, which solves Eq.
// at-flux-constraints (Table 1 for q = 2, 3, 4).
double at_coef(int k, int q, int i) {
  ld num = 1, den = 1;
  for (int m = 0; m < q; ++m) {
    if (m == i) continue;
    num *= (ld)(k + m);
    den *= (ld)(m - i);
  }
  return (double)(num / den);
}

// SplitMix64 output `idx` for `seed` (Steele, Lea and Flood 2014), mapped to [0, 1).
inline double splitmix_uniform(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

struct DelaySource {
  int P = 1, L = 1;
  uint64_t seed = 0;
  std::vector<double> edges;          // upper bin edges, summed left to right
  std::vector<uint8_t> caller;        // caller table (periodic) or empty
  int64_t caller_rows = 0;
  int caa = 0;                        // > 0: the communication-avoiding cycle (Section 6.3)

  void rows(int64_t first, int64_t count, uint8_t *out) const {
    for (int64_t r = 0; r < count; ++r) {
      const int64_t n = first + r;
      if (caa > 0) {
        const int m = (int)(n % (caa + L));
        std::memset(out + r * P, m < caa ? 0 : m - caa, P);
        continue;
      }
      if (!caller.empty()) {
        const int64_t cr = n % caller_rows;
        std::memcpy(out + r * P, caller.data() + cr * P, P);
        continue;
      }
      for (int j = 0; j < P; ++j) {
        const double u = splitmix_uniform(seed, (uint64_t)n * (uint64_t)P + (uint64_t)j);
        int k = L - 1;
        for (int b = 0; b < L; ++b)
          if (u < edges[b]) { k = b; break; }
        out[r * P + j] = (uint8_t)k;
      }
    }
  }
};

// 2N coefficients (A_s, B_s) in Williamson's form of the low-storage schemes (include/adg.h),
// as published fractions: forward Euler; Eq. dg2-rk2; Williamson's three-stage third-order
// scheme; Carpenter and Kennedy's five-stage fourth-order scheme.
struct Frac {
  long long n, d;
};
struct LsTable {
  int S;
  Frac A[adg::kMaxStages], B[adg::kMaxStages];
};

const LsTable *ls_table(int rk) {
  static const LsTable rk1 = {1, {{0, 1}}, {{1, 1}}};
  static const LsTable rk2 = {2, {{0, 1}, {-1, 1}}, {{1, 1}, {1, 2}}};
  static const LsTable lsrk3 = {3, {{0, 1}, {-5, 9}, {-153, 128}}, {{1, 3}, {15, 16}, {8, 15}}};
  static const LsTable lsrk4 = {
      5,
      {{0, 1}, {-567301805773LL, 1357537059087LL}, {-2404267990393LL, 2016746695238LL},
       {-3550918686646LL, 2091501179385LL}, {-1275806237668LL, 842570457699LL}},
      {{1432997174477LL, 9575080441755LL}, {5161836677717LL, 13612068292357LL},
       {1720146321549LL, 2090206949498LL}, {3134564353537LL, 4481467310338LL},
       {2277821191437LL, 14882151754819LL}}};
  switch (rk) {
    case ADG_RK1: return &rk1;
    case ADG_RK2: return &rk2;
    case ADG_LSRK3: return &lsrk3;
    case ADG_LSRK4: return &lsrk4;
    default: return nullptr;
  }
}

std::string check_config(const adg_config *c) {
  if (!c) return "cfg is NULL";
  if (c->pde != ADG_ADVECTION && c->pde != ADG_BURGERS && c->pde != ADG_EULER)
    return "pde must be ADG_ADVECTION, ADG_BURGERS or ADG_EULER";
  if (c->pde == ADG_EULER) {
    if (c->flux != ADG_LLF) return "Euler uses flux ADG_LLF";
    if (!(std::isfinite(c->dt) && c->dt > 0)) return "Euler needs dt > 0";
    if (c->rk != ADG_RK1 && c->rk != ADG_RK2 && c->rk != ADG_SSPRK3)
      return "Euler takes rk ADG_RK1, ADG_RK2 or ADG_SSPRK3";
    if (c->limiter != 0 && c->limiter != 1) return "limiter must be 0 or 1";
    if (!std::isfinite(c->tvb_m) || c->tvb_m < 0) return "tvb_m must be finite and >= 0";
  }
  if (c->pde == ADG_ADVECTION && c->flux != ADG_UPWIND) return "advection uses flux ADG_UPWIND";
  if (c->pde == ADG_BURGERS && c->flux != ADG_LLF) return "Burgers uses flux ADG_LLF";
  if (c->rk < ADG_RK1 || c->rk > ADG_LSRK4) return "rk must be one of ADG_RK1 .. ADG_LSRK4";
  if (c->p < 1 || c->p > ADG_MAX_P) return "p must be in 1..4";
  if (c->K < 1 || c->K > (1 << 30)) return "K must be in 1..2^30";
  if (c->P < 1 || c->K % c->P != 0) return "P must be >= 1 and divide K";
  if (!std::isfinite(c->x0) || !std::isfinite(c->x1) || !(c->x1 > c->x0)) return "need finite x0 < x1";
  if (c->pde == ADG_ADVECTION && (!std::isfinite(c->a) || c->a == 0.0)) return "advection speed a must be finite and nonzero";
  if (!std::isfinite(c->dt) || c->dt < 0) return "dt must be finite and >= 0";
  if (c->dt == 0 && !(std::isfinite(c->cfl) && c->cfl > 0)) return "cfl must be > 0 when dt == 0";
  if (c->mode != ADG_SYNC && c->mode != ADG_ASYNC && c->mode != ADG_ASYNC_AT) return "bad mode";
  if (c->caa_sync < 0 || c->caa_sync > 64) return "caa_sync must be in 0..64";
  if (!std::isfinite(c->nu) || c->nu < 0) return "nu must be finite and >= 0";
  if (c->nu > 0 && c->pde != ADG_BURGERS) return "nu > 0 needs pde ADG_BURGERS";
  if (c->caa_sync > 0 && c->delay_table) return "caa_sync and a caller delay table exclude each other";
  if (c->L < 1 || c->L > ADG_MAX_L) return "L must be in 1..16";
  if (c->at_order < 0 || c->at_order > ADG_MAX_Q) return "at_order must be in 0..5";
  if (c->variant < ADG_VARIANT_AUTO || c->variant > ADG_VARIANT_COMPOSED_FIXED) return "bad variant";
  if (c->ept != 0 && c->ept != 1 && c->ept != 2 && c->ept != 4) return "ept must be 0, 1, 2 or 4";
  if (c->probs) {
    double s = 0;
    for (int k = 0; k < c->L; ++k) {
      if (!std::isfinite(c->probs[k]) || c->probs[k] < 0) return "probs must be finite and >= 0";
      s += c->probs[k];
    }
    if (std::fabs(s - 1.0) > 1e-9) return "probs must sum to 1";
  }
  if (c->delay_table) {
    if (c->table_steps < 1) return "table_steps must be >= 1 with a delay_table";
    const int64_t n = c->table_steps * (int64_t)c->P;
    for (int64_t t = 0; t < n; ++t)
      if (c->delay_table[t] >= c->L) return "delay_table entries must be < L";
  }
  return "";
}

DelaySource make_delay_source(const adg_config *c) {
  DelaySource d;
  d.P = c->P;
  d.L = c->L;
  d.seed = c->seed;
  double s = 0;
  for (int k = 0; k < c->L; ++k) {
    s = s + (c->probs ? c->probs[k] : 1.0 / c->L);
    d.edges.push_back(s);
  }
  if (c->delay_table) {
    d.caller.assign(c->delay_table, c->delay_table + c->table_steps * (int64_t)c->P);
    d.caller_rows = c->table_steps;
  }
  d.caa = c->caa_sync;
  return d;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------
struct InstHost {
  adg_config cfg{};
  std::vector<double> probs;
  DelaySource delays;
  Ops ops;
  Inst I{};
  double dx = 0, dt = 0;
  int q_eff = 1;
  int64_t tbase = 0;
  int TR = 0;
  // device memory owned by this instance
  double *fields = nullptr;  // u | v1 | v2
  double2 *ring = nullptr;
  uint8_t *table = nullptr;
  double *coef = nullptr;
  double *w = nullptr, *M = nullptr;
  int stages = 3;            // stages per step of the RK scheme (the ring may keep more slots)
  double *qbuf = nullptr;    // viscous Burgers: q = u_x of the stage input
  double *ringq = nullptr;   // ... and the PE faces' q^+ traces
  adg::FxSlot *fx = nullptr; // scale slots of the fixed-point composed step
  double *fd = nullptr;      // ... and its PE faces' stage differences [2][P][3]
  bool fixed_ok = false;     // the composed coefficients fit the fixed-point bounds
  std::vector<uint8_t> host_rows;
};

// Parts of a uniform fixed-point batch advanced on separate streams (instances split by DOF;
// two, three and four parts measured 0.3404, 0.3368 and 0.3428 ms per batched step, and
// 0.3347, 0.3311 and 0.3310 once the fix-ups were launched at the highest priority).
constexpr int kBatchParts = 3;

struct adg_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  int device = 0;
  std::vector<InstHost> inst;
  bool batch = false;
  int64_t *meta = nullptr;      // [ninst][2], then one int64 holding `scan`
  int *scan = nullptr;          // the largest biased exponent of the field being loaded
  Inst *insts_dev = nullptr;
  int2 *work_dev = nullptr;
  int nwork = 0;
  int2 *fwork_dev = nullptr;   // (instance, first PE face) items of the batched face pass
  int nfwork = 0;
  int2 *fflat_dev = nullptr;   // (instance, PE face) of every PE face: the composed steps' fix-up
  int nflat = 0;
  bool batch_fused = false;     // every instance runs composed steps
  bool batch_fixed = false;     // ... in fixed point
  adg::BatchLite *lites_ept[3] = {};   // work records of 256, 512, 1024 elements (batch tuner)
  int nlites_ept[3] = {};
  // the same records and the PE-face list in kBatchParts parts of the instances (balanced by
  // DOF; pointers into lites_ept and fflat_dev, which hold the parts' entries in order),
  // advanced on separate streams so that the fix-up of one part overlaps the steps of the
  // others (uniform fixed-point batches launched directly)
  adg::BatchLite *lites_half[3][kBatchParts] = {};
  int nlites_half[3][kBatchParts] = {};
  int2 *fflat_half[kBatchParts] = {};
  int nflat_half[kBatchParts] = {};
  bool split = false;                          // the parts have their streams and events
  cudaStream_t side[kBatchParts] = {};         // side[0] unused: part 0 runs on `stream`
  cudaEvent_t fork_ev = nullptr, join_ev[kBatchParts] = {};
  bool batch_even = false;             // every instance has an even K (the paired kernel)
  std::unique_ptr<adg::BatchUniform> bu;   // shared coefficients per degree, when they are
  double *partials = nullptr, *red_out = nullptr;
  double *pinned = nullptr;
  cudaGraphExec_t gexec[4] = {};   // one graph of G steps per chunk kind (kChunk*)
  int fx_live = 0;                 // fixed-point state: 0 in u (FP64), 1 in v1, 2 in v2 (int64)
  bool u_fresh = true;             // u holds the state of step n (FP64)
  int G = 32;                      // steps per graph (128 measured slower: 78.5 against
                                   // 77.2 ms for 2000 steps of the adjoint workload)
  int64_t n = 0;
};

namespace {

int fail(adg_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, e_ == cudaErrorMemoryAllocation ? ADG_ENOMEM : ADG_ECUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

// The device address of a caller's host buffer where kernels can use it in place: pinned
// (page-locked, mapped) and managed memory give one, pageable memory gives null (the caller
// stages it through device memory). Device memory is refused: the _host entry points take host
// buffers, the others device buffers.
int host_view(adg_ctx *c, const void *p, const void **view) {
  *view = nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return ADG_OK;   // not known to the runtime: pageable
  }
  if (a.type == cudaMemoryTypeDevice)
    return fail(c, ADG_EINVAL, "a host buffer was expected, not device memory");
  if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged) *view = a.devicePointer;
  return ADG_OK;
}

// c2 a = -2 dt a / dx of upwind advection. With the step from the Courant number,
// dt = sigma dx / |a|, it is -2 sigma sign(a) exactly: folded from sigma, every instance with
// the same degree, sigma and sign of a gets the same constants (the rounded dt differs from
// sigma dx / |a| by one rounding, 1e-16 relatively).
long double advection_c2a(const InstHost &h) {
  const long double a = (long double)h.cfg.a;
  if (h.cfg.dt > 0) return -2.0L * (long double)h.dt * a / (long double)h.dx;
  return -2.0L * (long double)h.cfg.cfl * (a > 0 ? 1.0L : -1.0L);
}

void fold_constants(InstHost &h) {
  const Ops &o = h.ops;
  const int Np = o.Np;
  const ld c2 = -2.0L * (ld)h.dt / (ld)h.dx;
  const bool adv = h.cfg.pde == ADG_ADVECTION;
  const ld c2a = adv ? advection_c2a(h) : 0.0L;
  const ld alpha[3] = {0.0L, 0.75L, 1.0L / 3.0L};
  const ld beta[3] = {1.0L, 0.25L, 2.0L / 3.0L};
  // A 2N low-storage scheme uses one set, sc[0]: dt L alone (beta 1, no identity term).
  const bool ls = h.I.ls != 0;
  for (int s = 0; s < (ls ? 1 : kStages); ++s) {
    adg::StageConsts &C = h.I.sc[s];
    std::memset(&C, 0, sizeof(C));
    C.alpha = ls ? 0.0 : (double)alpha[s];
    C.beta = ls ? 0.0 : (double)beta[s];
    const ld b = ls ? 1.0L : beta[s];
    const ld id = ls ? 0.0L : 1.0L;
    for (int i = 0; i < Np; ++i) {
      for (int j = 0; j < Np; ++j) {
        const ld d = o.D[i * Np + j];
        C.A[i * Np + j] = adv ? (double)(b * ((i == j ? id : 0.0L) + c2a * d))
                              : (double)(b * c2 * 0.5L * d);
      }
      const ld sc = adv ? b * c2a : b * c2;
      C.lL[i] = (double)(sc * o.Minv[i * Np + 0]);
      C.lR[i] = (double)(-sc * o.Minv[i * Np + (Np - 1)]);
    }
  }
}

// Composed step constants (StepConsts in adg_internal.h), built in long double from the
// unrounded stage constants of upwind advection with a > 0.
// Butcher form (a, b) of the 2N scheme of rk (ls_table): with k_j = L(U_{j-1}), stage s+1's
// input U_s = u + dt sum_{j<=s} a_{s+1,j} k_j, a_{s+1,j} = sum_{r=j}^{s} B_r A_{j+1} ... A_r,
// and b_j the same sum for s = S.
void two_register_butcher(int rk, int &S, ld a[adg::kMaxStages][adg::kMaxStages],
                          ld b[adg::kMaxStages]) {
  const LsTable *t = ls_table(rk);
  S = t->S;
  ld A[adg::kMaxStages], B[adg::kMaxStages];
  for (int s = 0; s < S; ++s) {
    A[s] = (ld)t->A[s].n / (ld)t->A[s].d;
    B[s] = (ld)t->B[s].n / (ld)t->B[s].d;
  }
  auto coef = [&](int s, int j) {   // weight of dt k_j in U_s
    ld tot = 0;
    for (int r = j; r < s; ++r) {
      ld prod = 1;
      for (int m = j + 1; m <= r; ++m) prod *= A[m];
      tot += B[r] * prod;
    }
    return tot;
  };
  for (int s = 0; s < adg::kMaxStages; ++s) {
    b[s] = s < S ? coef(S, s) : 0;
    for (int jj = 0; jj < adg::kMaxStages; ++jj) a[s][jj] = (s < S && jj < s) ? coef(s, jj) : 0;
  }
}

// Block basis of the element operator for the fixed-point composed step. Every matrix of the
// composed step of upwind advection (G, and the stage maps behind h, r and R) is a polynomial
// in the element operator A = D + M^-1 e_0 e_0^T. In a basis of A-invariant subspaces of
// dimension two (a complex-conjugate pair of eigenvalues, or two real ones) and, for odd Np,
// one last eigenvector, G is block diagonal with 2 x 2 blocks, so each of its rows takes two
// multiply-adds instead of Np. Each pair's first vector has right trace 1 and its second
// trace 0 (a single vector: trace 1), so the right trace of u = T w is the sum of the even
// coordinates of w. Built in long double: eigenvalues as the roots of the characteristic
// polynomial (Faddeev-LeVerrier coefficients, Weierstrass iteration, Newton polishing),
// eigenvectors as null vectors of A - lambda I (elimination with complete pivoting). The
// basis is rejected (nodal values are kept) unless T^-1 A T is block diagonal to 1e-13 of
// its largest entry and cond_inf(T) <= 64: the fixed-point error of a step, relative to the
// field, grows with that condition number.
using cld = std::complex<ld>;

std::vector<ld> char_poly(const std::vector<ld> &A, int n) {
  // c[n] = 1; M_1 = I, c_{n-k} = -tr(A M_k) / k, M_{k+1} = A M_k + c_{n-k} I
  std::vector<ld> c(n + 1, 0.0L), M(n * n, 0.0L), AM(n * n);
  c[n] = 1;
  for (int i = 0; i < n; ++i) M[i * n + i] = 1;
  for (int k = 1; k <= n; ++k) {
    ld tr = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        ld a = 0;
        for (int l = 0; l < n; ++l) a += A[i * n + l] * M[l * n + j];
        AM[i * n + j] = a;
      }
    for (int i = 0; i < n; ++i) tr += AM[i * n + i];
    c[n - k] = -tr / k;
    M = AM;
    for (int i = 0; i < n; ++i) M[i * n + i] += c[n - k];
  }
  return c;
}

cld poly_at(const std::vector<ld> &c, cld z) {
  cld v = 0;
  for (int k = (int)c.size() - 1; k >= 0; --k) v = v * z + c[k];
  return v;
}

std::vector<cld> poly_roots(const std::vector<ld> &c) {
  const int n = (int)c.size() - 1;
  ld R = 1;
  for (int k = 0; k < n; ++k) R = std::max(R, 1 + fabsl(c[k]));
  std::vector<cld> z(n);
  cld zz = 1;
  for (int i = 0; i < n; ++i) {
    zz *= cld(0.4L, 0.9L);
    z[i] = zz * R;
  }
  for (int it = 0; it < 4000; ++it) {
    ld change = 0;
    for (int i = 0; i < n; ++i) {
      cld den = 1;
      for (int j = 0; j < n; ++j)
        if (j != i) den *= z[i] - z[j];
      if (std::abs(den) == 0) den = 1e-30L;
      const cld dz = poly_at(c, z[i]) / den;
      z[i] -= dz;
      change = std::max(change, std::abs(dz) / (1 + std::abs(z[i])));
    }
    if (change < 1e-30L) break;
  }
  std::vector<ld> dc(n);
  for (int k = 1; k <= n; ++k) dc[k - 1] = k * c[k];
  for (int i = 0; i < n; ++i)
    for (int it = 0; it < 3; ++it) {
      const cld d = poly_at(dc, z[i]);
      if (std::abs(d) > 0) z[i] -= poly_at(c, z[i]) / d;
    }
  return z;
}

// A null vector of A - lam I (unit 2-norm), or false.
bool null_vector(const std::vector<ld> &A, int n, cld lam, std::vector<cld> &v) {
  std::vector<cld> B(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B[i * n + j] = A[i * n + j] - (i == j ? lam : cld(0));
  std::vector<int> col(n);
  for (int j = 0; j < n; ++j) col[j] = j;
  for (int k = 0; k < n - 1; ++k) {
    int pi = k, pj = k;
    ld best = -1;
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j)
        if (std::abs(B[i * n + j]) > best) {
          best = std::abs(B[i * n + j]);
          pi = i;
          pj = j;
        }
    if (!(best > 0)) return false;
    for (int j = 0; j < n; ++j) std::swap(B[k * n + j], B[pi * n + j]);
    for (int i = 0; i < n; ++i) std::swap(B[i * n + k], B[i * n + pj]);
    std::swap(col[k], col[pj]);
    for (int i = k + 1; i < n; ++i) {
      const cld f = B[i * n + k] / B[k * n + k];
      for (int j = k; j < n; ++j) B[i * n + j] -= f * B[k * n + j];
    }
  }
  std::vector<cld> y(n);
  y[n - 1] = 1;
  for (int k = n - 2; k >= 0; --k) {
    cld acc = 0;
    for (int j = k + 1; j < n; ++j) acc += B[k * n + j] * y[j];
    y[k] = -acc / B[k * n + k];
  }
  v.assign(n, 0);
  ld nrm = 0;
  for (int k = 0; k < n; ++k) {
    v[col[k]] = y[k];
    nrm += std::norm(y[k]);
  }
  nrm = sqrtl(nrm);
  if (!(nrm > 0)) return false;
  for (auto &x : v) x /= nrm;
  return true;
}

// The blocks of the block basis: A = {0, 1} and B = {2, .., n-1} (a pair for n = 4, one
// vector for n = 3, a triple for n = 5); the first vector of each block has right trace 1.
bool same_block(int i, int j) { return (i < 2) == (j < 2); }

bool block_diagonal(const std::vector<ld> &X, int n, ld tol) {
  ld mx = 0, off = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      mx = std::max(mx, fabsl(X[i * n + j]));
      if (!same_block(i, j)) off = std::max(off, fabsl(X[i * n + j]));
    }
  return off <= tol * mx;
}

std::vector<ld> similar(const std::vector<ld> &Ti, const std::vector<ld> &X,
                        const std::vector<ld> &T, int n) {
  std::vector<ld> Y(n * n, 0.0L), Z(n * n, 0.0L);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) Y[i * n + j] += X[i * n + k] * T[k * n + j];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) Z[i * n + j] += Ti[i * n + k] * Y[k * n + j];
  return Z;
}

ld cond_inf(const std::vector<ld> &T, const std::vector<ld> &Ti, int n) {
  ld nt = 0, nti = 0;
  for (int i = 0; i < n; ++i) {
    ld a = 0, b = 0;
    for (int j = 0; j < n; ++j) {
      a += fabsl(T[i * n + j]);
      b += fabsl(Ti[i * n + j]);
    }
    nt = std::max(nt, a);
    nti = std::max(nti, b);
  }
  return nt * nti;
}

bool block_basis(const Ops &o, std::vector<ld> &T, std::vector<ld> &Ti) {
  const int n = o.Np, p = n - 1;
  std::vector<ld> A(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = o.D[i * n + j] + (j == 0 ? o.Minv[i * n + 0] : 0.0L);
  const std::vector<cld> lam = poly_roots(char_poly(A, n));
  ld anorm = 0;
  for (ld x : A) anorm = std::max(anorm, fabsl(x));
  // vectors spanning the invariant subspaces: complex pairs (Re v, Im v) first, then the real
  // eigenvectors two at a time, the last one alone for odd n
  std::vector<std::vector<ld>> span;
  std::vector<std::vector<ld>> reals;
  for (int i = 0; i < n; ++i) {
    const ld tol = 1e-9L * (1 + std::abs(lam[i]));
    std::vector<cld> v;
    if (!null_vector(A, n, lam[i], v)) return false;
    for (int r = 0; r < n; ++r) {   // residual
      cld acc = -lam[i] * v[r];
      for (int k = 0; k < n; ++k) acc += A[r * n + k] * v[k];
      if (std::abs(acc) > 1e-12L * (1 + anorm)) return false;
    }
    if (lam[i].imag() > tol) {
      std::vector<ld> re(n), im(n);
      for (int k = 0; k < n; ++k) {
        re[k] = v[k].real();
        im[k] = v[k].imag();
      }
      span.push_back(re);
      span.push_back(im);
    } else if (fabsl(lam[i].imag()) <= tol) {
      // a real eigenvalue: v is real up to a unit factor
      int km = 0;
      for (int k = 1; k < n; ++k)
        if (std::abs(v[k]) > std::abs(v[km])) km = k;
      const cld ph = v[km] / std::abs(v[km]);
      std::vector<ld> re(n);
      for (int k = 0; k < n; ++k) re[k] = (v[k] / ph).real();
      reals.push_back(re);
    }
  }
  std::vector<std::vector<ld>> pairs_re, pairs_im;   // the complex pairs
  for (size_t k = 0; k + 1 < span.size(); k += 2) {
    pairs_re.push_back(span[k]);
    pairs_im.push_back(span[k + 1]);
  }
  for (auto &r : reals) span.push_back(r);
  auto dot = [&](const std::vector<ld> &a, const std::vector<ld> &b) {
    ld s = 0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
  };
  // One block from the vectors spanning an invariant subspace (columns c0 .. of T): an
  // orthonormal basis Q of it (Gram-Schmidt), traces t = Q^T e_p; the first column Q t / |t|^2
  // (trace 1), the others Q c / |t| for an orthonormal basis c of the complement of t (trace 0).
  auto put_block = [&](std::vector<std::vector<ld>> vs, int c0) {
    const int d = (int)vs.size();
    for (int a = 0; a < d; ++a) {
      const ld n0 = sqrtl(dot(vs[a], vs[a]));
      for (int b = 0; b < a; ++b) {
        const ld pr = dot(vs[b], vs[a]);
        for (int k = 0; k < n; ++k) vs[a][k] -= pr * vs[b][k];
      }
      const ld na = sqrtl(dot(vs[a], vs[a]));
      if (!(na > 1e-9L * n0)) return false;
      for (auto &x : vs[a]) x /= na;
    }
    std::vector<ld> t(d);
    ld tt = 0;
    for (int a = 0; a < d; ++a) {
      t[a] = vs[a][p];
      tt += t[a] * t[a];
    }
    if (!(tt > 1e-12L)) return false;
    const ld tn = sqrtl(tt);
    // orthonormal complement of t in R^d (Gram-Schmidt of the unit vectors against t / |t|)
    std::vector<std::vector<ld>> cs;
    std::vector<ld> th(d);
    for (int a = 0; a < d; ++a) th[a] = t[a] / tn;
    for (int e = 0; e < d && (int)cs.size() < d - 1; ++e) {
      std::vector<ld> c(d, 0.0L);
      c[e] = 1;
      ld pr = th[e];
      for (int a = 0; a < d; ++a) c[a] -= pr * th[a];
      for (auto &o2 : cs) {
        ld q = 0;
        for (int a = 0; a < d; ++a) q += o2[a] * c[a];
        for (int a = 0; a < d; ++a) c[a] -= q * o2[a];
      }
      ld cn = 0;
      for (int a = 0; a < d; ++a) cn += c[a] * c[a];
      cn = sqrtl(cn);
      if (cn < 0.5L) continue;
      for (auto &x : c) x /= cn;
      cs.push_back(c);
    }
    if ((int)cs.size() != d - 1) return false;
    for (int k = 0; k < n; ++k) {
      ld f = 0;
      for (int a = 0; a < d; ++a) f += t[a] * vs[a][k];
      T[k * n + c0] = f / tt;
      for (int b = 0; b + 1 < d; ++b) {
        ld g = 0;
        for (int a = 0; a < d; ++a) g += cs[b][a] * vs[a][k];
        T[k * n + c0 + 1 + b] = g / tn;
      }
    }
    return true;
  };
  // the layouts: n = 2: one pair; n = 3: a pair (a complex pair, else two real vectors) and
  // the remaining real vector; n = 4: two pairs; n = 5: a complex pair and a triple (the other
  // complex pair with the real vector), whichever pair goes first gives the smaller cond_inf
  std::vector<std::vector<std::vector<ld>>> layouts;   // candidate: block A vectors, block B
  if ((int)span.size() != n) return false;
  if (n == 5) {
    if (pairs_re.size() != 2 || reals.size() != 1) return false;
    for (int f = 0; f < 2; ++f)
      layouts.push_back({pairs_re[f], pairs_im[f], pairs_re[1 - f], pairs_im[1 - f], reals[0]});
  } else {
    layouts.push_back(span);
  }
  std::vector<ld> bestT, bestTi;
  ld bestc = -1;
  for (auto &vs : layouts) {
    T.assign(n * n, 0.0L);
    bool ok = put_block({vs[0], vs[1]}, 0);
    if (ok && n > 2) {
      std::vector<std::vector<ld>> rest(vs.begin() + 2, vs.end());
      if (rest.size() == 1) {
        const std::vector<ld> &v = rest[0];
        ok = fabsl(v[p]) > 1e-6L * sqrtl(dot(v, v));
        if (ok)
          for (int k = 0; k < n; ++k) T[k * n + 2] = v[k] / v[p];
      } else {
        ok = put_block(rest, 2);
      }
    }
    if (!ok) continue;
    for (int j = 0; j < n; ++j) T[p * n + j] = (j == 0 || j == 2) ? 1.0L : 0.0L;
    std::vector<ld> Tinv;
    if (!invert(T, n, Tinv)) continue;
    if (!block_diagonal(similar(Tinv, A, T, n), n, 1e-13L)) continue;
    const ld cnd = cond_inf(T, Tinv, n);
    if (bestc < 0 || cnd < bestc) {
      bestc = cnd;
      bestT = T;
      bestTi = Tinv;
    }
  }
  if (bestc < 0) return false;
  T = bestT;
  Ti = bestTi;
  return bestc <= 64.0L;
}

// Composed step constants (StepConsts in adg_internal.h) of upwind advection with a > 0, in
// long double: from the SSP-RK3 stages in Shu and Osher's form, or, for the low-storage
// schemes (one to five stages), from their Butcher form (unused channels are zero).
void fold_step_constants(InstHost &h, bool allow_basis) {
  const Ops &o = h.ops;
  const int Np = o.Np;
  const ld c2a = advection_c2a(h);
  constexpr int CS = adg::kMaxCS;
  typedef std::vector<ld> Mat;
  auto mul = [&](const Mat &X, const Mat &Y) {
    Mat Z(Np * Np, 0);
    for (int i = 0; i < Np; ++i)
      for (int k = 0; k < Np; ++k)
        for (int j = 0; j < Np; ++j) Z[i * Np + j] += X[i * Np + k] * Y[k * Np + j];
    return Z;
  };
  auto mulv = [&](const Mat &X, const std::vector<ld> &v) {
    std::vector<ld> z(Np, 0);
    for (int i = 0; i < Np; ++i)
      for (int k = 0; k < Np; ++k) z[i] += X[i * Np + k] * v[k];
    return z;
  };
  const int p = Np - 1;
  // the step's constants: u'^e = G u^e + sum_t h_t P_t, channel scalars
  // Y_s p = r_s . u + sum_{t<s} k_st P_t, PE-face responses R and rho
  int S = 3;
  Mat Gl(Np * Np, 0);
  std::vector<ld> rl[CS], hl[CS];
  for (int s = 0; s < CS; ++s) {
    rl[s].assign(Np, 0);
    hl[s].assign(Np, 0);
  }
  ld kl[CS][CS] = {}, rhol[CS][CS] = {};
  ld Rl[CS][CS + 1][adg::kMaxNp] = {};

  if (h.cfg.rk == ADG_SSPRK3) {
    const ld alpha[3] = {0.0L, 0.75L, 1.0L / 3.0L};
    const ld beta[3] = {1.0L, 0.25L, 2.0L / 3.0L};
    Mat M[3];
    std::vector<ld> cv[3];
    for (int s = 0; s < 3; ++s) {
      M[s].assign(Np * Np, 0);
      cv[s].assign(Np, 0);
      for (int i = 0; i < Np; ++i) {
        const ld lL = beta[s] * c2a * o.Minv[i * Np + 0];
        for (int j = 0; j < Np; ++j)
          M[s][i * Np + j] = beta[s] * ((i == j ? 1.0L : 0.0L) + c2a * o.D[i * Np + j]);
        M[s][i * Np + 0] += lL;
        cv[s][i] = -lL;
      }
    }
    Mat M10 = mul(M[1], M[0]);
    Mat inner = M10;
    for (int i = 0; i < Np; ++i) inner[i * Np + i] += alpha[1];
    Gl = mul(M[2], inner);
    for (int i = 0; i < Np; ++i) Gl[i * Np + i] += alpha[2];
    hl[0] = mulv(mul(M[2], M[1]), cv[0]);
    hl[1] = mulv(M[2], cv[1]);
    hl[2] = cv[2];
    std::vector<ld> M1c0 = mulv(M[1], cv[0]);
    for (int i = 0; i < Np; ++i) {
      rl[1][i] = M[0][p * Np + i];
      rl[2][i] = M10[p * Np + i] + (i == p ? alpha[1] : 0.0L);
    }
    kl[1][0] = cv[0][p];
    kl[2][0] = M1c0[p];
    kl[2][1] = cv[1][p];
    // PE-face correction responses: inject lL_s at element e and lR_s at element e-1 after
    // stage s, then apply the remaining stages' perturbation maps
    // dx'^m = M_t dx^m + c_t dx^{m-1}_p (t = s+1 .. 2) on elements e-1 .. e+2; rho collects
    // the right trace of element e-1 seen by the later stages.
    for (int st = 0; st < 3; ++st) {
      std::vector<ld> d(4 * Np, 0.0L);   // elements e-1 .. e+2
      const ld sc = beta[st] * c2a;
      for (int i = 0; i < Np; ++i) {
        d[1 * Np + i] = sc * o.Minv[i * Np + 0];
        d[0 * Np + i] = -sc * o.Minv[i * Np + p];
      }
      for (int t = st + 1; t < 3; ++t) {
        rhol[t][st] = d[0 * Np + p];
        std::vector<ld> nd(4 * Np, 0.0L);
        for (int m = 0; m < 4; ++m)
          for (int i = 0; i < Np; ++i) {
            ld acc = 0;
            for (int k = 0; k < Np; ++k) acc += M[t][i * Np + k] * d[m * Np + k];
            if (m > 0) acc += cv[t][i] * d[(m - 1) * Np + p];
            nd[m * Np + i] = acc;
          }
        d = nd;
      }
      for (int m = 0; m < 4; ++m)
        for (int i = 0; i < Np; ++i) Rl[st][m][i] = d[m * Np + i];
    }
  } else {
    // Butcher form of a low-storage scheme: k_s = W Y_s + w P_s (stage s with all faces
    // synchronous, P_s = the left neighbour's Y_s trace), Y_s = u + sum_{j<s} a_sj k_j,
    // u' = u + sum_j b_j k_j. Every quantity is kept as A u + sum_t H_t P_t.
    ld a[adg::kMaxStages][adg::kMaxStages], b[adg::kMaxStages];
    two_register_butcher(h.cfg.rk, S, a, b);
    Mat W(Np * Np, 0);
    std::vector<ld> w(Np);
    for (int i = 0; i < Np; ++i) {
      for (int j = 0; j < Np; ++j)
        W[i * Np + j] = c2a * (o.D[i * Np + j] + (j == 0 ? o.Minv[i * Np + 0] : 0.0L));
      w[i] = -c2a * o.Minv[i * Np + 0];
    }
    Mat I(Np * Np, 0);
    for (int i = 0; i < Np; ++i) I[i * Np + i] = 1;
    struct Rep {
      Mat A;
      std::vector<ld> H[CS];
    };
    Rep Y[CS], Kr[CS];
    for (int s = 0; s < CS; ++s)
      for (int t = 0; t < CS; ++t) {
        Y[s].H[t].assign(Np, 0);
        Kr[s].H[t].assign(Np, 0);
      }
    Y[0].A = I;
    auto combine = [&](int s, const ld *coef) {   // I u + sum_{j<s} coef_j k_j
      Rep r;
      r.A = I;
      for (int t = 0; t < CS; ++t) r.H[t].assign(Np, 0);
      for (int j = 0; j < s; ++j) {
        for (int x = 0; x < Np * Np; ++x) r.A[x] += coef[j] * Kr[j].A[x];
        for (int t = 0; t < CS; ++t)
          for (int i = 0; i < Np; ++i) r.H[t][i] += coef[j] * Kr[j].H[t][i];
      }
      return r;
    };
    for (int s = 0; s < S; ++s) {
      Kr[s].A = mul(W, Y[s].A);
      for (int t = 0; t < CS; ++t) Kr[s].H[t] = mulv(W, Y[s].H[t]);
      for (int i = 0; i < Np; ++i) Kr[s].H[s][i] += w[i];
      if (s + 1 < S) Y[s + 1] = combine(s + 1, a[s + 1]);
    }
    Rep U = combine(S, b);
    Gl = U.A;
    for (int t = 0; t < S; ++t) hl[t] = U.H[t];
    for (int s = 1; s < S; ++s) {
      for (int i = 0; i < Np; ++i) rl[s][i] = Y[s].A[p * Np + i];
      for (int t = 0; t < s; ++t) kl[s][t] = Y[s].H[t][p];
    }
    // PE-face responses: the stage-st correction d enters k_st as c2a M^{-1} e_0 d at element e
    // and -c2a M^{-1} e_p d at element e-1 and spreads through the later stages on elements
    // e-1 .. e+S-1 (one element further per stage); rho is the right trace of element e-1's
    // later stage inputs.
    const int nw = S + 1;
    for (int st = 0; st < S; ++st) {
      std::vector<ld> dK[CS];
      for (auto &v : dK) v.assign((size_t)nw * Np, 0.0L);
      for (int i = 0; i < Np; ++i) {
        dK[st][1 * Np + i] = c2a * o.Minv[i * Np + 0];
        dK[st][0 * Np + i] = -c2a * o.Minv[i * Np + p];
      }
      for (int t = st + 1; t < S; ++t) {
        std::vector<ld> dY((size_t)nw * Np, 0.0L);
        for (int jj = st; jj < t; ++jj)
          for (int x = 0; x < nw * Np; ++x) dY[x] += a[t][jj] * dK[jj][x];
        rhol[t][st] = dY[0 * Np + p];
        for (int m = 0; m < nw; ++m)
          for (int i = 0; i < Np; ++i) {
            ld acc = 0;
            for (int k = 0; k < Np; ++k) acc += W[i * Np + k] * dY[m * Np + k];
            if (m > 0) acc += w[i] * dY[(m - 1) * Np + p];
            dK[t][m * Np + i] = acc;
          }
      }
      for (int m = 0; m < nw; ++m)
        for (int i = 0; i < Np; ++i) {
          ld acc = 0;
          for (int jj = st; jj < S; ++jj) acc += b[jj] * dK[jj][m * Np + i];
          Rl[st][m][i] = acc;
        }
    }
  }
  // the composed kernels keep S slots per ring level: three for schemes of up to three stages
  // (unused channels zero), five for the five-stage scheme
  h.I.ns = S <= 3 ? 3 : adg::kMaxCS;

  adg::StepConsts &Sc = h.I.st;
  std::memset(&Sc, 0, sizeof(Sc));
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) Sc.G[i * Np + j] = (double)Gl[i * Np + j];
  for (int s = 0; s < CS; ++s) {
    for (int i = 0; i < Np; ++i) {
      Sc.r[s][i] = (double)rl[s][i];
      Sc.h[s][i] = (double)hl[s][i];
    }
    for (int t = 0; t < CS; ++t) {
      Sc.k[s][t] = (double)kl[s][t];
      Sc.rho[s][t] = (double)rhol[s][t];
    }
    for (int m = 0; m <= CS; ++m)
      for (int i = 0; i < Np; ++i) Sc.R[s][m][i] = (double)Rl[s][m][i];
  }

  // The fixed-point step's coordinates: the block basis of the element operator for a single
  // instance where it is well conditioned (G block diagonal, h, R times T^-1, r times T), else
  // nodal values.
  h.I.basis = 0;
  h.I.fxh = 0;
  h.I.fxe = 0;
  std::memset(h.I.Tb, 0, sizeof(h.I.Tb));
  std::memset(h.I.Tbi, 0, sizeof(h.I.Tbi));
  std::vector<ld> Tm, Tim;
  bool basis = allow_basis && block_basis(o, Tm, Tim);
  Mat Gc = Gl;
  std::vector<ld> hc[CS], rc[CS];
  ld Rc[CS][CS + 1][adg::kMaxNp] = {};
  for (int s = 0; s < CS; ++s) {
    hc[s] = hl[s];
    rc[s] = rl[s];
    for (int m = 0; m <= CS; ++m)
      for (int i = 0; i < Np; ++i) Rc[s][m][i] = Rl[s][m][i];
  }
  int gshift[adg::kMaxNp / 2] = {};
  if (basis) {
    Gc = similar(Tim, Gl, Tm, Np);
    if (!block_diagonal(Gc, Np, 1e-13L)) basis = false;
  }
  if (basis) {
    // Within a 2 x 2 block two parameters of the basis are free: the trace-1 vector f may take
    // any multiple of its trace-0 partner g, and g any scale. f' = f + alpha g, g' = beta g
    // with alpha = -(G - I)_11 / (G - I)_12 and beta = 2^-k / (G - I)_12 make the block's first
    // row of G exactly (1, 2^-k) (k the nearest power of two, so beta is near 1): a row of
    // shifts and adds in the kernel.
    // The 3 x 3 block at p = 4 likewise: f' = f + a1 g1 + a2 g2 with (a1, a2) the smallest
    // solution of (G - I)_11 + (G - I)_12 a1 + (G - I)_13 a2 = 0, g1' = (n12 g1 + n13 g2)
    // 2^-k / |n|^2 and g2' = (n13 g1 - n12 g2) / |n|, n = ((G - I)_12, (G - I)_13): its first
    // row becomes (1, 2^-k, 0); where that basis is worse conditioned than allowed the triple
    // keeps its dense rows.
    auto shear = [&](bool triple, std::vector<ld> &Ts, std::vector<ld> &Tis, Mat &Gs, int *gsh) {
      Ts = Tm;
      gsh[0] = gsh[1] = 0;
      auto k_of = [](ld x) { return fabsl(x) > 0 ? (int)lroundl(-log2l(fabsl(x))) : -1; };
      for (int m = 0; m <= (Np == 4 ? 2 : 0); m += 2) {   // the 2 x 2 blocks
        const ld n11 = Gc[m * Np + m] - 1.0L, n12 = Gc[m * Np + m + 1];
        const int k = k_of(n12);
        if (k < 1 || k > 27) return false;
        const ld al = -n11 / n12, be = ldexpl(1.0L, -k) / n12;
        for (int r = 0; r < Np; ++r) {
          const ld f = Ts[r * Np + m], g = Ts[r * Np + m + 1];
          Ts[r * Np + m] = f + al * g;
          Ts[r * Np + m + 1] = be * g;
        }
        gsh[m / 2] = 29 - k;
      }
      if (triple) {
        const ld n11 = Gc[2 * Np + 2] - 1.0L, n12 = Gc[2 * Np + 3], n13 = Gc[2 * Np + 4];
        const ld nn2 = n12 * n12 + n13 * n13, nn = sqrtl(nn2);
        const int k = k_of(nn);
        if (k < 1 || k > 27) return false;
        const ld a1 = -n11 * n12 / nn2, a2 = -n11 * n13 / nn2, sc = ldexpl(1.0L, -k) / nn2;
        for (int r = 0; r < Np; ++r) {
          const ld f = Ts[r * Np + 2], g1 = Ts[r * Np + 3], g2 = Ts[r * Np + 4];
          Ts[r * Np + 2] = f + a1 * g1 + a2 * g2;
          Ts[r * Np + 3] = (n12 * g1 + n13 * g2) * sc;
          Ts[r * Np + 4] = (n13 * g1 - n12 * g2) / nn;
        }
        gsh[1] = 29 - k;
      }
      if (!invert(Ts, Np, Tis) || cond_inf(Ts, Tis, Np) > 64.0L) return false;
      Gs = similar(Tis, Gl, Ts, Np);
      bool rows = block_diagonal(Gs, Np, 1e-13L);
      for (int m = 0; m <= (Np >= 4 ? 2 : 0); m += 2) {
        if (m == 2 && Np == 5 && !triple) break;
        const ld t = ldexpl(1.0L, gsh[m / 2] - 29);
        rows = rows && fabsl(Gs[m * Np + m] - 1.0L) < 1e-15L &&
               fabsl(Gs[m * Np + m + 1] - t) < 1e-15L * t;
        if (m == 2 && Np == 5) rows = rows && fabsl(Gs[2 * Np + 4]) < 1e-15L * t;
      }
      return rows;
    };
    std::vector<ld> Ts, Tis;
    Mat Gs;
    int gsh[2] = {0, 0};
    const bool ok = (Np == 5 && shear(true, Ts, Tis, Gs, gsh)) || shear(false, Ts, Tis, Gs, gsh);
    if (ok) {
      Tm = Ts;
      Tim = Tis;
      Gc = Gs;
      gshift[0] = gsh[0];
      gshift[1] = gsh[1];
      for (int m = 0; m <= (Np >= 4 ? 2 : 0); m += 2) {
        if (gshift[m / 2] == 0) continue;   // the triple without its shear
        Gc[m * Np + m] = 1.0L;
        Gc[m * Np + m + 1] = ldexpl(1.0L, gshift[m / 2] - 29);
        if (m == 2 && Np == 5) Gc[2 * Np + 4] = 0.0L;
      }
    } else {
      basis = false;
    }
  }
  if (basis) {
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < Np; ++j)
        if (!same_block(i, j)) Gc[i * Np + j] = 0;
    auto times_ti = [&](const std::vector<ld> &v) {
      std::vector<ld> z(Np, 0.0L);
      for (int i = 0; i < Np; ++i)
        for (int k = 0; k < Np; ++k) z[i] += Tim[i * Np + k] * v[k];
      return z;
    };
    for (int s = 0; s < CS; ++s) {
      hc[s] = times_ti(hl[s]);
      for (int j = 0; j < Np; ++j) {
        ld a = 0;
        for (int i = 0; i < Np; ++i) a += rl[s][i] * Tm[i * Np + j];
        rc[s][j] = a;
      }
      for (int m = 0; m <= CS; ++m) {
        std::vector<ld> v(Rl[s][m], Rl[s][m] + Np);
        const std::vector<ld> z = times_ti(v);
        for (int i = 0; i < Np; ++i) Rc[s][m][i] = z[i];
      }
    }
  }

  // Fixed-point limbs of the same coefficients (from the long double values): C =
  // round(c 2^58) in balanced limbs C = ch 2^29 + cl (adg_fixed.cuh); every |c| < 2 keeps
  // both within 32 bits.
  adg::StepFixed &F = h.I.sf;
  std::memset(&F, 0, sizeof(F));
  bool ok = true;
  auto limbs = [&](ld c) {
    if (!(fabsl(c) < 1.999L)) ok = false;
    const long long C = ok ? llroundl(ldexpl(c, 58)) : 0;
    const long long cl = ((C + (1ll << 28)) & ((1ll << 29) - 1)) - (1ll << 28);
    int2 r;
    r.x = (int)((C - cl) >> 29);
    r.y = (int)cl;
    return r;
  };
  // Bounds of one fixed-point sum of terms c_m x_m whose multiplicands are below g_m 2^57,
  // so |xh| <= g 2^28 and 0 <= xl < 2^29: a = sum ch xh and b = 2^28 + sum (ch xl + cl xh)
  // below 2^62, and the result, below sum |c| g 2^57 + n, below 2^61.
  auto sum_ok = [&](const std::vector<std::pair<ld, ld>> &terms) {
    ld ab = 0, bb = ldexpl(1.0L, 28), rb = 0;
    for (auto &cg : terms) {
      const ld c = fabsl(cg.first), g = cg.second;
      const ld ch = c * ldexpl(1.0L, 29) + 1.0L, xh = g * ldexpl(1.0L, 28) + 1.0L;
      ab += ch * xh;
      bb += ch * ldexpl(1.0L, 29) + ldexpl(1.0L, 28) * xh;
      rb += c * g;
    }
    return ab < ldexpl(1.0L, 62) && bb < ldexpl(1.0L, 62) && rb < 15.9L;
  };
  // Inputs below 2^(57 - hb) (g = 2^-hb); the right trace, a sum of nb of them (nb = 1 for
  // nodal values, the number of blocks in the block basis); channel scalars Y_s below B_s 2^57
  // with B_s = sum |r_s| 2^-hb + |k_s0| g_0 + sum_{t>=1} |k_st| B_t. Nodal values keep the
  // bound B_s < 2 (multiplicands below 2^58); block-basis coordinates, whose channel scalars
  // are sums of about nb coordinates, take B_s < 7.9 (below 2^60, so the high limb
  // X >> 29 fits 32 bits), every sum then checked with its terms' own bounds. The smallest
  // headroom hb that passes every check (0 for nodal values).
  const int nb = basis ? (Np > 2 ? 2 : 1) : 1;
  auto checks = [&](int hb) {
    const ld gin = ldexpl(1.0L, -hb), g0 = nb * gin, blim = basis ? 7.9L : 1.999L;
    bool good = true;
    ld B[CS] = {g0};
    auto gch = [&](int t) { return basis ? B[t] : (t == 0 ? g0 : 2.0L); };
    for (int s = 1; s < S; ++s) {
      std::vector<std::pair<ld, ld>> sm;
      B[s] = 0;
      for (int i = 0; i < Np; ++i) {
        sm.push_back({rc[s][i], gin});
        B[s] += fabsl(rc[s][i]) * gin;
      }
      for (int t = 0; t < s; ++t) {
        sm.push_back({kl[s][t], gch(t)});
        B[s] += fabsl(kl[s][t]) * B[t];
      }
      good = good && sum_ok(sm) && B[s] < blim;
    }
    for (int i = 0; i < Np; ++i) {
      std::vector<std::pair<ld, ld>> row;
      for (int j = 0; j < Np; ++j)
        if (Gc[i * Np + j] != 0 || !basis) row.push_back({Gc[i * Np + j], gin});
      for (int t = 0; t < S; ++t) row.push_back({hc[t][i], gch(t)});
      good = good && sum_ok(row);
    }
    return good;
  };
  int hb = 0;
  while (hb < (basis ? 4 : 1) && !checks(hb)) ++hb;
  const bool sums = hb < (basis ? 4 : 1);
  for (int i = 0; i < Np; ++i) {
    for (int j = 0; j < Np; ++j) F.G[i * Np + j] = limbs(Gc[i * Np + j]);
    for (int t = 0; t < S; ++t) F.h[t][i] = limbs(hc[t][i]);
  }
  for (int s = 1; s < S; ++s) {
    for (int i = 0; i < Np; ++i) F.r[s][i] = limbs(rc[s][i]);
    for (int t = 0; t < s; ++t) F.k[s][t] = limbs(kl[s][t]);
  }
  h.fixed_ok = ok && sums;
  if (basis)
    for (int m = 0; m < 2; ++m) F.gs[m] = gshift[m];
  if (basis && h.fixed_ok) {
    // FP64 inputs: w = T^-1 u in FP64 is below ||T^-1||_inf 2^(E - 1022) (1 + 2^-40)
    ld nti = 0;
    for (int i = 0; i < Np; ++i) {
      ld a = 0;
      for (int j = 0; j < Np; ++j) a += fabsl(Tim[i * Np + j]);
      nti = std::max(nti, a);
    }
    h.I.basis = 1;
    h.I.fxh = hb;
    h.I.fxe = hb + (int)ceill(log2l(nti * (1.0L + ldexpl(1.0L, -40))));
    for (int i = 0; i < Np * Np; ++i) {
      h.I.Tb[i] = (double)Tm[i];
      h.I.Tbi[i] = (double)Tim[i];
    }
  }
  // the PE-face responses likewise (from the long double values), for the integer correction
  // of differences below 2^57
  std::memset(h.I.Rf, 0, sizeof(h.I.Rf));
  ok = true;
  bool rsums = true;
  for (int m = 0; m <= S; ++m)
    for (int i = 0; i < Np; ++i) {
      std::vector<std::pair<ld, ld>> row;
      for (int st = 0; st < S; ++st) {
        h.I.Rf[st][m][i] = limbs(Rc[st][m][i]);
        row.push_back({Rc[st][m][i], 1.0L});
      }
      rsums = rsums && sum_ok(row);
    }
  ok = ok && rsums;
  h.I.face_fx = ok ? 1 : 0;
}

int reduce(adg_ctx *c, InstHost &h, int kind, const double *g, double scale, double *host_out,
           const double *field = nullptr) {
  if (!c->partials) {
    // allocated at the first reduction (in adg_init that is the check of u0, after the
    // layout kernel has started reading it): 1024 partial sums and the result
    CK(cudaMalloc(&c->partials, 1025 * sizeof(double)));
    c->red_out = c->partials + 1024;
  }
  if (!c->pinned) CK(cudaMallocHost(&c->pinned, 8 * sizeof(double)));
  const int nb = adg::reduce_blocks(h.I.K);
  const double *wm = kind == 3 ? h.M : h.w;
  CK(adg::launch_reduce(kind, field ? field : h.I.u, g, h.I.K, h.I.Np, wm, scale, c->partials, nb,
                        c->red_out, c->stream));
  CK(cudaMemcpyAsync(c->pinned, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *host_out = c->pinned[0];
  return ADG_OK;
}

// Refill the device delay table of h with the rows of steps [first, first+TR).
int fill_table(adg_ctx *c, InstHost &h, int64_t first) {
  h.tbase = first;
  const DelaySource &d = h.delays;
  if (d.caller.empty()) {
    // seeded rows and the communication-avoiding cycle are generated on the device
    // seeded rows are generated on the device (the host generator's arithmetic, with the bin
    // edges as exact integer thresholds: u < e  <=>  (z >> 11) < ceil(e 2^53))
    adg::DelayGen g{};
    g.seed = d.seed;
    g.L = d.L;
    g.P = d.P;
    g.caa = d.caa;
    for (int b = 0; b < d.L; ++b) {
      const double t = std::ceil(std::ldexp(d.edges[b], 53));
      g.T[b] = t >= 18446744073709551616.0 ? ~0ull : (t <= 0 ? 0ull : (uint64_t)t);
    }
    CK(adg::launch_fill_delays(h.table, first, h.TR, g, c->stream));
  } else {
    h.host_rows.resize((size_t)h.TR * h.I.P);
    d.rows(first, h.TR, h.host_rows.data());
    CK(cudaMemcpyAsync(h.table, h.host_rows.data(), h.host_rows.size(), cudaMemcpyHostToDevice,
                       c->stream));
  }
  int64_t tb = first;
  CK(cudaMemcpyAsync((void *)(h.I.meta + 1), &tb, sizeof(int64_t), cudaMemcpyHostToDevice,
                     c->stream));
  return ADG_OK;
}

// Make the device delay table of h cover steps [n, n+count) (forward runs).
int ensure_table(adg_ctx *c, InstHost &h, int64_t n, int64_t count) {
  if (!h.I.async) return ADG_OK;
  if (n >= h.tbase && n + count <= h.tbase + h.TR) return ADG_OK;
  return fill_table(c, h, n);
}

// Make it cover step n for a sweep that runs backwards (the window ends at n).
int ensure_table_back(adg_ctx *c, InstHost &h, int64_t n) {
  if (!h.I.async) return ADG_OK;
  if (n >= h.tbase && n < h.tbase + h.TR) return ADG_OK;
  return fill_table(c, h, std::max<int64_t>(0, n - h.TR + 1));
}

// Scale slots of the fixed-point composed step for the current state: slot (n mod 3) gets
// the largest biased exponent of u^n (FP64), the other two are cleared.
// from_scan: u was just loaded, and the layout kernel's exponent in scan is taken instead
// of a pass over u.
int reset_exponent(adg_ctx *c, InstHost &h, bool from_scan = false) {
  if (h.I.fused != 2) return ADG_OK;
  if (from_scan) {
    CK(cudaMemsetAsync(h.fx, 0, 3 * sizeof(adg::FxSlot), c->stream));
    CK(cudaMemcpyAsync(&h.fx[(int)(c->n % 3)].E, c->scan, sizeof(int), cudaMemcpyDeviceToDevice,
                       c->stream));
    return ADG_OK;
  }
  CK(adg::launch_fixed_reset(h.I.u, (size_t)h.I.K * h.I.Np, h.fx, c->n, c->stream));
  return ADG_OK;
}

// Elements per thread of the composed-step kernel. The FP64 composed step times one, two and
// four on a copy of u0 held in the instance's v1/v2 fields (free at this point) and keeps the
// fastest; the fixed-point step takes two for even K, which measured faster in every timing
// of both (223.6 against 255.3 us per step on 2^24 elements), without timing them at init
// (a run's end-to-end cost includes adg_init). Every choice computes every element with the
// same arithmetic, so results do not depend on it.
int autotune_fused(adg_ctx *c, InstHost &h) {
  Inst &I = h.I;
  const size_t nd = (size_t)I.K * I.Np;
  if (h.cfg.ept > 0) {   // forced by the caller
    if (I.fused == 2 && (h.cfg.ept > 2 || (h.cfg.ept == 2 && I.K % 2)))
      return fail(c, ADG_EINVAL, "the fixed-point composed step takes ept 1, or 2 for even K");
    I.ept = h.cfg.ept;
    return ADG_OK;
  }
  if (I.K < 4 * 2 * adg::kTile) return ADG_OK;   // tiny meshes: one element per thread
  if (I.fused == 2) {
    I.ept = I.K % 2 ? 1 : 2;
    return ADG_OK;
  }
  CK(cudaMemcpyAsync(I.v1, I.u, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  int best_ept = 1;
  // Per choice one untimed launch, then two timed ones (the choices differ by about 10% on
  // large meshes, far above the event resolution; the autotuner runs inside adg_init, so it is
  // kept short).
  for (int ept = 1; ept <= 4; ept *= 2) {
    Inst T = I;
    T.ept = ept;
    CK(adg::launch_fused_step(T, I.v1, I.v2, 0, c->stream, false, 0));
    cudaEventRecord(a, c->stream);
    for (int k = 0; k < 2; ++k)
      CK(adg::launch_fused_step(T, k ? I.v1 : I.v2, k ? I.v2 : I.v1, 0, c->stream, false, 0));
    cudaEventRecord(b, c->stream);
    CK(cudaEventSynchronize(b));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) {
      best = ms;
      best_ept = ept;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  I.ept = best_ept;
  return ADG_OK;
}

int setup_instance(adg_ctx *c, InstHost &h, const adg_config *cfg, const double *u0,
                   int64_t *meta_slot, bool u0_host = false) {
  h.cfg = *cfg;
  if (cfg->probs) {
    h.probs.assign(cfg->probs, cfg->probs + cfg->L);
    h.cfg.probs = h.probs.data();
  }
  h.delays = make_delay_source(cfg);
  h.cfg.delay_table = nullptr;  // the DelaySource keeps the copy
  h.ops = make_ops(cfg->p);
  const int K = cfg->K, Np = cfg->p + 1;
  h.dx = (cfg->x1 - cfg->x0) / K;
  Inst &I = h.I;
  I.K = K;
  I.Np = Np;
  I.P = cfg->P;
  I.Kpe = K / cfg->P;
  I.pde = cfg->pde;
  I.a = cfg->pde == ADG_ADVECTION ? cfg->a : 0.0;
  I.async = (cfg->mode != ADG_SYNC && cfg->P > 1) ? 1 : 0;
  h.q_eff = cfg->mode == ADG_ASYNC_AT ? (cfg->at_order > 0 ? cfg->at_order : std::min(cfg->p + 1, ADG_MAX_Q)) : 1;
  I.q = h.q_eff;
  I.L = cfg->L;
  I.R = (cfg->L - 1) + h.q_eff;
  {
    const LsTable *lt = cfg->rk == ADG_SSPRK3 ? nullptr : ls_table(cfg->rk);
    I.ls = lt ? 1 : 0;
    I.ns = lt ? lt->S : kStages;
    h.stages = I.ns;
    for (int s = 0; s < adg::kMaxStages; ++s) {
      I.lsA[s] = lt && s < lt->S ? (double)((ld)lt->A[s].n / (ld)lt->A[s].d) : 0.0;
      I.lsB[s] = lt && s < lt->S ? (double)((ld)lt->B[s].n / (ld)lt->B[s].d) : 0.0;
    }
  }
  I.meta = meta_slot;
  I.visc = cfg->nu > 0 ? 1 : 0;
  I.nu = cfg->nu;
  I.euler = cfg->pde == ADG_EULER ? 1 : 0;
  if (I.euler) {
    // SSP Runge-Kutta in Shu and Osher's form (stage constants below), the limiter's weights
    I.ls = 0;
    I.ns = cfg->rk == ADG_RK1 ? 1 : (cfg->rk == ADG_RK2 ? 2 : 3);
    h.stages = I.ns;
    I.limiter = cfg->limiter;
    I.tvb_m = cfg->tvb_m;
    I.dx = h.dx;
    const Ops &o = h.ops;
    for (int j = 0; j < Np; ++j) {
      ld a = 0, b = 0;
      for (int i = 0; i < Np; ++i) {
        a += o.M[i * Np + j];
        b += o.M[j * Np + i] * o.x[i];
      }
      I.avg_w[j] = (double)(0.5L * a);
      I.p1_w[j] = (double)(1.5L * b);
      I.xi[j] = (double)o.x[j];
    }
  }
  if (I.visc || I.euler) {
    // q = (2/dx) [ D v + M^{-1} e_p (uhat_R - v_p) - M^{-1} e_0 (uhat_L - v_0) ]
    const Ops &o = h.ops;
    const ld s2 = 2.0L / (ld)h.dx;
    for (int i = 0; i < Np; ++i) {
      for (int j = 0; j < Np; ++j) I.QD[i * Np + j] = (double)(s2 * o.D[i * Np + j]);
      I.qlR[i] = (double)(s2 * o.Minv[i * Np + (Np - 1)]);
      I.qlL[i] = (double)(-s2 * o.Minv[i * Np + 0]);
    }
  }

  const size_t nd = (size_t)K * Np;
  if (I.visc) {
    CK(cudaMalloc(&h.qbuf, nd * sizeof(double)));
    I.qbuf = h.qbuf;
  }
  // u | v1 | v2 (| w: Euler's raw stage output under the limiter), ncomp components each
  const int ncomp = I.euler ? 3 : 1;
  const size_t fnd = ncomp * nd;
  const int nfields = (I.euler && I.limiter) ? 4 : 3;
  CK(cudaMalloc(&h.fields, nfields * fnd * sizeof(double)));
  I.u = h.fields;
  I.unext = h.fields;
  I.v1 = h.fields + fnd;
  I.v2 = h.fields + 2 * fnd;
  I.w = nfields == 4 ? h.fields + 3 * fnd : nullptr;
  // the initial field into node planes: from device memory, from pinned host memory over the
  // host link (the layout kernel reads it in place), or from pageable host memory through v1
  const double *src = u0;
  if (u0_host) {
    const void *view = nullptr;
    int r0 = host_view(c, u0, &view);
    if (r0) return r0;
    if (view) {
      src = static_cast<const double *>(view);
    } else {
      CK(cudaMemcpyAsync(I.v1, u0, fnd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      src = I.v1;
    }
  }
  // the layout kernel also raises scan to u0's largest biased exponent (its finiteness and
  // the fixed-point step's first scale, without another pass over u0)
  CK(cudaMemsetAsync(c->scan, 0, sizeof(int), c->stream));
  for (int comp = 0; comp < ncomp; ++comp)
    CK(adg::launch_to_internal(src + comp * nd, I.u + comp * nd, K, Np, c->stream, c->scan));
  CK(cudaMemsetAsync(I.v1, 0, (nfields - 1) * fnd * sizeof(double), c->stream));

  // weights and mass matrix for reductions, the ring's AT coefficients; uploaded (pageable
  // sources, which may wait for the stream) and u0 checked for NaN and Inf (a reduction read
  // on the host) where the setup first needs u0's values on the host: for the time step of
  // Burgers from max|u0|, else at the end, so that the host work in between overlaps the
  // layout kernel (which reads a host u0 over the host link)
  std::vector<double> wd(Np), Md(Np * Np), coef;
  for (int i = 0; i < Np; ++i) wd[i] = (double)h.ops.w[i];
  for (int i = 0; i < Np * Np; ++i) Md[i] = (double)h.ops.M[i];
  CK(cudaMalloc(&h.w, Np * sizeof(double)));
  CK(cudaMalloc(&h.M, Np * Np * sizeof(double)));
  auto upload_and_check = [&]() -> int {
    CK(cudaMemcpyAsync(h.w, wd.data(), Np * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(h.M, Md.data(), Np * Np * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    if (!coef.empty())
      CK(cudaMemcpyAsync(h.coef, coef.data(), coef.size() * sizeof(double),
                         cudaMemcpyHostToDevice, c->stream));
    if (!c->pinned) CK(cudaMallocHost(&c->pinned, 8 * sizeof(double)));
    int *emax = reinterpret_cast<int *>(c->pinned);
    CK(cudaMemcpyAsync(emax, c->scan, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (*emax >= 2047) return fail(c, ADG_EINVAL, "u0 holds NaN or Inf");
    return ADG_OK;
  };
  const bool dt_from_data = !(cfg->dt > 0) && cfg->pde == ADG_BURGERS;
  int r = ADG_OK;
  if (dt_from_data) {
    r = upload_and_check();
    if (r) return r;
  }

  if (cfg->dt > 0) {
    h.dt = cfg->dt;
  } else {
    double speed = std::fabs(cfg->a);
    if (cfg->pde == ADG_BURGERS) {
      r = reduce(c, h, 1, nullptr, 1.0, &speed);
      if (r) return r;
      if (!(speed > 0)) return fail(c, ADG_EINVAL, "Burgers needs max|u0| > 0 to set dt from cfl");
    }
    h.dt = (cfg->cfl * h.dx) / speed;
  }
  I.dt = h.dt;
  fold_constants(h);
  if (I.euler) {
    const double so[3][3][2] = {{{0.0, 1.0}}, {{0.0, 1.0}, {0.5, 0.5}},
                                {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}}};
    for (int s = 0; s < I.ns; ++s) {
      I.sc[s].alpha = so[I.ns - 1][s][0];
      I.sc[s].beta = so[I.ns - 1][s][1];
    }
  }
  {
    // the composed step: SSP-RK3, or a low-storage scheme (five stages: fixed point only).
    // With PE faces the correction windows of the composed step's S stages (elements e-S ..
    // e+S-1 of face e) must not overlap: K/P >= 8, and >= 10 for five stages.
    const int S = (I.ls && I.ns > kStages) ? adg::kMaxCS : kStages;
    const bool eligible = cfg->pde == ADG_ADVECTION && cfg->a > 0 && K >= 8 &&
                          (!I.async || I.Kpe >= (S == kStages ? 8 : 10)) &&
                          (!I.ls || I.ns <= adg::kMaxCS) && !I.visc && !I.euler;
    const bool want_composed = cfg->variant == ADG_VARIANT_COMPOSED ||
                               cfg->variant == ADG_VARIANT_COMPOSED_FIXED;
    if (want_composed && !eligible)
      return fail(c, ADG_EINVAL, "the composed step needs advection with a > 0, K >= 8 and "
                                 "K/P >= 8 (10 for the five-stage scheme)");
    if (cfg->variant == ADG_VARIANT_COMPOSED && S != kStages)
      return fail(c, ADG_EINVAL, "the FP64 composed step takes schemes of at most three "
                                 "stages; the five-stage scheme composes in fixed point");
    I.fused = (eligible && cfg->variant != ADG_VARIANT_STAGED) ? 1 : 0;
    I.ept = 1;
    const int ls0 = I.ls, ns0 = I.ns;
    if (I.fused) {
      I.ls = 0;
      // sets I.ns to the composed kernels' stage slots, and the block basis where it applies
      fold_step_constants(h, true);
      if (cfg->variant == ADG_VARIANT_COMPOSED_FIXED && !h.fixed_ok)
        return fail(c, ADG_EINVAL,
                    "the fixed-point composed step needs every composed coefficient "
                    "below 2 in magnitude (a smaller Courant number)");
      const bool fixed = h.fixed_ok && (cfg->variant == ADG_VARIANT_AUTO ||
                                        cfg->variant == ADG_VARIANT_COMPOSED_FIXED);
      if (!fixed && S != kStages) {
        // five stages without the fixed-point bounds: the staged 2N kernels
        I.fused = 0;
        I.ls = ls0;
        I.ns = ns0;
      }
    }
    if (I.fused) {
      const bool fixed = h.fixed_ok && (cfg->variant == ADG_VARIANT_AUTO ||
                                        cfg->variant == ADG_VARIANT_COMPOSED_FIXED);
      if (fixed) {
        I.fused = 2;
        CK(cudaMalloc(&h.fx, 3 * sizeof(adg::FxSlot)));
        I.fx = h.fx;
        if (I.async && !c->batch) {
          CK(cudaMalloc(&h.fd, (size_t)2 * I.P * I.ns * sizeof(double)));
          I.fd = h.fd;
        }
        int r2 = reset_exponent(c, h, true);
        if (r2) return r2;
      }
      if (!c->batch) {
        int r2 = autotune_fused(c, h);
        if (r2) return r2;
      }
    }
  }

  if (I.async) {
    const int q = h.q_eff, L = cfg->L;
    std::vector<double> cf((size_t)L * q * q, 0.0);
    for (int k = 0; k < L; ++k)
      for (int qe = 1; qe <= q; ++qe)
        for (int i = 0; i < qe; ++i) cf[((size_t)k * q + (qe - 1)) * q + i] = at_coef(k, qe, i);
    CK(cudaMalloc(&h.coef, cf.size() * sizeof(double)));
    I.coef = h.coef;
    if (dt_from_data)
      CK(cudaMemcpyAsync(h.coef, cf.data(), cf.size() * sizeof(double), cudaMemcpyHostToDevice,
                         c->stream));
    else
      coef = std::move(cf);   // uploaded with the weights below
    const size_t ring_n = (size_t)I.R * I.ns * I.P * (I.euler ? 3 : 1);
    CK(cudaMalloc(&h.ring, ring_n * sizeof(double2)));
    CK(cudaMemsetAsync(h.ring, 0, ring_n * sizeof(double2), c->stream));
    I.ring = h.ring;
    if (I.visc) {
      CK(cudaMalloc(&h.ringq, ring_n * sizeof(double)));
      CK(cudaMemsetAsync(h.ringq, 0, ring_n * sizeof(double), c->stream));
      I.ringq = h.ringq;
    }
    h.TR = std::max(512, 2 * c->G);
    CK(cudaMalloc(&h.table, (size_t)h.TR * I.P));
    I.table = h.table;
    I.table_rows = h.TR;
    h.tbase = -(int64_t)1 << 40;   // force a fill
  }
  if (!dt_from_data) return upload_and_check();
  return ADG_OK;
}

// Chunks of steps. The fixed-point step (single instance or batch) keeps the state in int64
// from step to step, across chunks and adg_step calls: the chunk kind is the field that
// holds the state when the chunk starts (0: u in FP64, 1: v1, 2: v2 in int64); every step
// writes the other int64 field, so a chunk of m steps from field k ends in fixed_end(k, m).
// Every other path reads and writes u (kind kChunkFP64). The FP64 field u is formed from the
// int64 state when something reads it (sync_state).
constexpr int kChunkFP64 = 3;
// Steps per directly launched chunk (at most half the delay-table window of 512 rows).
constexpr int kDirectChunk = 256;

int fixed_end(int from, int64_t m) {
  if (m == 0) return from;
  if (from == 0) return (m % 2) ? 1 : 2;
  return (m % 2) ? 3 - from : from;
}

// The context's steps run in fixed point (single instance or batch).
bool fixed_state(const adg_ctx *c) {
  return c->batch ? c->batch_fixed : c->inst[0].I.fused == 2;
}

// Writes the FP64 state of step n into every instance's u when it lives in int64 (after
// fixed-point steps); entry points that read u call it first.
int sync_state(adg_ctx *c) {
  if (!fixed_state(c) || c->fx_live == 0 || c->u_fresh) return ADG_OK;
  for (auto &h : c->inst) {
    const Inst &I = h.I;
    const long long *X = reinterpret_cast<const long long *>(c->fx_live == 1 ? I.v1 : I.v2);
    CK(adg::launch_fixed_to_fp64(I, X, c->n, c->stream));
  }
  c->u_fresh = true;
  return ADG_OK;
}

// Instance h's state as element-major FP64 rows in dst (device, pinned or managed memory):
// converted straight from the int64 state while that is newer than u (after fixed-point
// steps; the values sync_state would give, without writing u), else copied from u.
int state_rows(adg_ctx *c, InstHost &h, double *dst) {
  const Inst &I = h.I;
  if (fixed_state(c) && c->fx_live != 0 && !c->u_fresh) {
    const void *X = c->fx_live == 1 ? I.v1 : I.v2;
    CK(adg::launch_state_rows(I, X, true, c->n, dst, c->stream));
    return ADG_OK;
  }
  const size_t nd = (size_t)I.K * I.Np;
  for (int comp = 0; comp < (I.euler ? 3 : 1); ++comp)
    CK(adg::launch_state_rows(I, I.u + comp * nd, false, 0, dst + comp * nd, c->stream));
  return ADG_OK;
}

int launch_fused_steps(adg_ctx *c, int nsteps, int kind);

// Steps are launched directly (not through CUDA graphs) from 2^20 DOF in all: a step there
// takes hundreds of microseconds, and programmatic launches overlapped better outside a graph
// (0.2315 -> 0.2276 ms per fixed-point step on the 2^26-DOF mesh). Below, the host's launch
// rate is the bound: 2000 staged Burgers steps on 262144 DOF took 99.6 ms launched directly
// and 77.1 ms as graphs.
bool direct_launches(const adg_ctx *c) {
  int64_t dof = 0;
  for (const auto &h : c->inst) dof += (int64_t)h.I.K * h.I.Np;
  return dof >= (int64_t(1) << 20);
}

int launch_steps(adg_ctx *c, int nsteps, int kind = kChunkFP64) {
  if (!c->batch && c->inst[0].I.fused) return launch_fused_steps(c, nsteps, kind);
  if (c->batch && c->batch_fixed && c->bu && c->split && direct_launches(c)) {
    // the parts of the instances on the context's stream and the side streams (forked and
    // joined around the chunk); each part's chain as below
    const int k = c->bu->ept == 4 ? 2 : c->bu->ept - 1;
    CK(cudaEventRecord(c->fork_ev, c->stream));
    for (int q = 1; q < kBatchParts; ++q) CK(cudaStreamWaitEvent(c->side[q], c->fork_ev, 0));
    adg::BatchUniform part = *c->bu;
    int in = kind == kChunkFP64 ? 0 : kind;
    for (int rel = 0; rel < nsteps; ++rel) {
      const int out = in == 1 ? 2 : 1;
      const int fmt = (in != 0 ? adg::kFmtInFixed : 0) | adg::kFmtOutFixed;
      for (int q = 0; q < kBatchParts; ++q) {
        part.items_dev = c->lites_half[k][q];
        part.nitems = c->nlites_half[k][q];
        CK(adg::launch_batch_fused_step(c->insts_dev, c->work_dev, c->nwork, c->fflat_half[q],
                                        c->nflat_half[q], in, out, fmt, true, rel,
                                        q ? c->side[q] : c->stream, &part, rel > 0));
      }
      in = out;
    }
    for (int q = 1; q < kBatchParts; ++q) {
      CK(cudaEventRecord(c->join_ev[q], c->side[q]));
      CK(cudaStreamWaitEvent(c->stream, c->join_ev[q], 0));
    }
    CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
    return ADG_OK;
  }
  if (c->batch && c->batch_fixed) {
    // as launch_fused_steps: fields 0 (u, FP64), 1 and 2 (v1, v2, int64); each step carries
    // its own PE-face correction
    int in = kind == kChunkFP64 ? 0 : kind;
    for (int rel = 0; rel < nsteps; ++rel) {
      const int out = in == 1 ? 2 : 1;
      const int fmt = (in != 0 ? adg::kFmtInFixed : 0) | adg::kFmtOutFixed;
      // steps after the first are programmatic dependents of the fix-up (or step) before them
      CK(adg::launch_batch_fused_step(c->insts_dev, c->work_dev, c->nwork, c->fflat_dev, c->nflat,
                                      in, out, fmt, true, rel, c->stream, c->bu.get(), rel > 0));
      in = out;
    }
    CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
    return ADG_OK;
  }
  if (c->batch && c->batch_fused) {
    for (int rel = 0; rel < nsteps; ++rel)
      CK(adg::launch_batch_fused_step(c->insts_dev, c->work_dev, c->nwork, c->fflat_dev, c->nflat,
                                      rel % 2, 1 - rel % 2, 0, c->batch_fixed, rel, c->stream,
                                      c->batch_fixed ? c->bu.get() : nullptr));
    if (nsteps % 2) CK(adg::launch_batch_copy_back(c->insts_dev, c->work_dev, c->nwork, c->stream));
    CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
    return ADG_OK;
  }
  if (!c->batch && c->inst[0].I.euler) {
    // Euler: each stage from its input (u, v1, v2) into the raw buffer w and the limiter into
    // the stage's field (v1, v2; u for the last), or straight into it without the limiter (a
    // single stage goes through v1: it reads its input's neighbours)
    const Inst &I = c->inst[0].I;
    const size_t fbytes = 3 * (size_t)I.K * I.Np * sizeof(double);
    for (int rel = 0; rel < nsteps; ++rel) {
      for (int s = 0; s < I.ns; ++s) {
        double *dst = (s == I.ns - 1) ? I.u : (s == 0 ? I.v1 : I.v2);
        if (I.limiter) {
          CK(adg::launch_euler_stage(I, s, rel, I.w, c->stream));
          CK(adg::launch_euler_limit(I, I.w, dst, c->stream));
        } else if (I.ns == 1) {
          CK(adg::launch_euler_stage(I, 0, rel, I.v1, c->stream));
          CK(cudaMemcpyAsync(I.u, I.v1, fbytes, cudaMemcpyDeviceToDevice, c->stream));
        } else {
          CK(adg::launch_euler_stage(I, s, rel, dst, c->stream));
        }
      }
    }
    CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
    return ADG_OK;
  }
  if (!c->batch && c->inst[0].I.ls) {
    // 2N low-storage step: U_0 = u, dU in v1, U_s alternately in v2 and u (each stage reads
    // its input's neighbours, so it writes the other field); an odd stage count ends in v2
    const Inst &I = c->inst[0].I;
    for (int rel = 0; rel < nsteps; ++rel) {
      const double *in = I.u;
      for (int s = 0; s < I.ns; ++s) {
        double *out = (s % 2 == 0) ? I.v2 : I.u;
        if (I.visc) CK(adg::launch_ldg_q(I, in, s, rel, c->stream));
        CK(adg::launch_lsrk_stage(I, s, rel, in, out, c->stream));
        in = out;
      }
      if (I.ns % 2)
        CK(cudaMemcpyAsync(I.u, I.v2, (size_t)I.K * I.Np * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
    return ADG_OK;
  }
  for (int rel = 0; rel < nsteps; ++rel) {
    for (int s = 0; s < kStages; ++s) {
      if (c->batch) {
        CK(adg::launch_batch_stage(c->insts_dev, c->work_dev, c->nwork, s, rel, adg::kTile, c->stream));
        if (c->nfwork > 0)
          CK(adg::launch_batch_faces(c->insts_dev, c->fwork_dev, c->nfwork, s, rel, c->stream));
      } else {
        const Inst &I = c->inst[0].I;
        if (I.visc) CK(adg::launch_ldg_q(I, s == 0 ? I.u : (s == 1 ? I.v1 : I.v2), s, rel, c->stream));
        // a programmatic dependent of the stage before it on runs launched without graphs
        // (the first of the chunk follows other work; the viscous stage follows its q pass).
        // Inside the graphs of small runs programmatic launches measured slower (the adjoint
        // workload's forward 78 -> 95 ms), on the 2^20-element Burgers mesh 1.6% faster.
        CK(adg::launch_stage(I, s, rel, c->stream,
                             direct_launches(c) && !I.visc && (rel > 0 || s > 0)));
      }
    }
  }
  CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
  return ADG_OK;
}

// Composed steps. FP64: they ping-pong between u and v1; an odd count ends with a copy back
// into u. Fixed point: the chunk reads the state from the field its kind names (u in FP64 or
// v1 / v2 in int64) and alternates v1 and v2.
int launch_fused_steps(adg_ctx *c, int nsteps, int kind) {
  const Inst &I = c->inst[0].I;
  if (I.fused == 2) {
    // With PE faces, one face kernel before the chunk's first step forms its differences,
    // one between consecutive steps adds the earlier step's correction and forms the next
    // step's differences, and one after the last step adds its correction, so that the int64
    // state is complete at the end of every chunk.
    const bool faces = I.async != 0;
    if (faces && !I.fd)
      return fail(c, ADG_EINVAL, "internal: fixed-point step with PE faces lacks its buffer");
    const int from = kind == kChunkFP64 ? 0 : kind;
    void *in = from == 0 ? static_cast<void *>(I.u) : (from == 1 ? static_cast<void *>(I.v1)
                                                                 : static_cast<void *>(I.v2));
    int cur = from, fin_prev = 1;
    for (int rel = 0; rel < nsteps; ++rel) {
      const int nxt = cur == 1 ? 2 : 1;
      void *out = nxt == 1 ? static_cast<void *>(I.v1) : static_cast<void *>(I.v2);
      const bool fin = cur != 0;
      const int fmt = (fin ? adg::kFmtInFixed : 0) | adg::kFmtOutFixed;
      // Within the chunk every kernel after the first is a programmatic dependent of the one
      // before it (launch_maybe_pdl): its blocks start while that one drains.
      if (faces) {
        if (rel == 0)
          CK(adg::launch_face_step(I, in, 0, fin ? 1 : 0, 0, adg::kFaceDiff, c->stream));
        else
          CK(adg::launch_face_step(I, in, rel, 1, fin_prev, adg::kFaceApply | adg::kFaceDiff,
                                   c->stream, true));
      }
      CK(adg::launch_fixed_step(I, in, out, rel, fmt, c->stream, faces || rel > 0));
      fin_prev = fin ? 1 : 0;
      in = out;
      cur = nxt;
    }
    if (faces && nsteps > 0)
      CK(adg::launch_face_step(I, in, nsteps, 1, fin_prev, adg::kFaceApply, c->stream, true));
  } else {
    for (int rel = 0; rel < nsteps; ++rel) {
      const double *uin = (rel % 2 == 0) ? I.u : I.v1;
      double *uout = (rel % 2 == 0) ? I.v1 : I.u;
      CK(adg::launch_fused_step(I, uin, uout, rel, c->stream));
    }
    if (nsteps % 2)
      CK(cudaMemcpyAsync(I.u, I.v1, (size_t)I.K * I.Np * sizeof(double), cudaMemcpyDeviceToDevice,
                         c->stream));
  }
  CK(adg::launch_advance(c->meta, 2, (int)c->inst.size(), nsteps, c->stream));
  return ADG_OK;
}

int build_graph(adg_ctx *c, int kind) {
  cudaStream_t user = c->stream;
  c->stream = c->cap;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    c->stream = user;
    return fail(c, ADG_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  int r = launch_steps(c, c->G, kind);
  cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
  c->stream = user;
  if (r) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e2 != cudaSuccess) return fail(c, ADG_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&c->gexec[kind], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec[kind] = nullptr;
    return fail(c, ADG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  return ADG_OK;
}

int begin_ctx(adg_ctx *c, void *stream) {
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1)
    return fail(c, ADG_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  CK(cudaGetDevice(&c->device));
  c->stream = (cudaStream_t)stream;
  CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  return ADG_OK;
}

// Device memory owned for the duration of one adg_grad call.
struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  double *d() const { return static_cast<double *>(p); }
};

int dev_alloc(adg_ctx *c, DevBuf &b, size_t bytes) {
  if (bytes == 0) return ADG_OK;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return fail(c, ADG_ENOMEM, std::string("adg_grad: cudaMalloc: ") + cudaGetErrorString(e));
  }
  return ADG_OK;
}

int set_step(adg_ctx *c, InstHost &h, int64_t n) {
  int64_t v = n;
  CK(cudaMemcpyAsync((void *)h.I.meta, &v, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  c->n = n;
  return ADG_OK;
}

// Graph of one segment sweep, captured on the context's capture stream.
struct GraphExec {
  cudaGraphExec_t g = nullptr;
  ~GraphExec() {
    if (g) cudaGraphExecDestroy(g);
  }
};

template <class F>
int capture(adg_ctx *c, GraphExec &out, F &&body) {
  cudaStream_t user = c->stream;
  c->stream = c->cap;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    c->stream = user;
    return fail(c, ADG_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  int r = body();
  cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
  c->stream = user;
  if (r) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e2 != cudaSuccess) return fail(c, ADG_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&out.g, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    out.g = nullptr;
    return fail(c, ADG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  return ADG_OK;
}

// Forward over one segment of `len` steps starting at meta[0], recording the stage inputs
// of step t in slot t of `seg` (u^n, v1, v2); slot t+1's u receives u^{n+1}, so slot 0's u
// must hold the segment's first state and slot len's u holds the last.
// rel0 shifts the step indices: a segment that starts rel0 steps after meta[0] (the
// overlapped recompute runs the segment before the one meta[0] names, rel0 = -len).
int sweep_recompute(adg_ctx *c, InstHost &h, double *seg, int len, int rel0 = 0) {
  const size_t nd = (size_t)h.I.K * h.I.Np;
  for (int t = 0; t < len; ++t) {
    double *slot = seg + (size_t)t * kStages * nd;
    Inst I = h.I;
    I.u = slot;
    I.v1 = slot + nd;
    I.v2 = slot + 2 * nd;
    I.unext = slot + kStages * nd;
    for (int s = 0; s < kStages; ++s) {
      CK(adg::launch_stage(I, s, rel0 + t, c->stream));
    }
  }
  return ADG_OK;
}

// Adjoint sweep over one segment, steps len-1 .. 0 after meta[0]; lam[0..1] hold the
// adjoint of u at the segment's end on entry (index `par`) and of u at its start on exit.
int sweep_reverse(adg_ctx *c, InstHost &h, const double *seg, double *lam, double *lring, int len,
                  int par) {
  Inst &I = h.I;
  const size_t nd = (size_t)I.K * I.Np;
  const int dir = I.a >= 0.0 ? 1 : -1;
  double *Lv = lam + 2 * nd, *Lv2 = lam + 3 * nd;
  for (int t = len - 1; t >= 0; --t) {
    double *Lu = lam + (size_t)par * nd, *Lacc = lam + (size_t)(1 - par) * nd;
    const double *slot = seg ? seg + (size_t)t * kStages * nd : nullptr;
    for (int s = kStages - 1; s >= 0; --s) {
      adg::AdjStage A;
      A.w = s == 2 ? Lu : (s == 1 ? Lv : Lv2);
      A.v = slot ? slot + (size_t)s * nd : nullptr;
      A.lv = s == 2 ? Lv : (s == 1 ? Lv2 : nullptr);
      A.lacc = Lacc;
      A.K = I.K;
      A.Np = I.Np;
      A.C = I.sc[s];
      A.lring = lring;
      A.table = I.table;
      A.meta = I.meta;
      A.coef = I.coef;
      A.rel = t;
      A.stage = s;
      A.P = I.P;
      A.Kpe = I.Kpe;
      A.R = I.R;
      A.q = I.q;
      A.faces = (I.async && I.Kpe >= 8) ? 1 : 0;
      CK(adg::launch_adj_stage(A, I.pde, s, dir, c->stream));
      if (I.async && !A.faces) {
        adg::AdjFace F;
        F.w = A.w;
        F.v = A.v;
        F.target = s == 0 ? Lacc : A.lv;
        F.lring = lring;
        F.table = I.table;
        F.meta = I.meta;
        F.coef = I.coef;
        F.rel = t;
        F.K = I.K;
        F.Np = I.Np;
        F.P = I.P;
        F.Kpe = I.Kpe;
        F.R = I.R;
        F.q = I.q;
        F.stage = s;
        for (int i = 0; i < adg::kMaxNp; ++i) {
          F.lL[i] = I.sc[s].lL[i];
          F.lR[i] = I.sc[s].lR[i];
        }
        CK(adg::launch_adj_faces(F, I.pde, dir, c->stream));
      }
    }
    par = 1 - par;
  }
  return ADG_OK;
}

// Second stream and events of the overlapped recompute (released on every exit path).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t meta_set = nullptr, rec_done = nullptr;
  ~SideStream() {
    if (meta_set) cudaEventDestroy(meta_set);
    if (rec_done) cudaEventDestroy(rec_done);
    if (s) cudaStreamDestroy(s);
  }
};

// adg_grad: forward with checkpoints every C steps, misfit, then segments in reverse: restore
// the checkpoint, recompute the segment recording the stage inputs (Burgers; the linear
// advection adjoint needs no forward state), and run the adjoint stages from the last step
// of the segment to its first. The state of the context is restored at the end.
//
// Burgers with two or more segments: the recompute of segment s-1 runs on a second stream
// into a second segment buffer while the adjoint of segment s runs on the context's stream
// (the two share only read-only data, the delay table and meta[0]; the recompute's step
// indices are taken relative to segment s's start, so meta[0] changes only once both are
// done). Order per segment s on the context's stream: wait for the recompute of s, refill
// the delay table if it does not cover steps [start(s) - C, end(s)), set meta[0] = start(s),
// record `meta_set`, run the adjoint of s; on the second stream: wait for `meta_set` (which
// also orders it after the adjoint of s+1, the last reader of the buffer it overwrites),
// restore checkpoint s-1 and its ring, recompute s-1, record `rec_done`. Without room for
// the second buffer, or with 2C larger than the delay table, segments run one after the
// other on the context's stream.
int run_gradient(adg_ctx *c, const double *target_dev, int64_t nsteps, int C, double *grad_dev,
                 double *J_out) {
  InstHost &h = c->inst[0];
  Inst &I = h.I;
  const int K = I.K, Np = I.Np;
  const size_t nd = (size_t)K * Np;
  const int64_t n0 = c->n;
  const int64_t nseg = nsteps == 0 ? 0 : (nsteps + C - 1) / C;
  const bool states = I.pde == ADG_BURGERS;
  const int64_t nck = states ? nseg : std::min<int64_t>(nseg, 1);
  const size_t ring_n = I.async ? (size_t)I.R * kStages * I.P : 0;
  const int dir = I.a >= 0.0 ? 1 : -1;

  DevBuf g, ck_u, ck_ring, seg, lam, lring, ck_fx;
  // the fixed-point state (int64 field and its scale slots) is put back exactly at the end
  const int live0 = c->fx_live;
  int r = ADG_OK;
  if (live0) {
    r = dev_alloc(c, ck_fx, nd * sizeof(long long) + 3 * sizeof(adg::FxSlot));
    if (r) return r;
    CK(cudaMemcpyAsync(ck_fx.p, live0 == 1 ? I.v1 : I.v2, nd * sizeof(long long),
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(static_cast<char *>(ck_fx.p) + nd * sizeof(long long), I.fx,
                       3 * sizeof(adg::FxSlot), cudaMemcpyDeviceToDevice, c->stream));
  }
  r = dev_alloc(c, g, nd * sizeof(double));
  if (!r) r = dev_alloc(c, ck_u, (size_t)nck * nd * sizeof(double));
  if (!r) r = dev_alloc(c, ck_ring, (size_t)nck * ring_n * sizeof(double2));
  if (!r && states) r = dev_alloc(c, seg, ((size_t)C * kStages + 1) * nd * sizeof(double));
  if (!r) r = dev_alloc(c, lam, 4 * nd * sizeof(double));
  if (!r) r = dev_alloc(c, lring, ring_n * sizeof(double));
  if (r) return r;
  CK(adg::launch_to_internal(target_dev, g.d(), K, Np, c->stream));

  // Forward pass with checkpoints (u^n and the forward ring at each segment start). The last
  // segment's stage inputs are recorded on the way, so it is not recomputed.
  GraphExec rec_full, rec_last;
  const int64_t last_len = nseg > 0 ? nsteps - (nseg - 1) * C : 0;
  for (int64_t sidx = 0; sidx < nseg; ++sidx) {
    if (sidx < nck) {
      CK(cudaMemcpyAsync(ck_u.d() + sidx * nd, I.u, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      if (ring_n)
        CK(cudaMemcpyAsync(static_cast<double2 *>(ck_ring.p) + sidx * ring_n, I.ring,
                           ring_n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    }
    const int len = (int)std::min<int64_t>(C, nsteps - sidx * C);
    if (states && sidx == nseg - 1) {
      r = ensure_table(c, h, c->n, len);
      if (!r) r = set_step(c, h, c->n);
      if (r) return r;
      CK(cudaMemcpyAsync(seg.d(), I.u, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      GraphExec &ge = len == C ? rec_full : rec_last;
      r = capture(c, ge, [&] { return sweep_recompute(c, h, seg.d(), len); });
      if (r) return r;
      CK(cudaGraphLaunch(ge.g, c->stream));
      CK(cudaMemcpyAsync(I.u, seg.d() + (size_t)len * kStages * nd, nd * sizeof(double),
                         cudaMemcpyDeviceToDevice, c->stream));
      r = set_step(c, h, c->n + len);
      if (r) return r;
    } else {
      r = adg_step(c, len);
      if (r) return r;
    }
  }
  double J = 0.0;
  r = sync_state(c);
  if (!r) r = reduce(c, h, 3, g.d(), 0.5 * (h.dx / 2.0), &J);
  if (r) return r;

  CK(adg::launch_adj_init(I.u, g.d(), K, Np, h.M, h.dx / 2.0, lam.d(), c->stream));
  if (ring_n) CK(cudaMemsetAsync(lring.p, 0, ring_n * sizeof(double), c->stream));

  // Overlapped recompute: a second segment buffer and stream when there is room for them.
  DevBuf seg2;
  SideStream side;
  bool overlap = states && nseg >= 2 && (!I.async || 2 * (int64_t)C <= h.TR);
  if (overlap) {
    if (cudaMalloc(&seg2.p, ((size_t)C * kStages + 1) * nd * sizeof(double)) != cudaSuccess) {
      seg2.p = nullptr;
      (void)cudaGetLastError();   // clear the failed allocation; run segments serially
      overlap = false;
    }
  }
  if (overlap) {
    CK(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&side.meta_set, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&side.rec_done, cudaEventDisableTiming));
  }
  double *segb[2] = {seg.d(), seg2.d()};

  // Segment sweeps replay graphs captured once per (segment length, buffer parity, segment
  // buffer); the overlapped recompute has one graph per segment buffer.
  GraphExec rev[2][2][2], rec_prev[2];
  int par = 0, cur = 0;
  for (int64_t sidx = nseg - 1; sidx >= 0; --sidx) {
    const int64_t start = n0 + sidx * C;
    const int len = (int)std::min<int64_t>(C, nsteps - sidx * C);
    const bool is_last = sidx == nseg - 1 && last_len != C;
    if (overlap) {
      if (sidx != nseg - 1) CK(cudaStreamWaitEvent(c->stream, side.rec_done, 0));
      if (I.async) {
        const int64_t lo = sidx > 0 ? start - C : start, hi = start + len;
        if (!(lo >= h.tbase && hi <= h.tbase + h.TR)) {
          r = fill_table(c, h, std::max<int64_t>(0, hi - h.TR));
          if (r) return r;
        }
      }
      r = set_step(c, h, start);
      if (r) return r;
      if (sidx > 0) {
        // recompute of segment sidx-1 (full length C) into the other buffer
        double *nb = segb[1 - cur];
        CK(cudaEventRecord(side.meta_set, c->stream));
        CK(cudaStreamWaitEvent(side.s, side.meta_set, 0));
        CK(cudaMemcpyAsync(nb, ck_u.d() + (sidx - 1) * nd, nd * sizeof(double),
                           cudaMemcpyDeviceToDevice, side.s));
        if (ring_n)
          CK(cudaMemcpyAsync(I.ring, static_cast<double2 *>(ck_ring.p) + (sidx - 1) * ring_n,
                             ring_n * sizeof(double2), cudaMemcpyDeviceToDevice, side.s));
        GraphExec &gp = rec_prev[1 - cur];
        if (!gp.g) {
          r = capture(c, gp, [&] { return sweep_recompute(c, h, nb, C, -C); });
          if (r) return r;
        }
        CK(cudaGraphLaunch(gp.g, side.s));
        CK(cudaEventRecord(side.rec_done, side.s));
      }
    } else {
      r = ensure_table(c, h, start, len);
      if (r) return r;
      r = set_step(c, h, start);
      if (r) return r;
      if (states && sidx != nseg - 1) {
        CK(cudaMemcpyAsync(seg.d(), ck_u.d() + sidx * nd, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        if (ring_n)
          CK(cudaMemcpyAsync(I.ring, static_cast<double2 *>(ck_ring.p) + sidx * ring_n,
                             ring_n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        GraphExec &ge = is_last ? rec_last : rec_full;
        if (!ge.g) {
          r = capture(c, ge, [&] { return sweep_recompute(c, h, seg.d(), len); });
          if (r) return r;
        }
        CK(cudaGraphLaunch(ge.g, c->stream));
      }
    }
    double *sb = states ? segb[cur] : nullptr;
    GraphExec &gr = rev[is_last ? 1 : 0][par][cur];
    if (!gr.g) {
      r = capture(c, gr, [&] { return sweep_reverse(c, h, sb, lam.d(), lring.d(), len, par); });
      if (r) return r;
    }
    CK(cudaGraphLaunch(gr.g, c->stream));
    if (len % 2) par = 1 - par;
    if (overlap) cur = 1 - cur;
  }
  double *Lu = lam.d() + (size_t)par * nd;
  CK(adg::launch_to_external(Lu, grad_dev, K, Np, c->stream));
  if (nseg > 0) {
    CK(cudaMemcpyAsync(I.u, ck_u.d(), nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (ring_n)
      CK(cudaMemcpyAsync(I.ring, ck_ring.p, ring_n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    r = set_step(c, h, n0);
    if (!r) r = reset_exponent(c, h);
    if (r) return r;
    c->fx_live = live0;
    c->u_fresh = true;
    if (live0) {
      CK(cudaMemcpyAsync(live0 == 1 ? I.v1 : I.v2, ck_fx.p, nd * sizeof(long long),
                         cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(I.fx, static_cast<char *>(ck_fx.p) + nd * sizeof(long long),
                         3 * sizeof(adg::FxSlot), cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  *J_out = J;
  return ADG_OK;
}

}  // namespace

namespace adg {
void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }
void lgl_weights(int p, double *w) {
  Ops o = make_ops(p);
  for (int i = 0; i <= p; ++i) w[i] = (double)o.w[i];
}
}  // namespace adg

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

void adg_config_default(adg_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->pde = ADG_ADVECTION;
  cfg->flux = ADG_UPWIND;
  cfg->rk = ADG_SSPRK3;
  cfg->K = 64;
  cfg->p = 2;
  cfg->P = 1;
  cfg->x0 = 0.0;
  cfg->x1 = 6.283185307179586;
  cfg->a = 1.0;
  cfg->cfl = 0.1;
  cfg->mode = ADG_SYNC;
  cfg->L = 1;
  cfg->limiter = 1;
}

int adg_comm_stats(const adg_ctx *c, int32_t index, int64_t *steps_out, int64_t *exchanges_out,
                   int64_t *sync_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (index < 0 || index >= (int)c->inst.size()) return fail(nullptr, ADG_EINVAL, "bad instance index");
  const InstHost &h = c->inst[index];
  const int64_t n = c->n;
  const int64_t per_step = h.I.async ? (int64_t)h.stages * h.I.P : 0;
  int64_t comm = n;
  if (h.delays.caa > 0) {   // whole periods, then the partial one
    const int64_t per = h.delays.caa + h.delays.L;
    comm = (n / per) * h.delays.caa + std::min<int64_t>(n % per, h.delays.caa);
  }
  if (steps_out) *steps_out = n;
  if (exchanges_out) *exchanges_out = comm * per_step;
  if (sync_out) *sync_out = n * per_step;
  return ADG_OK;
}

const char *adg_last_error(const adg_ctx *c) {
  return c ? c->err.c_str() : g_last_error.c_str();
}

void adg_destroy(adg_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto &ge : c->gexec)
    if (ge) cudaGraphExecDestroy(ge);
  for (auto &h : c->inst) {
    cudaFree(h.fields);
    cudaFree(h.ring);
    cudaFree(h.table);
    cudaFree(h.coef);
    cudaFree(h.w);
    cudaFree(h.M);
    cudaFree(h.fx);
    cudaFree(h.fd);
    cudaFree(h.qbuf);
    cudaFree(h.ringq);
  }
  cudaFree(c->meta);
  cudaFree(c->insts_dev);
  for (auto *l : c->lites_ept) cudaFree(l);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  for (auto e : c->join_ev)
    if (e) cudaEventDestroy(e);
  for (auto st : c->side)
    if (st) cudaStreamDestroy(st);
  cudaFree(c->work_dev);
  cudaFree(c->fwork_dev);
  cudaFree(c->fflat_dev);
  cudaFree(c->partials);   // red_out lies inside it
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

static int init_one(const adg_config *cfg, const double *u0, bool u0_host, void *stream,
                    adg_ctx **out) {
  if (!out) return fail(nullptr, ADG_EINVAL, "out is NULL");
  *out = nullptr;
  std::string bad = check_config(cfg);
  if (!bad.empty()) return fail(nullptr, ADG_EINVAL, bad);
  if (!u0) return fail(nullptr, ADG_EINVAL, u0_host ? "u0_host is NULL" : "u0_dev is NULL");
  adg_ctx *c = new (std::nothrow) adg_ctx();
  if (!c) return fail(nullptr, ADG_ENOMEM, "host allocation failed");
  int r = begin_ctx(c, stream);
  if (!r) {
    if (cudaMalloc(&c->meta, 3 * sizeof(int64_t)) != cudaSuccess)
      r = fail(c, ADG_ENOMEM, "cudaMalloc(meta)");
    else if (cudaMemsetAsync(c->meta, 0, 3 * sizeof(int64_t), c->stream) != cudaSuccess)
      r = fail(c, ADG_ECUDA, "cudaMemsetAsync(meta)");
    else
      c->scan = reinterpret_cast<int *>(c->meta + 2);
  }
  if (!r) {
    c->inst.resize(1);
    r = setup_instance(c, c->inst[0], cfg, u0, c->meta, u0_host);
  }
  if (!r) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) r = fail(c, ADG_ECUDA, cudaGetErrorString(e));
  }
  if (r) {
    g_last_error = c->err;
    adg_destroy(c);
    return r;
  }
  *out = c;
  return ADG_OK;
}

int adg_init(const adg_config *cfg, const double *u0_dev, void *stream, adg_ctx **out) {
  return init_one(cfg, u0_dev, false, stream, out);
}

int adg_init_host(const adg_config *cfg, const double *u0_host, void *stream, adg_ctx **out) {
  return init_one(cfg, u0_host, true, stream, out);
}

// Batch state at step 0 from the callers' initial fields (after the tuner's timing steps): u
// from u0, step counters and rings cleared, delay tables refilled on the next step, scale slots
// of the fixed-point step reset.
int reset_batch(adg_ctx *c, const double *const *u0_devs) {
  const int n = (int)c->inst.size();
  CK(cudaMemsetAsync(c->meta, 0, 2 * sizeof(int64_t) * n, c->stream));
  for (int i = 0; i < n; ++i) {
    InstHost &h = c->inst[i];
    CK(adg::launch_to_internal(u0_devs[i], h.I.u, h.I.K, h.I.Np, c->stream));
    if (h.ring)
      CK(cudaMemsetAsync(h.ring, 0, (size_t)h.I.R * h.I.ns * h.I.P * sizeof(double2), c->stream));
    h.tbase = -(int64_t)1 << 40;
    if (h.fx) CK(adg::launch_fixed_reset(h.I.u, (size_t)h.I.K * h.I.Np, h.fx, 0, c->stream));
  }
  c->n = 0;
  c->fx_live = 0;
  c->u_fresh = true;
  return ADG_OK;
}

// Selects the kind of batched step (2: fixed point, 1: FP64 composed, 0: staged) and the
// elements per thread of the fixed-point kernel, and uploads the instances' descriptors.
int apply_batch_kind(adg_ctx *c, int kind, int ept) {
  c->batch_fused = kind >= 1;
  c->batch_fixed = kind == 2;
  std::vector<Inst> hi;
  for (auto &h : c->inst) {
    h.I.fused = kind;
    h.I.ept = kind == 2 ? ept : 1;
    hi.push_back(h.I);
  }
  if (kind == 2 && c->bu) {
    const int k = ept == 4 ? 2 : ept - 1;
    c->bu->items_dev = c->lites_ept[k];
    c->bu->nitems = c->nlites_ept[k];
    c->bu->ept = ept;

  }
  CK(cudaMemcpy(c->insts_dev, hi.data(), sizeof(Inst) * hi.size(), cudaMemcpyHostToDevice));
  return ADG_OK;
}

// The batch autotuner: every kind of step all instances admit (or the one their configs
// force) and, for the fixed-point step with shared coefficients, work items of 256, 512 and
// 1024 elements (one, two or four per thread; or the forced ept), timed over four steps after
// two untimed ones on the batch itself; the fastest is kept and the state is reset to the
// initial fields. Batches below 2^20 elements skip the timing and take fixed point, else the
// FP64 composed step, else the staged kernels, with two elements per thread.
int tune_batch(adg_ctx *c, const double *const *u0_devs) {
  struct Cand {
    int kind, ept;
  };
  int maxkind = 2, forced = -1, ept_forced = 0;
  int64_t elements = 0;
  for (auto &h : c->inst) {
    maxkind = std::min(maxkind, h.I.fused);
    if (h.cfg.variant == ADG_VARIANT_STAGED) forced = 0;
    if (h.cfg.variant == ADG_VARIANT_COMPOSED) forced = 1;
    if (h.cfg.variant == ADG_VARIANT_COMPOSED_FIXED) forced = 2;
    if (h.cfg.ept) ept_forced = h.cfg.ept;
    elements += h.I.K;
  }
  std::vector<Cand> cands;
  for (int kind = maxkind; kind >= 0; --kind) {
    if (forced >= 0 && kind != forced) continue;
    if (kind == 2 && c->bu) {
      for (int ept : {2, 1, 4})
        if ((!ept_forced || ept == ept_forced) && (ept != 2 || c->batch_even))
          cands.push_back({kind, ept});
    } else {
      cands.push_back({kind, 1});
    }
  }
  if (cands.empty()) return fail(c, ADG_EINVAL, "no kind of batched step fits every instance");
  Cand best = cands[0];
  if (cands.size() > 1 && elements >= (1 << 20)) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best_ms = 1e30f;
    int r = ADG_OK;
    for (const Cand &cd : cands) {
      r = apply_batch_kind(c, cd.kind, cd.ept);
      if (!r) r = reset_batch(c, u0_devs);
      for (auto &h : c->inst)
        if (!r) r = ensure_table(c, h, 0, 6);
      if (!r) r = launch_steps(c, 2, kChunkFP64);
      if (r) break;
      cudaEventRecord(a, c->stream);
      r = launch_steps(c, 4, cd.kind == 2 ? fixed_end(0, 2) : kChunkFP64);
      if (r) break;
      cudaEventRecord(b, c->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) {
        r = fail(c, ADG_ECUDA, "batch tuner: cudaEventSynchronize");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best_ms) {
        best_ms = ms;
        best = cd;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r) return r;
  }
  int r = apply_batch_kind(c, best.kind, best.ept);
  if (!r) r = reset_batch(c, u0_devs);
  return r;
}

int adg_batch_init(const adg_config *cfgs, const double *const *u0_devs, int32_t n, void *stream,
                   adg_ctx **out) {
  if (!out) return fail(nullptr, ADG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || !u0_devs || n < 1) return fail(nullptr, ADG_EINVAL, "need n >= 1 configs and fields");
  for (int i = 0; i < n; ++i) {
    std::string bad = check_config(&cfgs[i]);
    if (!bad.empty()) return fail(nullptr, ADG_EINVAL, "instance " + std::to_string(i) + ": " + bad);
    if (cfgs[i].pde != ADG_ADVECTION) return fail(nullptr, ADG_EINVAL, "batched runs take advection instances");
    if (!u0_devs[i]) return fail(nullptr, ADG_EINVAL, "u0_devs[i] is NULL");
  }
  adg_ctx *c = new (std::nothrow) adg_ctx();
  if (!c) return fail(nullptr, ADG_ENOMEM, "host allocation failed");
  c->batch = true;
  int r = begin_ctx(c, stream);
  if (!r) {
    cudaError_t e = cudaMalloc(&c->meta, sizeof(int64_t) * (2 * n + 1));
    if (e != cudaSuccess) r = fail(c, ADG_ENOMEM, "cudaMalloc(meta)");
    else if (cudaMemsetAsync(c->meta, 0, sizeof(int64_t) * (2 * n + 1), c->stream) != cudaSuccess)
      r = fail(c, ADG_ECUDA, "cudaMemsetAsync(meta)");
    else
      c->scan = reinterpret_cast<int *>(c->meta + 2 * n);
  }
  if (!r) {
    c->inst.resize(n);
    for (int i = 0; i < n && !r; ++i) r = setup_instance(c, c->inst[i], &cfgs[i], u0_devs[i], c->meta + 2 * i);
  }
  if (!r) {
    std::vector<Inst> hi(n);
    std::vector<int2> work, fwork, fflat;
    // the kinds of step every instance admits (a batch runs one kind for all instances):
    // fixed point, the FP64 composed step, the staged kernels; a variant forced by the
    // instances' configs leaves only that kind
    bool all_fixed = true, all_fused = true;
    int forced = ADG_VARIANT_AUTO, ept_forced = 0;
    for (int i = 0; i < n && !r; ++i) {
      const InstHost &h = c->inst[i];
      all_fused = all_fused && h.I.fused;
      all_fixed = all_fixed && h.I.fused == 2;
      if (h.cfg.rk != ADG_SSPRK3)
        r = fail(c, ADG_EINVAL, "instance " + std::to_string(i) + ": batches need rk = ADG_SSPRK3");
      else if (h.I.visc || h.I.euler)
        r = fail(c, ADG_EINVAL, "instance " + std::to_string(i) + ": batches take the inviscid scalar equations");
      const int v = h.cfg.variant;
      if (!r && v != ADG_VARIANT_AUTO) {
        if (forced != ADG_VARIANT_AUTO && forced != v)
          r = fail(c, ADG_EINVAL, "instances of one batch force different variants");
        forced = v;
      }
      if (!r && h.cfg.ept) {
        if (ept_forced && ept_forced != h.cfg.ept)
          r = fail(c, ADG_EINVAL, "instances of one batch force different ept");
        ept_forced = h.cfg.ept;
      }
    }
    if (!r && forced == ADG_VARIANT_COMPOSED_FIXED && !all_fixed)
      r = fail(c, ADG_EINVAL, "the fixed-point composed step needs every instance of the batch to admit it");
    if (!r && forced == ADG_VARIANT_COMPOSED && !all_fused)
      r = fail(c, ADG_EINVAL, "the composed step needs every instance of the batch to admit it");
    // the parts of the instances: largest first, each to the part with the fewest DOF
    std::vector<int> half(n, 0), order(n);
    {
      for (int i = 0; i < n; ++i) order[i] = i;
      auto dof = [&](int i) { return (int64_t)c->inst[i].I.K * c->inst[i].I.Np; };
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dof(a) > dof(b); });
      int64_t load[kBatchParts] = {};
      for (int i : order) {
        int best = 0;
        for (int q = 1; q < kBatchParts; ++q)
          if (load[q] < load[best]) best = q;
        half[i] = best;
        load[best] += dof(i);
      }
    }
    // the FP64 composed step of instances that admit fixed point (their I.fused is 2)
    for (int i = 0; i < n && !r; ++i) {
      InstHost &h = c->inst[i];
      h.I.ept = 1;
      hi[i] = h.I;
      for (int e0 = 0; e0 < hi[i].K; e0 += adg::kTile) work.push_back(make_int2(i, e0));
      if (hi[i].async)
        for (int j0 = 0; j0 < hi[i].P; j0 += 256) fwork.push_back(make_int2(i, j0));
    }
    int nflat_part[kBatchParts] = {};
    for (int hh = 0; hh < kBatchParts; ++hh)
      for (int i = 0; i < n; ++i)
        if (half[i] == hh && hi[i].async) {
          for (int j = 0; j < hi[i].P; ++j) fflat.push_back(make_int2(i, j));
          nflat_part[hh] += hi[i].P;
        }
    // every instance of a degree with the same fixed-point coefficients: pass them per degree,
    // with one record per work item of ept tiles (ept elements per thread)
    if (!r && all_fixed) {
      bool uniform = true;
      const Inst *ref[adg::kMaxNp - 1] = {nullptr, nullptr, nullptr, nullptr};
      for (int i = 0; i < n && uniform; ++i) {
        const Inst &I = c->inst[i].I;
        const int d = I.Np - 2;
        if (!ref[d]) ref[d] = &I;
        else
          uniform = std::memcmp(&ref[d]->sf, &I.sf, sizeof(I.sf)) == 0 &&
                    ref[d]->basis == I.basis && ref[d]->fxh == I.fxh && ref[d]->fxe == I.fxe &&
                    std::memcmp(ref[d]->Tbi, I.Tbi, sizeof(I.Tbi)) == 0;
      }
      if (uniform) {
        c->bu.reset(new (std::nothrow) adg::BatchUniform());
        if (!c->bu) r = fail(c, ADG_ENOMEM, "host allocation failed");
        for (int k = 0; k < 3 && !r; ++k) {
          const int ept = 1 << k;
          if (ept_forced && ept != ept_forced) continue;
          std::vector<adg::BatchLite> lites;
          int nlite_part[kBatchParts] = {};
          for (int hh = 0; hh < kBatchParts; ++hh)
          for (int i = 0; i < n; ++i) {
            if (half[i] != hh) continue;
            const Inst &I = c->inst[i].I;
            nlite_part[hh] += (I.K + ept * adg::kTile - 1) / (ept * adg::kTile);
            for (int e0 = 0; e0 < I.K; e0 += ept * adg::kTile) {
              adg::BatchLite L;
              L.f[0] = I.u;
              L.f[1] = I.v1;
              L.f[2] = I.v2;
              L.meta = I.meta;
              L.fx = I.fx;
              L.K = I.K;
              L.Np = I.Np;
              L.e0 = e0;
              L.pad = 0;
              lites.push_back(L);
            }
          }
          if (cudaMalloc(&c->lites_ept[k], sizeof(adg::BatchLite) * lites.size()) != cudaSuccess ||
              cudaMemcpy(c->lites_ept[k], lites.data(), sizeof(adg::BatchLite) * lites.size(),
                         cudaMemcpyHostToDevice) != cudaSuccess)
            r = fail(c, ADG_ENOMEM, "cudaMalloc(batch records)");
          c->nlites_ept[k] = (int)lites.size();
          int off = 0;
          for (int q = 0; q < kBatchParts; ++q) {
            c->lites_half[k][q] = c->lites_ept[k] + off;
            c->nlites_half[k][q] = nlite_part[q];
            off += nlite_part[q];
          }
        }
        // the parts' streams and fork / join events (batches of at least kBatchParts)
        if (!r && n >= kBatchParts) {
          bool ok = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
          for (int q = 1; q < kBatchParts && ok; ++q)
            ok = cudaStreamCreateWithFlags(&c->side[q], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->join_ev[q], cudaEventDisableTiming) == cudaSuccess;
          if (!ok) r = fail(c, ADG_ENOMEM, "batch side streams");
          c->split = ok;
        }
        if (!r) {
          std::memset(&c->bu->uf, 0, sizeof(c->bu->uf));
          for (int d = 0; d < adg::kMaxNp - 1; ++d)
            if (ref[d]) {
              adg::UniformFixed &uf = c->bu->uf;
              uf.sf[d] = ref[d]->sf;
              uf.basis[d] = ref[d]->basis;
              uf.fxh[d] = ref[d]->fxh;
              uf.fxe[d] = ref[d]->fxe;
              std::memcpy(uf.Tbi[d], ref[d]->Tbi, sizeof(uf.Tbi[d]));
            }
        }
      }
    }
    bool all_even = true;
    for (int i = 0; i < n; ++i) all_even = all_even && c->inst[i].I.K % 2 == 0;
    c->batch_even = all_even;
    if (!r && ept_forced && ept_forced != 1 && !(all_fixed && c->bu && forced != ADG_VARIANT_COMPOSED &&
                                                  forced != ADG_VARIANT_STAGED))
      r = fail(c, ADG_EINVAL, "ept > 1 in a batch needs the fixed-point step with shared coefficients");
    if (!r && ept_forced == 2 && !all_even)
      r = fail(c, ADG_EINVAL, "ept 2 in a batch needs an even K in every instance");
    c->nwork = (int)work.size();
    c->nfwork = (int)fwork.size();
    c->nflat = (int)fflat.size();
    if (!r && (cudaMalloc(&c->fflat_dev, sizeof(int2) * std::max<size_t>(1, fflat.size())) != cudaSuccess ||
               (!fflat.empty() && cudaMemcpy(c->fflat_dev, fflat.data(), sizeof(int2) * fflat.size(),
                                             cudaMemcpyHostToDevice) != cudaSuccess)))
      r = fail(c, ADG_ENOMEM, "cudaMalloc(batch face list)");
    {
      int off = 0;
      for (int q = 0; q < kBatchParts; ++q) {
        c->fflat_half[q] = c->fflat_dev + off;
        c->nflat_half[q] = nflat_part[q];
        off += nflat_part[q];
      }
    }
    if (cudaMalloc(&c->insts_dev, sizeof(Inst) * n) != cudaSuccess ||
        cudaMalloc(&c->work_dev, sizeof(int2) * work.size()) != cudaSuccess ||
        cudaMalloc(&c->fwork_dev, sizeof(int2) * std::max<size_t>(1, fwork.size())) != cudaSuccess)
      r = fail(c, ADG_ENOMEM, "cudaMalloc(batch descriptors)");
    else if (cudaMemcpy(c->insts_dev, hi.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(c->work_dev, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             (!fwork.empty() && cudaMemcpy(c->fwork_dev, fwork.data(), sizeof(int2) * fwork.size(), cudaMemcpyHostToDevice) != cudaSuccess))
      r = fail(c, ADG_ECUDA, "cudaMemcpy(batch descriptors)");
  }
  if (!r) r = tune_batch(c, u0_devs);
  if (!r && cudaStreamSynchronize(c->stream) != cudaSuccess) r = fail(c, ADG_ECUDA, "sync");
  if (r) {
    g_last_error = c->err;
    adg_destroy(c);
    return r;
  }
  *out = c;
  return ADG_OK;
}

int adg_step(adg_ctx *c, int64_t nsteps) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(c, ADG_EINVAL, "nsteps must be >= 0");
  // the fixed-point step carries its int64 state from chunk to chunk and call to call
  const bool carry = fixed_state(c);
  // CUDA graphs of G steps where launches dominate; larger runs launch chunks of up to
  // kDirectChunk steps directly (direct_launches)
  const bool graphs = !direct_launches(c);
  int64_t left = nsteps;
  while (left > 0) {
    const int chunk = (int)std::min<int64_t>(left, graphs ? c->G : kDirectChunk);
    const int kind = carry ? c->fx_live : kChunkFP64;
    for (auto &h : c->inst) {
      int r = ensure_table(c, h, c->n, chunk);
      if (r) return r;
    }
    if (graphs && chunk == c->G) {
      if (!c->gexec[kind]) {
        int r = build_graph(c, kind);
        if (r) return r;
      }
      CK(cudaGraphLaunch(c->gexec[kind], c->stream));
    } else {
      int r = launch_steps(c, chunk, kind);
      if (r) return r;
    }
    if (carry) {
      c->fx_live = fixed_end(kind, chunk);
      c->u_fresh = false;
    }
    c->n += chunk;
    left -= chunk;
  }
  return ADG_OK;
}

int adg_run(adg_ctx *c, double t_end) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (!std::isfinite(t_end)) return fail(c, ADG_EINVAL, "t_end must be finite");
  const double dt = c->inst[0].dt;
  const int64_t target = (int64_t)std::ceil(t_end / dt - 1e-9);
  return target > c->n ? adg_step(c, target - c->n) : ADG_OK;
}

int adg_get_state(adg_ctx *c, int32_t index, double *u_dev, int64_t *step_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (index < 0 || index >= (int)c->inst.size()) return fail(c, ADG_EINVAL, "bad instance index");
  if (!u_dev) return fail(c, ADG_EINVAL, "u_dev is NULL");
  {
    int r0 = state_rows(c, c->inst[index], u_dev);
    if (r0) return r0;
  }
  CK(cudaStreamSynchronize(c->stream));
  if (step_out) *step_out = c->n;
  return ADG_OK;
}

int adg_get_state_host(adg_ctx *c, int32_t index, double *u_host, int64_t *step_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (index < 0 || index >= (int)c->inst.size()) return fail(c, ADG_EINVAL, "bad instance index");
  if (!u_host) return fail(c, ADG_EINVAL, "u_host is NULL");
  const void *view = nullptr;
  {
    int r0 = host_view(c, u_host, &view);
    if (r0) return r0;
  }
  InstHost &h = c->inst[index];
  const size_t n = (size_t)(h.I.euler ? 3 : 1) * h.I.K * h.I.Np;
  // pinned memory: the rows kernel writes it over the host link; pageable memory: through
  // the field that holds no state (v2 while the fixed-point state is in v1, else v1) and one
  // copy
  double *dst = view ? static_cast<double *>(const_cast<void *>(view))
                     : (c->fx_live == 1 ? h.I.v2 : h.I.v1);
  {
    int r0 = state_rows(c, h, dst);
    if (r0) return r0;
  }
  if (!view)
    CK(cudaMemcpyAsync(u_host, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (step_out) *step_out = c->n;
  return ADG_OK;
}

int adg_get_dt(adg_ctx *c, int32_t index, double *dt_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (index < 0 || index >= (int)c->inst.size() || !dt_out) return fail(c, ADG_EINVAL, "bad argument");
  *dt_out = c->inst[index].dt;
  return ADG_OK;
}

int adg_get_variant(adg_ctx *c, int32_t index, int32_t *variant_out, int32_t *ept_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (index < 0 || index >= (int)c->inst.size()) return fail(c, ADG_EINVAL, "bad argument");
  const Inst &I = c->inst[index].I;
  if (variant_out)
    *variant_out = I.fused == 2 ? ADG_VARIANT_COMPOSED_FIXED
                                : (I.fused == 1 ? ADG_VARIANT_COMPOSED : ADG_VARIANT_STAGED);
  if (ept_out) *ept_out = I.fused ? I.ept : 1;
  return ADG_OK;
}

int adg_get_fixed_basis(adg_ctx *c, int32_t index, int32_t *basis_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (index < 0 || index >= (int)c->inst.size() || !basis_out)
    return fail(c, ADG_EINVAL, "bad argument");
  const Inst &I = c->inst[index].I;
  *basis_out = ((c->batch ? c->batch_fixed : I.fused == 2) && I.basis) ? 1 : 0;
  return ADG_OK;
}

int adg_integral(adg_ctx *c, int32_t index, double *out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  {
    int r0 = sync_state(c);
    if (r0) return r0;
  }
  if (index < 0 || index >= (int)c->inst.size() || !out) return fail(c, ADG_EINVAL, "bad argument");
  InstHost &h = c->inst[index];
  return reduce(c, h, 0, nullptr, h.dx / 2.0, out);
}

int adg_misfit(adg_ctx *c, int32_t index, const double *target_dev, double *J_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  {
    int r0 = sync_state(c);
    if (r0) return r0;
  }
  if (index < 0 || index >= (int)c->inst.size() || !target_dev || !J_out)
    return fail(c, ADG_EINVAL, "bad argument");
  InstHost &h = c->inst[index];
  const size_t nd = (size_t)h.I.K * h.I.Np;
  DevBuf g;
  int r = dev_alloc(c, g, nd * sizeof(double));
  if (r) return r;
  CK(adg::launch_to_internal(target_dev, g.d(), h.I.K, h.I.Np, c->stream));
  return reduce(c, h, 3, g.d(), 0.5 * (h.dx / 2.0), J_out);
}

int adg_check_finite(adg_ctx *c) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  {
    int r0 = sync_state(c);
    if (r0) return r0;
  }
  for (size_t i = 0; i < c->inst.size(); ++i) {
    InstHost &h = c->inst[i];
    for (int comp = 0; comp < (h.I.euler ? 3 : 1); ++comp) {
      double cnt = 0;
      int r = reduce(c, h, 2, nullptr, 1.0, &cnt, h.I.u + (size_t)comp * h.I.K * h.I.Np);
      if (r) return r;
      if (cnt != 0) return fail(c, ADG_ENONFINITE, "instance " + std::to_string(i) + " holds NaN or Inf");
    }
  }
  return ADG_OK;
}

int adg_delay_table(const adg_config *cfg, int64_t first_step, int64_t steps, uint8_t *out_host) {
  std::string bad = check_config(cfg);
  if (!bad.empty()) return fail(nullptr, ADG_EINVAL, bad);
  if (first_step < 0 || steps < 0 || (steps > 0 && !out_host)) return fail(nullptr, ADG_EINVAL, "bad range or NULL output");
  make_delay_source(cfg).rows(first_step, steps, out_host);
  return ADG_OK;
}

int adg_eval_modes(const adg_config *cfg, int32_t nmodes, const double *amp, const double *kappa,
                   const double *phase, double offset, double *u_dev, void *stream) {
  std::string bad = check_config(cfg);
  if (!bad.empty()) return fail(nullptr, ADG_EINVAL, bad);
  if (nmodes < 0 || nmodes > 16) return fail(nullptr, ADG_EINVAL, "nmodes must be in 0..16");
  if (nmodes > 0 && (!amp || !kappa || !phase)) return fail(nullptr, ADG_EINVAL, "NULL mode arrays");
  if (!u_dev) return fail(nullptr, ADG_EINVAL, "u_dev is NULL");
  Ops o = make_ops(cfg->p);
  double xi[kMaxNp];
  for (int i = 0; i <= cfg->p; ++i) xi[i] = (double)o.x[i];
  const double dx = (cfg->x1 - cfg->x0) / cfg->K;
  cudaError_t e = adg::launch_eval_modes(u_dev, cfg->K, cfg->p + 1, cfg->x0, dx, xi, nmodes, amp,
                                         kappa, phase, offset, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, ADG_ECUDA, std::string("eval_modes: ") + cudaGetErrorString(e));
  return ADG_OK;
}

int adg_lgl_nodes(int32_t p, double *nodes_host, double *weights_host) {
  if (p < 1 || p > ADG_MAX_P) return fail(nullptr, ADG_EINVAL, "p must be in 1..4");
  Ops o = make_ops(p);
  for (int i = 0; i <= p; ++i) {
    if (nodes_host) nodes_host[i] = (double)o.x[i];
    if (weights_host) weights_host[i] = (double)o.w[i];
  }
  return ADG_OK;
}

int adg_grad(adg_ctx *c, const double *target_dev, int64_t nsteps, int32_t ckpt_every,
             double *grad_u0_dev, double *J_out) {
  if (!c) return fail(nullptr, ADG_EINVAL, "ctx is NULL");
  if (c->batch) return fail(c, ADG_ESTATE, "adg_grad takes a single-instance context");
  if (c->inst[0].cfg.rk != ADG_SSPRK3) return fail(c, ADG_EINVAL, "adg_grad needs rk = ADG_SSPRK3");
  if (c->inst[0].I.visc || c->inst[0].I.euler)
    return fail(c, ADG_EINVAL, "adg_grad covers the inviscid scalar equations");
  if (nsteps < 0 || ckpt_every < 1) return fail(c, ADG_EINVAL, "need nsteps >= 0 and ckpt_every >= 1");
  if (!target_dev || !grad_u0_dev || !J_out) return fail(c, ADG_EINVAL, "NULL target, gradient or J");
  int r = sync_state(c);
  if (r) return r;
  return run_gradient(c, target_dev, nsteps, ckpt_every, grad_u0_dev, J_out);
}

}  // extern "C"
