// adg_integral_noalloc: the discrete integral of a caller's nodal field computed with a
// fixed scratch area that lives inside the library, for callers that cannot allocate
// device memory at the point of the call (see include/adg.h).
#include "adg.h"
#include "adg_internal.h"

#include <cmath>
#include <mutex>
#include <string>

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;   // partial sums held by the scratch area
constexpr int kMaxDevices = 64;

// The scratch area: one partial sum per block of the first pass. Every GPU that loads the
// library holds these 8 KiB until the process exits; all calls share them.
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks];

std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};

struct Weights {
  double w[adg::kMaxNp];
};

// First pass: grid-stride sums over elements of w^T u^e, u row-major (K, Np).
__global__ void __launch_bounds__(kThreads)
    k_integral_rowmajor(const double *__restrict__ u, int K, int Np, Weights wt, double *partials) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < Np; ++i) s = fma(wt.w[i], u[(size_t)e * Np + i], s);
    acc += s;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Second pass: one block adds the partials of this call in a fixed order.
__global__ void __launch_bounds__(kThreads)
    k_integral_final(const double *partials, int n, double scale, double *out) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) acc += partials[t];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

int fail(int code, const std::string &msg) {
  adg::set_last_error(msg.c_str());
  return code;
}

// Device address of the scratch area for the current device, looked up once per device
// (cudaGetSymbolAddress with that device current) and cached.
int scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ADG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(ADG_ECUDA, "device index beyond the scratch table");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      return fail(ADG_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch[dev] = static_cast<double *>(p);
  }
  *out = g_scratch[dev];
  return ADG_OK;
}

}  // namespace

extern "C" int adg_integral_noalloc(int32_t p, int32_t K, double dx, const double *u_dev,
                                    double *out_dev, void *stream) {
  if (p < 1 || p > ADG_MAX_P) return fail(ADG_EINVAL, "adg_integral_noalloc: p must be in 1..4");
  if (K < 1 || K > (1 << 30)) return fail(ADG_EINVAL, "adg_integral_noalloc: K must be in 1..2^30");
  if (!(dx > 0.0 && std::isfinite(dx)))
    return fail(ADG_EINVAL, "adg_integral_noalloc: dx must be finite and > 0");
  if (!u_dev || !out_dev) return fail(ADG_EINVAL, "adg_integral_noalloc: NULL field or output");
  double *scratch = nullptr;
  int r = scratch_for_current_device(&scratch);
  if (r) return r;
  Weights wt{};
  adg::lgl_weights(p, wt.w);
  int blocks = (K + kThreads - 1) / kThreads;
  if (blocks > kMaxBlocks) blocks = kMaxBlocks;
  cudaStream_t s = (cudaStream_t)stream;
  // Every block of the first pass writes its partial, so no clearing is needed: the second
  // pass reads exactly the partials this call wrote.
  k_integral_rowmajor<<<blocks, kThreads, 0, s>>>(u_dev, K, p + 1, wt, scratch);
  k_integral_final<<<1, kThreads, 0, s>>>(scratch, blocks, dx / 2.0, out_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ADG_ECUDA, std::string("adg_integral_noalloc launch: ") + cudaGetErrorString(e));
  return ADG_OK;
}
