// hfx_term_noalloc: one exchange term contracted with no device allocation.
//
// Some callers cannot allocate device memory when they call into this
// library: a host framework that owns the GPU's memory through its own pool
// and forbids direct cudaMalloc, a latency-critical loop where cudaMalloc /
// cudaFree (which can synchronize the device) are not allowed, or a process
// whose device memory is already fully reserved by another allocator so that a
// new allocation would fail.  hfx_build allocates its working memory inside
// the context; this entry point does not.  It evaluates the same staged
// product as the build's Y, D-stage and final contraction kernels, but keeps
// its two intermediates in the fixed static array below instead of allocated
// scratch.  The caller passes inputs and the output as device pointers.
#include <algorithm>
#include <mutex>

#include "hfx_internal.h"

namespace {

// Two intermediates of at most kHalf doubles each (2 MiB in total).  Every GPU
// that loads the library holds this array until the process exits.
constexpr int64_t kHalf = 131072;
static __device__ __align__(256) double g_noalloc_scratch[2 * kHalf];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the CUDA context the address was looked up in (its process-wide
// unique id, 0 = none yet) and the address.  A static __device__ array has one
// copy per context, so a cached address is only valid in the context it came
// from: after cudaDeviceReset (a new primary context) or under another context
// made current with the driver API, the address is looked up again.
unsigned long long g_scratch_ctx[kMaxDevices] = {0};
double *g_scratch_ptr[kMaxDevices] = {nullptr};

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Id of the current context (0 when none is current or the driver calls are
// unavailable; the lookup then runs on every call).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = (CtxGetCurrentFn)f1;
      get_id = (CtxGetIdFn)f2;
    }
    resolved = true;
  }
  if (!get_current || !get_id) return 0;
  void *c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
  return id;
}

// Y[al][j][l] = sum_be V[al][be] cB[be][j][l]
__global__ void k_term_y(int pA, int pB, int nj, int nl, const double *V, const double *cB,
                         double *Y) {
  const int n = nj * nl;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < pA * n;
       idx += gridDim.x * blockDim.x) {
    const int al = idx / n, c = idx - al * n;
    double s = 0.0;
    for (int be = 0; be < pB; ++be) s = fma(V[al * pB + be], cB[be * n + c], s);
    Y[idx] = s;
  }
}

// T[al][j][k] = sum_l Y[al][j][l] D[k][l]
__global__ void k_term_t(int pA, int nj, int nk, int nl, const double *Y, const double *D,
                         double *T) {
  const int n = nj * nk;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < pA * n;
       idx += gridDim.x * blockDim.x) {
    const int al = idx / n, r = idx - al * n, j = r / nk, k = r - j * nk;
    const double *y = Y + ((int64_t)al * nj + j) * nl;
    const double *d = D + (int64_t)k * nl;
    double s = 0.0;
    for (int l = 0; l < nl; ++l) s = fma(y[l], d[l], s);
    T[idx] = s;
  }
}

// out[i][j] = sum_{al,k} cA[al][i][k] T[al][j][k]
__global__ void k_term_out(int pA, int ni, int nj, int nk, const double *cA, const double *T,
                           double *out) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ni * nj;
       idx += gridDim.x * blockDim.x) {
    const int i = idx / nj, j = idx - i * nj;
    double s = 0.0;
    for (int al = 0; al < pA; ++al) {
      const double *a = cA + ((int64_t)al * ni + i) * nk;
      const double *t = T + ((int64_t)al * nj + j) * nk;
      for (int k = 0; k < nk; ++k) s = fma(a[k], t[k], s);
    }
    out[idx] = s;
  }
}

// Device address of the static array in the current context, looked up once
// per device and context (host code may not use the array's name as a device
// pointer).  The first call on a device, and the first after a device reset,
// does the lookup; make it outside stream capture.
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
    void *p = nullptr;
    // makes the device's primary context current when no context is
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double *)p;
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" hfx_status hfx_term_noalloc(int32_t nabf_a, int32_t nabf_b, int32_t nao_i,
                                       int32_t nao_k, int32_t nao_j, int32_t nao_l,
                                       const double *cA, const double *V, const double *cB,
                                       const double *D, double *out, void *cuda_stream) {
  if (!cA || !V || !cB || !D || !out) return HFX_E_ARG;
  if (nabf_a < 1 || nabf_b < 1 || nao_i < 1 || nao_k < 1 || nao_j < 1 || nao_l < 1)
    return HFX_E_ARG;
  // both intermediates must fit their half of the static array
  if ((int64_t)nabf_a * nao_j * nao_l > kHalf || (int64_t)nabf_a * nao_j * nao_k > kHalf)
    return HFX_E_SHAPE;
  // the output kernel indexes ni * nj outputs in 32-bit arithmetic
  if ((int64_t)nao_i * nao_j > 2147483647ll) return HFX_E_SHAPE;
  double *scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return HFX_E_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *Y = scratch, *T = scratch + kHalf;
  const int threads = 256;
  auto blocks = [&](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 4096)); };
  k_term_y<<<blocks((int64_t)nabf_a * nao_j * nao_l), threads, 0, st>>>(nabf_a, nabf_b, nao_j,
                                                                          nao_l, V, cB, Y);
  k_term_t<<<blocks((int64_t)nabf_a * nao_j * nao_k), threads, 0, st>>>(nabf_a, nao_j, nao_k,
                                                                          nao_l, Y, D, T);
  k_term_out<<<blocks((int64_t)nao_i * nao_j), threads, 0, st>>>(nabf_a, nao_i, nao_j, nao_k, cA,
                                                                 T, out);
  return cudaGetLastError() == cudaSuccess ? HFX_OK : HFX_E_CUDA;
}
