// Sigma finalisation and E_X (Algorithm 5, "Calculate E^X"), plus the block
// gather used when packing input blocks.
//
// Sigma arrives as two fixed-point words per element (see fx_add), so the
// conversion to FP64 is exact up to one final rounding and independent of the
// order contributions arrived in.  E_X = 1/2 sum over Sigma keys that are also
// D keys of sum_ij D[i][j] Sigma[i][j]: one partial per Sigma block in a fixed
// in-block order, then one block reduces the partials in a fixed order.
#include "hfx_internal.h"

namespace {

__global__ void k_fx_to_double(const unsigned long long *acc, int64_t n, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fx_value((long long)acc[2 * i], (long long)acc[2 * i + 1]);
}

// One warp per Sigma block: partial = sum D . Sigma in a fixed lane/shuffle order.
__global__ void k_ex_partials(const double *sigma, const uint64_t *skeys, const int64_t *soffs,
                              int64_t nsig, DevBlocks D, DevHash dhash, double *partials) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nsig) return;
  const int64_t d = dh_find(dhash, skeys[w]);
  double s = 0.0;
  if (d >= 0) {
    const double *db = D.data + D.offs[d];
    const int64_t len = soffs[w + 1] - soffs[w];
    const double *sb = sigma + soffs[w];
    for (int64_t t = lane; t < len; t += 32) s = fma(db[t], sb[t], s);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) partials[w] = s;
}

// Single block: thread t sums a contiguous slice, then a fixed tree.
__global__ void k_ex_reduce(const double *partials, int64_t n, double *ex) {
  __shared__ double red[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  double s = 0.0;
  for (int64_t i = t * per; i < n && i < (t + 1) * per; ++i) s += partials[i];
  red[t] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h; h >>= 1) {
    if (t < h) red[t] += red[t + h];
    __syncthreads();
  }
  if (t == 0) *ex = 0.5 * red[0];
}

// One warp per block: dst[dst_off[e] ...] = src[e][0 .. len[e]).
__global__ void k_gather(const double *const *src, const int64_t *dst_off, const int64_t *len,
                         int64_t nblk, double *dst) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nblk) return;
  const double *s = src[w];
  double *d = dst + dst_off[w];
  for (int64_t t = lane; t < len[w]; t += 32) d[t] = s[t];
}

// One warp per block e with nrow rows: block[mirror[e]] must equal block[e]^T.
__global__ void k_check_mirror(const double *data, const int64_t *offs, const int64_t *mirror,
                               const int32_t *rows, int64_t nblk, unsigned *bad) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nblk) return;
  const int64_t m = mirror[w];
  if (m < 0) {
    if (lane == 0) atomicOr(bad, 1u);
    return;
  }
  const int64_t len = offs[w + 1] - offs[w];
  const int nr = rows[w], nc = (int)(len / nr);
  const double *x = data + offs[w], *y = data + offs[m];
  bool diff = (offs[m + 1] - offs[m]) != len;
  for (int64_t t = lane; !diff && t < len; t += 32) {
    const int r = (int)(t / nc), c = (int)(t - (int64_t)r * nc);
    diff |= x[t] != y[(int64_t)c * nr + r];
  }
  if (__any_sync(0xffffffffu, diff) && lane == 0) atomicOr(bad, 1u);
}

}  // namespace

cudaError_t launch_check_mirror(const double *data, const int64_t *offs, const int64_t *mirror,
                                const int32_t *rows, int64_t nblk, unsigned *bad,
                                cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  k_check_mirror<<<(unsigned)((nblk * 32 + 255) / 256), 256, 0, st>>>(data, offs, mirror, rows,
                                                                      nblk, bad);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const unsigned long long *acc, int64_t nelem, double *sigma,
                            const uint64_t *skeys, const int64_t *soffs, int64_t nsig,
                            DevBlocks D, DevHash dhash, double *partials, double *ex,
                            cudaStream_t st) {
  if (nelem > 0)
    k_fx_to_double<<<(unsigned)((nelem + 255) / 256), 256, 0, st>>>(acc, nelem, sigma);
  if (nsig > 0)
    k_ex_partials<<<(unsigned)((nsig * 32 + 255) / 256), 256, 0, st>>>(sigma, skeys, soffs, nsig,
                                                                       D, dhash, partials);
  k_ex_reduce<<<1, 1024, 0, st>>>(partials, nsig, ex);
  return cudaGetLastError();
}

cudaError_t launch_ex_reduce(const double *partials, int64_t n, double *ex, cudaStream_t st) {
  k_ex_reduce<<<1, 1024, 0, st>>>(partials, n, ex);
  return cudaGetLastError();
}

cudaError_t launch_gather(const double *const *src, const int64_t *dst_off, const int64_t *len,
                          int64_t nblk, double *dst, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  k_gather<<<(unsigned)((nblk * 32 + 255) / 256), 256, 0, st>>>(src, dst_off, len, nblk, dst);
  return cudaGetLastError();
}
