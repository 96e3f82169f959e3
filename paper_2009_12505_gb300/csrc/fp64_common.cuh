// Device helpers shared by the FP64 contraction and adjoint kernels.
#pragma once

#include "hfx_internal.h"

namespace fp64 {

constexpr int kThreads = 256;
constexpr int kChunk = 4096;     // doubles of shared staging per chunk
constexpr int kMaxOut = 16;      // outputs per thread: nao*nao <= 4096

struct PairLoc {
  int64_t w;   // work item (absolute index)
  int idx;     // g or f within the item
};

// (w, g) or (w, f) pair p of the wave -> item and index (binary search).
__device__ inline PairLoc locate(const ContractArgs &A, int64_t p, bool by_g) {
  const int64_t base = by_g ? A.wg_base : A.wf_base;
  int64_t lo = A.w0, hi = A.w1 - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    const int64_t off = (by_g ? A.items[mid].wg_off : A.items[mid].wf_off) - base;
    if (off <= p) lo = mid; else hi = mid - 1;
  }
  const int64_t off = (by_g ? A.items[lo].wg_off : A.items[lo].wf_off) - base;
  return PairLoc{lo, (int)(p - off)};
}

__device__ inline bool mask_bit(const ContractArgs &A, const WorkItem &it, int g, int v, int f) {
  const uint32_t w = A.masks[it.mask_off + ((int64_t)g * 4 + v) * it.nFw + (f >> 5)];
  return (w >> (f & 31)) & 1u;
}

__device__ inline int64_t sig_offset(const ContractArgs &A, int i, int j, int n0, int n1, int n2) {
  const int64_t off = dh_find(A.shash, hk_pack(i, j, n0, n1, n2));
  if (off < 0) atomicOr(A.err, HFX_DEV_ERR_MISSING);
  return off;
}

// Ordered list of the indices x in [0, n) with bit(x) set, built by warp 0
// with ballots so the order is ascending (deterministic).  Returns the count.
template <class Bit>
__device__ inline int ordered_select(int n, Bit bit, int *list, int *count_smem) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int c = 0;
    for (int x0 = 0; x0 < n; x0 += 32) {
      const int x = x0 + lane;
      const bool b = x < n && bit(x);
      const uint32_t bal = __ballot_sync(0xffffffffu, b);
      if (b) list[c + __popc(bal & ((1u << lane) - 1u))] = x;
      c += __popc(bal);
    }
    if (lane == 0) *count_smem = c;
  }
  __syncthreads();
  return *count_smem;
}

}  // namespace fp64

using namespace fp64;
