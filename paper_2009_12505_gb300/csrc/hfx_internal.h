// Internal declarations shared by libhfx's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hfx.h"

// ---------------------------------------------------------------------------
// Keys: (i, j, n1, n2, n3) packed into 64 bits; i, j < 2^20, |n| <= 127.
// The +128 offsets make the packed order the lexicographic (i, j, n) order.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t hk_pack(int i, int j, int n1, int n2, int n3) {
  return ((uint64_t)(uint32_t)i << 44) | ((uint64_t)(uint32_t)j << 24) |
         ((uint64_t)((n1 + 128) & 0xFF) << 16) | ((uint64_t)((n2 + 128) & 0xFF) << 8) |
         (uint64_t)((n3 + 128) & 0xFF);
}
__host__ __device__ inline void hk_unpack(uint64_t k, int32_t out[5]) {
  out[0] = (int32_t)(k >> 44);
  out[1] = (int32_t)((k >> 24) & 0xFFFFF);
  out[2] = (int32_t)((k >> 16) & 0xFF) - 128;
  out[3] = (int32_t)((k >> 8) & 0xFF) - 128;
  out[4] = (int32_t)(k & 0xFF) - 128;
}
constexpr uint64_t HK_EMPTY = ~0ull;

// SplitMix64 finaliser (Steele, Lea, Flood 2014) as the slot hash.
__host__ __device__ inline uint64_t hk_mix(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// Read-only open-addressing table on the device: key -> int64 value.
struct DevHash {
  const uint64_t *keys;
  const int64_t *vals;
  uint64_t mask;  // capacity - 1 (capacity a power of two, load <= 1/2)
};

__device__ inline int64_t dh_find(const DevHash &h, uint64_t k) {
  uint64_t s = hk_mix(k) & h.mask;
  for (uint64_t probe = 0; probe <= h.mask; ++probe) {  // bounded: table never full
    uint64_t cur = h.keys[s];
    if (cur == k) return h.vals[s];
    if (cur == HK_EMPTY) return -1;
    s = (s + 1) & h.mask;
  }
  return -1;
}

// One neighbour entry of atom x: the C(x, y, m) block.
struct NbrEntry {
  int32_t other;     // atom y
  int32_t n[3];      // lattice vector m of y relative to x
  int32_t aopre;     // sum of nao over the earlier entries of x's list
  int32_t pad;
  int64_t cblk;      // index of the C block (key order)
};

// One <A,B> work item: A = (a, 0), B = (b, n), the V(a, b, n) block.
struct WorkItem {
  int32_t a, b, n[3];
  int32_t nF, nG, nFw;   // |N[a]|, |N[b]|, 32-bit words per F-bitmask
  int64_t vblk;          // V block index
  int64_t dab;           // D(a, b, n) block index or -1
  int64_t fbase, gbase;  // first neighbour entry of a and of b
  int64_t mask_off;      // first mask word: [g][variant][nFw]
  int64_t wg_off;        // first (w, g) flag index
  int64_t wf_off;        // first (w, f) flag index
  int32_t role;          // 0: B is A itself; 1: canonical pair; 2: mirror of a canonical pair
  int32_t pad;
};

// Device view of one block kind.
struct DevBlocks {
  const double *data;
  const int64_t *offs;
  const double *maxabs;
};

// ---------------------------------------------------------------------------
// Deterministic FP64 accumulation: two int64 fixed-point words per element.
// x is split as hi * 2^-32 + lo * 2^-64 with hi = rint(x 2^32) and
// lo = rint((x 2^32 - hi) 2^32); both are added with integer atomics, which
// are associative, so the sum does not depend on the order of arrival.
// |x| < 2^31 per contribution; the per-contribution error is <= 2^-65.  A
// contribution outside that range (or NaN) is not added: the adder records
// HFX_DEV_ERR_BOUNDS in *err and the build fails with an error status.
// ---------------------------------------------------------------------------
__device__ inline void fx_add(unsigned long long *hi_lo, double x, unsigned *err) {
  if (!(fabs(x) < 2147483648.0)) {
    atomicOr(err, 8u);  // HFX_DEV_ERR_BOUNDS
    return;
  }
  double s = x * 4294967296.0;  // exact
  double h = rint(s);
  double r = (s - h) * 4294967296.0;  // s - h exact
  long long hi = (long long)h;
  long long lo = (long long)rint(r);
  if (hi) atomicAdd(hi_lo, (unsigned long long)hi);
  if (lo) atomicAdd(hi_lo + 1, (unsigned long long)lo);
}

__host__ __device__ inline double fx_value(long long hi, long long lo) {
  return (double)hi * 2.3283064365386963e-10 + (double)lo * 5.4210108624275222e-20;
}

// Error words written by kernels (bitwise OR); checked by the host after a build.
enum : unsigned {
  HFX_DEV_ERR_HASH_FULL = 1u,   // Sigma key table overflow (retry with a larger table)
  HFX_DEV_ERR_NONFINITE = 2u,   // NaN/Inf in an input block
  HFX_DEV_ERR_MISSING = 4u,     // a Sigma key looked up by a contraction is absent
  HFX_DEV_ERR_BOUNDS = 8u,      // a size exceeded a kernel's compiled limit
  HFX_DEV_ERR_TIMEOUT = 16u,    // a bounded device wait expired
};

// Limits of the FP64 kernels' shared-memory staging.
constexpr int HFX_MAX_NAO = 64;
constexpr int HFX_MAX_NABF = 256;

struct ScreenArgs {
  const WorkItem *items;
  int64_t nitems;
  int64_t nwg;             // total (w, g) pairs
  const NbrEntry *nbr;
  const int32_t *nao, *nabf;
  DevBlocks C, V, D;
  DevHash dhash;
  double theta;
  uint32_t *masks;
  uint8_t *wg_flags;       // per (w,g): bit v = some F survives variant v
  uint32_t *wf_flags;      // per (w,f): bit v = some G survives variant v
  unsigned long long *sig_keys;
  uint64_t sig_mask;
  unsigned long long *sig_count;
  unsigned long long sig_limit;
  unsigned long long *counters;  // [0..3] survivors per variant, [4] active (A,B,G), [5] canonical MACs,
                                 // [16..19] canonical MACs per piece, [20] Y MACs,
                                 // [21] quadruples (A,B,F,G) removed by the ERI screen
  const double *eri_sq;    // per C block sqrt(max(Q, 0)) of the ERI screen; null: screen off
  double eps_eri;
  const double *theta_atom;  // per central atom threshold (batched cells); null: theta
  unsigned *err;
};


// Arguments of the contraction kernels for one wave of work items [w0, w1).
struct ContractArgs {
  const WorkItem *items;
  int64_t w0, w1;
  int64_t wg_base, wf_base;  // items[w0].wg_off, items[w0].wf_off
  int64_t nwg, nwf;          // (w,g) and (w,f) pairs in the wave
  const NbrEntry *nbr;
  const int32_t *nao, *nabf;
  const int32_t *ncol;       // per atom: sum of nao over its neighbour list
  DevBlocks C, V, D;
  DevHash dhash;             // D keys -> block index
  DevHash shash;             // Sigma keys -> element offset
  const uint32_t *masks;
  const uint8_t *wg_flags;
  const uint32_t *wf_flags;
  double *scratch;
  const int64_t *y_off, *p_off, *t3_off, *q_off;  // per item of the wave, into scratch
  unsigned long long *acc;   // Sigma fixed-point words, 2 per element
  unsigned long long *macs;  // executed multiply-adds per kernel class (7 slots)
  unsigned *err;
  int sym;                   // inputs Hermitian: use the mirror pieces (see hfx_fp64.cu)
  unsigned skip;             // kernels not to launch: bit q = launch order q (0 = Y ... 6 = D_AB)
  int no_p;                  // the D-stage leaves P (the D_AB piece's T) to the split path
  unsigned long long *dcacc; // adjoint: fixed-point dE/dC (2 words per C element)
  double *dv;                // adjoint: dE/dV in the V block layout
};

cudaError_t launch_maxabs(const double *data, const int64_t *offs, int64_t nblk, double *out,
                          unsigned *err, cudaStream_t st);
cudaError_t launch_screen(const ScreenArgs &a, cudaStream_t st);
// Cauchy-Schwarz ERI screen: per C block e (atoms cxy[2e], cxy[2e+1]) the
// largest diagonal ERI of its AO pairs under the LRI expansion, from the V
// blocks meta[5e .. 5e+3] (XX, XY, YX, YY; -1 = absent) and the partner C
// block meta[5e+4] (-1 = absent or the same site); writes sqrt(max(Q, 0)).
cudaError_t launch_diag_eri(const double *Cd, const int64_t *Co, const double *Vd,
                            const int64_t *Vo, const int64_t *meta, const int32_t *cxy,
                            const int32_t *nao, const int32_t *nabf, int64_t nC, double *sq,
                            cudaStream_t st);
cudaError_t launch_collect_keys(const unsigned long long *keys, uint64_t cap,
                                unsigned long long *out, unsigned long long *n, cudaStream_t st);
// Launches the seven FP64 contraction kernels; ev (8 events or null) is recorded
// before the first and after each kernel.  Returns the number of launches in *nl.
cudaError_t launch_contract_fp64(const ContractArgs &a, cudaStream_t st, cudaEvent_t *ev, int *nl);
// Adjoint kernels for one wave (Y in y_off, R in p_off).
cudaError_t launch_adjoint(const ContractArgs &a, cudaStream_t st);
cudaError_t launch_fx_to_double(const unsigned long long *acc, int64_t n, double *out,
                                cudaStream_t st);
// E_X = 1/2 the sum of n per-block partials, in the fixed order of the build.
cudaError_t launch_ex_reduce(const double *partials, int64_t n, double *ex, cudaStream_t st);
cudaError_t launch_finalize(const unsigned long long *acc, int64_t nelem, double *sigma,
                            const uint64_t *skeys, const int64_t *soffs, int64_t nsig,
                            DevBlocks D, DevHash dhash, double *partials, double *ex,
                            cudaStream_t st);
// Bitwise check that every block has its mirror (index mirror[e], -1 when
// absent) equal to its transpose; sets *bad on the first mismatch.
cudaError_t launch_check_mirror(const double *data, const int64_t *offs, const int64_t *mirror,
                                const int32_t *rows, int64_t nblk, unsigned *bad,
                                cudaStream_t st);
cudaError_t launch_gather(const double *const *src, const int64_t *dst_off, const int64_t *len,
                          int64_t nblk, double *dst, cudaStream_t st);
// Density-matrix blocks from eigenvectors and Sigma at k points (hfx_fourier.cu).
cudaError_t launch_density(int nk, const double *kfrac, int nb, int nbands, const double *coef,
                           const double *occ, int64_t nkeys, const int32_t *keys,
                           const int32_t *aoff, const int32_t *nao, const int64_t *doff,
                           double *out, unsigned long long *maxim, cudaStream_t st);
cudaError_t launch_sigma_k(int nk, const double *kfrac, int natoms, const int32_t *aoff,
                           const int32_t *nao, int64_t nkeys, const uint64_t *skeys,
                           const int64_t *soffs, const double *sigma, int64_t nb, double *out,
                           cudaStream_t st);
