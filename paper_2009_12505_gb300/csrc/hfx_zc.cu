// HFX_OZAKI: the D_FG and D_FB pieces of Algorithm 3 on the tensor cores.
//
// For a pair <A,B> and a neighbour G of B, with F running over the neighbours
// of A that survive the screen for the piece,
//   D_FG piece:  Z_G[(al,a)][g] = sum_F sum_f C_AF[al][a][f] D_FG[f][g]
//                Sigma_AB[a][b] -= sum_{al,g} Z_G[(al,a)][g] Y_G[al][b][g]
//   D_FB piece:  X_G[(al,a)][b] = sum_F sum_f C_AF[al][a][f] D_FB[f][b]
//                Sigma_AG[a][g] -= sum_{al,b} X_G[(al,a)][b] Y_G[al][b][g]
// These are Algorithm 3's T and Ht stages contracted D-first: the sums over F
// and the final contraction are reassociations of exact sums.
//
// Column blocks and jobs.  A column block is one (G, piece) with survivors:
// its Z columns are the rows of the transposed D blocks D_FG^T (piece 1) or
// D_FB^T (piece 2), 16 or 32 of them.  Consecutive blocks of a pair (in G
// order, D_FG before D_FB) are packed into groups of 32 columns; a job is one
// group and a run of the union of its blocks' surviving F with at most 640 K
// (so every digit-order group sum stays an exact f32 integer), over every
// 128-row tile of (al, a).  Within a job, a D block that is screened out for
// one of the blocks is a zero tile.
//
// Digit-stacked products.  A (C of atom A, rows (al,a), K = F blocks) and B
// (D blocks, transposed) are split into KS balanced base-128 digits, exact in
// bf16.  In shared memory each column block's B digits of one K step are
// stacked along N (digit j at rows R j .. R j + R - 1, R = 16 or 32 rows), so
// one tcgen05.mma with A digit i, N = R (KS - i) and accumulator column offset
// R i adds every product of digit order i + j into the block's TMEM columns
// [R (i + j), R (i + j + 1)): KS MMAs per block and K step instead of
// KS (KS + 1) / 2 narrow ones, and one bulk copy per block (the D tiles are
// stored digit-major).  The epilogue adds the order groups (exact f32
// integers times powers of two) in packed double-float arithmetic.
//
// Roles (one CTA per SM, persistent over the job list, which the plan writes
// longest first and the CTAs deal out among themselves in snake order; each
// CTA records its busy time so the host can report the load balance):
// warp 8 streams A and B tiles with 1-D bulk copies into a ring of shared
// stages; warp 9 issues the MMAs into one of two TMEM accumulators; warp 10
// copies the Y rows of each tile (f32 pairs, laid out [16-column block][al]
// [b][16] so a tile's rows are contiguous) into one of two shared buffers;
// warps 0-7 read an accumulator (warp w: TMEM lanes 32 (w % 4).., columns
// 16 (w / 4)..), turn Z into f32 pairs, contract with Y in packed (f32x2)
// double-float arithmetic, reduce over al through shared memory in a fixed
// order and add
// each finished block to the fixed-point Sigma (and its mirror for Hermitian
// inputs) once per job.  Every wait is bounded; on expiry the kernel records
// HFX_DEV_ERR_TIMEOUT, drains its copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "hfx_split.h"
#include "split_common.cuh"

namespace split {

constexpr int ZC_COLS = 32;                      // Z columns per job
constexpr int ZC_KMAX = 640;                     // K per job: exact f32 group sums

// Epilogue geometry for EPI epilogue warps (8 or 16): 4 warps cover the 128
// TMEM lanes, so there are EPI / 4 column groups of 32 / (EPI / 4) columns.
template <int EPI>
struct ZcGeo {
  static constexpr int NQ = EPI / 4;                 // column groups
  static constexpr int CW = ZC_COLS / NQ;            // Z columns per epilogue warp
  static constexpr int ET = EPI * 32;                // epilogue threads
  static constexpr int THREADS = (EPI + 3) * 32;     // + A/B loader, MMA issuer, Y loader
  static constexpr int OWN = 2 * 32 * 32 / ET;       // owned outputs per epilogue thread
};
constexpr long long ZC_WAIT = 2000000000ll;      // cycles per bounded wait
// Staged Y rows of one al are padded by ZC_YPAD pairs, so the rows of the
// few al a warp touches fall in different shared-memory banks.
constexpr int ZC_YPAD = 2;

__host__ __device__ __forceinline__ int kb_of(int nao) { return nao <= 16 ? 16 : 32; }

// element offset of (r, c) in an [R x kb] K-major core-matrix tile
__device__ __forceinline__ int tile_off_kb(int r, int c, int kb) {
  return ((r >> 3) * (kb >> 3) + (c >> 3)) * 64 + (r & 7) * 8 + (c & 7);
}

// ---------------------------------------------------------------- operands

// C of atom x as rows (al, a), K = F blocks (one exponent per row).
template <int KS>
__global__ void k_slice_cz(SplitShared S) {
  const int64_t grow = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (grow >= S.cz_rowpre[S.natoms]) return;
  int lo = 0, hi = S.natoms - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S.cz_rowpre[mid] <= grow) lo = mid; else hi = mid - 1;
  }
  const int x = lo;
  const int r = (int)(grow - S.cz_rowpre[x]);
  const int nx = S.nao[x], px = S.nabf[x];
  const bool live = r < px * nx;
  const int64_t base = S.nc_start[x];
  const int n = (int)(S.nc_start[x + 1] - base);
  const int ktot = S.ktotZ[x];
  long long mbits = 0;
  if (live)
    for (int q = 0; q < n; ++q) {
      const NbrEntry &e = S.nbr[base + q];
      const int nf = S.nao[e.other];
      for (int f = lane; f < nf; f += 32)
        mbits = max(mbits, __double_as_longlong(S.Cd[S.Co[e.cblk] + (int64_t)r * nf + f]) &
                               0x7FFFFFFFFFFFFFFFll);
    }
  for (int o = 16; o; o >>= 1) mbits = max(mbits, __shfl_xor_sync(0xffffffffu, mbits, o));
  const int ex = row_exponent(mbits);
  if (lane == 0) S.cz_e[grow] = (int16_t)max(-30000, ex);
  const int mt = r / 128, rr = r - mt * 128;
  __nv_bfloat16 *tile0 = S.cz + S.cz_base[x] + (int64_t)mt * ktot * KS * 128;
  for (int q = 0; q < n; ++q) {
    const NbrEntry &e = S.nbr[base + q];
    const int nf = S.nao[e.other], kb = kb_of(nf);
    __nv_bfloat16 *tile = tile0 + (int64_t)S.kofs[base + q] * KS * 128;
    for (int f = lane; f < kb; f += 32) {
      const double v = (live && f < nf) ? S.Cd[S.Co[e.cblk] + (int64_t)r * nf + f] : 0.0;
      int d[KS];
      to_digits<KS>(v, ex, d);
#pragma unroll
      for (int s = 0; s < KS; ++s)
        tile[(int64_t)s * kb * 128 + tile_off_kb(rr, f, kb)] = __int2bfloat16_rn(d[s]);
    }
  }
}

// Column maxima of D: de[aoff[j] + y] = max over every block (i, j, n) and x of
// |D[x][y]| (bit pattern; nonnegative doubles order as integers).
__global__ void k_dz_exp(SplitShared S) {
  const int64_t e = blockIdx.x;
  const int i = S.dij[2 * e], j = S.dij[2 * e + 1];
  const int nr = S.nao[i], nc = S.nao[j];
  const double *D = S.Dd + S.Do[e];
  for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
    const int y = idx % nc;
    const unsigned long long b =
        (unsigned long long)(__double_as_longlong(D[idx]) & 0x7FFFFFFFFFFFFFFFll);
    atomicMax(S.de + S.aoff[j] + y, b);
  }
}

// D block (i, j, n) as the transposed digit tile [digit][R x kb]: rows y of
// atom j (R = 16 or 32), K = x of atom i (kb = 16 or 32), exponent per y.
template <int KS>
__global__ void k_dz_slice(SplitShared S) {
  const int64_t e = blockIdx.x;
  const int i = S.dij[2 * e], j = S.dij[2 * e + 1];
  const int nr = S.nao[i], nc = S.nao[j];
  const int R = nc <= 16 ? 16 : 32, kb = kb_of(nr);
  const double *D = S.Dd + S.Do[e];
  __nv_bfloat16 *t = S.dz + S.dz_off[e];
  for (int idx = threadIdx.x; idx < R * kb; idx += blockDim.x) {
    const int y = idx / kb, x = idx - y * kb;
    const bool live = y < nc && x < nr;
    const double v = live ? D[x * nc + y] : 0.0;
    const int ex = y < nc ? row_exponent((long long)S.de[S.aoff[j] + y]) : -1000;
    int d[KS];
    to_digits<KS>(v, ex, d);
#pragma unroll
    for (int s = 0; s < KS; ++s)
      t[(int64_t)s * R * kb + tile_off_kb(y, x, kb)] = __int2bfloat16_rn(d[s]);
  }
}

// ---------------------------------------------------------------- job plan

// Cost key of a job (Algorithm 6's processing time, in 256 buckets): row
// tiles x operand stages of 16 K, a quarter per bucket.  The plan's count
// pass histograms the keys, the host turns the histogram into descending
// start offsets, and the fill pass places each job in its key's range, so the
// list runs longest first (longest-processing-time order).
constexpr int ZC_NCOST = 256;
constexpr int ZC_NKEYS = 2 * ZC_NCOST;
__device__ __forceinline__ int zc_cost_key(int mtz, int k) {
  return min(ZC_NCOST - 1, (mtz * (k / 16) + 3) / 4);
}
// Size class of a job: small when atom A and every block it touches have at
// most 16 AOs (outputs, Z columns and F entries), so its Y rows fit the
// staging buffers of the fastest kernel variant and its job sums fit fewer
// registers; small jobs take keys [0, 256), the others [256, 512), and the
// host places the small class first, so each class is a contiguous,
// longest-first range launched with its own variant.
__device__ __forceinline__ int zc_key(int mtz, int k, bool small) {
  return zc_cost_key(mtz, k) + (small ? 0 : ZC_NCOST);
}

// Job handed to CTA b in round r of the persistent loop: rounds alternate
// direction (snake order), so over a longest-first list every CTA gets a
// similar mix of long and short jobs.  The last round is partial.
__device__ __forceinline__ int zc_job_of(int r, int b, int G) {
  return r * G + ((r & 1) ? G - 1 - b : b);
}

// Runs of the union of a group's surviving F with at most ZC_KMAX K each: one
// job per run.  Called by one lane per group.  fill == 0 only counts.
__device__ void zc_plan_group(const SplitShared &S, const SplitWave &W, const WorkItem &it,
                              int32_t w, const int (&bg)[2], const int (&bp)[2], int nblk,
                              int mtz, int fill, unsigned long long &macs,
                              unsigned long long &umacs) {
  const uint32_t *mr[2] = {nullptr, nullptr};
  for (int q = 0; q < nblk; ++q)
    mr[q] = S.masks + it.mask_off + ((int64_t)bg[q] * 4 + (bp[q] - 1)) * it.nFw;
  int64_t eg_n[2][4];
  int ncv[2] = {0, 0};  // Z columns of each block
  for (int q = 0; q < nblk; ++q) {
    const NbrEntry eg = S.nbr[it.gbase + bg[q]];
    eg_n[q][0] = eg.other;
    eg_n[q][1] = eg.n[0];
    eg_n[q][2] = eg.n[1];
    eg_n[q][3] = eg.n[2];
    ncv[q] = bp[q] == 1 ? S.nao[eg.other] : S.nao[it.b];
  }
  const unsigned long long rows = (unsigned long long)S.nabf[it.a] * S.nao[it.a];
  // outputs and Z columns of both pieces are nao(B) and nao(G); the small
  // class also bounds atom A (the outputs an epilogue thread owns)
  bool small = S.nao[it.b] <= 16 && S.nao[it.a] <= 16;
  for (int q = 0; q < nblk; ++q) small = small && S.nao[(int)eg_n[q][0]] <= 16;
  // cursor over the union bits: word wd, remaining bits u
  int wd = 0;
  uint32_t u = 0;
  auto next = [&](int &f) -> bool {
    while (!u) {
      if (wd >= it.nFw) return false;
      for (int q = 0; q < nblk; ++q) u |= mr[q][wd];
      ++wd;
      if (!u) continue;
    }
    const int b = __ffs(u) - 1;
    u &= u - 1;
    f = (wd - 1) * 32 + b;
    return true;
  };
  int f;
  bool more = next(f);
  while (more) {
    // this run: F from f on while K <= ZC_KMAX (scan ahead on a copy of the cursor)
    const int wd0 = wd;
    const uint32_t u0 = u;
    const int f0 = f;
    int n = 0, k = 0, kbm = 16;
    int fa = f;
    bool ma = true;
    while (ma) {
      const int kb = kb_of(S.nao[S.nbr[it.fbase + fa].other]);
      if (k + kb > ZC_KMAX) break;
      k += kb;
      kbm = max(kbm, kb);
      ++n;
      ma = next(fa);
    }
    macs += (unsigned long long)mtz * 128 * ZC_COLS * k;
    const int key = zc_key(mtz, k, small && kbm == 16);
    int64_t eo = 0;
    if (!fill) {
      atomicAdd(W.njobs + 2, 1);
      atomicAdd(W.njobs + 3, n);
      atomicAdd(W.zc_keys + key, 1);
    } else {
      atomicAdd(W.njobs + 2, 1);
      const int js = atomicAdd(W.zc_keys + key, 1);  // next slot of this key's range
      eo = (int64_t)atomicAdd(W.njobs + 3, n);
      ZcJob jb{};
      jb.w = w;
      jb.nblk = (int8_t)nblk;
      for (int q = 0; q < 2; ++q) {
        jb.g[q] = (int16_t)(q < nblk ? bg[q] : -1);
        jb.piece[q] = (int8_t)(q < nblk ? bp[q] : 0);
      }
      jb.nent = n;
      jb.ent = eo;
      W.zc_jobs[js] = jb;
      // entries: rewind to the run start
      wd = wd0;
      u = u0;
      int fe = f0;
      for (int q = 0; q < n; ++q) {
        const NbrEntry ef = S.nbr[it.fbase + fe];
        ZcEnt en{};
        en.kofs = S.kofs[it.fbase + fe];
        en.kb = kb_of(S.nao[ef.other]);
        for (int c = 0; c < 2; ++c) {
          en.dz[c] = -1;
          if (c >= nblk || !((mr[c][fe >> 5] >> (fe & 31)) & 1u)) continue;
          int64_t d;
          if (bp[c] == 1)
            d = dh_find(S.dhash, hk_pack(ef.other, (int)eg_n[c][0],
                                         it.n[0] + (int)eg_n[c][1] - ef.n[0],
                                         it.n[1] + (int)eg_n[c][2] - ef.n[1],
                                         it.n[2] + (int)eg_n[c][3] - ef.n[2]));
          else
            d = dh_find(S.dhash, hk_pack(ef.other, it.b, it.n[0] - ef.n[0], it.n[1] - ef.n[1],
                                         it.n[2] - ef.n[2]));
          if (d < 0) {
            atomicOr(S.err, HFX_DEV_ERR_MISSING);
          } else {
            en.dz[c] = S.dz_off[d];
            // products that are not padding or zero tiles
            umacs += rows * (unsigned long long)S.nao[ef.other] * ncv[c];
          }
        }
        W.zc_ents[eo + q] = en;
        if (q + 1 < n) next(fe);
      }
      // leave the cursor after the run
      more = next(fe);
      f = fe;
      continue;
    }
    more = ma;
    f = fa;
  }
}

// One warp per work item of the wave.  Lane 0 walks the column blocks in G
// order (D_FG before D_FB) and packs them into groups of at most 32 columns,
// 32 groups at a time; the lanes then plan one group each.  With fill == 0
// only counts jobs and entries (W.njobs[2], W.njobs[3]).
__global__ void __launch_bounds__(128) k_zc_plan(SplitShared S, SplitWave W, int fill) {
  __shared__ int sgrp[4][32][5];  // g0, p0, g1, p1, nblk
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wl = blockIdx.x * 4 + wib;
  if (wl >= W.nw) return;
  const WorkItem it = S.items[W.w0 + wl];
  const int pA = S.nabf[it.a], na = S.nao[it.a], nb = S.nao[it.b];
  const int mtz = (pA * na + 127) / 128;
  unsigned long long macs = 0, umacs = 0;
  // lane 0 state: cursor (g, piece) and the open group
  int g = 0, piece = 1, nblk = 0, rows = 0, cg[2] = {0, 0}, cp[2] = {0, 0};
  bool finished = false;
  while (true) {
    int cnt = 0;
    if (lane == 0) {
      while (cnt < 32) {
        // next block
        int R = 0;
        bool found = false;
        while (g < it.nG) {
          const unsigned bits = S.wg[it.wg_off + g];
          const bool on = (bits & (piece == 1 ? 1u : 2u)) &&
                          !(piece == 1 && S.sym && it.role == 2);
          if (on) {
            const int ncb = piece == 1 ? S.nao[S.nbr[it.gbase + g].other] : nb;
            R = ncb <= 16 ? 16 : 32;
            found = true;
            break;
          }
          if (++piece > 2) { piece = 1; ++g; }
        }
        if (!found) {
          if (nblk) {
            int *o = sgrp[wib][cnt++];
            o[0] = cg[0]; o[1] = cp[0]; o[2] = cg[1]; o[3] = cp[1]; o[4] = nblk;
            nblk = 0;
            rows = 0;
          }
          finished = true;
          break;
        }
        if (rows + R > ZC_COLS && nblk) {
          int *o = sgrp[wib][cnt++];
          o[0] = cg[0]; o[1] = cp[0]; o[2] = cg[1]; o[3] = cp[1]; o[4] = nblk;
          nblk = 0;
          rows = 0;
        }
        cg[nblk] = g;
        cp[nblk] = piece;
        ++nblk;
        rows += R;
        if (++piece > 2) { piece = 1; ++g; }
      }
    }
    cnt = __shfl_sync(0xffffffffu, cnt, 0);
    const bool fin = __shfl_sync(0xffffffffu, (int)finished, 0) != 0;
    __syncwarp();
    if (lane < cnt) {
      const int *o = sgrp[wib][lane];
      const int bg[2] = {o[0], o[2]}, bp[2] = {o[1], o[3]};
      zc_plan_group(S, W, it, (int32_t)(W.w0 + wl), bg, bp, o[4], mtz, fill, macs, umacs);
    }
    __syncwarp();
    if (fin) break;
  }
  for (int o = 16; o; o >>= 1) {
    macs += __shfl_xor_sync(0xffffffffu, macs, o);
    umacs += __shfl_xor_sync(0xffffffffu, umacs, o);
  }
  if (fill && lane == 0 && macs) atomicAdd(W.tmacs + 2, macs);
  if (fill && lane == 0 && umacs) atomicAdd(W.tmacs + 3, umacs);
}

// ---------------------------------------------------------------- product

// Epilogue data of one job, written to shared memory by a few lanes when its
// pair starts and read by every epilogue thread on each of the job's tiles.
struct ZcEpiJob {
  int64_t czrow0;    // first row of atom A's C exponents
  int64_t y2off;     // the work item's Y pairs in the wave scratch
  int64_t sg[2][2];  // block q: Sigma offset of its outputs, of their mirror (-1: none)
  int pA, na, nb, mtz, nblk, R0b;
  int nout[2], ncv[2], pc[2], gcb[2];
};

struct ZcSmem {
  uint64_t full[8], empty[8], tfull[2], tempty[2], yfull[2], yempty[2], drain;
  unsigned long long t_start;  // globaltimer at the start of the roles
  uint32_t tslot;
  int abort_f;
  int stkb[8];  // K of the entry in each operand stage (16 or 32)
  int ecol[2][ZC_COLS];  // column exponents of the pair's jobs (column group q at q * CW)
  ZcEpiJob ej[2][2];     // [pair parity][job of the pair]
};

// Number of jobs CTA b receives from zc_job_of over a list of njobs.
__device__ __forceinline__ int zc_cta_jobs(int njobs, int b, int G) {
  const int full = njobs / G, rem = njobs - full * G;
  return full + (((full & 1) ? G - 1 - b : b) < rem ? 1 : 0);
}

// Tile order of a CTA.  Its jobs r = 0 .. n - 1 run heaviest first (operand
// stages x row tiles).  With PAIR, pair p is job n - 1 - p (light) and job p
// (heavy), and their row tiles alternate while both have some: the MMAs of a
// long tile then run beside the epilogue of a short one, where one job after
// the other leaves the epilogue idle through the long tiles and the tensor
// pipe idle through the short ones.  Without PAIR, pair p is job p alone.
// Every role walks the same order.
template <bool PAIR>
struct ZcPair {
  int r0, r1, m0, m1, t0, t1, last;
  bool two;
  __device__ __forceinline__ void begin(int p, int n) {
    r0 = PAIR ? n - 1 - p : p;
    r1 = PAIR ? p : -1;
    two = PAIR && r1 < r0;
    m0 = m1 = t0 = t1 = 0;
    last = 1;
  }
  // next tile: job x of the pair (0: r0, 1: r1) and its row tile mt
  __device__ __forceinline__ bool next(int &x, int &mt) {
    const bool a = t0 < m0, b = t1 < m1;
    if (!a && !b) return false;
    x = (a && (!b || last == 1)) ? 0 : 1;
    last = x;
    mt = x ? t1++ : t0++;
    return true;
  }
};

template <class T>
__device__ __forceinline__ void zc_swap(T &a, T &b) {
  const T t = a;
  a = b;
  b = t;
}

__device__ __forceinline__ ZcJob zc_job(const SplitWave &W, int jbeg, int r) {
  return W.zc_jobs[jbeg + zc_job_of(r, blockIdx.x, gridDim.x)];
}

// rows of a job's lone column block (16 or 32); two blocks have 16 each
__device__ __forceinline__ int zc_rows(const SplitShared &S, const ZcJob &jb, const WorkItem &it) {
  if (jb.nblk != 1) return 16;
  const int ncb = jb.piece[0] == 1 ? S.nao[S.nbr[it.gbase + jb.g[0]].other] : S.nao[it.b];
  return ncb <= 16 ? 16 : 32;
}

// block and first column cq of column group q of width CW: two 16-column
// blocks take half the groups each; one block takes the groups below its R
template <int CW>
__device__ __forceinline__ int zc_group_block(int nblk, int R0b, int q, int &cq) {
  const int jc = q * CW;
  if (nblk == 2) { cq = jc & 15; return jc >> 4; }
  cq = jc;
  return jc < R0b ? 0 : -1;
}

// Epilogue data of job r, by one whole warp: lanes 0 .. 3 look up the Sigma
// offsets of block lane / 2 (odd lanes: the mirror), lane 4 the scalars.  A
// missing Sigma key fails the build, and the block is not added.
__device__ __forceinline__ void zc_epi_job(const SplitShared &S, const SplitWave &W, int jbeg,
                                           int r, int lane, ZcEpiJob &e) {
  const ZcJob jb = zc_job(W, jbeg, r);
  const WorkItem it = S.items[jb.w];
  const int q = (lane >> 1) & 1, m = lane & 1;
  int64_t t = -1;
  bool miss = false;
  if (lane < 4 && q < jb.nblk) {
    const int pcb = q ? jb.piece[1] : jb.piece[0];
    const bool mir = S.sym && (pcb == 2 || it.role == 1);
    if (m == 0 || mir) {
      if (pcb == 1) {
        t = m == 0 ? dh_find(S.shash, hk_pack(it.a, it.b, it.n[0], it.n[1], it.n[2]))
                   : dh_find(S.shash, hk_pack(it.b, it.a, -it.n[0], -it.n[1], -it.n[2]));
      } else {
        const NbrEntry eg = S.nbr[it.gbase + (q ? jb.g[1] : jb.g[0])];
        const int n0 = it.n[0] + eg.n[0], n1 = it.n[1] + eg.n[1], n2 = it.n[2] + eg.n[2];
        t = m == 0 ? dh_find(S.shash, hk_pack(it.a, eg.other, n0, n1, n2))
                   : dh_find(S.shash, hk_pack(eg.other, it.a, -n0, -n1, -n2));
      }
      miss = t < 0;
      if (miss) atomicOr(S.err, HFX_DEV_ERR_MISSING);
    }
  }
  const bool bad = __shfl_sync(0xffffffffu, (int)miss, lane & ~1) |
                   __shfl_sync(0xffffffffu, (int)miss, lane | 1);
  if (lane < 4) e.sg[q][m] = bad ? -1 : t;
  if (lane == 4) {
    const int pA = S.nabf[it.a], na = S.nao[it.a], nb = S.nao[it.b];
    e.czrow0 = S.cz_rowpre[it.a];
    e.y2off = W.y2_off[(int)(jb.w - W.w0)];
    e.pA = pA;
    e.na = na;
    e.nb = nb;
    e.mtz = (pA * na + 127) / 128;
    e.nblk = jb.nblk;
    e.R0b = 16;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      e.nout[b] = e.ncv[b] = e.pc[b] = e.gcb[b] = 0;
      if (b < jb.nblk) {
        const int ng = S.nao[S.nbr[it.gbase + jb.g[b]].other];
        e.pc[b] = jb.piece[b];
        e.gcb[b] = S.kofs[it.gbase + jb.g[b]] / 16;
        e.ncv[b] = jb.piece[b] == 1 ? ng : nb;
        e.nout[b] = jb.piece[b] == 1 ? nb : ng;
      }
    }
    if (jb.nblk > 0) e.R0b = e.ncv[0] <= 16 ? 16 : 32;
  }
}

// Column exponents of job r's column group hf (CW columns), by lanes < CW.
template <int CW>
__device__ __forceinline__ void zc_epi_ecol(const SplitShared &S, const SplitWave &W, int jbeg,
                                            int r, int hf, int lane, int *ecol) {
  if (lane >= CW) return;
  const ZcJob jb = zc_job(W, jbeg, r);
  const WorkItem it = S.items[jb.w];
  int ncv0 = 0, R0b = 16;
  if (jb.nblk > 0) {
    ncv0 = jb.piece[0] == 1 ? S.nao[S.nbr[it.gbase + jb.g[0]].other] : S.nao[it.b];
    R0b = ncv0 <= 16 ? 16 : 32;
  }
  int c0 = 0;
  const int hb = zc_group_block<CW>(jb.nblk, R0b, hf, c0);
  int e = -1000;
  if (hb >= 0) {
    const int pc = hb ? jb.piece[1] : jb.piece[0], g = hb ? jb.g[1] : jb.g[0];
    const int at = pc == 1 ? S.nbr[it.gbase + g].other : it.b;
    const int ncvh = S.nao[at];  // piece 1: nao(G); piece 2: nao(B)
    const int cc = c0 + lane;
    if (cc < ncvh) e = row_exponent((long long)S.de[S.aoff[at] + cc]);
  }
  ecol[hf * CW + lane] = e;
}

// Launch shape of k_zc: ybytes = shared bytes per staged Y block (0: the
// epilogue reads Y from global memory), rs = outputs per block held in the
// reduction buffer (16 or 32; the buffer is [column group][output][row]).
struct ZcCfg {
  int ybytes, rs;
  int jbeg, jend;  // the launch's range of the job list
  int cta0;        // first slot of its CTAs' busy times
};

// Y rows al in [al0, al0 + nal) of the 16-column block cb: [al][b][16] pairs.
__device__ __forceinline__ const float2 *zc_y_global(const float2 *Y2, int cb, int pA, int nb,
                                                     int al) {
  return Y2 + (((int64_t)cb * pA + al) * nb) * 16;
}

// One operand stage's MMAs (K = KB): for each K step of 16 and block b, A
// digit i times the block's B digits 0 .. KS - 1 - i stacked along N
// (N = R (KS - i)) into TMEM columns b 16 KS + i R ..  Descriptors are the
// stage's two base descriptors plus constant offsets (the 14-bit start field
// cannot carry: shared addresses stay below 2^18).
template <int KS, int KB>
__device__ __forceinline__ void zc_stage_mmas(uint32_t a0, uint32_t b0, uint32_t dcol, int nblk,
                                              int R, const uint32_t (&id16)[KS],
                                              const uint32_t (&id32)[KS], bool first) {
  constexpr uint32_t SBO = KB / 8 * 128;
  const uint64_t adesc = umma::smem_desc(a0, 128, SBO);
  const uint64_t bdesc = umma::smem_desc(b0, 128, SBO);
#pragma unroll
  for (int ks = 0; ks < KB / 16; ++ks)
    for (int b = 0; b < nblk; ++b) {
      const uint64_t bd = bdesc + (uint64_t)((b * (KS * 16 * KB * 2) + ks * 256) >> 4);
#pragma unroll
      for (int i = 0; i < KS; ++i) {
        const uint64_t ad = adesc + (uint64_t)((i * (128 * KB * 2) + ks * 256) >> 4);
        umma::mma_bf16(dcol + (uint32_t)(b * 16 * KS + i * R), ad, bd,
                       R == 16 ? id16[i] : id32[i], (!first || ks || i) ? 1u : 0u);
      }
    }
}

// One row's contraction with Y in double-float: out[o] = sum_{c < cend} z[c]
// yb[o so + c sc] for o < no, four outputs at a time; out[o] is stored at
// outp[o 128] (the reduction buffer is output-major, so a warp's 32 rows
// store to consecutive addresses).  The even and the odd columns are summed
// separately and added at the end, in exactly the order of the packed form
// below (zc_contract2), so the kernel variants that read Y from global memory
// and from shared memory give the same bits: which variant runs depends on
// the largest atom of the whole system, and a cell must not change its result
// when it is built together with other cells.
template <int CW>
__device__ __forceinline__ void zc_contract(const float2 (&z)[CW], int cend,
                                            const float2 *__restrict__ yb, int so, int sc, int no,
                                            float2 *__restrict__ outp) {
  const int no4 = no & ~3;
  for (int o0 = 0; o0 < no4; o0 += 4) {
    float eh[4] = {0.f, 0.f, 0.f, 0.f}, el[4] = {0.f, 0.f, 0.f, 0.f};
    float oh[4] = {0.f, 0.f, 0.f, 0.f}, ol[4] = {0.f, 0.f, 0.f, 0.f};
    const float2 *y0 = yb + o0 * so;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      if (c >= cend) break;
      const float2 *yc = y0 + c * sc;
      const float2 v[4] = {yc[0], yc[so], yc[2 * so], yc[3 * so]};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (c & 1) df_mac(oh[u], ol[u], z[c], v[u]);
        else df_mac(eh[u], el[u], z[c], v[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      df_add(eh[u], el[u], make_float2(oh[u], ol[u]));
      outp[(o0 + u) * 128] = make_float2(eh[u], el[u]);
    }
  }
  for (int o = no4; o < no; ++o) {
    float eh = 0.f, el = 0.f, oh = 0.f, ol = 0.f;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      if (c >= cend) break;
      if (c & 1) df_mac(oh, ol, z[c], yb[o * so + c * sc]);
      else df_mac(eh, el, z[c], yb[o * so + c * sc]);
    }
    df_add(eh, el, make_float2(oh, ol));
    outp[o * 128] = make_float2(eh, el);
  }
}

// The same contraction with packed f32x2 arithmetic: lane 0 sums the even
// columns, lane 1 the odd ones, and the two double-float sums are added at the
// end.  zh / nzh / nzl hold column pairs (2j, 2j + 1) of the high words, their
// negatives and the negated low words, zero from column cend on (an odd last
// pair repeats its column's Y, times zero).  Y words are loaded one by one
// into the two lanes.  P1: so = 16, sc = 1; otherwise so = 1, sc = 16.
template <int NP, bool P1>
__device__ __forceinline__ void zc_contract2(const uint64_t (&zh)[NP], const uint64_t (&nzh)[NP],
                                             const uint64_t (&nzl)[NP], int cend,
                                             const float2 *__restrict__ yb, int no,
                                             float2 *__restrict__ outp) {
  const float *yf = reinterpret_cast<const float *>(yb);
  constexpr int SO = P1 ? 32 : 2, SC = P1 ? 2 : 32;  // float words per output, column
  const int npair = (cend + 1) >> 1;
  auto put = [&](int o, uint64_t h2, uint64_t l2) {
    const float2 h = f2_un(h2), l = f2_un(l2);
    float sh = h.x, sl = l.x;
    df_add(sh, sl, make_float2(h.y, l.y));
    outp[o * 128] = make_float2(sh, sl);
  };
  const int no4 = no & ~3;
  for (int o0 = 0; o0 < no4; o0 += 4) {
    uint64_t sh[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      if (j >= npair) break;
      const int d1 = 2 * j + 1 < cend ? SC : 0;  // the pair's second column
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float *y = yf + (o0 + u) * SO + 2 * j * SC;
        df_mac2(sh[u], sl[u], zh[j], nzh[j], nzl[j], f2_pk(y[0], y[d1]), f2_pk(y[1], y[d1 + 1]));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) put(o0 + u, sh[u], sl[u]);
  }
  for (int o = no4; o < no; ++o) {
    uint64_t sh = 0, sl = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      if (j >= npair) break;
      const int d1 = 2 * j + 1 < cend ? SC : 0;
      const float *y = yf + o * SO + 2 * j * SC;
      df_mac2(sh, sl, zh[j], nzh[j], nzl[j], f2_pk(y[0], y[d1]), f2_pk(y[1], y[d1 + 1]));
    }
    put(o, sh, sl);
  }
}

// Loader-warp view of a job: operand bases, its entries (lane l holds entry
// held + l) and the B rows per block.
struct ZcLd {
  const __nv_bfloat16 *A;
  int64_t ktot, ent;
  int nent, nblk, Rl, mtz, held;
  ZcEnt mine;
};

__device__ __forceinline__ void zc_ld_job(const SplitShared &S, const SplitWave &W, int jbeg,
                                          int r, ZcLd &L) {
  const ZcJob jb = zc_job(W, jbeg, r);
  const WorkItem it = S.items[jb.w];
  L.A = S.cz + S.cz_base[it.a];
  L.ktot = S.ktotZ[it.a];
  L.ent = jb.ent;
  L.nent = jb.nent;
  L.nblk = jb.nblk;
  L.Rl = zc_rows(S, jb, it);
  L.mtz = (S.nabf[it.a] * S.nao[it.a] + 127) / 128;
  L.held = -1;
  L.mine = ZcEnt{0, 0, {-1, -1}};
}

// Y-loader view of a job: its Y pairs, sizes and the 16-column blocks of Y
// columns of each column block.
struct ZcYJob {
  const float2 *Y2;
  int pA, na, nb, mtz, nblk, ncb0, ncb1, cb0, cb1;
};

__device__ __forceinline__ void zc_y_job(const SplitShared &S, const SplitWave &W, int jbeg,
                                         int r, ZcYJob &Y) {
  const ZcJob jb = zc_job(W, jbeg, r);
  const WorkItem it = S.items[jb.w];
  Y.Y2 = reinterpret_cast<const float2 *>(W.scratch + W.y2_off[(int)(jb.w - W.w0)]);
  Y.pA = S.nabf[it.a];
  Y.na = S.nao[it.a];
  Y.nb = S.nao[it.b];
  Y.mtz = (Y.pA * Y.na + 127) / 128;
  Y.nblk = jb.nblk;
  Y.ncb0 = Y.ncb1 = Y.cb0 = Y.cb1 = 0;
  if (jb.nblk > 0) {
    Y.ncb0 = (S.nao[S.nbr[it.gbase + jb.g[0]].other] + 15) / 16;
    Y.cb0 = S.kofs[it.gbase + jb.g[0]] / 16;
  }
  if (jb.nblk > 1) {
    Y.ncb1 = (S.nao[S.nbr[it.gbase + jb.g[1]].other] + 15) / 16;
    Y.cb1 = S.kofs[it.gbase + jb.g[1]] / 16;
  }
}

template <int KS, int KBM, int NST, int EPI, bool YST, bool PAIR>
__global__ void __launch_bounds__(ZcGeo<EPI>::THREADS, 1)
    k_zc(SplitShared S, SplitWave W, ZcCfg cfg) {
  constexpr int ZC_EPI = EPI, ZC_NQ = ZcGeo<EPI>::NQ, ZC_CW = ZcGeo<EPI>::CW,
                ZC_ET = ZcGeo<EPI>::ET;
  // owned outputs per epilogue thread, for the job sums of both paired jobs:
  // na x (outputs of the job's blocks), at most 16 x 32 in the small class
  // (atom A and blocks of at most 16 AOs), else 32 x 64 (two blocks of 16
  // columns of piece 1 have nao(B) outputs each)
  constexpr int ZC_OWN = PAIR && KBM == 16 ? (16 * 32 + ZC_ET - 1) / ZC_ET : ZcGeo<EPI>::OWN;
  constexpr int A_BYTES = KS * 128 * KBM * 2;
  constexpr int B_BYTES = KS * ZC_COLS * KBM * 2;
  constexpr int STG = A_BYTES + B_BYTES;
  constexpr int SH = 7 * (KS + 1);
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *ybuf = smem + NST * STG;                                     // [2][2][ybytes]
  float2 *red = reinterpret_cast<float2 *>(ybuf + 4 * cfg.ybytes);     // [ZC_NQ][rs][128]
  ZcSmem *ctl = reinterpret_cast<ZcSmem *>(red + ZC_NQ * 128 * cfg.rs);
  volatile int *abort_f = &ctl->abort_f;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int njobs = cfg.jend - cfg.jbeg;
  // this CTA's jobs and pairs
  const int ncj = zc_cta_jobs(njobs, blockIdx.x, gridDim.x);
  const int npair = PAIR ? (ncj + 1) / 2 : ncj;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      umma::mbar_init(&ctl->full[s], 1);
      umma::mbar_init(&ctl->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(&ctl->tfull[b], 1);
      umma::mbar_init(&ctl->tempty[b], ZC_EPI);
      umma::mbar_init(&ctl->yfull[b], 1);
      umma::mbar_init(&ctl->yempty[b], ZC_EPI);
    }
    umma::mbar_init(&ctl->drain, 1);
    ctl->abort_f = 0;
    umma::fence_barrier_init();
  }
  if (warp == 0) {
    umma::tmem_alloc(&ctl->tslot, 512);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = ctl->tslot;
  if (threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    ctl->t_start = t;  // in shared memory: no register held across the roles
  }

  if (warp == ZC_EPI) {
    // ------------------------------------------------------------ A / B loader
    // the whole warp walks the steps.  Lane l holds entry q0 + l of the job
    // (fetched 32 at a time, off the per-stage path); lane 0 waits and arms
    // the stage, then lane 0 copies the A tile and lanes 1 .. nblk one whole
    // B block each
    long long step = 0;
    bool ok = true;
    for (int p = 0; p < npair && ok; ++p) {
      // one decision for the whole warp
      if (__shfl_sync(0xffffffffu, lane == 0 ? *abort_f : 0, 0)) break;
      ZcPair<PAIR> pr;
      pr.begin(p, ncj);
      ZcLd L, Lo;  // L: the job of the current tile, Lo: the pair's other job
      zc_ld_job(S, W, cfg.jbeg, pr.r0, L);
      pr.m0 = L.mtz;
      if (pr.two) {
        zc_ld_job(S, W, cfg.jbeg, pr.r1, Lo);
        pr.m1 = Lo.mtz;
      }
      int cur = 0, x, mt;
      while (ok && pr.next(x, mt)) {
        if (x != cur) {
          zc_swap(L, Lo);
          cur = x;
        }
        const int cb = lane - 1;
        const bool has_b = lane >= 1 && lane <= L.nblk;
        for (int q0 = 0; q0 < L.nent && ok; q0 += 32) {
          if (L.held != q0) {
            if (q0 + lane < L.nent) L.mine = W.zc_ents[L.ent + q0 + lane];
            L.held = q0;
          }
          const int nq = min(32, L.nent - q0);
          for (int qq = 0; qq < nq; ++qq, ++step) {
            const int kofs = __shfl_sync(0xffffffffu, L.mine.kofs, qq);
            const int kb = __shfl_sync(0xffffffffu, L.mine.kb, qq);
            const long long d0 = __shfl_sync(0xffffffffu, (long long)L.mine.dz[0], qq);
            const long long d1 = __shfl_sync(0xffffffffu, (long long)L.mine.dz[1], qq);
            const int s = (int)(step % NST);
            bool w = true;
            if (lane == 0) {
              if (step >= NST)
                w = umma::mbar_wait(&ctl->empty[s], (uint32_t)((step / NST - 1) & 1), S.err,
                                    ZC_WAIT);
              w = w && !*abort_f;
            }
            w = __shfl_sync(0xffffffffu, (int)w, 0) != 0;
            if (!w) {
              if (lane == 0) *abort_f = 1;
              ok = false;
              break;
            }
            uint8_t *st = smem + s * STG;
            const uint32_t abytes = (uint32_t)(KS * 128 * kb * 2);
            const uint32_t bbytes = (uint32_t)(KS * kb * 2) * (uint32_t)(L.nblk * L.Rl);
            if (lane == 0) {
              ctl->stkb[s] = kb;  // read by the MMA issuer after the stage lands
              umma::mbar_arrive_expect_tx(&ctl->full[s], abytes + bbytes);
            }
            __syncwarp();
            if (lane == 0) {
              umma::bulk_g2s(st, L.A + ((int64_t)mt * L.ktot + kofs) * KS * 128, abytes,
                             &ctl->full[s]);
            } else if (has_b) {
              // B stage block-major: block b's KS digits of Rl rows x kb at b KS 16 kb
              const int64_t dz = cb == 0 ? d0 : d1;
              const __nv_bfloat16 *src = dz >= 0 ? S.dz + dz : S.dzero;
              umma::bulk_g2s(st + A_BYTES + cb * (KS * 16 * kb * 2), src,
                             (uint32_t)(KS * L.Rl * kb * 2), &ctl->full[s]);
            }
          }
        }
      }
    }
    // drain: the last stages issued must have landed before the CTA exits
    if (lane == 0) {
      const long long first = step > NST ? step - NST : 0;
      for (long long t = first; t < step; ++t)
        umma::mbar_wait(&ctl->full[t % NST], (uint32_t)((t / NST) & 1), S.err, ZC_WAIT);
    }
  } else if (warp == ZC_EPI + 2) {
    // ------------------------------------------------------------ Y loader
    if constexpr (YST) {
      long long hand = 0;
      bool ok = true;
      for (int p = 0; p < npair && ok; ++p) {
        if (__shfl_sync(0xffffffffu, lane == 0 ? *abort_f : 0, 0)) break;
        ZcPair<PAIR> pr;
        pr.begin(p, ncj);
        ZcYJob Y, Yo;
        zc_y_job(S, W, cfg.jbeg, pr.r0, Y);
        pr.m0 = Y.mtz;
        if (pr.two) {
          zc_y_job(S, W, cfg.jbeg, pr.r1, Yo);
          pr.m1 = Yo.mtz;
        }
        int cur = 0, x, mt;
        while (pr.next(x, mt)) {
          if (x != cur) {
            zc_swap(Y, Yo);
            cur = x;
          }
          const int tb = (int)(hand & 1);
          const long long use = hand >> 1;
          bool w = true;
          if (lane == 0) {
            if (use >= 1)
              w = umma::mbar_wait(&ctl->yempty[tb], (uint32_t)((use - 1) & 1), S.err, ZC_WAIT);
            w = w && !*abort_f;
          }
          if (!__shfl_sync(0xffffffffu, (int)w, 0)) {
            if (lane == 0) *abort_f = 1;
            ok = false;
            break;
          }
          ++hand;
          const int al0 = mt * 128 / Y.na, al1 = min(Y.pA - 1, (mt * 128 + 127) / Y.na);
          const int nal = al1 - al0 + 1;
          const uint32_t run = (uint32_t)(Y.nb * 16 * 8);  // one al's [b][16] pairs
          const int n0 = Y.ncb0 * nal, ncopy = n0 + (Y.nblk > 1 ? Y.ncb1 * nal : 0);
          if (lane == 0) umma::mbar_arrive_expect_tx(&ctl->yfull[tb], (uint32_t)ncopy * run);
          __syncwarp();
          for (int q = lane; q < ncopy; q += 32) {
            const int b = q < n0 ? 0 : 1;
            const int r = q - (b ? n0 : 0), k = r / nal, al = al0 + r - k * nal;
            uint8_t *dst = ybuf + (tb * 2 + b) * cfg.ybytes +
                           ((int64_t)(k * nal + (al - al0)) * (Y.nb * 16 + ZC_YPAD)) * 8;
            umma::bulk_g2s(dst, zc_y_global(Y.Y2, (b ? Y.cb1 : Y.cb0) + k, Y.pA, Y.nb, al), run,
                           &ctl->yfull[tb]);
          }
        }
      }
    }
  } else if (warp == ZC_EPI + 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long step = 0, hand = 0;
      // N = R (KS - i) for a block of R rows (16 or 32), 16 KS at most 192
      uint32_t idesc16[KS], idesc32[KS];
#pragma unroll
      for (int i = 0; i < KS; ++i) {
        idesc16[i] = umma::idesc_bf16_f32(128, 16 * (KS - i));
        idesc32[i] = umma::idesc_bf16_f32(128, 32 * (KS - i));
      }
      const uint32_t sbase = umma::smem_u32(smem);
      bool ok = true;
      for (int p = 0; p < npair && ok && !*abort_f; ++p) {
        ZcPair<PAIR> pr;
        pr.begin(p, ncj);
        // entries, blocks and rows per block of the pair's two jobs
        int ne0, nk0, R0, ne1 = 0, nk1 = 0, R1 = 16;
        {
          const ZcJob jb = zc_job(W, cfg.jbeg, pr.r0);
          const WorkItem it = S.items[jb.w];
          ne0 = jb.nent;
          nk0 = jb.nblk;
          R0 = zc_rows(S, jb, it);
          pr.m0 = (S.nabf[it.a] * S.nao[it.a] + 127) / 128;
        }
        if (pr.two) {
          const ZcJob jb = zc_job(W, cfg.jbeg, pr.r1);
          const WorkItem it = S.items[jb.w];
          ne1 = jb.nent;
          nk1 = jb.nblk;
          R1 = zc_rows(S, jb, it);
          pr.m1 = (S.nabf[it.a] * S.nao[it.a] + 127) / 128;
        }
        int x, mt;
        while (ok && !*abort_f && pr.next(x, mt)) {
          const int nent = x ? ne1 : ne0, nblk = x ? nk1 : nk0, R = x ? R1 : R0;
          const int tb = (int)(hand & 1);
          const long long use = hand >> 1;
          if (use >= 1 &&
              !umma::mbar_wait(&ctl->tempty[tb], (uint32_t)((use - 1) & 1), S.err, ZC_WAIT)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          const uint32_t dcol = tbase + (uint32_t)(tb * 256);
          for (int q = 0; q < nent; ++q, ++step) {
            const int s = (int)(step % NST);
            if (!umma::mbar_wait(&ctl->full[s], (uint32_t)((step / NST) & 1), S.err, ZC_WAIT)) {
              ok = false;
              break;
            }
            umma::fence_after_sync();
            const uint32_t a0 = sbase + (uint32_t)(s * STG);
            if (KBM == 16 || ctl->stkb[s] == 16)
              zc_stage_mmas<KS, 16>(a0, a0 + A_BYTES, dcol, nblk, R, idesc16, idesc32, q == 0);
            else
              zc_stage_mmas<KS, 32>(a0, a0 + A_BYTES, dcol, nblk, R, idesc16, idesc32, q == 0);
            umma::mma_commit(&ctl->empty[s]);
          }
          if (!ok) break;
          umma::mma_commit(&ctl->tfull[tb]);
          ++hand;
        }
      }
      if (!ok) *abort_f = 1;
      umma::mma_commit(&ctl->drain);
      umma::mbar_wait(&ctl->drain, 0, S.err, ZC_WAIT);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q4 = warp & 3, hf = warp >> 2;  // TMEM lane quarter, column group
    const int row = q4 * 32 + lane;
    const int et = threadIdx.x;  // 0 .. ZC_ET - 1
    const int rs = cfg.rs;
    long long hand = 0;
    bool aborted = false;
    for (int p = 0; p < npair && !aborted; ++p) {
      const int pp = p & 1;
      ZcPair<PAIR> pr;
      pr.begin(p, ncj);
      // the pair's epilogue data: warps 0 and 1 the jobs' scalars and Sigma
      // offsets, warps 2 + x + 4 hf the column exponents of job x's column
      // group hf.  The previous pair's reads of the column exponents are
      // behind its tile barriers, and its data sit in the other parity.
      if (q4 < 2) {
        if (hf == 0 && (q4 == 0 || pr.two))
          zc_epi_job(S, W, cfg.jbeg, q4 ? pr.r1 : pr.r0, lane, ctl->ej[pp][q4]);
      } else if (q4 == 2 || pr.two) {
        zc_epi_ecol<ZC_CW>(S, W, cfg.jbeg, q4 == 3 ? pr.r1 : pr.r0, hf, lane, ctl->ecol[q4 - 2]);
      }
      asm volatile("bar.sync 1, %0;" ::"r"(ZC_ET) : "memory");
      pr.m0 = ctl->ej[pp][0].mtz;
      if (pr.two) pr.m1 = ctl->ej[pp][1].mtz;
      // job sums of the owned outputs (f32 pairs): jh / jl of the current
      // tile's job, oh / ol of the pair's other job
      float jh[ZC_OWN], jl[ZC_OWN], oh[ZC_OWN], ol[ZC_OWN];
#pragma unroll
      for (int k = 0; k < ZC_OWN; ++k) jh[k] = jl[k] = oh[k] = ol[k] = 0.f;
      int cur = 0, x, mt;
      while (pr.next(x, mt)) {
        if (x != cur) {
#pragma unroll
          for (int k = 0; k < ZC_OWN; ++k) {
            zc_swap(jh[k], oh[k]);
            zc_swap(jl[k], ol[k]);
          }
          cur = x;
        }
        const ZcEpiJob &ej = ctl->ej[pp][x];
        const int pA = ej.pA, na = ej.na, nb = ej.nb;
        const int tb = (int)(hand & 1);
        const uint32_t par = (uint32_t)((hand >> 1) & 1);
        ++hand;
        // this row's exponent, read before the wait so its latency is hidden
        const int eA = (mt * 128 + row < pA * na) ? S.cz_e[ej.czrow0 + mt * 128 + row] : 0;
        // this warp's column group: block hb, its first column c0
        int c0 = 0;
        const int hb = zc_group_block<ZC_CW>(ej.nblk, ej.R0b, hf, c0);
        const int hq = hb > 0 ? 1 : 0;
        const int piece = hb >= 0 ? ej.pc[hq] : 0;
        const int Rh = hq ? 16 : ej.R0b;
        const int noh = ej.nout[hq], ncvh = ej.ncv[hq], gcbh = ej.gcb[hq];
        const int *ecol = ctl->ecol[x] + hf * ZC_CW;
        const float2 *Y2 = reinterpret_cast<const float2 *>(W.scratch + ej.y2off);
        bool okw = umma::mbar_wait(&ctl->tfull[tb], par, S.err, ZC_WAIT);
        if constexpr (YST) {
          if (okw) okw = umma::mbar_wait(&ctl->yfull[tb], par, S.err, ZC_WAIT);
        }
        // the same decision in every epilogue warp
        if (umma::bar_any(!okw || *abort_f, ZC_ET)) {
          *abort_f = 1;
          aborted = true;
          break;
        }
        umma::fence_after_sync();
        const int rowZ = mt * 128 + row;
        const bool rvalid = rowZ < pA * na;
        const int al = rvalid ? rowZ / na : 0;
        const int al0 = mt * 128 / na, al1 = min(pA - 1, (mt * 128 + 127) / na);
        const int nal = al1 - al0 + 1;
        // the order groups (exact f32 integers) summed in double-float, columns
        // (2j, 2j + 1) in the two f32x2 lanes
        constexpr int NP = ZC_CW / 2;
        uint64_t ds[NP], dr[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) ds[j] = dr[j] = 0;
        if (hb >= 0) {
          // the digit-order groups, three loads in flight per wait
          // block hb's order g occupies TMEM columns hb 16 KS + g R .. + R
          const uint32_t ta = tbase + (uint32_t)(tb * 256) + ((uint32_t)(q4 * 32) << 16) +
                              (uint32_t)(hb * 16 * KS + c0);
#pragma unroll
          for (int g0 = 0; g0 < KS; g0 += 3) {
            uint32_t r[3][ZC_CW];
#pragma unroll
            for (int u = 0; u < 3; ++u)
              if (g0 + u < KS) {
                if constexpr (ZC_CW == 8)
                  umma::tmem_ld8_nowait(ta + (uint32_t)((g0 + u) * Rh), r[u]);
                else
                  umma::tmem_ld16_nowait(ta + (uint32_t)((g0 + u) * Rh), r[u]);
              }
            umma::tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              if (g0 + u >= KS) break;
              const float cg = __int_as_float((7 * (KS - 1 - g0 - u) + 127) << 23);
              const uint64_t c2 = f2_pk(cg, cg);
#pragma unroll
              for (int j = 0; j < NP; ++j)
                df_acc2(ds[j], dr[j],
                        f2_mul(f2_pk(__uint_as_float(r[u][2 * j]), __uint_as_float(r[u][2 * j + 1])),
                               c2));
            }
          }
        }
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&ctl->tempty[tb]);
        // Y rows of this thread's al in 16-column block k of G: [b][16] pairs
        auto yrow = [&](int k) -> const float2 * {
          if constexpr (YST)
            return reinterpret_cast<const float2 *>(ybuf + (tb * 2 + hb) * cfg.ybytes) +
                   ((int64_t)k * nal + (al - al0)) * (nb * 16 + ZC_YPAD);
          else
            return zc_y_global(Y2, gcbh + k, pA, nb, al);
        };
        // a tile of at most 32 valid rows (the last of an atom of 13 AOs and 60
        // ABFs holds 12): its rows are all in TMEM lane quarter 0, so that
        // quarter's warps stage Z in rows 32 .. 63 of the reduction buffer
        // (unused by such a tile) and all epilogue warps share the contraction
        const int rv = min(128, pA * na - mt * 128);
        if (PAIR && YST && KBM == 16 && rv <= 32) {
          constexpr int NPT = ZC_CW / 2;
          if (q4 == 0 && hb >= 0 && rvalid) {
            float2 *zs = red + (int64_t)hf * rs * 128 + 32 + row;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
              float2 z0, z1;
              df_fin2(ds[j], dr[j], eA + ecol[2 * j] - SH, eA + ecol[2 * j + 1] - SH, z0, z1);
              const int cend = min(ZC_CW, ncvh - c0);
              zs[(2 * j) * 128] = 2 * j < cend ? z0 : make_float2(0.f, 0.f);
              zs[(2 * j + 1) * 128] = 2 * j + 1 < cend ? z1 : make_float2(0.f, 0.f);
            }
          }
          asm volatile("bar.sync 1, %0;" ::"r"(ZC_ET) : "memory");
          // items (row r, column group q, output o), rows fastest; each output
          // takes the same operations as in the row-per-thread form below
          for (int idx = et; idx < ZC_NQ * 16 * 32; idx += ZC_ET) {
            const int r = idx & 31, qo = idx >> 5, q = qo >> 4, o = qo & 15;
            int cq = 0;
            const int bq = zc_group_block<ZC_CW>(ej.nblk, ej.R0b, q, cq);
            if (r >= rv || bq < 0) continue;
            const int bqi = bq > 0 ? 1 : 0;
            if (o >= ej.nout[bqi]) continue;
            const int cend = min(ZC_CW, ej.ncv[bqi] - cq);
            const float2 *zs = red + (int64_t)q * rs * 128 + 32 + r;
            uint64_t zh[NPT], nzh[NPT], nzl[NPT];
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
              const float2 z0 = zs[(2 * j) * 128], z1 = zs[(2 * j + 1) * 128];
              zh[j] = f2_pk(z0.x, z1.x);
              nzh[j] = f2_pk(-z0.x, -z1.x);
              nzl[j] = f2_pk(-z0.y, -z1.y);
            }
            const int alr = (mt * 128 + r) / na;
            const float2 *yq = reinterpret_cast<const float2 *>(ybuf + (tb * 2 + bq) * cfg.ybytes);
            float2 *outp = red + ((int64_t)q * rs + o) * 128 + r;
            if (ej.pc[bqi] == 1) {
              const float2 *yb = yq + ((int64_t)(cq >> 4) * nal + (alr - al0)) * (nb * 16 + ZC_YPAD);
              zc_contract2<NPT, true>(zh, nzh, nzl, cend, yb + (cq & 15) + o * 16, 1, outp);
            } else {
              const float2 *yb = yq + ((int64_t)(o >> 4) * nal + (alr - al0)) * (nb * 16 + ZC_YPAD);
              zc_contract2<NPT, false>(zh, nzh, nzl, cend, yb + cq * 16 + (o & 15), 1, outp);
            }
          }
        } else if (hb >= 0 && rvalid) {
          const int cend = min(ZC_CW, ncvh - c0);
          float2 *rr = red + (int64_t)hf * rs * 128 + row;
          // Z = (order-group sum) 2^(eA + ecol - SH) as f32 pairs; zero from cend on
          float2 zp[NP][2];
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            df_fin2(ds[j], dr[j], eA + ecol[2 * j] - SH, eA + ecol[2 * j + 1] - SH, zp[j][0],
                    zp[j][1]);
            if (2 * j >= cend) zp[j][0] = make_float2(0.f, 0.f);
            if (2 * j + 1 >= cend) zp[j][1] = make_float2(0.f, 0.f);
          }
          if constexpr (YST) {
            // Z as column pairs for the packed contraction
            uint64_t zh[NP], nzh[NP], nzl[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
              zh[j] = f2_pk(zp[j][0].x, zp[j][1].x);
              nzh[j] = f2_pk(-zp[j][0].x, -zp[j][1].x);
              nzl[j] = f2_pk(-zp[j][0].y, -zp[j][1].y);
            }
            if (piece == 1) {
              // out b: Y[al][b][G, g = c0 + c]
              zc_contract2<NP, true>(zh, nzh, nzl, cend, yrow(c0 >> 4) + (c0 & 15), noh, rr);
            } else {
              // out g: Y[al][b = c0 + c][G, g], one 16-column block of g at a time
              for (int k = 0; 16 * k < noh; ++k)
                zc_contract2<NP, false>(zh, nzh, nzl, cend, yrow(k) + c0 * 16,
                                        min(16, noh - 16 * k), rr + 16 * k * 128);
            }
          } else {
            float2 z[ZC_CW];
#pragma unroll
            for (int c = 0; c < ZC_CW; ++c) z[c] = zp[c >> 1][c & 1];
            if (piece == 1) {
              zc_contract<ZC_CW>(z, cend, yrow(c0 >> 4) + (c0 & 15), 16, 1, noh, rr);
            } else {
              for (int k = 0; 16 * k < noh; ++k)
                zc_contract<ZC_CW>(z, cend, yrow(k) + c0 * 16, 1, 16, min(16, noh - 16 * k),
                                   rr + 16 * k * 128);
            }
          }
        }
        __syncwarp();
        if constexpr (YST) {
          if (lane == 0) umma::mbar_arrive(&ctl->yempty[tb]);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ZC_ET) : "memory");
        // owners: (block, a, o) summed over the tile's rows (al, a) and the
        // block's column groups, in a fixed order
        const int nout0 = ej.nout[0];
        const int own0 = na * nout0, nown = own0 + na * ej.nout[1];
        unsigned qm0 = 0, qm1 = 0;  // column groups feeding block 0 and block 1 (bit q)
#pragma unroll
        for (int q = 0; q < ZC_NQ; ++q) {
          int cq;
          const int bq = zc_group_block<ZC_CW>(ej.nblk, ej.R0b, q, cq);
          qm0 |= (bq == 0 ? 1u : 0u) << q;
          qm1 |= (bq == 1 ? 1u : 0u) << q;
        }
        const int r0 = mt * 128, rend = min(pA * na, r0 + 128);
        const int ph = r0 % na;
#pragma unroll
        for (int k = 0; k < ZC_OWN; ++k) {
          const int idx = et + k * ZC_ET;
          if (idx >= nown) break;
          const bool b1 = idx >= own0;
          const int rem = idx - (b1 ? own0 : 0);
          const int o = rem / na, a = rem - o * na;  // consecutive owners: consecutive a
          const unsigned qm = b1 ? qm1 : qm0;
          int d = a - ph;
          if (d < 0) d += na;
          float h = jh[k], l = jl[k];
#pragma unroll
          for (int q = 0; q < ZC_NQ; ++q) {
            if (!((qm >> q) & 1u)) continue;
            const float2 *rq = red + ((int64_t)q * rs + o) * 128;
            int lr = d;
            // two rows per step: both loads in flight before the adds
            for (; lr + na < rend - r0; lr += 2 * na) {
              const float2 v0 = rq[lr], v1 = rq[lr + na];
              df_add(h, l, v0);
              df_add(h, l, v1);
            }
            if (lr < rend - r0) df_add(h, l, rq[lr]);
          }
          jh[k] = h;
          jl[k] = l;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ZC_ET) : "memory");
        if (mt + 1 < ej.mtz) continue;
        // the job's last tile: add its finished blocks to Sigma (and mirrors);
        // a sum outside the fixed-point range is not added and fails the build
        bool inrange = true;
#pragma unroll
        for (int k = 0; k < ZC_OWN; ++k)
          if (et + k * ZC_ET < nown) inrange = inrange && fx_df_in_range(jh[k]);
        if (!inrange) atomicOr(S.err, HFX_DEV_ERR_BOUNDS);
#pragma unroll
        for (int k = 0; k < ZC_OWN && inrange; ++k) {
          const int idx = et + k * ZC_ET;
          if (idx >= nown) break;
          const int b1 = idx >= own0 ? 1 : 0;
          const int nob = ej.nout[b1];
          const int rem = idx - (b1 ? own0 : 0);
          const int o = rem / na, a = rem - o * na;
          const int64_t t0 = ej.sg[b1][0], t1 = ej.sg[b1][1];
          if (t0 < 0) continue;  // missing key: recorded when the pair started
          const float2 v = make_float2(jh[k], jl[k]);
          fx_add_df(S.acc + 2 * (t0 + (int64_t)a * nob + o), v, true);
          if (t1 >= 0) fx_add_df(S.acc + 2 * (t1 + (int64_t)o * na + a), v, true);
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, 512);
  if (threadIdx.x == 0) {
    unsigned long long t_end;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
    W.cta_ns[cfg.cta0 + blockIdx.x] = (long long)(t_end - ctl->t_start);
  }
}

// Y staged in shared memory (two buffers per block) with a shorter operand
// ring, or read from global memory with a deeper ring.
constexpr bool ZC_STAGE_Y = true;

template <int KS>
cudaError_t zc_range_t(const SplitShared &S, const SplitWave &W, const ZcPlanShape &P, int nsm,
                       int jbeg, int jend, int cta0, bool small, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(jend - jbeg, nsm);
  if (blocks <= 0) return cudaSuccess;
  constexpr size_t kMax = 227 * 1024;
  const int rs = P.nout_max <= 16 ? 16 : 32;
  auto smem_of = [&](int nst, int kbm, int ybytes, int nq) {
    return (size_t)nst * KS * (128 + ZC_COLS) * kbm * 2 + 4 * (size_t)ybytes +
           (size_t)nq * 128 * rs * sizeof(float2) + sizeof(ZcSmem) + 64;
  };
  auto launch = [&](auto kern, int threads, int nst, int kbm, int ybytes, int nq) -> cudaError_t {
    const size_t smem = smem_of(nst, kbm, ybytes, nq);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, st>>>(S, W, ZcCfg{ybytes, rs, jbeg, jend, cta0});
    return cudaGetLastError();
  };
  // 8 epilogue warps (2 column groups of 16).  16 warps (4 groups of 8) leave
  // room for only two operand stages next to the staged Y and were slower.
  constexpr int T8 = ZcGeo<8>::THREADS;
  // Jobs are taken in heavy/light pairs by the small class's four-stage
  // variant (every block and atom A of at most 16 AOs) and by both variants
  // of the large-block class; the small class's fallbacks, for cells whose
  // staged Y does not fit next to four stages, keep one job at a time.
  if (P.kbmax <= 16) {
    if (ZC_STAGE_Y && smem_of(4, 16, P.ybytes, 2) <= kMax) {
      if (small) return launch(k_zc<KS, 16, 4, 8, true, true>, T8, 4, 16, P.ybytes, 2);
      return launch(k_zc<KS, 16, 4, 8, true, false>, T8, 4, 16, P.ybytes, 2);
    }
    if (ZC_STAGE_Y && smem_of(3, 16, P.ybytes, 2) <= kMax)
      return launch(k_zc<KS, 16, 3, 8, true, false>, T8, 3, 16, P.ybytes, 2);
    return launch(k_zc<KS, 16, 3, 8, false, false>, T8, 3, 16, 0, 2);
  }
  if (ZC_STAGE_Y && smem_of(2, 32, P.ybytes, 2) <= kMax)
    return launch(k_zc<KS, 32, 2, 8, true, true>, T8, 2, 32, P.ybytes, 2);
  return launch(k_zc<KS, 32, 2, 8, false, true>, T8, 2, 32, 0, 2);
}

// The wave's small-class jobs [0, nsmall) with the shape of blocks of at most
// 16 AOs, then the others with the system's shape.
template <int KS>
cudaError_t zc_run_t(const SplitShared &S, const SplitWave &W, const ZcPlanShape &P, int nsm,
                     int nsmall, cudaStream_t st) {
  const int njobs = (int)W.h_zc_jobs;
  if (nsmall > 0) {
    const ZcPlanShape Q{16, 16, P.ybytes_small, P.ybytes_small};
    cudaError_t e = zc_range_t<KS>(S, W, Q, nsm, 0, nsmall, 0, true, st);
    if (e != cudaSuccess) return e;
  }
  if (njobs > nsmall)
    return zc_range_t<KS>(S, W, P, nsm, nsmall, njobs, nsm, false, st);
  return cudaSuccess;
}

template <int KS>
cudaError_t dz_prepare_t(const SplitShared &S, cudaStream_t st) {
  if (S.h_nd <= 0) return cudaSuccess;
  k_dz_exp<<<(unsigned)S.h_nd, 128, 0, st>>>(S);
  k_dz_slice<KS><<<(unsigned)S.h_nd, 128, 0, st>>>(S);
  return cudaGetLastError();
}

template <int KS>
cudaError_t slice_cz_t(const SplitShared &S, cudaStream_t st) {
  if (S.h_cz_rows > 0)
    k_slice_cz<KS><<<(unsigned)((S.h_cz_rows * 32 + 255) / 256), 256, 0, st>>>(S);
  return cudaGetLastError();
}

}  // namespace split

cudaError_t split_zc_plan(const SplitShared &S, const SplitWave &W, int fill, cudaStream_t st) {
  if (W.nw <= 0) return cudaSuccess;
  split::k_zc_plan<<<(unsigned)((W.nw + 3) / 4), 128, 0, st>>>(S, W, fill);
  return cudaGetLastError();
}

cudaError_t split_zc_run(const SplitShared &S, const SplitWave &W, int ks, const ZcPlanShape &P,
                         int nsm, int nsmall, cudaStream_t st) {
  switch (ks) {
    case 2: return split::zc_run_t<2>(S, W, P, nsm, nsmall, st);
    case 4: return split::zc_run_t<4>(S, W, P, nsm, nsmall, st);
    case 5: return split::zc_run_t<5>(S, W, P, nsm, nsmall, st);
    case 6: return split::zc_run_t<6>(S, W, P, nsm, nsmall, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t split_dz_prepare(const SplitShared &S, int ks, cudaStream_t st) {
  switch (ks) {
    case 2: return split::dz_prepare_t<2>(S, st);
    case 4: return split::dz_prepare_t<4>(S, st);
    case 5: return split::dz_prepare_t<5>(S, st);
    case 6: return split::dz_prepare_t<6>(S, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t split_slice_cz(const SplitShared &S, int ks, cudaStream_t st) {
  switch (ks) {
    case 2: return split::slice_cz_t<2>(S, st);
    case 4: return split::slice_cz_t<4>(S, st);
    case 5: return split::slice_cz_t<5>(S, st);
    case 6: return split::slice_cz_t<6>(S, st);
    default: return cudaErrorInvalidValue;
  }
}
