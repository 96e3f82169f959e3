// HFX_OZAKI: the Y = V C product and the D_AB piece (Sigma_FG -= C_AF^T P_G)
// of Algorithm 3 as exact split-precision tcgen05 products, in one persistent
// kernel per wave.
//
// A job is a 128-row x 64-column output tile over all its K tiles of 32.
// The MMAs hand the accumulator to the epilogue after every 20 K tiles (so
// every digit-order group sum stays an exact f32 integer), and the epilogue
// adds up the chunks before it writes the tile once: in int64 for D_AB, in
// packed double-float for Y (whose result is an f32 pair anyway):
//   Y job:    rows (b, G, g) of C_B transposed, columns al of V_AB, K = beta;
//   D_AB job: rows (F, f) of C_A, columns (G, g) of P, K = (al, a).
// Both operands are stored as KS balanced base-128 bf16 digits, one exponent
// per row; the B digits of a K tile are contiguous, so one MMA with A digit i
// covers up to four B digits j stacked along N at TMEM column 64 (i + j): 9
// MMAs per K step of 16 instead of KS (KS + 1) / 2 = 21 for KS = 6.
//
// Roles (one CTA per SM, static round-robin over the wave's jobs; warp
// numbers of Y jobs, those of D_AB jobs in parentheses): warp 16 (8) copies
// each K tile's A and B digits (lanes 0 and 1, 1-D bulk copies) into a ring
// of shared stages; warp 18 (10) writes each job's epilogue data into one of
// two shared slots, off the epilogue's and the loader's paths (Y jobs: row
// exponents and Y2 offsets, column exponents; D_AB jobs: the rows' (F, f) and
// columns' (G, g) decoding with their exponents and the tile's Sigma_FG
// offsets per block pair); warp 17 (9) issues the MMAs into the TMEM
// accumulator; warps 0-15 (0-7), TMEM lanes 32 (w % 4).. and columns 16 (32)
// (w / 4).., drain the accumulator into those sums, release it to the next
// job's MMAs, and then write Y (f32 pairs, and FP64 where read) or add the
// surviving Sigma_FG blocks to the fixed-point Sigma.  Every wait is bounded:
// on expiry the kernel records HFX_DEV_ERR_TIMEOUT, drains its copies and
// MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "hfx_split.h"
#include "split_common.cuh"

namespace split {

// Epilogue warps: 4 TMEM lane quarters x EPI / 4 groups of CW columns.  Y
// jobs take 16 warps of 16 columns (96 registers, the budget of 20 warps, as
// warps are placed four per scheduler): with 8 the epilogue had two warps per
// scheduler to hide its latencies.  D_AB jobs keep 8 warps of 32 columns.
template <int JOB>
struct PgGeo {
  static constexpr int EPI = JOB == 0 ? 16 : 8;
  static constexpr int CW = NT / (EPI / 4);
  static constexpr int THREADS = (EPI + 3) * 32;  // + loader, MMA and job-data warps
  // job-data slots: Y jobs are short, so their data run further ahead
  static constexpr int NMS = JOB == 0 ? 4 : 2;
};
constexpr int PG_NST = 3;                      // operand stages
constexpr long long PG_WAIT = 2000000000ll;    // cycles per bounded wait

struct PgSmem {
  uint64_t full[PG_NST], empty[PG_NST], tfull, tempty, drain;
  uint64_t mfull[4], mempty[4];  // the epilogue-data ring (PgMetaY / PgMetaD slots)
  uint32_t tslot;
  int abort_f;
};

constexpr int PG_CTL_BYTES = (int)((sizeof(PgSmem) + 15) / 16 * 16);

// One Y job's epilogue data, written by the job-data warp ahead of the job into
// one of two slots, so the epilogue reads shared memory instead of running a
// chain of dependent global loads per job.
struct PgMetaY {
  int64_t y2base;     // scratch offset (doubles) of the pair's Y2 region
  int64_t y64base;    // scratch offset of the pair's FP64 Y region
  int32_t pA, nbY, nrowY, pad;
  int32_t y2row[TM];  // Y2 offset (pairs) of each row, -1: the row is not stored;
                      // below 2^31: at most 512 blocks of 16 x 256 x 32 x 16 pairs
  int16_t ea[TM];     // row exponents
  int16_t eb[NT];     // column exponents (0 beyond nabf(A))
};

// One D_AB job's epilogue data, written by the job-data warp ahead of the job:
// the row (F, f) and column (G, g) decoding of the tile and, when the tile
// spans at most PG_TBL (F block, G block) pairs, each pair's Sigma_FG offset
// and that of its mirror (-1: no surviving term or no mirror).
constexpr int PG_TBL = 160;
struct PgMetaD {
  int32_t fb0, gb0, nfb, ngb;  // first F and G neighbour index of the tile, block counts
  int32_t tbl, mir, pad0, pad1;  // tbl: the offset table is filled; mir: mirror adds
  int16_t fi[TM];     // row's F - fb0, -1: row past the atom's neighbour columns
  int8_t f[TM], nf[TM];
  int16_t ea[TM];     // row exponents
  int16_t gi[NT];     // column's G - gb0, -1: column past the pair's columns
  int8_t g[NT], ng[NT];
  int16_t eb[NT];     // column exponents
  int64_t off[PG_TBL], moff[PG_TBL];  // [fi * ngb + gi]
};

// Fill m for D_AB job jb (the whole job-data warp); loads issued level by level.
__device__ __forceinline__ void dab_meta_fill(const SplitShared &S, const SplitWave &W,
                                              const Job &jb, const WorkItem &it, PgMetaD &m,
                                              int lane) {
  constexpr int RPL = TM / 32, CPL = NT / 32;
  const int wl = (int)(jb.w - W.w0);
  const int ncolA = S.ncol[it.a], ncolB = S.ncol[it.b];
  const int64_t coloffA = S.coloff[it.a], coloffB = S.coloff[it.b];
  const int16_t *ea_p = S.c4_e + S.c4_rowpre[it.a] + jb.mt * TM;
  const int16_t *eb_p = W.ps_e + W.p_rowpre[wl] + jb.nt * NT;
  int F[RPL], G[CPL];
  bool rv[RPL], cv[CPL];
  int16_t ea[RPL], eb[CPL];
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int rF = jb.mt * TM + lane + 32 * u;
    rv[u] = rF < ncolA;
    F[u] = rv[u] ? S.colG[coloffA + rF] : 0;
    ea[u] = ea_p[lane + 32 * u];
  }
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int cG = jb.nt * NT + lane + 32 * u;
    cv[u] = cG < ncolB;
    G[u] = cv[u] ? S.colG[coloffB + cG] : 0;
    eb[u] = cv[u] ? eb_p[lane + 32 * u] : (int16_t)0;
  }
  NbrEntry ef[RPL], eg[CPL];
#pragma unroll
  for (int u = 0; u < RPL; ++u) ef[u] = S.nbr[it.fbase + F[u]];
#pragma unroll
  for (int u = 0; u < CPL; ++u) eg[u] = S.nbr[it.gbase + G[u]];
  int fmax = 0, gmax = 0;
#pragma unroll
  for (int u = 0; u < RPL; ++u) fmax = max(fmax, rv[u] ? F[u] : 0);
#pragma unroll
  for (int u = 0; u < CPL; ++u) gmax = max(gmax, cv[u] ? G[u] : 0);
  for (int o = 16; o; o >>= 1) {
    fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
    gmax = max(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  }
  // rows and columns are ordered by neighbour index: row 0 and column 0 hold
  // the first blocks (a job's tile always starts inside the pair's columns)
  const int fb0 = __shfl_sync(0xffffffffu, F[0], 0), gb0 = __shfl_sync(0xffffffffu, G[0], 0);
  const int nfb = fmax - fb0 + 1, ngb = gmax - gb0 + 1;
  const bool tbl = nfb * ngb <= PG_TBL;
  const bool mir = S.sym && it.role == 1;
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int r = lane + 32 * u;
    m.fi[r] = rv[u] ? (int16_t)(F[u] - fb0) : (int16_t)-1;
    m.f[r] = (int8_t)(rv[u] ? jb.mt * TM + r - ef[u].aopre : 0);
    m.nf[r] = (int8_t)(rv[u] ? S.nao[ef[u].other] : 0);
    m.ea[r] = ea[u];
  }
#pragma unroll
  for (int u = 0; u < CPL; ++u) {
    const int c = lane + 32 * u;
    m.gi[c] = cv[u] ? (int16_t)(G[u] - gb0) : (int16_t)-1;
    m.g[c] = (int8_t)(cv[u] ? jb.nt * NT + c - eg[u].aopre : 0);
    m.ng[c] = (int8_t)(cv[u] ? S.nao[eg[u].other] : 0);
    m.eb[c] = eb[u];
  }
  if (lane == 0) {
    m.fb0 = fb0;
    m.gb0 = gb0;
    m.nfb = nfb;
    m.ngb = ngb;
    m.tbl = tbl ? 1 : 0;
    m.mir = mir ? 1 : 0;
  }
  if (!tbl) return;
  // Sigma_FG offsets of the tile's (F, G) block pairs with a surviving D_AB term
  for (int q = lane; q < nfb * ngb; q += 32) {
    const int Fq = fb0 + q / ngb, Gq = gb0 + q % ngb;
    const NbrEntry a = S.nbr[it.fbase + Fq], b = S.nbr[it.gbase + Gq];
    const uint32_t mw = S.masks[it.mask_off + ((int64_t)Gq * 4 + 3) * it.nFw + (Fq >> 5)];
    int64_t off = -1, moff = -1;
    if ((mw >> (Fq & 31)) & 1u) {
      const int n0 = it.n[0] + b.n[0] - a.n[0], n1 = it.n[1] + b.n[1] - a.n[1],
                n2 = it.n[2] + b.n[2] - a.n[2];
      off = dh_find(S.shash, hk_pack(a.other, b.other, n0, n1, n2));
      if (mir) moff = dh_find(S.shash, hk_pack(b.other, a.other, -n0, -n1, -n2));
      if (off < 0 || (mir && moff < 0)) {
        atomicOr(S.err, HFX_DEV_ERR_MISSING);
        off = moff = -1;
      }
    }
    m.off[q] = off;
    m.moff[q] = moff;
  }
}

// Sigma_FG offset and mirror offset of the block pair (F, G) of job jb (-1:
// no surviving term), for tiles whose pairs do not fit the slot's table.
__device__ __noinline__ void dab_lookup(const SplitShared &S, const Job &jb, int Fa, int Ga,
                                        bool mir, int64_t &off, int64_t &moff) {
  const WorkItem it = S.items[jb.w];
  const NbrEntry ef = S.nbr[it.fbase + Fa], eg = S.nbr[it.gbase + Ga];
  const uint32_t mw = S.masks[it.mask_off + ((int64_t)Ga * 4 + 3) * it.nFw + (Fa >> 5)];
  off = moff = -1;
  if (!((mw >> (Fa & 31)) & 1u)) return;
  const int n0 = it.n[0] + eg.n[0] - ef.n[0], n1 = it.n[1] + eg.n[1] - ef.n[1],
            n2 = it.n[2] + eg.n[2] - ef.n[2];
  off = dh_find(S.shash, hk_pack(ef.other, eg.other, n0, n1, n2));
  if (mir) moff = dh_find(S.shash, hk_pack(eg.other, ef.other, -n0, -n1, -n2));
  if (off < 0 || (mir && moff < 0)) {
    atomicOr(S.err, HFX_DEV_ERR_MISSING);
    off = moff = -1;
  }
}

// Fill m for Y job jb (the whole job-data warp; lane l takes rows l, l + 32,
// l + 64, l + 96).  The loads are issued level by level for the four rows at
// once, so the dependent chain is three loads deep, not twelve.
__device__ __forceinline__ void y_meta_fill(const SplitShared &S, const SplitWave &W,
                                            const Job &jb, const WorkItem &it, PgMetaY &m,
                                            int lane) {
  constexpr int RPL = TM / 32;  // rows per lane
  const int wl = (int)(jb.w - W.w0);
  const int nbY = S.nao[it.b], ncol = S.ncol[it.b], pA = S.nabf[it.a];
  const int64_t coloff = S.coloff[it.b];
  const int16_t *ea_p = S.cy_e + S.cy_rowpre[it.b] + jb.mt * TM;
  const int16_t *eb_p = S.vs_e + S.v_rowpre[it.vblk] + jb.nt * NT;
  const int nrowY = nbY * ncol;
  if (lane == 0) {
    m.y2base = W.y2_on ? W.y2_off[wl] : 0;
    m.y64base = W.y_off[wl];
    m.pA = pA;
    m.nbY = nbY;
    m.nrowY = nrowY;
  }
  int b[RPL], col[RPL], G[RPL];
  bool live[RPL];
  int16_t ea[RPL];
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int rowY = jb.mt * TM + lane + 32 * u;
    live[u] = rowY < nrowY && W.y2_on;
    b[u] = live[u] ? rowY / ncol : 0;
    col[u] = live[u] ? rowY - b[u] * ncol : 0;
    ea[u] = ea_p[lane + 32 * u];  // padded rows hold the slicing's exponent too
  }
#pragma unroll
  for (int u = 0; u < RPL; ++u) G[u] = live[u] ? S.colG[coloff + col[u]] : 0;
  int aopre[RPL], kofs[RPL];
  unsigned bits[RPL];
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    aopre[u] = live[u] ? S.nbr[it.gbase + G[u]].aopre : 0;
    kofs[u] = live[u] ? S.kofs[it.gbase + G[u]] : 0;
    bits[u] = live[u] ? S.wg[it.wg_off + G[u]] : 0u;
  }
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    // only rows of G with survivors are read: the f32 pairs by the D_FG /
    // D_FB products and by P of the D_AB piece
    int32_t y2 = -1;
    if (live[u] && (bits[u] & 11u)) {
      const int g = col[u] - aopre[u];
      y2 = (((kofs[u] / 16 + g / 16) * pA) * nbY + b[u]) * 16 + (g & 15);
    }
    m.y2row[lane + 32 * u] = y2;
    m.ea[lane + 32 * u] = ea[u];
  }
  const int ncl = pA - jb.nt * NT;
#pragma unroll
  for (int u = 0; u < NT / 32; ++u) {
    const int c = lane + 32 * u;
    m.eb[c] = c < ncl ? eb_p[c] : (int16_t)0;
  }
}

// Operand tiles, exponents and K range of job jb.
template <int KS, int JOB>
__device__ __forceinline__ void pg_operands(const SplitShared &S, const SplitWave &W,
                                            const Job &jb, const WorkItem &it,
                                            const __nv_bfloat16 *&Ab, const __nv_bfloat16 *&Bb,
                                            const int16_t *&ea_p, const int16_t *&eb_p) {
  const int wl = (int)(jb.w - W.w0);
  if (JOB == 0) {
    const int kt = S.ktY[it.b];
    Ab = S.cy + S.cy_base[it.b] + ((int64_t)jb.mt * kt + jb.k0) * KS * TM * TK;
    Bb = S.vs + S.vs_base[it.vblk] + ((int64_t)jb.nt * kt + jb.k0) * KS * NT * TK;
    ea_p = S.cy_e + S.cy_rowpre[it.b] + jb.mt * TM;
    eb_p = S.vs_e + S.v_rowpre[it.vblk] + jb.nt * NT;
  } else {
    const int kt = S.kt4[it.a];
    Ab = S.c4 + S.c4_base[it.a] + ((int64_t)jb.mt * kt + jb.k0) * KS * TM * TK;
    Bb = W.ps + W.ps_base[wl] + ((int64_t)jb.nt * kt + jb.k0) * KS * NT * TK;
    ea_p = S.c4_e + S.c4_rowpre[it.a] + jb.mt * TM;
    eb_p = W.ps_e + W.p_rowpre[wl] + jb.nt * NT;
  }
}

template <int KS, int JOB>
__global__ void __launch_bounds__(PgGeo<JOB>::THREADS, 1) k_pgemm(SplitShared S, SplitWave W) {
  constexpr int PG_EPI = PgGeo<JOB>::EPI, PG_CW = PgGeo<JOB>::CW, PG_NMS = PgGeo<JOB>::NMS;
  constexpr int A_BYTES = KS * TM * TK * 2;
  constexpr int B_BYTES = KS * NT * TK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr int SH = 7 * (KS + 1);
  extern __shared__ __align__(1024) uint8_t smem[];
  PgSmem *ctl = reinterpret_cast<PgSmem *>(smem + PG_NST * STAGE);
  PgMetaY *meta = reinterpret_cast<PgMetaY *>(smem + PG_NST * STAGE + PG_CTL_BYTES);
  PgMetaD *metaD = reinterpret_cast<PgMetaD *>(smem + PG_NST * STAGE + PG_CTL_BYTES);
  volatile int *abort_f = &ctl->abort_f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int njobs = W.njobs[JOB];
  const Job *jobs = JOB == 0 ? W.jobs : W.jobs4;

  if (threadIdx.x == 0) {
    for (int s = 0; s < PG_NST; ++s) {
      umma::mbar_init(&ctl->full[s], 1);
      umma::mbar_init(&ctl->empty[s], 1);
    }
    umma::mbar_init(&ctl->tfull, 1);
    umma::mbar_init(&ctl->tempty, PG_EPI);
    umma::mbar_init(&ctl->drain, 1);
    for (int m = 0; m < PG_NMS; ++m) {
      umma::mbar_init(&ctl->mfull[m], 1);
      umma::mbar_init(&ctl->mempty[m], PG_EPI);
    }
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

  if (warp == PG_EPI) {
    // ------------------------------------------------------------ loader
    long long step = 0;
    // descriptors two jobs ahead and work items one job ahead, so a job's
    // operand addresses wait on one level of loads (Y jobs have two K tiles)
    const int G = (int)gridDim.x;
    const int j0 = blockIdx.x;
    Job jn1 = j0 < njobs ? jobs[j0] : Job{};
    Job jn2 = j0 + G < njobs ? jobs[j0 + G] : Job{};
    WorkItem itn1 = j0 < njobs ? S.items[jn1.w] : WorkItem{};
    for (int j = j0; j < njobs; j += G) {
      if (__shfl_sync(0xffffffffu, lane == 0 ? *abort_f : 0, 0)) break;
      const Job jb = jn1;
      const WorkItem it = itn1;
      jn1 = jn2;
      if (j + G < njobs) itn1 = S.items[jn1.w];
      if (j + 2 * G < njobs) jn2 = jobs[j + 2 * G];
      const __nv_bfloat16 *Ab, *Bb;
      const int16_t *ea_p, *eb_p;
      pg_operands<KS, JOB>(S, W, jb, it, Ab, Bb, ea_p, eb_p);
      bool ok = true;
      for (int kt = 0; kt < jb.nk; ++kt, ++step) {
        const int s = (int)(step % PG_NST);
        bool w = true;
        if (lane == 0) {
          if (step >= PG_NST)
            w = umma::mbar_wait(&ctl->empty[s], (uint32_t)((step / PG_NST - 1) & 1), S.err,
                                PG_WAIT);
          w = w && !*abort_f;
        }
        w = __shfl_sync(0xffffffffu, (int)w, 0) != 0;
        if (!w) {
          if (lane == 0) *abort_f = 1;
          ok = false;
          break;
        }
        uint8_t *st = smem + s * STAGE;
        if (lane == 0) umma::mbar_arrive_expect_tx(&ctl->full[s], STAGE);
        __syncwarp();
        if (lane == 0)
          umma::bulk_g2s(st, Ab + (int64_t)kt * KS * TM * TK, A_BYTES, &ctl->full[s]);
        else if (lane == 1)
          umma::bulk_g2s(st + A_BYTES, Bb + (int64_t)kt * KS * NT * TK, B_BYTES, &ctl->full[s]);
      }
      if (!ok) break;
    }
    // drain: the last stages issued must have landed before the CTA exits
    if (lane == 0) {
      const long long first = step > PG_NST ? step - PG_NST : 0;
      for (long long t = first; t < step; ++t)
        umma::mbar_wait(&ctl->full[t % PG_NST], (uint32_t)((t / PG_NST) & 1), S.err, PG_WAIT);
    }
  } else if (warp == PG_EPI + 2) {
    // ------------------------------------------------------------ job data
    // each job with K tiles gets its epilogue data in slot mcount % NMS once the
    // slot's previous job is done with it; this warp waits on nothing but the
    // epilogue, so the loader's copies never wait for these loads
    long long mcount = 0;
    Job jnext = blockIdx.x < njobs ? jobs[blockIdx.x] : Job{};  // a job ahead
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
      if (__shfl_sync(0xffffffffu, lane == 0 ? *abort_f : 0, 0)) break;
      const Job jb = jnext;
      if (j + (int)gridDim.x < njobs) jnext = jobs[j + gridDim.x];
      if (jb.nk == 0) continue;  // the epilogue skips it too
      const WorkItem it = S.items[jb.w];
      const int ms = (int)(mcount % PG_NMS);
      const long long use = mcount / PG_NMS;
      bool w = true;
      if (lane == 0) {
        if (use >= 1)
          w = umma::mbar_wait(&ctl->mempty[ms], (uint32_t)((use - 1) & 1), S.err, PG_WAIT);
        w = w && !*abort_f;
      }
      if (!__shfl_sync(0xffffffffu, (int)w, 0)) {
        if (lane == 0) *abort_f = 1;
        break;
      }
      if constexpr (JOB == 0) y_meta_fill(S, W, jb, it, meta[ms], lane);
      else dab_meta_fill(S, W, jb, it, metaD[ms], lane);
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&ctl->mfull[ms]);
      ++mcount;
    }
  } else if (warp == PG_EPI + 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long step = 0, hand = 0;
      // MMA i, chunk c: A digit i times B digits [4c, 4c + n), n = min(4, KS - i - 4c)
      uint32_t idesc[4];
#pragma unroll
      for (int n = 1; n <= 4; ++n) idesc[n - 1] = umma::idesc_bf16_f32(TM, NT * n);
      Job jnext = blockIdx.x < njobs ? jobs[blockIdx.x] : Job{};  // a job ahead
      for (int j = blockIdx.x; j < njobs && !*abort_f; j += gridDim.x) {
        const Job jb = jnext;
        if (j + (int)gridDim.x < njobs) jnext = jobs[j + gridDim.x];
        if (jb.nk == 0) continue;  // an empty job (a skipped candidate tile)
        bool ok = true;
        // K chunks of at most KT_CHUNK tiles, one accumulator handoff each
        for (int k0 = 0; k0 < jb.nk && ok; k0 += KT_CHUNK) {
        if (hand >= 1 &&
            !umma::mbar_wait(&ctl->tempty, (uint32_t)((hand - 1) & 1), S.err, PG_WAIT)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const int k1 = min(jb.nk, k0 + KT_CHUNK);
        for (int kt = k0; kt < k1; ++kt, ++step) {
          const int s = (int)(step % PG_NST);
          if (!umma::mbar_wait(&ctl->full[s], (uint32_t)((step / PG_NST) & 1), S.err, PG_WAIT)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          const uint32_t a0 = umma::smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
          for (int ks = 0; ks < TK / 16; ++ks)
#pragma unroll
            for (int i = 0; i < KS; ++i)
#pragma unroll
              for (int c = 0; c * 4 < KS - i; ++c) {
                const int n = min(4, KS - i - 4 * c);
                const uint64_t ad = umma::smem_desc(a0 + i * TM * TK * 2 + ks * 256, 128, 512);
                const uint64_t bd =
                    umma::smem_desc(b0 + 4 * c * NT * TK * 2 + ks * 256, 128, 512);
                // the two MMAs of digit 0 write every column of a chunk's first step
                umma::mma_bf16(tbase + (uint32_t)((i + 4 * c) * NT), ad, bd, idesc[n - 1],
                               ((kt - k0) | ks | i) ? 1u : 0u);
              }
          umma::mma_commit(&ctl->empty[s]);
        }
        if (!ok) break;
        umma::mma_commit(&ctl->tfull);
        ++hand;
        }
        if (!ok) { *abort_f = 1; break; }
      }
      umma::mma_commit(&ctl->drain);
      umma::mbar_wait(&ctl->drain, 0, S.err, PG_WAIT);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q4 = warp & 3, hf = warp >> 2;
    const int row = q4 * 32 + lane;
    const int c0 = hf * PG_CW;  // this warp's PG_CW of the 64 columns
    long long hand = 0;
    long long mcount = 0;
    // the next job's descriptor is loaded a job ahead
    Job jnext = blockIdx.x < njobs ? jobs[blockIdx.x] : Job{};
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
      const Job jb = jnext;
      if (j + (int)gridDim.x < njobs) jnext = jobs[j + gridDim.x];
      if (jb.nk == 0) continue;  // no MMAs, no accumulator handoff
      int ea;
      // Y: the column exponents (pairs of int16)
      uint32_t ebp[JOB == 0 ? PG_CW / 2 : 1];
      bool valid;
      // Y job: row (b, G, g) of Y, Y2 row, FP64 need, Y regions
      int64_t yrow = 0, y2row = -1, nrowY = 0, y2base = 0, y64base = 0;
      bool need64 = false;
      int pA = 0, nbY = 0;
      // D_AB job: row (F - fb0, f) and the slot holding the job's data
      int F = 0, nf = 0, f = 0, dms = 0;
      if constexpr (JOB == 0) {
        // the job-data warp wrote this job's data into slot mcount % NMS
        const int ms = (int)(mcount % PG_NMS);
        const bool okm = umma::mbar_wait(&ctl->mfull[ms], (uint32_t)((mcount / PG_NMS) & 1), S.err,
                                         PG_WAIT);
        ++mcount;
        if (umma::bar_any(!okm || *abort_f, PG_EPI * 32)) {
          *abort_f = 1;
          break;
        }
        const PgMetaY &m = meta[ms];
        ea = m.ea[row];
#pragma unroll
        for (int p = 0; p < PG_CW / 2; ++p)
          ebp[p] = (uint32_t)(uint16_t)m.eb[c0 + 2 * p] |
                   ((uint32_t)(uint16_t)m.eb[c0 + 2 * p + 1] << 16);
        nbY = m.nbY;
        pA = m.pA;
        nrowY = m.nrowY;
        y2base = m.y2base;
        y64base = m.y64base;
        const int rowY = jb.mt * TM + row;
        valid = rowY < nrowY;
        yrow = rowY;
        need64 = W.y64_mode == 1;
        y2row = m.y2row[row];
        // the slot is free for the loader once every warp has read it
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&ctl->mempty[ms]);
      } else {
        // the job-data warp wrote this job's data into slot mcount % NMS; the slot
        // is held until the Sigma adds at the end of the job
        dms = (int)(mcount % PG_NMS);
        const bool okm = umma::mbar_wait(&ctl->mfull[dms], (uint32_t)((mcount / PG_NMS) & 1),
                                         S.err, PG_WAIT);
        ++mcount;
        if (umma::bar_any(!okm || *abort_f, PG_EPI * 32)) {
          *abort_f = 1;
          break;
        }
        const PgMetaD &m = metaD[dms];
        ea = m.ea[row];
        F = m.fi[row];
        valid = F >= 0;
        f = m.f[row];
        nf = m.nf[row];
      }

      // one accumulator handoff per K chunk.  D_AB: the chunks' exact sums add
      // in int64.  Y: the order groups (exact f32 integers times powers of two)
      // add in double-float, columns (2p, 2p + 1) in the two f32x2 lanes.
      long long Wv[JOB == 1 ? PG_CW : 1];
      uint64_t ds[JOB == 0 ? PG_CW / 2 : 1], dr[JOB == 0 ? PG_CW / 2 : 1];
#pragma unroll
      for (int i = 0; i < (JOB == 1 ? PG_CW : 1); ++i) Wv[i] = 0;
#pragma unroll
      for (int p = 0; p < (JOB == 0 ? PG_CW / 2 : 1); ++p) ds[p] = dr[p] = 0;
      bool aborted = false;
      for (int k0 = 0; k0 < jb.nk; k0 += KT_CHUNK) {
        const uint32_t par = (uint32_t)(hand & 1);
        ++hand;
        const bool okw = umma::mbar_wait(&ctl->tfull, par, S.err, PG_WAIT);
        if (umma::bar_any(!okw || *abort_f, PG_EPI * 32)) {
          *abort_f = 1;
          aborted = true;
          break;
        }
        umma::fence_after_sync();
#pragma unroll
        for (int g = 0; g < KS; ++g) {
          float v[PG_CW];
          const uint32_t ta = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * NT + c0);
          if constexpr (PG_CW == 32) umma::tmem_ld32(ta, v);
          else umma::tmem_ld16(ta, v);
          if constexpr (JOB == 0) {
            const float cg = __int_as_float((7 * (KS - 1 - g) + 127) << 23);
            const uint64_t c2 = f2_pk(cg, cg);
#pragma unroll
            for (int p = 0; p < PG_CW / 2; ++p)
              df_acc2(ds[p], dr[p], f2_mul(f2_pk(v[2 * p], v[2 * p + 1]), c2));
          } else {
            const long long sc = 1ll << (7 * (KS - 1 - g));
#pragma unroll
            for (int i = 0; i < PG_CW; ++i) Wv[i] += (long long)__float2int_rn(v[i]) * sc;
          }
        }
        // the accumulator is free for the next chunk's or job's MMAs
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&ctl->tempty);
      }
      if (aborted) break;
      // D_AB: every warp releases the job's slot after its adds, so a row
      // outside the atom's columns skips the adds but not the release
      if (!valid && JOB == 0) continue;

      if constexpr (JOB == 0) {
        // Y[al][b * ncol + col(G,g)] (FP64) and Y2 (f32 pairs) in 16-column
        // blocks [cb][al][b][16], cb = kofs(G) / 16 + g / 16
        double *Y = W.scratch + y64base;
        float2 *Y2 = reinterpret_cast<float2 *>(W.scratch + y2base);
#pragma unroll
        for (int p = 0; p < PG_CW / 2; ++p) {
          const int al = jb.nt * NT + c0 + 2 * p;
          if (al >= pA) break;
          float2 o[2];
          df_fin2(ds[p], dr[p], ea + (int)(int16_t)(ebp[p] & 0xFFFFu) - SH,
                  ea + (int)(int16_t)(ebp[p] >> 16) - SH, o[0], o[1]);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (al + u >= pA) break;
            if (need64)
              Y[(int64_t)(al + u) * nrowY + yrow] = (double)o[u].x + (double)o[u].y;
            if (y2row >= 0) Y2[y2row + (int64_t)(al + u) * nbY * 16] = o[u];
          }
        }
      } else {
        // Sigma_FG blocks: rows (F,f) of atom A, columns (G,g) of atom B; the
        // offsets come from the slot's table, or (a tile over more block pairs
        // than the table holds) from the same lookups done here
        const PgMetaD &m = metaD[dms];
        const int ilim = valid ? PG_CW : 0;
        int lastgi = -1;
        int64_t off = -1, moff = -1;
        int ng = 0;
        if (m.tbl) {
          // unrolled and free of calls, so the chunk sums stay in registers
#pragma unroll
          for (int i = 0; i < PG_CW; ++i) {
            const int c = c0 + i;
            const int gi = m.gi[c];
            if (i >= ilim || gi < 0) break;
            if (gi != lastgi) {
              lastgi = gi;
              ng = m.ng[c];
              off = m.off[F * m.ngb + gi];
              moff = m.moff[F * m.ngb + gi];
            }
            if (off < 0) continue;  // no surviving term in this block pair
            const int g = m.g[c];
            const int e = ea + m.eb[c] - SH;
            fx_add_scaled(S.acc + 2 * (off + (int64_t)f * ng + g), -Wv[i], e, S.err);
            if (moff >= 0)
              fx_add_scaled(S.acc + 2 * (moff + (int64_t)g * nf + f), -Wv[i], e, S.err);
          }
        } else if (valid) {
          // a tile over more block pairs than the table holds: the same adds
          // in the same order, the sums copied to a local array first so the
          // lookups' call does not hold them
          long long Wl[PG_CW];
#pragma unroll
          for (int i = 0; i < PG_CW; ++i) Wl[i] = Wv[i];
          for (int i = 0; i < PG_CW; ++i) {
            const int c = c0 + i;
            const int gi = m.gi[c];
            if (gi < 0) break;
            if (gi != lastgi) {
              lastgi = gi;
              ng = m.ng[c];
              dab_lookup(S, jb, m.fb0 + F, m.gb0 + gi, m.mir != 0, off, moff);
            }
            if (off < 0) continue;
            const int g = m.g[c];
            const int e = ea + m.eb[c] - SH;
            fx_add_scaled(S.acc + 2 * (off + (int64_t)f * ng + g), -Wl[i], e, S.err);
            if (moff >= 0)
              fx_add_scaled(S.acc + 2 * (moff + (int64_t)g * nf + f), -Wl[i], e, S.err);
          }
        }
      }
      if constexpr (JOB == 1) {
        // the slot is free for the loader once every warp is done with it
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&ctl->mempty[dms]);
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, 512);
}

template <int KS, int JOB>
cudaError_t launch_pgemm_t(const SplitShared &S, const SplitWave &W, int64_t maxjobs,
                           cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(maxjobs, S.nsm > 0 ? S.nsm : 1);
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = (size_t)PG_NST * KS * (TM + NT) * TK * 2 + PG_CTL_BYTES +
                      PgGeo<JOB>::NMS * (JOB == 0 ? sizeof(PgMetaY) : sizeof(PgMetaD)) + 64;
  cudaError_t e = cudaFuncSetAttribute(k_pgemm<KS, JOB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_pgemm<KS, JOB><<<blocks, PgGeo<JOB>::THREADS, smem, st>>>(S, W);
  return cudaGetLastError();
}

}  // namespace split

cudaError_t split_pgemm(const SplitShared &S, const SplitWave &W, int ks, int job,
                        int64_t maxjobs, cudaStream_t st) {
  switch (ks * 2 + job) {
    case 4: return split::launch_pgemm_t<2, 0>(S, W, maxjobs, st);
    case 5: return split::launch_pgemm_t<2, 1>(S, W, maxjobs, st);
    case 8: return split::launch_pgemm_t<4, 0>(S, W, maxjobs, st);
    case 9: return split::launch_pgemm_t<4, 1>(S, W, maxjobs, st);
    case 10: return split::launch_pgemm_t<5, 0>(S, W, maxjobs, st);
    case 11: return split::launch_pgemm_t<5, 1>(S, W, maxjobs, st);
    case 12: return split::launch_pgemm_t<6, 0>(S, W, maxjobs, st);
    case 13: return split::launch_pgemm_t<6, 1>(S, W, maxjobs, st);
    default: return cudaErrorInvalidValue;
  }
}
