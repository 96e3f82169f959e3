// HFX_OZAKI: the Y = V C product and the D_AB piece of Algorithm 3 on the
// tensor cores, as exact split-precision products (see hfx_ozaki.cu for the
// digit scheme and the tcgen05 pipeline it shares).
//
//   Y job  (one per 128 rows (b,G,g) of a work item <A,B>):
//       Y^T[(b,G,g)][al] = sum_be C_BG[be][b][g] V_AB[al][be]
//     A operand: C of atom B transposed (rows (b,G,g), K = be), sliced once
//     per build; B operand: V_AB (rows al, K = be), sliced once per build.
//     The epilogue stores Y[al][b][(G,g)] in FP64 for the remaining FP64
//     kernels and the D-stage.
//   D_AB job (128 rows (F,f) x 64 columns (G,g) of a pair, K chunk <= 640):
//       Sigma_FG[f][g] -= sum_{al,a} C_AF[al][a][f] P_G[al][a][g]
//     A operand: C of atom A as rows (F,f), K = (al,a), sliced once per
//     build; B operand: P of the pair as rows (G,g), K = (al,a), sliced per
//     wave.  The epilogue keeps only surviving (F,G) blocks and adds them to
//     the fixed-point Sigma accumulators with integer arithmetic.
// Tiles without any surviving block are not launched (device-built job list;
// Sigma accumulation is order-independent, so job order does not matter).
#include <cuda_bf16.h>

#include <algorithm>

#include "umma.cuh"

#include "split_common.cuh"
#include "hfx_split.h"

namespace split {

// ------------------------------------------------------------------ slicing
// One warp per padded operand row; lanes run over K.  Each source type gives
// the element (row, kappa) and the row/K extents.

template <int KS, class Src>
__device__ __forceinline__ void slice_row(const Src &src, int64_t row_global, int row_in_op,
                                          int rows_pt, int nrows, int K, int ktiles,
                                          __nv_bfloat16 *out, int16_t *eout) {
  const int lane = threadIdx.x & 31;
  long long mbits = 0;
  const bool live = row_in_op < nrows && src.row_live(row_in_op);
  if (live)
    for (int c = lane; c < K; c += 32)
      mbits = max(mbits, __double_as_longlong(src.get(row_in_op, c)) & 0x7FFFFFFFFFFFFFFFll);
  for (int o = 16; o; o >>= 1) mbits = max(mbits, __shfl_xor_sync(0xffffffffu, mbits, o));
  const int e = row_exponent(mbits);
  if (lane == 0) eout[row_global] = (int16_t)max(-30000, e);
  const int rt = row_in_op / rows_pt, rr = row_in_op - rt * rows_pt;
  for (int c = lane; c < ktiles * TK; c += 32) {
    const double x = (live && c < K && e > -1000) ? src.get(row_in_op, c) : 0.0;
    int d[KS];
    to_digits<KS>(x, e, d);
    const int kt = c / TK, cc = c - kt * TK;
    __nv_bfloat16 *base = out + ((int64_t)(rt * ktiles + kt) * KS) * rows_pt * TK;
#pragma unroll
    for (int s = 0; s < KS; ++s)
      base[(int64_t)s * rows_pt * TK + tile_off(rr, cc)] = __int2bfloat16_rn(d[s]);
  }
}

// C of atom x transposed for the Y product: row (b, G, g) = b * ncol + col(G,g), K = beta.
struct SrcCY {
  const double *Cd;
  const int64_t *Co;
  const NbrEntry *nbr;
  const int32_t *nao;
  int64_t base;
  int n, nb, ncol;
  __device__ bool row_live(int) const { return true; }
  __device__ double get(int r, int beta) const {
    const int b = r / ncol, c = r - b * ncol;
    const NbrEntry &e = nbr[base + entry_of(nbr, base, n, c)];
    const int ng = nao[e.other], g = c - e.aopre;
    return Cd[Co[e.cblk] + ((int64_t)beta * nb + b) * ng + g];
  }
};

// C of atom x as rows (F, f), K = (alpha, a).
struct SrcC4 {
  const double *Cd;
  const int64_t *Co;
  const NbrEntry *nbr;
  const int32_t *nao;
  int64_t base;
  int n;
  __device__ bool row_live(int) const { return true; }
  __device__ double get(int r, int kappa) const {
    const NbrEntry &e = nbr[base + entry_of(nbr, base, n, r)];
    const int nf = nao[e.other], f = r - e.aopre;
    return Cd[Co[e.cblk] + (int64_t)kappa * nf + f];
  }
};

// V block: rows alpha, K = beta.
struct SrcV {
  const double *V;
  int pB;
  __device__ bool row_live(int) const { return true; }
  __device__ double get(int r, int beta) const { return V[(int64_t)r * pB + beta]; }
};

// P of a pair: rows (G, g), K = (alpha, a); rows of G without D_AB survivors are zero.
struct SrcP {
  const double *P;
  const NbrEntry *nbr;
  const uint8_t *wg;
  int64_t gbase, wg_off;
  int nG, ncol;
  __device__ bool row_live(int r) const {
    return (wg[wg_off + entry_of(nbr, gbase, nG, r)] & 8u) != 0;
  }
  __device__ double get(int r, int kappa) const { return P[(int64_t)kappa * ncol + r]; }
};

template <int KS>
__global__ void k_slice_atoms(SplitShared S, int which /*0: CY, 1: C4*/) {
  const int64_t grow = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t *rowpre = which == 0 ? S.cy_rowpre : S.c4_rowpre;
  if (grow >= rowpre[S.natoms]) return;
  int lo = 0, hi = S.natoms - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rowpre[mid] <= grow) lo = mid; else hi = mid - 1;
  }
  const int x = lo;
  const int r = (int)(grow - rowpre[x]);
  const int nx = S.nao[x], px = S.nabf[x], ncol = S.ncol[x];
  const int64_t base = S.nc_start[x];
  const int n = (int)(S.nc_start[x + 1] - base);
  if (which == 0) {
    SrcCY src{S.Cd, S.Co, S.nbr, S.nao, base, n, nx, ncol};
    slice_row<KS>(src, grow, r, TM, nx * ncol, px, S.ktY[x], S.cy + S.cy_base[x], S.cy_e);
  } else {
    SrcC4 src{S.Cd, S.Co, S.nbr, S.nao, base, n};
    slice_row<KS>(src, grow, r, TM, ncol, px * nx, S.kt4[x], S.c4 + S.c4_base[x], S.c4_e);
  }
}

template <int KS>
__global__ void k_slice_v(SplitShared S) {
  const int64_t grow = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (grow >= S.v_rowpre[S.nv]) return;
  int64_t lo = 0, hi = S.nv - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (S.v_rowpre[mid] <= grow) lo = mid; else hi = mid - 1;
  }
  const int64_t e = lo;
  const int r = (int)(grow - S.v_rowpre[e]);
  const WorkItem &it = S.items[e];  // work items are the V blocks in key order
  const int pA = S.nabf[it.a], pB = S.nabf[it.b];
  SrcV src{S.Vd + S.Vo[e], pB};
  slice_row<KS>(src, grow, r, NT, pA, pB, S.ktY[it.b], S.vs + S.vs_base[e], S.vs_e);
}

template <int KS>
__global__ void k_slice_p(SplitShared S, SplitWave W) {
  const int64_t grow = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (grow >= W.p_rowpre[W.nw]) return;
  int lo = 0, hi = W.nw - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (W.p_rowpre[mid] <= grow) lo = mid; else hi = mid - 1;
  }
  const int wl = lo;
  if (W.ps_base[wl] < 0) return;  // no D_AB job for this pair
  const WorkItem &it = S.items[W.w0 + wl];
  const int r = (int)(grow - W.p_rowpre[wl]);
  const int pA = S.nabf[it.a], na = S.nao[it.a], ncol = S.ncol[it.b];
  SrcP src{W.scratch + W.p_off[wl], S.nbr, S.wg, it.gbase, it.wg_off, it.nG, ncol};
  slice_row<KS>(src, grow, r, NT, ncol, pA * na, S.kt4[it.a], W.ps + W.ps_base[wl], W.ps_e);
}

// ------------------------------------------------------------------- jobs
// Y jobs: every 128-row tile of every pair of the wave that has a surviving term.
__global__ void k_jobs_y(SplitShared S, SplitWave W) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= W.y_candpre[W.nw]) return;
  int lo = 0, hi = W.nw - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (W.y_candpre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int wl = lo;
  const WorkItem &it = S.items[W.w0 + wl];
  const int local = (int)(t - W.y_candpre[wl]);
  const int ntv = (S.nabf[it.a] + NT - 1) / NT;
  const int mt = local / ntv, nt = local - mt * ntv;
  // skip tiles whose rows (b, G, g) belong only to G without a surviving term
  const int ncol = S.ncol[it.b], nrow = S.nao[it.b] * ncol;
  const int r0 = mt * TM, r1 = min(nrow, r0 + TM) - 1;
  const int b0 = r0 / ncol, b1 = r1 / ncol;
  const int c0 = r0 - b0 * ncol, c1 = r1 - b1 * ncol;
  int G0 = entry_of(S.nbr, it.gbase, it.nG, c0), G1 = entry_of(S.nbr, it.gbase, it.nG, c1);
  bool any = false;
  if (b1 > b0 + 1 || (b1 == b0 + 1 && G1 >= G0)) {
    G0 = 0;
    G1 = it.nG - 1;
  }
  if (b1 == b0 || G0 == 0) {
    for (int g = G0; g <= G1 && !any; ++g) any = S.wg[it.wg_off + g] != 0;
  } else {  // wraps: [G0, nG) then [0, G1]
    for (int g = G0; g < it.nG && !any; ++g) any = S.wg[it.wg_off + g] != 0;
    for (int g = 0; g <= G1 && !any; ++g) any = S.wg[it.wg_off + g] != 0;
  }
  if (!any) return;
  const int j = atomicAdd(W.njobs, 1);
  W.jobs[j] = Job{W.w0 + wl, mt, nt, 0, S.ktY[it.b]};
  atomicAdd(W.tmacs, (unsigned long long)TM * NT * TK * S.ktY[it.b]);
}

// D_AB jobs: (F-tile, G-tile) pairs holding at least one surviving block.
__global__ void k_jobs_v4(SplitShared S, SplitWave W) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= W.v4_candpre[W.nw]) return;
  int lo = 0, hi = W.nw - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (W.v4_candpre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int wl = lo;
  if (W.ps_base[wl] < 0) return;
  const WorkItem &it = S.items[W.w0 + wl];
  const int local = (int)(t - W.v4_candpre[wl]);
  const int ncolA = S.ncol[it.a], ncolB = S.ncol[it.b];
  const int ntg = (ncolB + NT - 1) / NT;
  const int mt = local / ntg, nt = local - mt * ntg;
  const int r0 = mt * TM, r1 = min(ncolA, r0 + TM) - 1;
  const int c0 = nt * NT, c1 = min(ncolB, c0 + NT) - 1;
  const int F0 = entry_of(S.nbr, it.fbase, it.nF, r0), F1 = entry_of(S.nbr, it.fbase, it.nF, r1);
  const int G0 = entry_of(S.nbr, it.gbase, it.nG, c0), G1 = entry_of(S.nbr, it.gbase, it.nG, c1);
  bool any = false;
  for (int g = G0; g <= G1 && !any; ++g) {
    if (!(S.wg[it.wg_off + g] & 8u)) continue;
    const uint32_t *row = S.masks + it.mask_off + ((int64_t)g * 4 + 3) * it.nFw;
    for (int wd = F0 >> 5; wd <= (F1 >> 5) && !any; ++wd) {
      uint32_t m = row[wd];
      if (wd == (F0 >> 5)) m &= ~0u << (F0 & 31);
      if (wd == (F1 >> 5) && (F1 & 31) != 31) m &= (1u << ((F1 & 31) + 1)) - 1u;
      any = m != 0;
    }
  }
  if (!any) return;
  const int kt = S.kt4[it.a];
  for (int k0 = 0; k0 < kt; k0 += KT_CHUNK) {
    const int j = atomicAdd(W.njobs + 1, 1);
    W.jobs4[j] = Job{W.w0 + wl, mt, nt, k0, min(KT_CHUNK, kt - k0)};
    atomicAdd(W.tmacs + 1, (unsigned long long)TM * NT * TK * min(KT_CHUNK, kt - k0));
  }
}

// ------------------------------------------------------------------- GEMM
__host__ __device__ constexpr uint32_t tmem_cols(int ks) {
  return (uint32_t)(ks * NT <= 64 ? 64 : ks * NT <= 128 ? 128 : ks * NT <= 256 ? 256 : 512);
}

template <int KS, int JOB>
__global__ void __launch_bounds__(128, 1) k_gemm(SplitShared S, SplitWave W) {
  const int njobs = W.njobs[JOB];
  if ((int)blockIdx.x >= njobs) return;
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int A_BYTES = KS * TM * TK * 2;
  constexpr int B_BYTES = KS * NT * TK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = tmem_cols(KS);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + NSTAGE * STAGE);
  uint64_t *empty = full + NSTAGE;
  uint64_t *done = empty + NSTAGE;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);

  const Job jb = (JOB == 0 ? W.jobs : W.jobs4)[blockIdx.x];
  const WorkItem it = S.items[jb.w];
  const int wl = (int)(jb.w - W.w0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const __nv_bfloat16 *Ab, *Bb;
  const int16_t *ea_p, *eb_p;
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

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(done, 1);
    umma::fence_barrier_init();
  }
  if (warp == 0) {
    umma::tmem_alloc(tslot, TCOLS);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = *tslot;

  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = umma::idesc_bf16_f32(TM, NT);
    auto load = [&](int s, int kt) {
      umma::mbar_arrive_expect_tx(&full[s], STAGE);
      umma::bulk_g2s(smem + s * STAGE, Ab + (int64_t)kt * KS * TM * TK, A_BYTES, &full[s]);
      umma::bulk_g2s(smem + s * STAGE + A_BYTES, Bb + (int64_t)kt * KS * NT * TK, B_BYTES,
                     &full[s]);
    };
    for (int s = 0; s < NSTAGE && s < jb.nk; ++s) load(s, s);
    bool ok = true;
    for (int kt = 0; kt < jb.nk; ++kt) {
      const int s = kt % NSTAGE;
      const uint32_t ph = (uint32_t)(kt / NSTAGE) & 1u;
      if (!umma::mbar_wait(&full[s], ph, S.err)) { ok = false; break; }
      umma::fence_after_sync();
      const uint32_t a0 = umma::smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int j = 0; j < TK / 16; ++j)
#pragma unroll
        for (int g = 0; g < KS; ++g)
#pragma unroll
          for (int i = 0; i <= g; ++i) {
            const uint64_t ad = umma::smem_desc(a0 + i * TM * TK * 2 + j * 256, 128, 512);
            const uint64_t bd = umma::smem_desc(b0 + (g - i) * NT * TK * 2 + j * 256, 128, 512);
            umma::mma_bf16(tbase + g * NT, ad, bd, idesc, (kt | j | i) ? 1u : 0u);
          }
      umma::mma_commit(&empty[s]);
      if (kt + NSTAGE < jb.nk) {
        if (!umma::mbar_wait(&empty[s], ph, S.err)) { ok = false; break; }
        load(s, kt + NSTAGE);
      }
    }
    if (ok) umma::mma_commit(done);
    else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(done)) : "memory");
  }
  __syncwarp();
  const bool ready = umma::mbar_wait(done, 0, S.err);
  umma::fence_after_sync();

  const int row = warp * 32 + lane;
  const int ea = ea_p[row];
  constexpr int SH = 7 * (KS + 1);
  if (JOB == 0) {
    // Y[al][rowY] with rowY = b * ncol + col(G,g); columns al of this tile.
    // Y2 (f32 pairs) in 16-column blocks: [cb][al][b][16], cb = kofs(G) / 16 + g / 16
    const int nb = S.nao[it.b], ncol = S.ncol[it.b];
    const int nrow = nb * ncol;
    const int rowY = jb.mt * TM + row;
    const int pA = S.nabf[it.a];
    double *Y = W.scratch + W.y_off[wl];
    float2 *Y2 = reinterpret_cast<float2 *>(W.scratch + W.y2_off[wl]);
    int64_t y2row = -1;
    if (W.y2_on && rowY < nrow) {
      const int b = rowY / ncol, col = rowY - b * ncol;
      const int G = entry_of(S.nbr, it.gbase, it.nG, col);
      const int g = col - S.nbr[it.gbase + G].aopre;
      const int cb = S.kofs[it.gbase + G] / 16 + g / 16;
      y2row = (((int64_t)cb * pA) * nb + b) * 16 + (g & 15);
    }
    for (int c0 = 0; c0 < NT; c0 += 32) {
      long long Wv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) Wv[i] = 0;
#pragma unroll
      for (int g = 0; g < KS; ++g) {
        float v[32];
        umma::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * NT + c0), v);
        const long long sc = 1ll << (7 * (KS - 1 - g));
#pragma unroll
        for (int i = 0; i < 32; ++i) Wv[i] += (long long)__float2int_rn(v[i]) * sc;
      }
      if (ready && rowY < nrow) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int al = jb.nt * NT + c0 + i;
          if (al < pA) {
            const int e = ea + eb_p[c0 + i] - SH;
            Y[(int64_t)al * nrow + rowY] = scaled_i64(Wv[i], e);
            if (y2row >= 0) Y2[y2row + (int64_t)al * nb * 16] = pair_i64(Wv[i], e);
          }
        }
      }
    }
  } else {
    // Sigma_FG blocks: rows (F,f) of atom A, columns (G,g) of atom B
    const int ncolA = S.ncol[it.a], ncolB = S.ncol[it.b];
    const int rF = jb.mt * TM + row;
    const bool rvalid = ready && rF < ncolA;
    const int F = entry_of(S.nbr, it.fbase, it.nF, rvalid ? rF : 0);
    const NbrEntry ef = S.nbr[it.fbase + F];
    const int nf = S.nao[ef.other], f = rF - ef.aopre;
    const bool mir = S.sym && it.role == 1;
    int lastG = -1;
    bool live = false;
    int64_t off = -1, moff = -1;
    int ng = 0, gpre = 0;
    for (int c0 = 0; c0 < NT; c0 += 32) {
      long long Wv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) Wv[i] = 0;
#pragma unroll
      for (int g = 0; g < KS; ++g) {
        float v[32];
        umma::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * NT + c0), v);
        const long long sc = 1ll << (7 * (KS - 1 - g));
#pragma unroll
        for (int i = 0; i < 32; ++i) Wv[i] += (long long)__float2int_rn(v[i]) * sc;
      }
      if (!rvalid) continue;
#pragma unroll 1
      for (int i = 0; i < 32; ++i) {
        const int cG = jb.nt * NT + c0 + i;
        if (cG >= ncolB) break;
        if (cG >= gpre + ng || lastG < 0) {
          const int G = entry_of(S.nbr, it.gbase, it.nG, cG);
          const NbrEntry eg = S.nbr[it.gbase + G];
          lastG = G;
          ng = S.nao[eg.other];
          gpre = eg.aopre;
          const uint32_t m = S.masks[it.mask_off + ((int64_t)G * 4 + 3) * it.nFw + (F >> 5)];
          live = (m >> (F & 31)) & 1u;
          off = moff = -1;
          if (live) {
            const int n0 = it.n[0] + eg.n[0] - ef.n[0], n1 = it.n[1] + eg.n[1] - ef.n[1],
                      n2 = it.n[2] + eg.n[2] - ef.n[2];
            off = dh_find(S.shash, hk_pack(ef.other, eg.other, n0, n1, n2));
            if (mir) moff = dh_find(S.shash, hk_pack(eg.other, ef.other, -n0, -n1, -n2));
            if (off < 0 || (mir && moff < 0)) atomicOr(S.err, HFX_DEV_ERR_MISSING);
          }
        }
        if (!live) continue;
        const int g = cG - gpre;
        const int e = ea + eb_p[c0 + i] - SH;
        if (off >= 0) fx_add_scaled(S.acc + 2 * (off + (int64_t)f * ng + g), -Wv[i], e);
        if (moff >= 0) fx_add_scaled(S.acc + 2 * (moff + (int64_t)g * nf + f), -Wv[i], e);
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, TCOLS);
}

template <int KS, int JOB>
cudaError_t launch_gemm_t(const SplitShared &S, const SplitWave &W, int64_t maxjobs,
                          cudaStream_t st) {
  if (maxjobs <= 0) return cudaSuccess;
  constexpr int STAGE = KS * (TM + NT) * TK * 2;
  const size_t need = (size_t)NSTAGE * STAGE + 64;
  const int limit = 512 / (int)tmem_cols(KS);
  const size_t smem = std::max(need, (size_t)(233472 / (limit + 1)) + 1024);
  cudaError_t e = cudaFuncSetAttribute(k_gemm<KS, JOB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_gemm<KS, JOB><<<(unsigned)maxjobs, 128, smem, st>>>(S, W);
  return cudaGetLastError();
}

template <int KS>
cudaError_t slice_inputs_t(const SplitShared &S, cudaStream_t st) {
  const int64_t ry = S.h_cy_rows, r4 = S.h_c4_rows, rv = S.h_v_rows;
  if (ry > 0) k_slice_atoms<KS><<<(unsigned)((ry * 32 + 255) / 256), 256, 0, st>>>(S, 0);
  if (r4 > 0) k_slice_atoms<KS><<<(unsigned)((r4 * 32 + 255) / 256), 256, 0, st>>>(S, 1);
  if (rv > 0) k_slice_v<KS><<<(unsigned)((rv * 32 + 255) / 256), 256, 0, st>>>(S);
  return cudaGetLastError();
}

template <int KS>
cudaError_t wave_t(const SplitShared &S, const SplitWave &W, int phase, cudaStream_t st) {
  if (phase == 0) {  // Y jobs and Y products
    if (W.h_ycand > 0)
      k_jobs_y<<<(unsigned)((W.h_ycand + 255) / 256), 256, 0, st>>>(S, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_gemm_t<KS, 0>(S, W, W.h_ycand, st);
  }
  // phase 1: slice P, build D_AB jobs, run them
  if (W.h_prows > 0)
    k_slice_p<KS><<<(unsigned)((W.h_prows * 32 + 255) / 256), 256, 0, st>>>(S, W);
  if (W.h_v4cand > 0)
    k_jobs_v4<<<(unsigned)((W.h_v4cand + 255) / 256), 256, 0, st>>>(S, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gemm_t<KS, 1>(S, W, W.h_v4jobs_max, st);
}

}  // namespace split

cudaError_t split_slice_inputs(const SplitShared &S, int ks, cudaStream_t st) {
  switch (ks) {
    case 4: return split::slice_inputs_t<4>(S, st);
    case 5: return split::slice_inputs_t<5>(S, st);
    case 6: return split::slice_inputs_t<6>(S, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t split_wave(const SplitShared &S, const SplitWave &W, int ks, int phase,
                       cudaStream_t st) {
  switch (ks) {
    case 4: return split::wave_t<4>(S, W, phase, st);
    case 5: return split::wave_t<5>(S, W, phase, st);
    case 6: return split::wave_t<6>(S, W, phase, st);
    default: return cudaErrorInvalidValue;
  }
}
