// HFX_OZAKI: operand slicing and job lists for the Y = V C product and the
// D_AB piece of Algorithm 3, which run as exact split-precision tcgen05
// products in hfx_pgemm.cu (hfx_ozaki.cu documents the digit scheme).
//
//   Y job  (one per 128 rows (b,G,g) of a work item <A,B>):
//       Y^T[(b,G,g)][al] = sum_be C_BG[be][b][g] V_AB[al][be]
//     A operand: C of atom B transposed (rows (b,G,g), K = be), sliced once
//     per build; B operand: V_AB (rows al, K = be), sliced once per build.
//   D_AB job (128 rows (F,f) x 64 columns (G,g) of a pair, K chunk <= 640):
//       Sigma_FG[f][g] -= sum_{al,a} C_AF[al][a][f] P_G[al][a][g]
//     A operand: C of atom A as rows (F,f), K = (al,a), sliced once per
//     build; B operand: P of the pair as rows (G,g), K = (al,a), sliced per
//     wave.
// Tiles without any surviving block get no job (device-built job list;
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

// P of the D_AB piece, computed and sliced in one pass: one CTA per (pair, G)
// of the wave's pairs with a D_AB job and D_AB survivors for G.
//   P_G[(al,a)][g] = sum_b D_AB[a][b] Y[al][b][(G,g)]
// in double-float arithmetic from the f32 pairs of Y, held in shared memory
// for a chunk of g columns, then written as the digit rows (G,g) of the B
// operand, K = (al,a), with one exponent per row.  A digit expansion only has
// to be within one unit of the scaled value, so the integer is formed from
// the two halves of the pair separately.  Rows of G without D_AB survivors
// and the padding rows after the last G are not written: the D_AB epilogue
// adds only surviving (F, G) blocks, and each output column depends on its
// own B row alone, so whatever those rows hold never reaches Sigma.
constexpr int PD_THREADS = 256;

template <int KS>
__global__ void __launch_bounds__(PD_THREADS, 3) k_pdig(SplitShared S, SplitWave W) {
  extern __shared__ __align__(16) float2 Ps[];  // [gc][K], then the staged Y
  __shared__ int es[32];
  __shared__ float2 Dp[32 * 32];  // D_AB as f32 pairs
  const int64_t t = blockIdx.x;
  int lo = 0, hi = W.nw - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (W.pg_candpre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int wl = lo;
  if (W.ps_base[wl] < 0) return;
  const WorkItem &it = S.items[W.w0 + wl];
  const int G = (int)(t - W.pg_candpre[wl]);
  if (!(S.wg[it.wg_off + G] & 8u)) return;  // no D_AB survivor for this G
  const NbrEntry eg = S.nbr[it.gbase + G];
  const int pA = S.nabf[it.a], na = S.nao[it.a], nb = S.nao[it.b], ng = S.nao[eg.other];
  const int K = pA * na, ktiles = S.kt4[it.a], KT = ktiles * TK;
  const int cbG = S.kofs[it.gbase + G] / 16;
  __nv_bfloat16 *out = W.ps + W.ps_base[wl];
  int16_t *eout = W.ps_e + W.p_rowpre[wl];
  const float2 *Y2 = reinterpret_cast<const float2 *>(W.scratch + W.y2_off[wl]);
  const double *Dab = S.Dd + S.Do[it.dab];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < na * nb; i += PD_THREADS) {
    const double d = Dab[i];
    const float h = __double2float_rn(d);
    Dp[i] = make_float2(h, __double2float_rn(d - (double)h));
  }
  __syncthreads();
  // g columns per pass: 4 (one 32-byte sector of each Y2 row), else fewer
  const int nrow = pA * nb;
  const int cap = S.pd_pairs;  // >= K + nrow for every pair (sized on the host)
  const int gc = 4 * (K + nrow) <= cap ? 4 : 2 * (K + nrow) <= cap ? 2 : 1;
  float2 *Ys = Ps + gc * K;
  for (int g0 = 0; g0 < ng; g0 += gc) {
    const int gn = min(gc, ng - g0);
    // stage Y[al][b][g0 .. g0 + gc) (Y2 layout [cb][al][b][16]; g0 is a multiple
    // of gc, so the gc pairs stay inside one 16-column block and one sector)
    // staged as [al][b] rows of gc high words, then gc low words (gc > 1), so
    // two columns' high (low) words are one register pair
    const float2 *yb = Y2 + ((int64_t)(cbG + (g0 >> 4)) * pA * nb) * 16 + (g0 & 15);
    float *Yf = reinterpret_cast<float *>(Ys);
    for (int r = threadIdx.x; r < nrow; r += PD_THREADS) {
      const float2 *src = yb + (int64_t)r * 16;
      if (gc == 4) {
        const float4 u0 = reinterpret_cast<const float4 *>(src)[0];
        const float4 u1 = reinterpret_cast<const float4 *>(src)[1];
        reinterpret_cast<float4 *>(Yf + r * 8)[0] = make_float4(u0.x, u0.z, u1.x, u1.z);
        reinterpret_cast<float4 *>(Yf + r * 8)[1] = make_float4(u0.y, u0.w, u1.y, u1.w);
      } else if (gc == 2) {
        const float4 u0 = reinterpret_cast<const float4 *>(src)[0];
        reinterpret_cast<float4 *>(Yf + r * 4)[0] = make_float4(u0.x, u0.z, u0.y, u0.w);
      } else {
        Ys[r] = src[0];
      }
    }
    __syncthreads();
    if (gc == 1) {
      for (int kap = threadIdx.x; kap < K; kap += PD_THREADS) {
        const int al = kap / na, a = kap - al * na;
        const float2 *y = Ys + al * nb;
        const float2 *d = Dp + a * nb;
        float sh = 0.f, sl = 0.f;
        for (int b = 0; b < nb; ++b) df_mac(sh, sl, d[b], y[b]);
        Ps[kap] = make_float2(sh, sl);
      }
    } else {
      // all gn columns of one (al, a) per thread, two per packed (f32x2)
      // operation; each lane takes exactly the scalar df_mac's operations
      for (int kap = threadIdx.x; kap < K; kap += PD_THREADS) {
        const int al = kap / na, a = kap - al * na;
        const float *yr = Yf + (int64_t)al * nb * 2 * gc;
        const float2 *d = Dp + a * nb;
        uint64_t s0 = 0, r0 = 0, s1 = 0, r1 = 0;
        for (int b = 0; b < nb; ++b) {
          const float2 dv = d[b];
          const uint64_t ah = f2_pk(dv.x, dv.x), nah = f2_pk(-dv.x, -dv.x),
                         nal = f2_pk(-dv.y, -dv.y);
          if (gc == 4) {
            const float4 H = reinterpret_cast<const float4 *>(yr + b * 8)[0];
            const float4 L = reinterpret_cast<const float4 *>(yr + b * 8)[1];
            df_mac2(s0, r0, ah, nah, nal, f2_pk(H.x, H.y), f2_pk(L.x, L.y));
            df_mac2(s1, r1, ah, nah, nal, f2_pk(H.z, H.w), f2_pk(L.z, L.w));
          } else {
            const float4 V = reinterpret_cast<const float4 *>(yr + b * 4)[0];
            df_mac2(s0, r0, ah, nah, nal, f2_pk(V.x, V.y), f2_pk(V.z, V.w));
          }
        }
        const float2 S0 = f2_un(s0), R0 = f2_un(r0), S1 = f2_un(s1), R1 = f2_un(r1);
        Ps[kap] = make_float2(S0.x, R0.x);
        if (gn > 1) Ps[K + kap] = make_float2(S0.y, R0.y);
        if (gn > 2) Ps[2 * K + kap] = make_float2(S1.x, R1.x);
        if (gn > 3) Ps[3 * K + kap] = make_float2(S1.y, R1.y);
      }
    }
    __syncthreads();
    // one exponent per row (G, g0 + gi) over its K values
    for (int gi = warp; gi < gn; gi += PD_THREADS / 32) {
      float m = 0.f;
      for (int c = lane; c < K; c += 32) m = fmaxf(m, fabsf(Ps[gi * K + c].x));
      for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const int e = row_exponent(__double_as_longlong((double)m));
      if (lane == 0) {
        es[gi] = e;
        eout[eg.aopre + g0 + gi] = (int16_t)max(-30000, e);
      }
    }
    __syncthreads();
    // eight consecutive K of one row per thread: each digit plane gets one
    // 16-byte store (the eight are adjacent in the core-matrix tile)
    const int KT8 = KT / 8;
    for (int idx = threadIdx.x; idx < gn * KT8; idx += PD_THREADS) {
      const int gi = idx / KT8, c8 = (idx - gi * KT8) * 8;
      const int e = es[gi];
      // scale by 2^(7 KS - e) (|value| < 2^(e - 1)) in two exact steps
      const int sft = 7 * KS - e, s1 = sft / 2, s2 = sft - s1;
      const float f1 = __int_as_float((s1 + 127) << 23), f2 = __int_as_float((s2 + 127) << 23);
      uint32_t pk[KS][4];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int c = c8 + k;
        long long X = 0;
        if (c < K && e > -200) {  // below 2^-200 the row is dropped
          const float2 v = Ps[gi * K + c];
          X = __float2ll_rn(__fmul_rn(__fmul_rn(v.x, f1), f2)) +
              __float2ll_rn(__fmul_rn(__fmul_rn(v.y, f1), f2));
        }
        int d[KS];
        to_digits_i64<KS>(X, d);
#pragma unroll
        for (int sd = 0; sd < KS; ++sd) {
          const uint32_t b = __bfloat16_as_ushort(__int2bfloat16_rn(d[sd]));
          if (k & 1) pk[sd][k >> 1] |= b << 16;
          else pk[sd][k >> 1] = b;
        }
      }
      const int r = eg.aopre + g0 + gi;
      const int rt = r / NT, rr = r - rt * NT, kt = c8 / TK, cc = c8 - kt * TK;
      __nv_bfloat16 *base = out + ((int64_t)(rt * ktiles + kt) * KS) * NT * TK + tile_off(rr, cc);
#pragma unroll
      for (int sd = 0; sd < KS; ++sd)
        *reinterpret_cast<uint4 *>(base + (int64_t)sd * NT * TK) =
            make_uint4(pk[sd][0], pk[sd][1], pk[sd][2], pk[sd][3]);
    }
    __syncthreads();
  }
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
  // candidates are enumerated with the items grouped by atom B, and job t is
  // candidate t (an empty job when skipped), so jobs running side by side
  // read the same C_B tiles from L2
  const int wl = (int)W.y_perm[lo];
  if (t == 0) W.njobs[0] = (int)W.y_candpre[W.nw];
  const WorkItem &it = S.items[W.w0 + wl];
  const int local = (int)(t - W.y_candpre[lo]);
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
  W.jobs[t] = Job{W.w0 + wl, mt, nt, 0, any ? S.ktY[it.b] : 0};
  if (any) atomicAdd(W.tmacs, (unsigned long long)TM * NT * TK * S.ktY[it.b]);
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
  // one job over the whole K; the product hands the accumulator to the
  // epilogue after every KT_CHUNK tiles (exact group sums)
  const int j = atomicAdd(W.njobs + 1, 1);
  W.jobs4[j] = Job{W.w0 + wl, mt, nt, 0, kt};
  atomicAdd(W.tmacs + 1, (unsigned long long)TM * NT * TK * kt);
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
    return split_pgemm(S, W, KS, 0, W.h_ycand, st);
  }
  // phase 1: P digits, D_AB jobs, D_AB products
  if (W.h_pgcand > 0) {
    // P and the staged Y of up to 4 g columns (50 KB for 13 NAO / 60 ABF)
    const int smem = S.pd_pairs * (int)sizeof(float2);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_pdig<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    k_pdig<KS><<<(unsigned)W.h_pgcand, PD_THREADS, smem, st>>>(S, W);
  }
  if (W.h_v4cand > 0)
    k_jobs_v4<<<(unsigned)((W.h_v4cand + 255) / 256), 256, 0, st>>>(S, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return split_pgemm(S, W, KS, 1, W.h_v4jobs_max, st);
}

}  // namespace split

cudaError_t split_slice_inputs(const SplitShared &S, int ks, cudaStream_t st) {
  switch (ks) {
    case 2: return split::slice_inputs_t<2>(S, st);
    case 4: return split::slice_inputs_t<4>(S, st);
    case 5: return split::slice_inputs_t<5>(S, st);
    case 6: return split::slice_inputs_t<6>(S, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t split_wave(const SplitShared &S, const SplitWave &W, int ks, int phase,
                       cudaStream_t st) {
  switch (ks) {
    case 2: return split::wave_t<2>(S, W, phase, st);
    case 4: return split::wave_t<4>(S, W, phase, st);
    case 5: return split::wave_t<5>(S, W, phase, st);
    case 6: return split::wave_t<6>(S, W, phase, st);
    default: return cudaErrorInvalidValue;
  }
}
