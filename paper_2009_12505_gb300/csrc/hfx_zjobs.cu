// HFX_OZAKI: the D_FG and D_FB pieces of Algorithm 3 on the tensor cores.
//
// For a pair <A,B> and a neighbour G of B, with F running over the
// neighbours of A that survive the screen for the piece,
//   D_FG piece:  Z_G[(al,a)][g] = sum_F sum_f C_AF[al][a][f] D_FG[f][g]
//                Sigma_AB[a][b] -= sum_{al,g} Z_G[(al,a)][g] Y_G[al][b][g]
//   D_FB piece:  Z_G[(al,a)][b] = sum_F sum_f C_AF[al][a][f] D_FB[f][b]
//                Sigma_AG[a][g] -= sum_{al,b} Z_G[(al,a)][b] Y_G[al][b][g]
// (the same terms as Algorithm 3's T and Ht, contracted D-first; the sums
// over F and the final contraction are reassociations of exact sums).
//
// One job = one 128-row tile of (al,a) for one (pair, G, piece) and a chunk of
// the selected F.  Z is an exact split-precision product (bf16 digits,
// tcgen05): the A operand is C of atom A sliced once per build (rows (al,a),
// K = F blocks padded to 16 or 32), streamed by bulk copies; the B operand is
// the D blocks of the selected F, sliced in the kernel with one exponent per
// output column over those blocks.  The epilogue turns Z into f32 pairs,
// contracts with Y (f32 pairs from the Y product) in double-float
// arithmetic, reduces over al through shared memory in FP64 and adds the
// block to the fixed-point Sigma (and its mirror for Hermitian inputs).
#include <cuda_bf16.h>

#include <algorithm>

#include "hfx_split.h"
#include "split_common.cuh"

namespace split {

constexpr int ZF_MAX = 16;          // selected F per job
constexpr int ZB_BYTES = 64 * 1024; // shared bytes for the D digit tiles of one job

__host__ __device__ __forceinline__ int kb_of(int nao) { return nao <= 16 ? 16 : 32; }
__host__ __device__ __forceinline__ int nb_of(int n) { return n <= 16 ? 16 : 32; }

// element offset of (r, c) in an [R x kb] K-major core-matrix tile
__device__ __forceinline__ int tile_off_kb(int r, int c, int kb) {
  return ((r >> 3) * (kb >> 3) + (c >> 3)) * 64 + (r & 7) * 8 + (c & 7);
}

// C of atom x as rows (al, a), K = F blocks.
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
  // exponent over the whole row (every F block)
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

// Jobs: per (pair, G) candidate, per piece with survivors, per F chunk, per M tile.
__global__ void k_jobs_z(SplitShared S, SplitWave W) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= W.z_candpre[W.nw]) return;
  int lo = 0, hi = W.nw - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (W.z_candpre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int wl = lo;
  const WorkItem &it = S.items[W.w0 + wl];
  const int g = (int)(t - W.z_candpre[wl]);
  const unsigned bits = S.wg[it.wg_off + g];
  const int pA = S.nabf[it.a], na = S.nao[it.a];
  const int mtz = (pA * na + 127) / 128;
  const NbrEntry eg = S.nbr[it.gbase + g];
  for (int piece = 1; piece <= 2; ++piece) {
    if (!(bits & (piece == 1 ? 1u : 2u))) continue;
    if (piece == 1 && S.sym && it.role == 2) continue;  // mirror of a canonical pair
    const uint32_t *row = S.masks + it.mask_off + ((int64_t)g * 4 + (piece - 1)) * it.nFw;
    int cnt = 0;
    for (int wd = 0; wd < it.nFw; ++wd) cnt += __popc(row[wd]);
    if (!cnt) continue;
    const int ncolsB = piece == 1 ? S.nao[eg.other] : S.nao[it.b];
    const int nbB = nb_of(ncolsB);
    const int per_f = 6 * nbB * 32 * 2;  // worst-case digit-tile bytes per selected F
    const int chunk = max(1, min(ZF_MAX, ZB_BYTES / per_f));
    for (int r0 = 0; r0 < cnt; r0 += chunk) {
      const int nsel = min(chunk, cnt - r0);
      if (!W.zjobs) {
        atomicAdd(W.njobs + 2, mtz);
        continue;
      }
      for (int mt = 0; mt < mtz; ++mt) {
        const int j = atomicAdd(W.njobs + 2, 1);
        W.zjobs[j] = Job{W.w0 + wl, mt, g, r0, nsel | (piece << 16)};
      }
      atomicAdd(W.tmacs + 2, (unsigned long long)mtz * 128 * nbB * 16 * nsel);
    }
  }
}

template <int KS>
__global__ void __launch_bounds__(128, 1) k_zgemm(SplitShared S, SplitWave W) {
  if ((int)blockIdx.x >= W.njobs[2]) return;
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int A_STAGE = KS * 128 * 32 * 2;  // one F block of width <= 32
  uint8_t *Bsm = smem + 2 * A_STAGE;
  uint64_t *full = reinterpret_cast<uint64_t *>(Bsm + ZB_BYTES);
  uint64_t *empty = full + 2;
  uint64_t *done = empty + 2;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  int *flist = reinterpret_cast<int *>(tslot + 4);
  int *kbl = flist + ZF_MAX;
  int *boff = kbl + ZF_MAX;
  int *ecol = boff + ZF_MAX;           // 32 column exponents
  int64_t *dlist = reinterpret_cast<int64_t *>(ecol + 32);
  int64_t *tgt = dlist + ZF_MAX;       // [0] target offset, [1] mirror offset

  const Job jb = W.zjobs[blockIdx.x];
  const WorkItem it = S.items[jb.w];
  const int wl = (int)(jb.w - W.w0);
  const int piece = jb.nk >> 16, nsel = jb.nk & 0xFFFF, g_ = jb.nt, mt = jb.mt;
  const NbrEntry eg = S.nbr[it.gbase + g_];
  const int pA = S.nabf[it.a], na = S.nao[it.a], nb = S.nao[it.b], ng = S.nao[eg.other];
  const int ncolsB = piece == 1 ? ng : nb;   // columns of Z = rows of the D digit tiles
  const int NB = nb_of(ncolsB);
  const int nG0 = it.n[0] + eg.n[0], nG1 = it.n[1] + eg.n[1], nG2 = it.n[2] + eg.n[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t TCOLS = NB == 16 ? 128u : 256u;  // KS * NB columns

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
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
  if (warp == 1) {
    // selected F (ranks [k0, k0 + nsel) among the piece's survivors for G), in order
    const uint32_t *row = S.masks + it.mask_off + ((int64_t)g_ * 4 + (piece - 1)) * it.nFw;
    if (lane < ZF_MAX) flist[lane] = 0;
    __syncwarp();
    int seen = 0, c = 0;
    for (int f0 = 0; f0 < it.nF && c < nsel; f0 += 32) {
      const uint32_t m = row[f0 >> 5];
      const bool b = f0 + lane < it.nF && ((m >> lane) & 1u);
      const uint32_t bal = __ballot_sync(0xffffffffu, b);
      const int rank = seen + __popc(bal & ((1u << lane) - 1u));
      if (b && rank >= jb.k0 && rank < jb.k0 + nsel) flist[rank - jb.k0] = f0 + lane;
      seen += __popc(bal);
      c = max(0, min(nsel, seen - jb.k0));
    }
    __syncwarp();
    if (lane < nsel) {
      const NbrEntry ef = S.nbr[it.fbase + flist[lane]];
      const int nf = S.nao[ef.other];
      int64_t d;
      if (piece == 1)
        d = dh_find(S.dhash, hk_pack(ef.other, eg.other, nG0 - ef.n[0], nG1 - ef.n[1], nG2 - ef.n[2]));
      else
        d = dh_find(S.dhash, hk_pack(ef.other, it.b, it.n[0] - ef.n[0], it.n[1] - ef.n[1],
                                     it.n[2] - ef.n[2]));
      if (d < 0) atomicOr(S.err, HFX_DEV_ERR_MISSING);
      dlist[lane] = d;
      kbl[lane] = kb_of(nf);
    }
    __syncwarp();
    if (lane == 0) {
      int o = 0;
      for (int q = 0; q < nsel; ++q) {
        boff[q] = o;
        o += KS * NB * kbl[q] * 2;
      }
    }
    __syncwarp();
    // one exponent per Z column over the selected D blocks
    {
      long long mb = 0;
      if (lane < ncolsB)
        for (int q = 0; q < nsel; ++q) {
          if (dlist[q] < 0) continue;
          const NbrEntry ef = S.nbr[it.fbase + flist[q]];
          const int nf = S.nao[ef.other];
          const double *Db = S.Dd + S.Do[dlist[q]];
          for (int f = 0; f < nf; ++f)
            mb = max(mb, __double_as_longlong(Db[f * ncolsB + lane]) & 0x7FFFFFFFFFFFFFFFll);
        }
      ecol[lane] = row_exponent(mb);
    }
    __syncwarp();
    // D digit tiles: rows = Z columns c, K = f
    for (int q = 0; q < nsel; ++q) {
      const NbrEntry ef = S.nbr[it.fbase + flist[q]];
      const int nf = S.nao[ef.other], kb = kbl[q];
      const double *Db = dlist[q] >= 0 ? S.Dd + S.Do[dlist[q]] : nullptr;
      __nv_bfloat16 *bt = reinterpret_cast<__nv_bfloat16 *>(Bsm + boff[q]);
      for (int idx = lane; idx < NB * kb; idx += 32) {
        const int c = idx / kb, f = idx - c * kb;
        const double v = (Db && c < ncolsB && f < nf) ? Db[f * ncolsB + c] : 0.0;
        int d[KS];
        to_digits<KS>(v, ecol[c], d);
#pragma unroll
        for (int s = 0; s < KS; ++s)
          bt[s * NB * kb + tile_off_kb(c, f, kb)] = __int2bfloat16_rn(d[s]);
      }
    }
    umma::fence_proxy_async_smem();
  }
  if (threadIdx.x == 64) {
    // Sigma targets of this job (and mirrors)
    const bool mir = S.sym && (piece == 2 || it.role == 1);
    int64_t o, m = -1;
    if (piece == 1) {
      o = dh_find(S.shash, hk_pack(it.a, it.b, it.n[0], it.n[1], it.n[2]));
      if (mir) m = dh_find(S.shash, hk_pack(it.b, it.a, -it.n[0], -it.n[1], -it.n[2]));
    } else {
      o = dh_find(S.shash, hk_pack(it.a, eg.other, nG0, nG1, nG2));
      if (mir) m = dh_find(S.shash, hk_pack(eg.other, it.a, -nG0, -nG1, -nG2));
    }
    if (o < 0 || (mir && m < 0)) atomicOr(S.err, HFX_DEV_ERR_MISSING);
    tgt[0] = o;
    tgt[1] = m;
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = *tslot;

  if (threadIdx.x == 0) {
    const uint32_t idesc = umma::idesc_bf16_f32(128, NB);
    const __nv_bfloat16 *Abase =
        S.cz + S.cz_base[it.a] + (int64_t)mt * S.ktotZ[it.a] * KS * 128;
    auto load = [&](int s, int q) {
      const int kb = kbl[q];
      const int64_t koff = S.kofs[it.fbase + flist[q]];
      umma::mbar_arrive_expect_tx(&full[s], (uint32_t)(KS * kb * 128 * 2));
      umma::bulk_g2s(smem + s * A_STAGE, Abase + koff * KS * 128, (uint32_t)(KS * kb * 128 * 2),
                     &full[s]);
    };
    for (int s = 0; s < 2 && s < nsel; ++s) load(s, s);
    bool ok = true;
    for (int q = 0; q < nsel; ++q) {
      const int s = q & 1;
      const uint32_t ph = (uint32_t)(q >> 1) & 1u;
      if (!umma::mbar_wait(&full[s], ph, S.err)) { ok = false; break; }
      umma::fence_after_sync();
      const int kb = kbl[q];
      const uint32_t sbo = (uint32_t)(kb / 8) * 128;
      const uint32_t a0 = umma::smem_u32(smem + s * A_STAGE);
      const uint32_t b0 = umma::smem_u32(Bsm + boff[q]);
      for (int j = 0; j < kb / 16; ++j)
#pragma unroll
        for (int g = 0; g < KS; ++g)
#pragma unroll
          for (int i = 0; i <= g; ++i) {
            const uint64_t ad = umma::smem_desc(a0 + i * kb * 128 * 2 + j * 256, 128, sbo);
            const uint64_t bd = umma::smem_desc(b0 + (g - i) * NB * kb * 2 + j * 256, 128, sbo);
            umma::mma_bf16(tbase + g * NB, ad, bd, idesc, (q | j | i) ? 1u : 0u);
          }
      umma::mma_commit(&empty[s]);
      if (q + 2 < nsel) {
        if (!umma::mbar_wait(&empty[s], ph, S.err)) { ok = false; break; }
        load(s, q + 2);
      }
    }
    if (ok) umma::mma_commit(done);
    else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(done)) : "memory");
  }
  __syncwarp();
  const bool ready = umma::mbar_wait(done, 0, S.err);
  umma::fence_after_sync();

  // ---- epilogue
  const int row = warp * 32 + lane;
  const int rowZ = mt * 128 + row;              // (al, a) = al * na + a
  const bool rvalid = ready && rowZ < pA * na;
  const int al = rvalid ? rowZ / na : 0;
  const int eA = S.cz_e[S.cz_rowpre[it.a] + rowZ];
  constexpr int SH = 7 * (KS + 1);
  float2 z[32];
  for (int c0 = 0; c0 < NB; c0 += 16) {
    long long Wv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) Wv[i] = 0;
#pragma unroll
    for (int g = 0; g < KS; ++g) {
      float v[16];
      umma::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * NB + c0), v);
      const long long sc = 1ll << (7 * (KS - 1 - g));
#pragma unroll
      for (int i = 0; i < 16; ++i) Wv[i] += (long long)__float2int_rn(v[i]) * sc;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
      z[c0 + i] = (c0 + i < ncolsB && rvalid) ? pair_i64(Wv[i], eA + ecol[c0 + i] - SH)
                                              : make_float2(0.f, 0.f);
  }
  // contract with Y (f32 pairs): out[o] = sum_c Z[c] Y...[o, c]
  const int ncol = S.ncol[it.b];
  const float2 *Y2 = reinterpret_cast<const float2 *>(W.scratch + W.y2_off[wl]);
  const int nout = piece == 1 ? nb : ng;
  double outv[32];
  for (int o = 0; o < nout; ++o) {
    float sh = 0.f, sl = 0.f;
    if (rvalid) {
      if (piece == 1) {  // out b: sum_g Z[g] Y[al][b][G, g]
        const float2 *y = Y2 + ((int64_t)al * nb + o) * ncol + eg.aopre;
        for (int c = 0; c < ng; ++c) df_mac(sh, sl, z[c], y[c]);
      } else {           // out g: sum_b Z[b] Y[al][b][G, g]
        const float2 *y = Y2 + (int64_t)al * nb * ncol + eg.aopre + o;
        for (int c = 0; c < nb; ++c) df_mac(sh, sl, z[c], y[(int64_t)c * ncol]);
      }
    }
    outv[o] = (double)sh + (double)sl;
  }
  // reduce over al within the tile (shared memory reuses the operand ring)
  __syncthreads();
  double *red = reinterpret_cast<double *>(smem);  // [128][32]
  for (int o = 0; o < nout; ++o) red[row * 32 + o] = outv[o];
  __syncthreads();
  const int r0 = mt * 128;
  const int rend = min(pA * na, r0 + 128);
  for (int idx = threadIdx.x; idx < na * nout; idx += 128) {
    const int a = idx / nout, o = idx - a * nout;
    // rows r in [r0, rend) with r % na == a
    int r = r0 + ((a - r0 % na) % na + na) % na;
    double sacc = 0.0;
    bool any = false;
    for (; r < rend; r += na) {
      sacc += red[(r - r0) * 32 + o];
      any = true;
    }
    if (!any || !ready) continue;
    // piece 1: Sigma_AB[a][b = o]; piece 2: Sigma_AG[a][g = o]
    if (tgt[0] >= 0) fx_add(S.acc + 2 * (tgt[0] + (int64_t)a * nout + o), -sacc);
    if (tgt[1] >= 0) fx_add(S.acc + 2 * (tgt[1] + (int64_t)o * na + a), -sacc);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, TCOLS);
}

template <int KS>
cudaError_t zwave_t(const SplitShared &S, const SplitWave &W, cudaStream_t st) {
  if (W.h_zcand > 0) k_jobs_z<<<(unsigned)((W.h_zcand + 255) / 256), 256, 0, st>>>(S, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !W.zjobs || W.h_zjobs_max <= 0) return e;
  const size_t smem = 2 * (size_t)KS * 128 * 32 * 2 + ZB_BYTES + 64 + 16 +
                      (4 * ZF_MAX + 32) * 4 + (ZF_MAX + 2) * 8 + 64;
  e = cudaFuncSetAttribute(k_zgemm<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_zgemm<KS><<<(unsigned)W.h_zjobs_max, 128, smem, st>>>(S, W);
  return cudaGetLastError();
}

template <int KS>
cudaError_t slice_cz_t(const SplitShared &S, cudaStream_t st) {
  if (S.h_cz_rows > 0)
    k_slice_cz<KS><<<(unsigned)((S.h_cz_rows * 32 + 255) / 256), 256, 0, st>>>(S);
  return cudaGetLastError();
}

}  // namespace split

cudaError_t split_zwave(const SplitShared &S, const SplitWave &W, int ks, cudaStream_t st) {
  switch (ks) {
    case 4: return split::zwave_t<4>(S, W, st);
    case 5: return split::zwave_t<5>(S, W, st);
    case 6: return split::zwave_t<6>(S, W, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t split_slice_cz(const SplitShared &S, int ks, cudaStream_t st) {
  switch (ks) {
    case 4: return split::slice_cz_t<4>(S, st);
    case 5: return split::slice_cz_t<5>(S, st);
    case 6: return split::slice_cz_t<6>(S, st);
    default: return cudaErrorInvalidValue;
  }
}
