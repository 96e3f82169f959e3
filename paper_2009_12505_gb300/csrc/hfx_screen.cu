// Block upper limits and the per-term screen (Sec. III.B-C of the paper).
//
//  * k_maxabs: max|x| of every block (the upper limit of Sec. III.B), one warp
//    per block; flags NaN/Inf.
//  * k_screen: one warp per (work item <A,B>, G in N[B]).  For every F in N[A]
//    and each of the four placements of the ABF centres (Algorithm 2/3:
//    D_FG -> Sigma_AB, D_FB -> Sigma_AG, D_AG -> Sigma_FB, D_AB -> Sigma_FG)
//    it evaluates S = (max|C_AF| max|C_BG|)(max|V_AB| max|D_src|) with
//    round-to-nearest multiplies in that association and keeps the term iff
//    S > theta (strict, as Algorithm 4).  With the Cauchy-Schwarz ERI screen
//    on (Sec. III.C, Eq. CS-ERI) a quadruple (A,B,F,G) also needs
//    sqrt(Q_AF) sqrt(Q_BG) > eps_eri, else all four of its terms go.
//    Survivors become bits of four F-bitmasks per (A,B,G); their Sigma keys go
//    into a hash set.
//  * k_diag_eri: one block per C block, the largest diagonal ERI Q of its AO
//    pairs (phi_Xa phi_Yf | phi_Xa phi_Yf) under the LRI expansion of the pair
//    on the ABFs of X and of Y (Eq. LRI), in FP64.
#include "hfx_internal.h"

__global__ void k_maxabs(const double *__restrict__ data, const int64_t *__restrict__ offs,
                         int64_t nblk, double *__restrict__ out, unsigned *err) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nblk) return;
  const int64_t b0 = offs[warp], b1 = offs[warp + 1];
  double m = 0.0;
  bool bad = false;
  for (int64_t t = b0 + lane; t < b1; t += 32) {
    const double a = fabs(data[t]);
    bad |= !isfinite(a);
    m = fmax(m, a);
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, HFX_DEV_ERR_NONFINITE);
  if (lane == 0) out[warp] = m;
}

// u^T V w over one V block ([nu][nw] row-major, nullptr = absent), with u and
// w strided views into C blocks.
__device__ inline double vform(const double *V, const double *u, int64_t su, int nu,
                               const double *w, int64_t sw, int nw) {
  if (!V) return 0.0;
  double q = 0.0;
  for (int al = 0; al < nu; ++al) {
    const double *row = V + (int64_t)al * nw;
    double t = 0.0;
    for (int be = 0; be < nw; ++be) t = fma(row[be], w[be * sw], t);
    q = fma(u[al * su], t, q);
  }
  return q;
}

// The pair (X a, Y f) of C block (x, y, n) expands as sum_alpha C_XY[alpha][a][f]
// P_X alpha + sum_beta C_YX[beta][f][a] P_Y beta; its diagonal ERI is that
// vector's V-norm: u^T V_XX u + u^T V_XY w + w^T V_YX u + w^T V_YY w.
__global__ void __launch_bounds__(128) k_diag_eri(const double *Cd, const int64_t *Co,
                                                  const double *Vd, const int64_t *Vo,
                                                  const int64_t *meta, const int32_t *cxy,
                                                  const int32_t *nao, const int32_t *nabf,
                                                  double *sq) {
  __shared__ double red[4];
  const int64_t e = blockIdx.x;
  const int x = cxy[2 * e], y = cxy[2 * e + 1];
  const int px = nabf[x], py = nabf[y], nx = nao[x], ny = nao[y];
  const int64_t *m = meta + 5 * e;
  const double *VXX = m[0] >= 0 ? Vd + Vo[m[0]] : nullptr;
  const double *VXY = m[1] >= 0 ? Vd + Vo[m[1]] : nullptr;
  const double *VYX = m[2] >= 0 ? Vd + Vo[m[2]] : nullptr;
  const double *VYY = m[3] >= 0 ? Vd + Vo[m[3]] : nullptr;
  const double *CX = Cd + Co[e];
  const double *CY = m[4] >= 0 ? Cd + Co[m[4]] : nullptr;
  double qmax = -INFINITY;
  for (int c = threadIdx.x; c < nx * ny; c += blockDim.x) {
    const int a = c / ny, f = c - a * ny;
    const double *u = CX + c;                    // u[alpha] at alpha nx ny
    double q = vform(VXX, u, (int64_t)nx * ny, px, u, (int64_t)nx * ny, px);
    if (CY) {
      const double *w = CY + (int64_t)f * nx + a;  // w[beta] at beta ny nx
      q += vform(VXY, u, (int64_t)nx * ny, px, w, (int64_t)ny * nx, py);
      q += vform(VYX, w, (int64_t)ny * nx, py, u, (int64_t)nx * ny, px);
      q += vform(VYY, w, (int64_t)ny * nx, py, w, (int64_t)ny * nx, py);
    }
    qmax = fmax(qmax, q);
  }
  for (int o = 16; o; o >>= 1) qmax = fmax(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = qmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
    sq[e] = sqrt(q > 0.0 ? q : 0.0);
  }
}

// Insert k into the mutable Sigma key table (open addressing, linear probe).
__device__ inline void sig_insert(unsigned long long *keys, uint64_t mask, uint64_t k,
                                  unsigned long long *count, unsigned long long limit,
                                  unsigned *err) {
  uint64_t s = hk_mix(k) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long cur = *(volatile unsigned long long *)&keys[s];
    if (cur == k) return;
    if (cur == HK_EMPTY) {
      const unsigned long long prev = atomicCAS(&keys[s], HK_EMPTY, (unsigned long long)k);
      if (prev == HK_EMPTY) {
        if (atomicAdd(count, 1ull) + 1 > limit) atomicOr(err, HFX_DEV_ERR_HASH_FULL);
        return;
      }
      if (prev == k) return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, HFX_DEV_ERR_HASH_FULL);
}

// Index of the work item owning flat pair index p (items' wg_off ascending).
__device__ inline int64_t find_item(const WorkItem *items, int64_t nitems, int64_t p) {
  int64_t lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (items[mid].wg_off <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ inline int64_t dfind(const DevHash &h, int i, int j, int n0, int n1, int n2) {
  return dh_find(h, hk_pack(i, j, n0, n1, n2));
}

__global__ void __launch_bounds__(256, 3) k_screen(ScreenArgs A) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= A.nwg) return;
  const int64_t w = find_item(A.items, A.nitems, p);
  const WorkItem it = A.items[w];
  const int g = (int)(p - it.wg_off);
  const NbrEntry eg = A.nbr[it.gbase + g];
  const int gt = eg.other;
  const int nG0 = it.n[0] + eg.n[0], nG1 = it.n[1] + eg.n[1], nG2 = it.n[2] + eg.n[2];
  const bool g_is_b = (gt == it.b) && eg.n[0] == 0 && eg.n[1] == 0 && eg.n[2] == 0;
  const double mcBG = A.C.maxabs[eg.cblk];
  const double mv = A.V.maxabs[it.vblk];
  const double theta = A.theta_atom ? A.theta_atom[it.a] : A.theta;
  const int64_t dAG = dfind(A.dhash, it.a, gt, nG0, nG1, nG2);
  const double mvAG = dAG >= 0 ? __dmul_rn(mv, A.D.maxabs[dAG]) : 0.0;
  const double mvAB = it.dab >= 0 ? __dmul_rn(mv, A.D.maxabs[it.dab]) : 0.0;
  const int pA = A.nabf[it.a];
  const int na = A.nao[it.a], nb = A.nao[it.b], ng = A.nao[gt];
  unsigned cnt[4] = {0, 0, 0, 0};  // surviving F per piece (at most nF each)
  unsigned long long macs = 0, pm[4] = {0, 0, 0, 0};
  unsigned eri_cut = 0;
  const double sqBG = A.eri_sq ? A.eri_sq[eg.cblk] : 0.0;
  unsigned any = 0;
  uint32_t *mrow = A.masks + it.mask_off + (int64_t)g * 4 * it.nFw;
  for (int f0 = 0; f0 < it.nF; f0 += 32) {
    const int f = f0 + lane;
    bool b1 = false, b2 = false, b3 = false, b4 = false;
    int ft = 0, mF0 = 0, mF1 = 0, mF2 = 0, nf = 0;
    if (f < it.nF) {
      const NbrEntry ef = A.nbr[it.fbase + f];
      ft = ef.other; mF0 = ef.n[0]; mF1 = ef.n[1]; mF2 = ef.n[2];
      nf = A.nao[ft];
      const bool f_is_a = (ft == it.a) && mF0 == 0 && mF1 == 0 && mF2 == 0;
      const double cc = __dmul_rn(A.C.maxabs[ef.cblk], mcBG);
      // the Cauchy-Schwarz ERI screen removes the whole quadruple
      const bool eri_ok = !A.eri_sq || __dmul_rn(A.eri_sq[ef.cblk], sqBG) > A.eps_eri;
      eri_cut += eri_ok ? 0 : 1;
      if (eri_ok) {
        // variant 1: D_FG -> Sigma_AB
        const int64_t dFG = dfind(A.dhash, ft, gt, nG0 - mF0, nG1 - mF1, nG2 - mF2);
        if (dFG >= 0) b1 = __dmul_rn(cc, __dmul_rn(mv, A.D.maxabs[dFG])) > theta;
        // variant 2: D_FB -> Sigma_AG (not when G is B)
        if (!g_is_b) {
          const int64_t dFB = dfind(A.dhash, ft, it.b, it.n[0] - mF0, it.n[1] - mF1, it.n[2] - mF2);
          if (dFB >= 0) b2 = __dmul_rn(cc, __dmul_rn(mv, A.D.maxabs[dFB])) > theta;
        }
        // variant 3: D_AG -> Sigma_FB (not when F is A)
        if (!f_is_a && dAG >= 0) b3 = __dmul_rn(cc, mvAG) > theta;
        // variant 4: D_AB -> Sigma_FG (neither)
        if (!f_is_a && !g_is_b && it.dab >= 0) b4 = __dmul_rn(cc, mvAB) > theta;
      }
    }
    const uint32_t w1 = __ballot_sync(0xffffffffu, b1);
    const uint32_t w2 = __ballot_sync(0xffffffffu, b2);
    const uint32_t w3 = __ballot_sync(0xffffffffu, b3);
    const uint32_t w4 = __ballot_sync(0xffffffffu, b4);
    if (lane == 0) {
      const int wd = f0 >> 5;
      mrow[0 * it.nFw + wd] = w1;
      mrow[1 * it.nFw + wd] = w2;
      mrow[2 * it.nFw + wd] = w3;
      mrow[3 * it.nFw + wd] = w4;
    }
    cnt[0] += __popc(w1); cnt[1] += __popc(w2); cnt[2] += __popc(w3); cnt[3] += __popc(w4);
    any |= (w1 ? 1u : 0u) | (w2 ? 2u : 0u) | (w3 ? 4u : 0u) | (w4 ? 8u : 0u);
    if (f < it.nF) {
      const unsigned fb = (b1 ? 1u : 0u) | (b2 ? 2u : 0u) | (b3 ? 4u : 0u) | (b4 ? 8u : 0u);
      if (fb) atomicOr(&A.wf_flags[it.wf_off + f], fb);
      // Algorithm 3 multiply-adds per surviving term (T stage + Ht stage)
      if (b1) pm[0] += (unsigned long long)pA * nb * nf * (ng + na);
      if (b2) pm[1] += (unsigned long long)pA * nf * ng * (nb + na);
      if (b3) pm[2] += (unsigned long long)pA * na * nb * (ng + nf);
      if (b4) pm[3] += (unsigned long long)pA * na * ng * (nb + nf);
      if (b3) sig_insert(A.sig_keys, A.sig_mask,
                         hk_pack(ft, it.b, it.n[0] - mF0, it.n[1] - mF1, it.n[2] - mF2),
                         A.sig_count, A.sig_limit, A.err);
      if (b4) sig_insert(A.sig_keys, A.sig_mask, hk_pack(ft, gt, nG0 - mF0, nG1 - mF1, nG2 - mF2),
                         A.sig_count, A.sig_limit, A.err);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    for (int o = 16; o; o >>= 1) pm[v] += __shfl_xor_sync(0xffffffffu, pm[v], o);
    macs += pm[v];
  }
  for (int o = 16; o; o >>= 1) eri_cut += __shfl_xor_sync(0xffffffffu, eri_cut, o);
  if (lane == 0 && eri_cut) atomicAdd(&A.counters[21], (unsigned long long)eri_cut);
  if (lane == 0) {
    A.wg_flags[it.wg_off + g] = (uint8_t)any;
    if (any & 1u) sig_insert(A.sig_keys, A.sig_mask, hk_pack(it.a, it.b, it.n[0], it.n[1], it.n[2]),
                             A.sig_count, A.sig_limit, A.err);
    if (any & 2u) sig_insert(A.sig_keys, A.sig_mask, hk_pack(it.a, gt, nG0, nG1, nG2),
                             A.sig_count, A.sig_limit, A.err);
    for (int v = 0; v < 4; ++v)
      if (cnt[v]) atomicAdd(&A.counters[v], (unsigned long long)cnt[v]);
    if (any) {
      atomicAdd(&A.counters[4], 1ull);
      const int pB = A.nabf[it.b];
      const unsigned long long ym = (unsigned long long)pA * pB * nb * ng;
      macs += ym;  // Y = V C_BG once per active (A,B,G)
      atomicAdd(&A.counters[20], ym);
    }
    if (macs) atomicAdd(&A.counters[5], macs);
    for (int v = 0; v < 4; ++v)
      if (pm[v]) atomicAdd(&A.counters[16 + v], pm[v]);
  }
}

// Collect the occupied slots of the Sigma key table.
__global__ void k_collect_keys(const unsigned long long *keys, uint64_t cap,
                               unsigned long long *out, unsigned long long *n) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cap) return;
  const unsigned long long k = keys[s];
  if (k != HK_EMPTY) out[atomicAdd(n, 1ull)] = k;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_maxabs(const double *data, const int64_t *offs, int64_t nblk, double *out,
                          unsigned *err, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  const int64_t threads = nblk * 32;
  k_maxabs<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(data, offs, nblk, out, err);
  return cudaGetLastError();
}

cudaError_t launch_screen(const ScreenArgs &a, cudaStream_t st) {
  if (a.nwg <= 0) return cudaSuccess;
  const int64_t threads = a.nwg * 32;
  k_screen<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diag_eri(const double *Cd, const int64_t *Co, const double *Vd,
                            const int64_t *Vo, const int64_t *meta, const int32_t *cxy,
                            const int32_t *nao, const int32_t *nabf, int64_t nC, double *sq,
                            cudaStream_t st) {
  if (nC <= 0) return cudaSuccess;
  k_diag_eri<<<(unsigned)nC, 128, 0, st>>>(Cd, Co, Vd, Vo, meta, cxy, nao, nabf, sq);
  return cudaGetLastError();
}

cudaError_t launch_collect_keys(const unsigned long long *keys, uint64_t cap,
                                unsigned long long *out, unsigned long long *n, cudaStream_t st) {
  k_collect_keys<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(keys, cap, out, n);
  return cudaGetLastError();
}
