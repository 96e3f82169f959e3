// Adjoint of the exchange energy with the surviving-term set of the last
// build frozen: dE_X/dC and dE_X/dV (FP64, CUDA cores).
//
// With E_X = 1/2 sum D . Sigma and Sigma = - sum over surviving terms, every
// quadruple (A, B, F, G) of a pair <A,B> contributes
//   E = -1/2 sum C_AF[al][a][f] V_AB[al][be] C_BG[be][b][g] Omega[a][b][f][g],
//   Omega = w14 D_FG[f][g] D_AB[a][b] + w23 D_FB[f][b] D_AG[a][g],
// where w14 = m1 + m4 and w23 = m2 + m3 count the surviving pieces (ABFs on
// (I,J) and (K,L) read D_FG and D_AB, the other two read D_FB and D_AG; a
// missing D block is zero).  Hence, per pair and G,
//   Z1[al][a][g] = sum_F w14 sum_f C_AF[al][a][f] D_FG[f][g]
//   Z2[al][a][b] = sum_F w23 sum_f C_AF[al][a][f] D_FB[f][b]
//   R[al][b][g]  = sum_a D_AB[a][b] Z1[al][a][g] + sum_a D_AG[a][g] Z2[al][a][b]
//   dV_AB[al][be]   = -1/2 sum_{G,b,g} C_BG[be][b][g] R[al][b][g]
//   dC_BG[be][b][g] += -1/2 sum_al V_AB[al][be] R[al][b][g]          (C in the B role)
// and per pair and F, with Y = V_AB C_BG,
//   dC_AF[al][a][f] += -1/2 ( sum_b D_AB[a][b] sum_G w14 sum_g Y[al][b][g] D_FG[f][g]
//                           + sum_b D_FB[f][b] sum_G w23 sum_g D_AG[a][g] Y[al][b][g] )
// (C in the A role).  dC accumulates through the fixed-point adder, so the
// gradient is bitwise reproducible; each pair owns its V block.
#include "fp64_common.cuh"

namespace {

__device__ inline int64_t dblock(const ContractArgs &A, int i, int j, int n0, int n1, int n2) {
  return dh_find(A.dhash, hk_pack(i, j, n0, n1, n2));
}

// R[al][b][(G,g)] for one (pair, G), written over Y's layout in the R region.
__global__ void __launch_bounds__(kThreads) k_adj_r(ContractArgs A) {
  __shared__ int f14[512], f23[512];
  __shared__ int8_t w14[512], w23[512];
  __shared__ int64_t d14[512], d23[512];
  __shared__ int n14_s, n23_s;
  __shared__ double Z1[kChunk / 2], Z2[kChunk / 2];
  const PairLoc L = locate(A, blockIdx.x, true);
  const WorkItem it = A.items[L.w];
  const unsigned bits = A.wg_flags[it.wg_off + L.idx];
  if (!(bits & 0xFu)) return;
  if (it.nF > 512) { if (threadIdx.x == 0) atomicOr(A.err, HFX_DEV_ERR_BOUNDS); return; }
  const int g_ = L.idx;
  const NbrEntry eg = A.nbr[it.gbase + g_];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], ng = A.nao[eg.other];
  const int ncol = A.ncol[it.b];
  const int nG0 = it.n[0] + eg.n[0], nG1 = it.n[1] + eg.n[1], nG2 = it.n[2] + eg.n[2];
  const int64_t dAG = dblock(A, it.a, eg.other, nG0, nG1, nG2);
  const int n14 = ordered_select(
      it.nF, [&](int f) { return mask_bit(A, it, g_, 0, f) || mask_bit(A, it, g_, 3, f); }, f14,
      &n14_s);
  const int n23 = ordered_select(
      it.nF, [&](int f) { return mask_bit(A, it, g_, 1, f) || mask_bit(A, it, g_, 2, f); }, f23,
      &n23_s);
  for (int s = threadIdx.x; s < n14; s += kThreads) {
    const int f = f14[s];
    const NbrEntry ef = A.nbr[it.fbase + f];
    w14[s] = (int8_t)(mask_bit(A, it, g_, 0, f) + mask_bit(A, it, g_, 3, f));
    d14[s] = dblock(A, ef.other, eg.other, nG0 - ef.n[0], nG1 - ef.n[1], nG2 - ef.n[2]);
  }
  for (int s = threadIdx.x; s < n23; s += kThreads) {
    const int f = f23[s];
    const NbrEntry ef = A.nbr[it.fbase + f];
    w23[s] = (int8_t)(mask_bit(A, it, g_, 1, f) + mask_bit(A, it, g_, 2, f));
    d23[s] = dblock(A, ef.other, it.b, it.n[0] - ef.n[0], it.n[1] - ef.n[1], it.n[2] - ef.n[2]);
  }
  __syncthreads();
  const bool use14 = it.dab >= 0, use23 = dAG >= 0;
  const double *Dab = use14 ? A.D.data + A.D.offs[it.dab] : nullptr;
  const double *Dag = use23 ? A.D.data + A.D.offs[dAG] : nullptr;
  double *R = A.scratch + A.p_off[L.w - A.w0] + eg.aopre;  // R[al][b][ncol]
  const int per1 = na * ng, per2 = na * nb;
  const int ach = max(1, min(pA, (kChunk / 2) / max(per1, per2)));
  unsigned long long macs = 0;
  for (int al0 = 0; al0 < pA; al0 += ach) {
    const int ac = min(ach, pA - al0);
    for (int idx = threadIdx.x; idx < ac * per1; idx += kThreads) {
      const int al = idx / per1, r = idx - al * per1, a = r / ng, g = r - a * ng;
      double s = 0.0;
      if (use14)
        for (int q = 0; q < n14; ++q) {
          if (d14[q] < 0) continue;
          const NbrEntry ef = A.nbr[it.fbase + f14[q]];
          const int nf = A.nao[ef.other];
          const double *c = A.C.data + A.C.offs[ef.cblk] + ((int64_t)(al0 + al) * na + a) * nf;
          const double *d = A.D.data + A.D.offs[d14[q]] + g;
          double t = 0.0;
          for (int f = 0; f < nf; ++f) t = fma(c[f], d[f * ng], t);
          s = fma((double)w14[q], t, s);
        }
      Z1[idx] = s;
    }
    for (int idx = threadIdx.x; idx < ac * per2; idx += kThreads) {
      const int al = idx / per2, r = idx - al * per2, a = r / nb, b = r - a * nb;
      double s = 0.0;
      if (use23)
        for (int q = 0; q < n23; ++q) {
          if (d23[q] < 0) continue;
          const NbrEntry ef = A.nbr[it.fbase + f23[q]];
          const int nf = A.nao[ef.other];
          const double *c = A.C.data + A.C.offs[ef.cblk] + ((int64_t)(al0 + al) * na + a) * nf;
          const double *d = A.D.data + A.D.offs[d23[q]] + b;
          double t = 0.0;
          for (int f = 0; f < nf; ++f) t = fma(c[f], d[f * nb], t);
          s = fma((double)w23[q], t, s);
        }
      Z2[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ac * nb * ng; idx += kThreads) {
      const int al = idx / (nb * ng), r = idx - al * nb * ng, b = r / ng, g = r - b * ng;
      double s = 0.0;
      if (use14)
        for (int a = 0; a < na; ++a) s = fma(Dab[a * nb + b], Z1[(al * na + a) * ng + g], s);
      if (use23)
        for (int a = 0; a < na; ++a) s = fma(Dag[a * ng + g], Z2[(al * na + a) * nb + b], s);
      R[((int64_t)(al0 + al) * nb + b) * ncol + g] = s;
    }
    __syncthreads();
    macs += (unsigned long long)ac * na * (ng * n14 + nb * n23) * 13 + (unsigned long long)ac * nb * ng * na * 2;
  }
  if (threadIdx.x == 0) atomicAdd(A.macs + 0, macs);
}

// dV_AB[al][be] = -1/2 sum over active G of sum_{b,g} C_BG[be][b][g] R[al][b][(G,g)].
__global__ void __launch_bounds__(kThreads) k_adj_dv(ContractArgs A) {
  const int64_t w = A.w0 + blockIdx.x;
  if (w >= A.w1) return;
  const WorkItem it = A.items[w];
  const int pA = A.nabf[it.a], pB = A.nabf[it.b], nb = A.nao[it.b];
  const int ncol = A.ncol[it.b];
  const double *R = A.scratch + A.p_off[w - A.w0];
  double *out = A.dv + A.V.offs[it.vblk];
  for (int o = threadIdx.x; o < pA * pB; o += kThreads) {
    const int al = o / pB, be = o - al * pB;
    double s = 0.0;
    for (int g_ = 0; g_ < it.nG; ++g_) {
      if (!(A.wg_flags[it.wg_off + g_] & 0xFu)) continue;
      const NbrEntry eg = A.nbr[it.gbase + g_];
      const int ng = A.nao[eg.other];
      const double *c = A.C.data + A.C.offs[eg.cblk] + (int64_t)be * nb * ng;
      const double *r = R + (int64_t)al * nb * ncol + eg.aopre;
      for (int b = 0; b < nb; ++b)
        for (int g = 0; g < ng; ++g) s = fma(c[b * ng + g], r[(int64_t)b * ncol + g], s);
    }
    out[(int64_t)al * pB + be] = -0.5 * s;
  }
}

// dC_BG[be][b][g] += -1/2 sum_al V_AB[al][be] R[al][b][(G,g)]   (C in the B role)
__global__ void __launch_bounds__(kThreads) k_adj_dcb(ContractArgs A) {
  const PairLoc L = locate(A, blockIdx.x, true);
  const WorkItem it = A.items[L.w];
  if (!(A.wg_flags[it.wg_off + L.idx] & 0xFu)) return;
  const NbrEntry eg = A.nbr[it.gbase + L.idx];
  const int pA = A.nabf[it.a], pB = A.nabf[it.b], nb = A.nao[it.b], ng = A.nao[eg.other];
  const int ncol = A.ncol[it.b];
  const double *V = A.V.data + A.V.offs[it.vblk];
  const double *R = A.scratch + A.p_off[L.w - A.w0] + eg.aopre;
  unsigned long long *acc = A.dcacc + 2 * A.C.offs[eg.cblk];
  for (int o = threadIdx.x; o < pB * nb * ng; o += kThreads) {
    const int be = o / (nb * ng), r = o - be * nb * ng, b = r / ng, g = r - b * ng;
    double s = 0.0;
    for (int al = 0; al < pA; ++al)
      s = fma(V[(int64_t)al * pB + be], R[((int64_t)al * nb + b) * ncol + g], s);
    fx_add(acc + 2 * o, -0.5 * s, A.err);
  }
}

// dC_AF (C in the A role) for one (pair, F).
__global__ void __launch_bounds__(kThreads) k_adj_dca(ContractArgs A) {
  __shared__ int g14[512], g23[512];
  __shared__ int8_t w14[512], w23[512];
  __shared__ int64_t d14[512], d23[512];
  __shared__ int n14_s, n23_s;
  __shared__ double T1[kChunk / 2], Ts[kChunk / 2];
  const PairLoc L = locate(A, blockIdx.x, false);
  const WorkItem it = A.items[L.w];
  if (!(A.wf_flags[it.wf_off + L.idx] & 0xFu)) return;
  if (it.nG > 512) { if (threadIdx.x == 0) atomicOr(A.err, HFX_DEV_ERR_BOUNDS); return; }
  const int f_ = L.idx;
  const NbrEntry ef = A.nbr[it.fbase + f_];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], nf = A.nao[ef.other];
  const int ncol = A.ncol[it.b];
  const int64_t dFB = dblock(A, ef.other, it.b, it.n[0] - ef.n[0], it.n[1] - ef.n[1],
                             it.n[2] - ef.n[2]);
  const bool use14 = it.dab >= 0, use23 = dFB >= 0;
  const int n14 = ordered_select(
      it.nG, [&](int g) { return mask_bit(A, it, g, 0, f_) || mask_bit(A, it, g, 3, f_); }, g14,
      &n14_s);
  const int n23 = ordered_select(
      it.nG, [&](int g) { return mask_bit(A, it, g, 1, f_) || mask_bit(A, it, g, 2, f_); }, g23,
      &n23_s);
  for (int s = threadIdx.x; s < n14; s += kThreads) {
    const NbrEntry eg = A.nbr[it.gbase + g14[s]];
    w14[s] = (int8_t)(mask_bit(A, it, g14[s], 0, f_) + mask_bit(A, it, g14[s], 3, f_));
    d14[s] = dblock(A, ef.other, eg.other, it.n[0] + eg.n[0] - ef.n[0],
                    it.n[1] + eg.n[1] - ef.n[1], it.n[2] + eg.n[2] - ef.n[2]);
  }
  for (int s = threadIdx.x; s < n23; s += kThreads) {
    const NbrEntry eg = A.nbr[it.gbase + g23[s]];
    w23[s] = (int8_t)(mask_bit(A, it, g23[s], 1, f_) + mask_bit(A, it, g23[s], 2, f_));
    d23[s] = dblock(A, it.a, eg.other, it.n[0] + eg.n[0], it.n[1] + eg.n[1], it.n[2] + eg.n[2]);
  }
  __syncthreads();
  const double *Dab = use14 ? A.D.data + A.D.offs[it.dab] : nullptr;
  const double *Dfb = use23 ? A.D.data + A.D.offs[dFB] : nullptr;
  const double *Ybase = A.scratch + A.y_off[L.w - A.w0];
  unsigned long long *acc = A.dcacc + 2 * A.C.offs[ef.cblk];
  const int per1 = nb * nf, per2 = na * nb;
  const int ach = max(1, min(pA, (kChunk / 2) / max(per1, per2)));
  unsigned long long macs = 0;
  for (int al0 = 0; al0 < pA; al0 += ach) {
    const int ac = min(ach, pA - al0);
    // T1[al][b][f] = sum_G w14 sum_g Y[al][b][(G,g)] D_FG[f][g]
    for (int idx = threadIdx.x; idx < ac * per1; idx += kThreads) {
      const int ab = idx / nf, f = idx - ab * nf;
      double s = 0.0;
      if (use14)
        for (int q = 0; q < n14; ++q) {
          if (d14[q] < 0) continue;
          const NbrEntry eg = A.nbr[it.gbase + g14[q]];
          const int ng = A.nao[eg.other];
          const double *y = Ybase + ((int64_t)al0 * nb + ab) * ncol + eg.aopre;
          const double *d = A.D.data + A.D.offs[d14[q]] + f * ng;
          double t = 0.0;
          for (int g = 0; g < ng; ++g) t = fma(y[g], d[g], t);
          s = fma((double)w14[q], t, s);
        }
      T1[idx] = s;
    }
    // Ts[al][a][b] = sum_G w23 sum_g D_AG[a][g] Y[al][b][(G,g)]
    for (int idx = threadIdx.x; idx < ac * per2; idx += kThreads) {
      const int al = idx / per2, r = idx - al * per2, a = r / nb, b = r - a * nb;
      double s = 0.0;
      if (use23)
        for (int q = 0; q < n23; ++q) {
          if (d23[q] < 0) continue;
          const NbrEntry eg = A.nbr[it.gbase + g23[q]];
          const int ng = A.nao[eg.other];
          const double *y = Ybase + ((int64_t)(al0 + al) * nb + b) * ncol + eg.aopre;
          const double *d = A.D.data + A.D.offs[d23[q]] + a * ng;
          double t = 0.0;
          for (int g = 0; g < ng; ++g) t = fma(d[g], y[g], t);
          s = fma((double)w23[q], t, s);
        }
      Ts[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ac * na * nf; idx += kThreads) {
      const int al = idx / (na * nf), r = idx - al * na * nf, a = r / nf, f = r - a * nf;
      double s = 0.0;
      if (use14)
        for (int b = 0; b < nb; ++b) s = fma(Dab[a * nb + b], T1[(al * nb + b) * nf + f], s);
      if (use23)
        for (int b = 0; b < nb; ++b) s = fma(Dfb[f * nb + b], Ts[(al * na + a) * nb + b], s);
      fx_add(acc + 2 * ((int64_t)(al0 + al) * na * nf + r), -0.5 * s, A.err);
    }
    __syncthreads();
    macs += (unsigned long long)ac * (per1 + per2) * 13 * (n14 + n23);
  }
  if (threadIdx.x == 0) atomicAdd(A.macs + 1, macs);
}

__global__ void k_fx_to_double_adj(const unsigned long long *acc, int64_t n, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fx_value((long long)acc[2 * i], (long long)acc[2 * i + 1]);
}

}  // namespace

cudaError_t launch_adjoint(const ContractArgs &a, cudaStream_t st) {
  if (a.nwg > 0) {
    k_adj_r<<<(unsigned)a.nwg, kThreads, 0, st>>>(a);
    k_adj_dcb<<<(unsigned)a.nwg, kThreads, 0, st>>>(a);
  }
  if (a.w1 > a.w0) k_adj_dv<<<(unsigned)(a.w1 - a.w0), kThreads, 0, st>>>(a);
  if (a.nwf > 0) k_adj_dca<<<(unsigned)a.nwf, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fx_to_double(const unsigned long long *acc, int64_t n, double *out,
                                cudaStream_t st) {
  if (n > 0) k_fx_to_double_adj<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc, n, out);
  return cudaGetLastError();
}
