// FP64 contraction kernels: the staged C((VC)D) build of Algorithm 3 on CUDA
// cores, one wave of <A,B> work items at a time.
//
// Per work item w = <A,B> (A = (a,0), B = (b,n)), F in N[A], G in N[B]:
//   k_y      Y_G[al][b][g]  = sum_be V_AB[al][be] C_BG[be][b][g]       (Alg. 3, Y = V*C)
//   k_dstage P_G[al][a][g]  = sum_b  D_AB[a][b]  Y_G[al][b][g]         (T of the D_AB piece)
//            T3_G[al][a][b] = sum_g  D_AG[a][g]  Y_G[al][b][g]         (T of the D_AG piece)
//   k_q      Q_F[al][a][b]  = sum_f  C_AF[al][a][f] D_FB[f][b]
//   k_v1     Sigma_AB[a][b] -= sum_{al,f} C_AF[al][a][f] sum_{G in M1(F)} sum_g Y_G[al][b][g] D_FG[f][g]
//   k_v2     Sigma_AG[a][g] -= sum_{al,b} (sum_{F in M2(G)} Q_F[al][a][b]) Y_G[al][b][g]
//   k_v3     Sigma_FB[f][b] -= sum_{al,a} C_AF[al][a][f] (sum_{G in M3(F)} T3_G[al][a][b])
//   k_v4     Sigma_FG[f][g] -= sum_{al,a} C_AF[al][a][f] P_G[al][a][g]       for F in M4(G)
// Layouts in a work item's scratch (ncol = sum of nao over N[B], the G
// columns concatenated in neighbour order, column of (G,g) = aopre(G) + g):
//   Y[al][b][ncol], P[al][a][ncol], T3[G][al][a][b], Q[F][al][a][b].
// M_v are the surviving-term bitmasks from the screen.  Every term is the
// same multilinear form as Algorithm 3's Ht; the D_FB and D_AG pieces sum the
// masked F (G) contributions before the last contraction, which is exact
// reassociation (distributivity), not an approximation.
//
// Summation order inside a kernel is fixed (masks are scanned in index order),
// and Sigma receives each block through the deterministic fixed-point adder,
// so results are bitwise reproducible.
//
// Mirror pieces (A.sym, set only when every V and D block has its mirror
// block equal to its transpose): the D_AG piece of <A,B> at (F,G) is the
// transpose of the D_FB piece of <B,A> at (G,F) -- the same factors and the
// same screening product -- so k_v2 adds each block both to Sigma_AG and,
// transposed, to Sigma_GA, and k_v3 is not run.  Likewise the D_FG and D_AB
// pieces of the mirror pair <B,A> are the transposes of those of <A,B>: they
// run on canonical pairs only (role 1), adding each block and its transpose,
// and on pairs whose B is A itself (role 0) without a mirror.
#include "hfx_internal.h"

#include "fp64_common.cuh"

namespace {

__global__ void __launch_bounds__(kThreads) k_y(ContractArgs A) {
  const PairLoc L = locate(A, blockIdx.x, true);
  const WorkItem it = A.items[L.w];
  if (!(A.wg_flags[it.wg_off + L.idx] & 0xFu)) return;
  const NbrEntry eg = A.nbr[it.gbase + L.idx];
  const int pA = A.nabf[it.a], pB = A.nabf[it.b], nb = A.nao[it.b], ng = A.nao[eg.other];
  const double *V = A.V.data + A.V.offs[it.vblk];
  const double *Cb = A.C.data + A.C.offs[eg.cblk];
  const int ncol = A.ncol[it.b];
  double *Y = A.scratch + A.y_off[L.w - A.w0] + eg.aopre;
  const int N = nb * ng;
  for (int idx = threadIdx.x; idx < pA * N; idx += kThreads) {
    const int al = idx / N, c = idx - al * N, b = c / ng, g = c - b * ng;
    const double *v = V + (int64_t)al * pB;
    double s = 0.0;
    for (int be = 0; be < pB; ++be) s = fma(v[be], Cb[(int64_t)be * N + c], s);
    Y[((int64_t)al * nb + b) * ncol + g] = s;
  }
  if (threadIdx.x == 0) atomicAdd(A.macs + 0, (unsigned long long)pA * pB * N);
}

__global__ void __launch_bounds__(kThreads) k_dstage(ContractArgs A) {
  const PairLoc L = locate(A, blockIdx.x, true);
  const WorkItem it = A.items[L.w];
  const unsigned bits = A.wg_flags[it.wg_off + L.idx];
  if (!(bits & 0xCu)) return;
  const NbrEntry eg = A.nbr[it.gbase + L.idx];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], ng = A.nao[eg.other];
  const int ncol = A.ncol[it.b];
  const double *Y = A.scratch + A.y_off[L.w - A.w0] + eg.aopre;  // Y[al][b][ncol]
  unsigned long long macs = 0;
  if ((bits & 8u) && it.dab >= 0 && !(A.sym && it.role == 2) && !A.no_p) {
    // P_G[al][a][g] = sum_b D_AB[a][b] Y_G[al][b][g]
    const double *Dab = A.D.data + A.D.offs[it.dab];
    double *P = A.scratch + A.p_off[L.w - A.w0] + eg.aopre;  // P[al][a][ncol]
    const int per = na * ng;
    for (int idx = threadIdx.x; idx < pA * per; idx += kThreads) {
      const int al = idx / per, r = idx - al * per, a = r / ng, g = r - a * ng;
      const double *y = Y + (int64_t)al * nb * ncol + g;
      const double *d = Dab + a * nb;
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s = fma(d[b], y[(int64_t)b * ncol], s);
      P[((int64_t)al * na + a) * ncol + g] = s;
    }
    macs += (unsigned long long)pA * per * nb;
  }
  if ((bits & 4u) && !A.sym) {  // T3_G[al][a][b] = sum_g D_AG[a][g] Y_G[al][b][g]
    const int n0 = it.n[0] + eg.n[0], n1 = it.n[1] + eg.n[1], n2 = it.n[2] + eg.n[2];
    const int64_t dag = dh_find(A.dhash, hk_pack(it.a, eg.other, n0, n1, n2));
    if (dag < 0) { atomicOr(A.err, HFX_DEV_ERR_MISSING); return; }
    const double *Dag = A.D.data + A.D.offs[dag];
    double *T3 = A.scratch + A.t3_off[L.w - A.w0] + (int64_t)L.idx * pA * na * nb;
    const int per = na * nb;
    for (int idx = threadIdx.x; idx < pA * per; idx += kThreads) {
      const int al = idx / per, r = idx - al * per, a = r / nb, b = r - a * nb;
      const double *y = Y + ((int64_t)al * nb + b) * ncol;
      const double *d = Dag + a * ng;
      double s = 0.0;
      for (int g = 0; g < ng; ++g) s = fma(d[g], y[g], s);
      T3[idx] = s;
    }
    macs += (unsigned long long)pA * per * ng;
  }
  if (threadIdx.x == 0 && macs) atomicAdd(A.macs + 1, macs);
}

__global__ void __launch_bounds__(kThreads) k_q(ContractArgs A) {
  const PairLoc L = locate(A, blockIdx.x, false);
  const WorkItem it = A.items[L.w];
  if (!(A.wf_flags[it.wf_off + L.idx] & 2u)) return;
  const NbrEntry ef = A.nbr[it.fbase + L.idx];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], nf = A.nao[ef.other];
  const int64_t dfb = dh_find(A.dhash, hk_pack(ef.other, it.b, it.n[0] - ef.n[0],
                                               it.n[1] - ef.n[1], it.n[2] - ef.n[2]));
  if (dfb < 0) { atomicOr(A.err, HFX_DEV_ERR_MISSING); return; }
  const double *Dfb = A.D.data + A.D.offs[dfb];
  const double *Caf = A.C.data + A.C.offs[ef.cblk];
  double *Q = A.scratch + A.q_off[L.w - A.w0] + (int64_t)L.idx * pA * na * nb;
  const int per = na * nb;
  for (int idx = threadIdx.x; idx < pA * per; idx += kThreads) {
    const int al = idx / per, r = idx - al * per, a = r / nb, b = r - a * nb;
    const double *c = Caf + ((int64_t)al * na + a) * nf;
    double s = 0.0;
    for (int f = 0; f < nf; ++f) s = fma(c[f], Dfb[f * nb + b], s);
    Q[idx] = s;
  }
  if (threadIdx.x == 0) atomicAdd(A.macs + 2, (unsigned long long)pA * per * nf);
}

// Sigma_AB -= sum_{al,f} C_AF[al][a][f] T1[al][b][f],
// T1[al][b][f] = sum_{G in M1(F)} sum_g Y_G[al][b][g] D_FG[f][g].
__global__ void __launch_bounds__(kThreads) k_v1(ContractArgs A) {
  __shared__ int glist[1024];
  __shared__ int64_t dlist[1024];
  __shared__ int nsel_s;
  __shared__ double T1[kChunk];
  const PairLoc L = locate(A, blockIdx.x, false);
  const WorkItem it = A.items[L.w];
  if (!(A.wf_flags[it.wf_off + L.idx] & 1u)) return;
  if (A.sym && it.role == 2) return;
  if (it.nG > 1024) { if (threadIdx.x == 0) atomicOr(A.err, HFX_DEV_ERR_BOUNDS); return; }
  const int f_ = L.idx;
  const NbrEntry ef = A.nbr[it.fbase + f_];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], nf = A.nao[ef.other];
  const int nsel = ordered_select(it.nG, [&](int g) { return mask_bit(A, it, g, 0, f_); },
                                  glist, &nsel_s);
  for (int s = threadIdx.x; s < nsel; s += kThreads) {
    const NbrEntry eg = A.nbr[it.gbase + glist[s]];
    dlist[s] = dh_find(A.dhash, hk_pack(ef.other, eg.other, it.n[0] + eg.n[0] - ef.n[0],
                                        it.n[1] + eg.n[1] - ef.n[1], it.n[2] + eg.n[2] - ef.n[2]));
  }
  __syncthreads();
  const double *Caf = A.C.data + A.C.offs[ef.cblk];
  const double *Ybase = A.scratch + A.y_off[L.w - A.w0];
  const int ncol = A.ncol[it.b];
  const int nout = na * nb;
  double acc[kMaxOut];
#pragma unroll
  for (int q = 0; q < kMaxOut; ++q) acc[q] = 0.0;
  const int per = nb * nf;
  const int ach = max(1, min(pA, kChunk / per));
  unsigned long long macs = 0;
  for (int al0 = 0; al0 < pA; al0 += ach) {
    const int ac = min(ach, pA - al0);
    for (int idx = threadIdx.x; idx < ac * per; idx += kThreads) T1[idx] = 0.0;
    for (int s = 0; s < nsel; ++s) {
      const NbrEntry eg = A.nbr[it.gbase + glist[s]];
      const int ng = A.nao[eg.other];
      const int64_t dfg = dlist[s];
      if (dfg < 0) continue;
      const double *Dfg = A.D.data + A.D.offs[dfg];
      const double *Y = Ybase + eg.aopre + (int64_t)al0 * nb * ncol;
      for (int idx = threadIdx.x; idx < ac * per; idx += kThreads) {
        const int ab = idx / nf, f = idx - ab * nf;  // ab = al*nb + b
        const double *y = Y + (int64_t)ab * ncol;
        const double *d = Dfg + f * ng;
        double t = 0.0;
        for (int g = 0; g < ng; ++g) t = fma(y[g], d[g], t);
        T1[idx] += t;
      }
      macs += (unsigned long long)ac * per * ng;
    }
    __syncthreads();
    for (int q = 0; q < kMaxOut; ++q) {
      const int o = threadIdx.x + q * kThreads;
      if (o >= nout) break;
      const int a = o / nb, b = o - a * nb;
      double s = acc[q];
      for (int al = 0; al < ac; ++al) {
        const double *c = Caf + ((int64_t)(al0 + al) * na + a) * nf;
        const double *t = T1 + (al * nb + b) * nf;
        for (int f = 0; f < nf; ++f) s = fma(c[f], t[f], s);
      }
      acc[q] = s;
    }
    macs += (unsigned long long)ac * nout * nf;
    __syncthreads();
  }
  const int64_t off = sig_offset(A, it.a, it.b, it.n[0], it.n[1], it.n[2]);
  const int64_t moff = (A.sym && it.role == 1)
                           ? sig_offset(A, it.b, it.a, -it.n[0], -it.n[1], -it.n[2]) : -1;
  for (int q = 0; q < kMaxOut; ++q) {
    const int o = threadIdx.x + q * kThreads;
    if (o >= nout) break;
    if (off >= 0) fx_add(A.acc + 2 * (off + o), -acc[q], A.err);
    if (moff >= 0) fx_add(A.acc + 2 * (moff + (o % nb) * na + o / nb), -acc[q], A.err);
  }
  if (threadIdx.x == 0) atomicAdd(A.macs + 3, macs);
}

// Sigma_AG -= sum_{al,b} Qsum[al][a][b] Y_G[al][b][g],  Qsum = sum_{F in M2(G)} Q_F.
__global__ void __launch_bounds__(kThreads) k_v2(ContractArgs A) {
  __shared__ int flist[1024];
  __shared__ int nsel_s;
  __shared__ double Qs[kChunk];
  const PairLoc L = locate(A, blockIdx.x, true);
  const WorkItem it = A.items[L.w];
  if (!(A.wg_flags[it.wg_off + L.idx] & 2u)) return;
  if (it.nF > 1024) { if (threadIdx.x == 0) atomicOr(A.err, HFX_DEV_ERR_BOUNDS); return; }
  const int g_ = L.idx;
  const NbrEntry eg = A.nbr[it.gbase + g_];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], ng = A.nao[eg.other];
  const int nsel = ordered_select(it.nF, [&](int f) { return mask_bit(A, it, g_, 1, f); },
                                  flist, &nsel_s);
  const double *Qbase = A.scratch + A.q_off[L.w - A.w0];
  const int ncol = A.ncol[it.b];
  const double *Y = A.scratch + A.y_off[L.w - A.w0] + eg.aopre;  // Y[al][b][ncol]
  const int per = na * nb, nout = na * ng;
  double acc[kMaxOut];
#pragma unroll
  for (int q = 0; q < kMaxOut; ++q) acc[q] = 0.0;
  const int ach = max(1, min(pA, kChunk / per));
  unsigned long long macs = 0;
  for (int al0 = 0; al0 < pA; al0 += ach) {
    const int ac = min(ach, pA - al0);
    for (int idx = threadIdx.x; idx < ac * per; idx += kThreads) {
      double s = 0.0;
      for (int k = 0; k < nsel; ++k) s += Qbase[((int64_t)flist[k] * pA + al0) * per + idx];
      Qs[idx] = s;
    }
    macs += (unsigned long long)nsel * ac * per;
    __syncthreads();
    for (int q = 0; q < kMaxOut; ++q) {
      const int o = threadIdx.x + q * kThreads;
      if (o >= nout) break;
      const int a = o / ng, g = o - a * ng;
      double s = acc[q];
      for (int al = 0; al < ac; ++al) {
        const double *qq = Qs + (al * na + a) * nb;
        const double *y = Y + (int64_t)(al0 + al) * nb * ncol + g;
        for (int b = 0; b < nb; ++b) s = fma(qq[b], y[(int64_t)b * ncol], s);
      }
      acc[q] = s;
    }
    macs += (unsigned long long)ac * nout * nb;
    __syncthreads();
  }
  const int64_t off = sig_offset(A, it.a, eg.other, it.n[0] + eg.n[0], it.n[1] + eg.n[1],
                                 it.n[2] + eg.n[2]);
  const int64_t moff = A.sym ? sig_offset(A, eg.other, it.a, -(it.n[0] + eg.n[0]),
                                          -(it.n[1] + eg.n[1]), -(it.n[2] + eg.n[2]))
                             : -1;
  for (int q = 0; q < kMaxOut; ++q) {
    const int o = threadIdx.x + q * kThreads;
    if (o >= nout) break;
    if (off >= 0) fx_add(A.acc + 2 * (off + o), -acc[q], A.err);
    if (moff >= 0) fx_add(A.acc + 2 * (moff + (o % ng) * na + o / ng), -acc[q], A.err);
  }
  if (threadIdx.x == 0) atomicAdd(A.macs + 5, macs);
}

// Sigma_FB -= sum_{al,a} C_AF[al][a][f] Tsum[al][a][b],  Tsum = sum_{G in M3(F)} T3_G.
__global__ void __launch_bounds__(kThreads) k_v3(ContractArgs A) {
  __shared__ int glist[1024];
  __shared__ int nsel_s;
  __shared__ double Ts[kChunk];
  if (A.sym) return;  // obtained as the mirror of the D_FB piece
  const PairLoc L = locate(A, blockIdx.x, false);
  const WorkItem it = A.items[L.w];
  if (!(A.wf_flags[it.wf_off + L.idx] & 4u)) return;
  if (it.nG > 1024) { if (threadIdx.x == 0) atomicOr(A.err, HFX_DEV_ERR_BOUNDS); return; }
  const int f_ = L.idx;
  const NbrEntry ef = A.nbr[it.fbase + f_];
  const int pA = A.nabf[it.a], na = A.nao[it.a], nb = A.nao[it.b], nf = A.nao[ef.other];
  const int nsel = ordered_select(it.nG, [&](int g) { return mask_bit(A, it, g, 2, f_); },
                                  glist, &nsel_s);
  const double *Tbase = A.scratch + A.t3_off[L.w - A.w0];
  const double *Caf = A.C.data + A.C.offs[ef.cblk];
  const int per = na * nb, nout = nf * nb;
  double acc[kMaxOut];
#pragma unroll
  for (int q = 0; q < kMaxOut; ++q) acc[q] = 0.0;
  const int ach = max(1, min(pA, kChunk / per));
  unsigned long long macs = 0;
  for (int al0 = 0; al0 < pA; al0 += ach) {
    const int ac = min(ach, pA - al0);
    for (int idx = threadIdx.x; idx < ac * per; idx += kThreads) {
      double s = 0.0;
      for (int k = 0; k < nsel; ++k) s += Tbase[((int64_t)glist[k] * pA + al0) * per + idx];
      Ts[idx] = s;
    }
    macs += (unsigned long long)nsel * ac * per;
    __syncthreads();
    for (int q = 0; q < kMaxOut; ++q) {
      const int o = threadIdx.x + q * kThreads;
      if (o >= nout) break;
      const int f = o / nb, b = o - f * nb;
      double s = acc[q];
      for (int al = 0; al < ac; ++al)
        for (int a = 0; a < na; ++a)
          s = fma(Caf[((int64_t)(al0 + al) * na + a) * nf + f], Ts[(al * na + a) * nb + b], s);
      acc[q] = s;
    }
    macs += (unsigned long long)ac * nout * na;
    __syncthreads();
  }
  const int64_t off = sig_offset(A, ef.other, it.b, it.n[0] - ef.n[0], it.n[1] - ef.n[1],
                                 it.n[2] - ef.n[2]);
  if (off >= 0)
    for (int q = 0; q < kMaxOut; ++q) {
      const int o = threadIdx.x + q * kThreads;
      if (o >= nout) break;
      fx_add(A.acc + 2 * (off + o), -acc[q], A.err);
    }
  if (threadIdx.x == 0) atomicAdd(A.macs + 4, macs);
}

// Sigma_FG -= sum_{al,a} C_AF[al][a][f] P_G[al][a][g]   for every F in M4(G).
__global__ void __launch_bounds__(kThreads) k_v4(ContractArgs A) {
  __shared__ int flist[1024];
  __shared__ int nsel_s;
  const PairLoc L = locate(A, blockIdx.x, true);
  const WorkItem it = A.items[L.w];
  if (!(A.wg_flags[it.wg_off + L.idx] & 8u)) return;
  if (A.sym && it.role == 2) return;
  if (it.nF > 1024) { if (threadIdx.x == 0) atomicOr(A.err, HFX_DEV_ERR_BOUNDS); return; }
  const int g_ = L.idx;
  const NbrEntry eg = A.nbr[it.gbase + g_];
  const int pA = A.nabf[it.a], na = A.nao[it.a], ng = A.nao[eg.other];
  const int nsel = ordered_select(it.nF, [&](int f) { return mask_bit(A, it, g_, 3, f); },
                                  flist, &nsel_s);
  const int ncol = A.ncol[it.b];
  const double *P = A.scratch + A.p_off[L.w - A.w0] + eg.aopre;  // P[al][a][ncol]
  const int K = pA * na;
  const int nG0 = it.n[0] + eg.n[0], nG1 = it.n[1] + eg.n[1], nG2 = it.n[2] + eg.n[2];
  unsigned long long macs = 0;
  for (int k = 0; k < nsel; ++k) {
    const NbrEntry ef = A.nbr[it.fbase + flist[k]];
    const int nf = A.nao[ef.other];
    const double *Caf = A.C.data + A.C.offs[ef.cblk];
    const int nout = nf * ng;
    const int64_t off = sig_offset(A, ef.other, eg.other, nG0 - ef.n[0], nG1 - ef.n[1],
                                   nG2 - ef.n[2]);
    const int64_t moff = (A.sym && it.role == 1)
                             ? sig_offset(A, eg.other, ef.other, -(nG0 - ef.n[0]),
                                          -(nG1 - ef.n[1]), -(nG2 - ef.n[2]))
                             : -1;
    for (int o = threadIdx.x; o < nout; o += kThreads) {
      const int f = o / ng, g = o - f * ng;
      double s = 0.0;
      for (int r = 0; r < K; ++r) s = fma(Caf[(int64_t)r * nf + f], P[(int64_t)r * ncol + g], s);
      if (off >= 0) fx_add(A.acc + 2 * (off + o), -s, A.err);
      if (moff >= 0) fx_add(A.acc + 2 * (moff + g * nf + f), -s, A.err);
    }
    macs += (unsigned long long)nout * K;
  }
  if (threadIdx.x == 0 && macs) atomicAdd(A.macs + 6, macs);
}

}  // namespace

cudaError_t launch_contract_fp64(const ContractArgs &a, cudaStream_t st, cudaEvent_t *ev, int *nl) {
  int n = 0;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], st);
  };
  const unsigned gg = (unsigned)(a.nwg > 0 ? a.nwg : 0), gf = (unsigned)(a.nwf > 0 ? a.nwf : 0);
  mark(0);
  if (gg && !(a.skip & 1u)) { k_y<<<gg, kThreads, 0, st>>>(a); ++n; }
  mark(1);
  if (gg && !(a.skip & 2u)) { k_dstage<<<gg, kThreads, 0, st>>>(a); ++n; }
  mark(2);
  if (gf && !(a.skip & 4u)) { k_q<<<gf, kThreads, 0, st>>>(a); ++n; }
  mark(3);
  if (gf && !(a.skip & 8u)) { k_v1<<<gf, kThreads, 0, st>>>(a); ++n; }
  mark(4);
  if (gf && !(a.skip & 16u)) { k_v3<<<gf, kThreads, 0, st>>>(a); ++n; }
  mark(5);
  if (gg && !(a.skip & 32u)) { k_v2<<<gg, kThreads, 0, st>>>(a); ++n; }
  mark(6);
  if (gg && !(a.skip & 64u)) { k_v4<<<gg, kThreads, 0, st>>>(a); ++n; }
  mark(7);
  if (nl) *nl = n;
  return cudaGetLastError();
}
