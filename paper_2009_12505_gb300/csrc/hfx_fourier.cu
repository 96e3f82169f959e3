// The two steps next to the exchange build, in FP64 on CUDA cores:
//
// Real-space density matrix from Kohn-Sham eigenvectors (Eq. DM_realspace).
// With the block key (K, L, n) = sites (K, 0) and (L, n), so that
// R_K - R_L = -R_n,
//   D_{Kk,Ll}(n) = (1/N_k) sum_q sum_b f_qb c_q[Kk][b] conj(c_q[Ll][b])
//                  exp(2 pi i kappa_q . n),
// kappa_q the q-th k point in fractional reciprocal coordinates.  D is real
// when the k set and the eigenvectors are time-reversal symmetric; the largest
// |imaginary part| is reported so a caller can check that.
//
// Exchange matrix at k points (Eq. Ham_rs2kspace):
//   Sigma_{Ii,Jj}(k) = sum_{keys (I, J, n)} exp(2 pi i kappa . n) Sigma(I, J, n)_{ij}.
//
// Both are gathers: each output element is a fixed-order sum, so results are
// deterministic.  The phases come from sincospi of 2 kappa . n.
#include <cuda_runtime.h>

#include "hfx_internal.h"

namespace {

// One block per requested key; threads over the block's elements.
__global__ void k_density(int nk, const double *__restrict__ kfrac, int nb, int nbands,
                          const double *__restrict__ coef, const double *__restrict__ occ,
                          const int32_t *__restrict__ keys, const int32_t *__restrict__ aoff,
                          const int32_t *__restrict__ nao, const int64_t *__restrict__ doff,
                          double *__restrict__ out, unsigned long long *__restrict__ maxim) {
  const int64_t e = blockIdx.x;
  const int K = keys[5 * e], L = keys[5 * e + 1];
  const double n0 = keys[5 * e + 2], n1 = keys[5 * e + 3], n2 = keys[5 * e + 4];
  const int nK = nao[K], nL = nao[L];
  const double inv = 1.0 / nk;
  for (int t = threadIdx.x; t < nK * nL; t += blockDim.x) {
    const int kk = t / nL, ll = t - kk * nL;
    const int64_t rk = aoff[K] + kk, rl = aoff[L] + ll;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < nk; ++q) {
      const double *cK = coef + ((int64_t)q * nb + rk) * nbands * 2;
      const double *cL = coef + ((int64_t)q * nb + rl) * nbands * 2;
      const double *f = occ + (int64_t)q * nbands;
      double zr = 0.0, zi = 0.0;  // sum_b f c_K conj(c_L)
      for (int b = 0; b < nbands; ++b) {
        const double ar = cK[2 * b], ai = cK[2 * b + 1], br = cL[2 * b], bi = cL[2 * b + 1];
        zr += f[b] * (ar * br + ai * bi);
        zi += f[b] * (ai * br - ar * bi);
      }
      double s, c;
      sincospi(2.0 * (kfrac[3 * q] * n0 + kfrac[3 * q + 1] * n1 + kfrac[3 * q + 2] * n2), &s, &c);
      re += zr * c - zi * s;
      im += zr * s + zi * c;
    }
    out[doff[e] + t] = re * inv;
    // nonnegative doubles order as their bit patterns
    atomicMax(maxim, (unsigned long long)__double_as_longlong(fabs(im * inv)));
  }
}

// One block per (k point, I, J); the keys of (I, J) are the sorted range
// [lower_bound(I, J), ...) of the build's key list.
__global__ void k_sigma_k(int nk, const double *__restrict__ kfrac, int natoms,
                          const int32_t *__restrict__ aoff, const int32_t *__restrict__ nao,
                          int64_t nkeys, const uint64_t *__restrict__ skeys,
                          const int64_t *__restrict__ soffs, const double *__restrict__ sigma,
                          int64_t nb, double *__restrict__ out) {
  const int64_t bid = blockIdx.x;
  const int q = (int)(bid / ((int64_t)natoms * natoms));
  const int64_t ij = bid - (int64_t)q * natoms * natoms;
  const int I = (int)(ij / natoms), J = (int)(ij - (int64_t)I * natoms);
  // first key of (I, J)
  const uint64_t k0 = hk_pack(I, J, -128, -128, -128);
  int64_t lo = 0, hi = nkeys;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (skeys[mid] < k0) lo = mid + 1; else hi = mid;
  }
  const int nI = nao[I], nJ = nao[J];
  const double kx = kfrac[3 * q], ky = kfrac[3 * q + 1], kz = kfrac[3 * q + 2];
  for (int t = threadIdx.x; t < nI * nJ; t += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int64_t e = lo; e < nkeys; ++e) {
      int32_t k[5];
      hk_unpack(skeys[e], k);
      if (k[0] != I || k[1] != J) break;
      double s, c;
      sincospi(2.0 * (kx * k[2] + ky * k[3] + kz * k[4]), &s, &c);
      const double v = sigma[soffs[e] + t];
      re += v * c;
      im += v * s;
    }
    const int i = t / nJ, j = t - i * nJ;
    double *o = out + (((int64_t)q * nb + aoff[I] + i) * nb + aoff[J] + j) * 2;
    o[0] = re;
    o[1] = im;
  }
}

}  // namespace

cudaError_t launch_density(int nk, const double *kfrac, int nb, int nbands, const double *coef,
                           const double *occ, int64_t nkeys, const int32_t *keys,
                           const int32_t *aoff, const int32_t *nao, const int64_t *doff,
                           double *out, unsigned long long *maxim, cudaStream_t st) {
  if (nkeys <= 0) return cudaSuccess;
  k_density<<<(unsigned)nkeys, 256, 0, st>>>(nk, kfrac, nb, nbands, coef, occ, keys, aoff, nao,
                                              doff, out, maxim);
  return cudaGetLastError();
}

cudaError_t launch_sigma_k(int nk, const double *kfrac, int natoms, const int32_t *aoff,
                           const int32_t *nao, int64_t nkeys, const uint64_t *skeys,
                           const int64_t *soffs, const double *sigma, int64_t nb, double *out,
                           cudaStream_t st) {
  const int64_t nblk = (int64_t)nk * natoms * natoms;
  if (nblk <= 0) return cudaSuccess;
  k_sigma_k<<<(unsigned)nblk, 256, 0, st>>>(nk, kfrac, natoms, aoff, nao, nkeys, skeys, soffs,
                                             sigma, nb, out);
  return cudaGetLastError();
}
