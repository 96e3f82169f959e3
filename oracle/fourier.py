"""CPU oracle for the two steps next to the exchange build (test infrastructure).

Only the test suite uses this module; the library never imports it.  Plain
numpy, FP64 and complex128, one explicit loop per sum of the definitions:

- ``density``: the real-space density matrix from Kohn-Sham eigenvectors
  (Sec. II, Eq. DM_realspace).  With the block key (K, L, n) for sites (K, 0)
  and (L, n), the phase e^{-i k.(R_K - R_L)} is e^{2 pi i kappa.n}, kappa in
  fractional reciprocal coordinates.
- ``sigma_k``: the exchange matrix at k points (Eq. Ham_rs2kspace),
  Sigma(k) = sum over the real-space keys of e^{2 pi i kappa.n} Sigma(R_n).
"""
from __future__ import annotations

import numpy as np


def basis_offsets(nao) -> np.ndarray:
    """First basis index of each atom: rows (K, k) -> offset[K] + k."""
    nao = np.asarray(nao, np.int64)
    return np.concatenate([[0], np.cumsum(nao)])


def density(nao, kfrac, coef, occ, keys):
    """Eq. DM_realspace for each key (K, L, n1, n2, n3).

    coef: complex (nk, nbasis, nbands); occ: (nk, nbands); kfrac: (nk, 3).
    Returns (list of complex blocks [nao(K)][nao(L)], in key order)."""
    off = basis_offsets(nao)
    kfrac = np.asarray(kfrac, np.float64).reshape(-1, 3)
    coef = np.asarray(coef, np.complex128)
    occ = np.asarray(occ, np.float64)
    nk = kfrac.shape[0]
    blocks = []
    for K, L, n1, n2, n3 in np.asarray(keys, np.int64).reshape(-1, 5).tolist():
        rows = slice(off[K], off[K + 1])
        cols = slice(off[L], off[L + 1])
        acc = np.zeros((off[K + 1] - off[K], off[L + 1] - off[L]), np.complex128)
        for q in range(nk):
            phase = np.exp(2j * np.pi * (kfrac[q, 0] * n1 + kfrac[q, 1] * n2 + kfrac[q, 2] * n3))
            # sum over bands of f c_K conj(c_L)
            p = (coef[q, rows, :] * occ[q][None, :]) @ np.conj(coef[q, cols, :]).T
            acc += phase * p
        blocks.append(acc / nk)
    return blocks


def sigma_k(nao, keys, blocks, kfrac):
    """Eq. Ham_rs2kspace: dense complex (nk, nbasis, nbasis) from real-space
    blocks {key (I, J, n1, n2, n3): [nao(I)][nao(J)]}."""
    off = basis_offsets(nao)
    nb = int(off[-1])
    kfrac = np.asarray(kfrac, np.float64).reshape(-1, 3)
    out = np.zeros((kfrac.shape[0], nb, nb), np.complex128)
    for key, blk in zip(np.asarray(keys, np.int64).reshape(-1, 5).tolist(), blocks):
        I, J, n1, n2, n3 = key
        blk = np.asarray(blk, np.float64).reshape(off[I + 1] - off[I], off[J + 1] - off[J])
        for q in range(kfrac.shape[0]):
            phase = np.exp(2j * np.pi * (kfrac[q, 0] * n1 + kfrac[q, 1] * n2 + kfrac[q, 2] * n3))
            out[q, off[I]:off[I + 1], off[J]:off[J + 1]] += phase * blk
    return out
