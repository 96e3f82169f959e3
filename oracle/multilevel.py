"""CPU oracle for the multi-level Cauchy-Schwarz matrix screening (test
infrastructure; Sec. III.C, Eq. CS_upper_bounds and Algorithm 4).

Only the test suite uses this module; the library never imports it and does
not implement this screen yet.  Plain numpy, FP64, in the <A,B>-pair loop of
Algorithm 3 with its four pieces.

For one term, with the output element's AO indices fixed, the element is
    h = tr[X^T V Y D^T],  X (alpha x k) from C_AF, Y (beta x l) from C_BG,
    V = V_AB (alpha x beta), D the piece's source density block (k x l):
    piece 1 (D_FG -> Sigma_AB[a][b]): X = C_AF[:, a, :], Y = C_BG[:, b, :]
    piece 2 (D_FB -> Sigma_AG[a][g]): X = C_AF[:, a, :], Y = C_BG[:, :, g]
    piece 3 (D_AG -> Sigma_FB[f][b]): X = C_AF[:, :, f], Y = C_BG[:, b, :]
    piece 4 (D_AB -> Sigma_FG[f][g]): X = C_AF[:, :, f], Y = C_BG[:, :, g].
Algorithm 4 tests three upper bounds of |h| in turn and stops at the first
that is not above eps:
    L1 = |X|_4 |V|_4 |Y|_4 |D|_4,   L2 = |X|_4 |V Y| |D|_4,   L3 = |X| |(V Y) D^T|,
where |M| is the Frobenius norm and |M|_4 = sqrt(|M M^+|) (the Schatten-4
norm).  Reading: the paper does not name the norm; with the Frobenius norm all
three are Hoelder bounds (|tr ABCD| <= prod of Schatten-4 norms;
|tr[X^T W D^T]| <= |X|_4 |W| |D|_4; Cauchy-Schwarz), so each is a true bound.
The block screen of the library (block max-norm product > theta) is applied
first, as the first level of Algorithm 4; the Cauchy-Schwarz ERI screen
(Eq. CS-ERI, per quadruple of atoms) optionally before the element bounds.
A diagonal ERI can be negative when the synthetic V is not positive
semi-definite; the screen then uses 0 for it.
"""
from __future__ import annotations

import numpy as np


def s4(m: np.ndarray) -> float:
    """Schatten-4 norm sqrt(|M M^+|_F)."""
    m = np.asarray(m, np.float64)
    return float(np.sqrt(np.linalg.norm(m @ m.T)))


def _fro(m) -> float:
    return float(np.linalg.norm(m))


class _Sites:
    def __init__(self, wl):
        self.nao, self.nabf = wl.system.nao, wl.system.nabf
        self.C, self.V, self.D = wl.C.as_dict(), wl.V.as_dict(), wl.D.as_dict()
        self.Cnbr, self.Vnbr = {}, {}
        for (i, j, *n) in self.C:
            self.Cnbr.setdefault(i, []).append((j, tuple(n)))
        for (i, j, *n) in self.V:
            self.Vnbr.setdefault(i, []).append((j, tuple(n)))

    @staticmethod
    def key(x, y):
        return (x[0], y[0]) + tuple(int(q - p) for p, q in zip(x[1], y[1]))

    def c(self, x, y):
        return self.C[self.key(x, y)].reshape(int(self.nabf[x[0]]), int(self.nao[x[0]]),
                                              int(self.nao[y[0]]))


def diag_eri_max(wl) -> dict:
    """For every C key (A, F, n): the largest diagonal ERI
    (phi_Aa phi_Ff | phi_Aa phi_Ff) over a in A, f in F (Sec. III.C,
    Cauchy-Schwarz ERI screening).  By Eq. LRI the pair expands on the ABFs of
    A with C(A, F, n)[:, a, f] and, when F is another site, on those of F with
    C(F, A, -n)[:, f, a]; the ERI is that vector's V-norm with the V blocks
    between the two sites (a missing block is zero)."""
    S = _Sites(wl)
    out = {}
    for (A, F, n1, n2, n3), blk in S.C.items():
        n = (n1, n2, n3)
        pa, na, nf = int(S.nabf[A]), int(S.nao[A]), int(S.nao[F])
        cA = blk.reshape(pa, na, nf)
        vAA = S.V.get((A, A, 0, 0, 0))
        vAA = np.zeros((pa, pa)) if vAA is None else vAA.reshape(pa, pa)
        same = A == F and n == (0, 0, 0)
        q = np.einsum("xaf,xy,yaf->af", cA, vAA, cA)
        if not same:
            pf = int(S.nabf[F])
            m = (-n1, -n2, -n3)
            cF = S.C.get((F, A) + m)
            cF = np.zeros((pf, nf, na)) if cF is None else cF.reshape(pf, nf, na)
            vAF = S.V.get((A, F) + n)
            vAF = np.zeros((pa, pf)) if vAF is None else vAF.reshape(pa, pf)
            vFA = S.V.get((F, A) + m)
            vFA = np.zeros((pf, pa)) if vFA is None else vFA.reshape(pf, pa)
            vFF = S.V.get((F, F, 0, 0, 0))
            vFF = np.zeros((pf, pf)) if vFF is None else vFF.reshape(pf, pf)
            q = q + np.einsum("xaf,xy,yfa->af", cA, vAF, cF) \
                  + np.einsum("xfa,xy,yaf->af", cF, vFA, cA) \
                  + np.einsum("xfa,xy,yfa->af", cF, vFF, cF)
        out[(A, F) + n] = float(q.max())
    return out


def build(wl, theta: float, eps: float, eps_eri: float = None):
    """Sigma with the block screen at theta, the Cauchy-Schwarz ERI screen at
    eps_eri (a quadruple (A, F, B, G) is kept iff
    sqrt(Q(A,F)) sqrt(Q(B,G)) > eps_eri, Q from diag_eri_max; None skips it)
    and the three element-level bounds at eps.  Returns (Sigma {key: block},
    counts) where counts[0..2] are the elements stopped by L1, L2, L3,
    counts[3] the elements computed and counts[4] the quadruples the ERI
    screen removed."""
    S = _Sites(wl)
    qeri = diag_eri_max(wl) if eps_eri is not None else None
    mx = {k: float(np.abs(v).max()) for k, v in S.C.items()}
    mv = {k: float(np.abs(v).max()) for k, v in S.V.items()}
    md = {k: float(np.abs(v).max()) for k, v in S.D.items()}
    sig = {}
    stats = np.zeros(5, np.int64)
    z3 = (0, 0, 0)
    for a in range(wl.system.natoms):
        A = (a, z3)
        Fs = S.Cnbr.get(a, [])
        for (b, nb) in S.Vnbr.get(a, []):
            B = (b, nb)
            V = S.V[S.key(A, B)].reshape(int(S.nabf[a]), int(S.nabf[b]))
            v4 = s4(V)
            Gs = [(g, tuple(p + q for p, q in zip(nb, n))) for (g, n) in S.Cnbr.get(b, [])]
            for F in Fs:
                cAF = S.c(A, F)
                for G in Gs:
                    cBG = S.c(B, G)
                    if qeri is not None:
                        qa, qb = qeri[S.key(A, F)], qeri[S.key(B, G)]
                        if not np.sqrt(max(qa, 0.0)) * np.sqrt(max(qb, 0.0)) > eps_eri:
                            stats[4] += 1
                            continue
                    cc = mx[S.key(A, F)] * mx[S.key(B, G)]
                    for v, (dsrc, tx, tgt) in enumerate(((F, G, (A, B)), (F, B, (A, G)),
                                                         (A, G, (F, B)), (A, B, (F, G)))):
                        if v in (2, 3) and F == A:
                            continue  # {I,K} is one site (the on-site rule)
                        if v in (1, 3) and G == B:
                            continue
                        dk = S.key(dsrc, tx)
                        if dk not in S.D:
                            continue
                        if not cc * (mv[S.key(A, B)] * md[dk]) > theta:
                            continue  # the block screen
                        D = S.D[dk].reshape(int(S.nao[dsrc[0]]), int(S.nao[tx[0]]))
                        d4 = s4(D)
                        Xs = [cAF[:, i, :] for i in range(cAF.shape[1])] if v in (0, 1) else \
                             [cAF[:, :, f] for f in range(cAF.shape[2])]
                        Ys = [cBG[:, j, :] for j in range(cBG.shape[1])] if v in (0, 2) else \
                             [cBG[:, :, g] for g in range(cBG.shape[2])]
                        out = np.zeros((len(Xs), len(Ys)))
                        for j, Y in enumerate(Ys):
                            y4 = s4(Y)
                            VY = V @ Y
                            vy = _fro(VY)
                            W = VY @ D.T
                            w = _fro(W)
                            for i, X in enumerate(Xs):
                                x4 = s4(X)
                                if not x4 * v4 * y4 * d4 > eps:
                                    stats[0] += 1
                                elif not x4 * vy * d4 > eps:
                                    stats[1] += 1
                                elif not _fro(X) * w > eps:
                                    stats[2] += 1
                                else:
                                    stats[3] += 1
                                    out[i, j] = float(np.sum(X * W))  # tr[X^T (V Y) D^T]
                        tk = S.key(*tgt)
                        sig[tk] = sig.get(tk, 0.0) - out
    return sig, stats
