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
first, as the first level of Algorithm 4.
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


def build(wl, theta: float, eps: float):
    """Sigma with the block screen at theta and the three element-level bounds
    at eps.  Returns (Sigma {key: block}, kept {level: count}) where level 0..2
    counts elements stopped by L1, L2, L3 and level 3 the elements computed."""
    S = _Sites(wl)
    mx = {k: float(np.abs(v).max()) for k, v in S.C.items()}
    mv = {k: float(np.abs(v).max()) for k, v in S.V.items()}
    md = {k: float(np.abs(v).max()) for k, v in S.D.items()}
    sig = {}
    stats = np.zeros(4, np.int64)
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
