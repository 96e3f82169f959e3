"""Independent restatements of the exchange build used to pin the oracle.

Each function here is a different route to the same quantity as the oracle,
written from the paper's equations and never from the oracle's code:

* ``brute_sigma``: Eq. LRI as a linear map.  For a site X, the AO products
  phi_Xx phi_Yy (Y any partner) expand on ABFs with a coefficient matrix M_X;
  the four-centre ERIs between the pair spaces of X and J are M_X V M_J^T
  (Eq. ERI_split summed), and Sigma_XJ = -sum_{K,L} ERI D_KL (Eq. HFX_ERIs).
* ``cluster_sigma``: the same for a finite cluster with dense tensors and one
  numpy.einsum.
* ``ab_form``: Algorithm 3 -- pairs <A,B> outermost, F in N[A], G in N[B],
  Y = V C_BG, the four T contractions with D_FG, D_FB, D_AG, D_AB and the four
  Ht accumulations -- with the per-term screen and the on-site rule, plus the
  per-block bound sum_{dropped} (contracted dims) * S for the screening test.
"""
from __future__ import annotations

import itertools

import numpy as np


def _d(blocks):
    return blocks.as_dict()


class Sites:
    """Block lookups between sites (atom, cell) for a synth Workload."""

    def __init__(self, wl):
        self.wl = wl
        self.nao = wl.system.nao
        self.nabf = wl.system.nabf
        self.C = _d(wl.C)
        self.V = _d(wl.V)
        self.D = _d(wl.D)
        self.Cnbr = {}
        for (i, j, *n) in self.C:
            self.Cnbr.setdefault(i, []).append((j, tuple(n)))
        self.Vnbr = {}
        for (i, j, *n) in self.V:
            self.Vnbr.setdefault(i, []).append((j, tuple(n)))

    @staticmethod
    def key(x, y):
        (a, na), (b, nb) = x, y
        return (a, b) + tuple(int(q - p) for p, q in zip(na, nb))

    def c(self, x, y):
        blk = self.C.get(self.key(x, y))
        if blk is None:
            return None
        return blk.reshape(int(self.nabf[x[0]]), int(self.nao[x[0]]), int(self.nao[y[0]]))

    def v(self, x, y):
        blk = self.V.get(self.key(x, y))
        return None if blk is None else blk.reshape(int(self.nabf[x[0]]), int(self.nabf[y[0]]))

    def dm(self, x, y):
        blk = self.D.get(self.key(x, y))
        return None if blk is None else blk.reshape(int(self.nao[x[0]]), int(self.nao[y[0]]))

    def partners(self, x):
        """Sites Y with C(X,Y) or C(Y,X) present."""
        a, na = x
        out = set()
        for (j, n) in self.Cnbr.get(a, []):
            out.add((j, tuple(p + q for p, q in zip(na, n))))
        for (i, j, *n) in self.C:
            if j == a:
                out.add((i, tuple(p - q for p, q in zip(na, n))))
        return sorted(out)

    @staticmethod
    def shift(x, n):
        return (x[0], tuple(p + q for p, q in zip(x[1], n)))


def _lri_matrix(S: Sites, x, abf_index):
    """Rows (Y, x-AO, y-AO) for every partner Y of X; columns ABFs (Z, zeta).

    Eq. LRI: phi_Xx phi_Yy = sum_zeta C(X,Y)[zeta,x,y] P_{X zeta}
                           + [Y != X] sum_zeta C(Y,X)[zeta,y,x] P_{Y zeta}."""
    rows = []
    parts = S.partners(x)
    for y in parts:
        rows.append((y, int(S.nao[x[0]]), int(S.nao[y[0]])))
    nrow = sum(nx * ny for _, nx, ny in rows)
    ncol = max(v[1] for v in abf_index.values())
    M = np.zeros((nrow, ncol))
    r0 = 0
    for (y, nx, ny) in rows:
        cxy = S.c(x, y)
        if cxy is not None:
            c0, c1 = abf_index[x]
            M[r0:r0 + nx * ny, c0:c1] += cxy.transpose(1, 2, 0).reshape(nx * ny, -1)
        if y != x:
            cyx = S.c(y, x)
            if cyx is not None:
                c0, c1 = abf_index[y]
                M[r0:r0 + nx * ny, c0:c1] += cyx.transpose(2, 1, 0).reshape(nx * ny, -1)
        r0 += nx * ny
    return M, rows


def brute_sigma(wl, i: int, J):
    """Sigma block between site (i, 0) and site J, at theta = 0, by M_I V M_J^T."""
    S = Sites(wl)
    I = (i, (0, 0, 0))
    J = (J[0], tuple(J[1]))
    sites = set([I, J]) | set(S.partners(I)) | set(S.partners(J))
    sites = sorted(sites)
    abf_index = {}
    c = 0
    for s in sites:
        abf_index[s] = (c, c + int(S.nabf[s[0]]))
        c += int(S.nabf[s[0]])
    Vfull = np.zeros((c, c))
    for s in sites:
        for t in sites:
            vb = S.v(s, t)
            if vb is not None:
                Vfull[abf_index[s][0]:abf_index[s][1], abf_index[t][0]:abf_index[t][1]] = vb
    MI, rowsI = _lri_matrix(S, I, abf_index)
    MJ, rowsJ = _lri_matrix(S, J, abf_index)
    eri = MI @ Vfull @ MJ.T          # [(K, i, k), (L, j, l)]
    ni, nj = int(S.nao[i]), int(S.nao[J[0]])
    out = np.zeros((ni, nj))
    r0 = 0
    for (K, _, nk) in rowsI:
        q0 = 0
        for (L, _, nl) in rowsJ:
            dkl = S.dm(K, L)
            if dkl is not None:
                blk = eri[r0:r0 + ni * nk, q0:q0 + nj * nl].reshape(ni, nk, nj, nl)
                out -= np.einsum("ikjl,kl->ij", blk, dkl)
            q0 += nj * nl
        r0 += ni * nk
    return out


def cluster_sigma(wl):
    """Finite cluster (no periodic images within reach): dense einsum.

    Ctil[z, x, y] is the LRI coefficient of P_z in phi_x phi_y over the whole
    cluster; Sigma[i, j] = -sum Ctil[z,i,k] V[z,w] Ctil[w,j,l] D[k,l]."""
    S = Sites(wl)
    nat = wl.system.natoms
    ao = np.concatenate([[0], np.cumsum(S.nao)])
    ab = np.concatenate([[0], np.cumsum(S.nabf)])
    n, m = int(ao[-1]), int(ab[-1])
    z3 = (0, 0, 0)
    Ct = np.zeros((m, n, n))
    V = np.zeros((m, m))
    D = np.zeros((n, n))
    for a in range(nat):
        for b in range(nat):
            A, B = (a, z3), (b, z3)
            cab = S.c(A, B)
            if cab is not None:
                Ct[ab[a]:ab[a + 1], ao[a]:ao[a + 1], ao[b]:ao[b + 1]] += cab
                if a != b:
                    Ct[ab[a]:ab[a + 1], ao[b]:ao[b + 1], ao[a]:ao[a + 1]] += cab.transpose(0, 2, 1)
            vab = S.v(A, B)
            if vab is not None:
                V[ab[a]:ab[a + 1], ab[b]:ab[b + 1]] = vab
            dab = S.dm(A, B)
            if dab is not None:
                D[ao[a]:ao[a + 1], ao[b]:ao[b + 1]] = dab
    sig = -np.einsum("zik,zw,wjl,kl->ij", Ct, V, Ct, D, optimize=True)
    return sig, ao


def ab_form(wl, theta: float, atoms=None, each=None):
    """Algorithm 3 with the block-norm screen; returns ({key: block}, counts,
    {key: bound}) where bound sums (pA pB nK nL) * S over DROPPED terms.
    ``atoms`` limits the central atoms A; ``each(key, block)`` is called with
    every surviving term's contribution."""
    S = Sites(wl)
    mx = {k: float(np.max(np.abs(v))) for k, v in S.C.items()}
    mv = {k: float(np.max(np.abs(v))) for k, v in S.V.items()}
    md = {k: float(np.max(np.abs(v))) for k, v in S.D.items()}
    sig, bound = {}, {}
    counts = np.zeros(4, np.int64)
    z3 = (0, 0, 0)

    def add(dct, key, val):
        if key in dct:
            dct[key] = dct[key] + val
        else:
            dct[key] = val

    for a in range(wl.system.natoms):
        if atoms is not None and a not in atoms:
            continue
        A = (a, z3)
        Fs = [(f, n) for (f, n) in S.Cnbr.get(a, [])]
        for (b, nb) in S.Vnbr.get(a, []):
            B = (b, nb)
            vab = S.v(A, B)
            mvab = mv[S.key(A, B)]
            Gs = [(g, tuple(p + q for p, q in zip(nb, n))) for (g, n) in S.Cnbr.get(b, [])]
            for F in Fs:
                cAF = S.c(A, F)
                for G in Gs:
                    cBG = S.c(B, G)
                    Y = np.einsum("ab,bjl->ajl", vab, cBG)       # Y[alpha][b][g]
                    cc = mx[S.key(A, F)] * mx[S.key(B, G)]
                    # (source D, target pair, contraction) per variant
                    for v, (dsrc, tx, ty) in enumerate(((F, G, (A, B)), (F, B, (A, G)),
                                                        (A, G, (F, B)), (A, B, (F, G)))):
                        if v in (2, 3) and F == A:
                            continue   # {I,K} is one site: counted as ABFs on I
                        if v in (1, 3) and G == B:
                            continue
                        dk = S.key(dsrc, tx)
                        if dk not in S.D:
                            continue
                        s = cc * (mvab * md[dk])
                        dblk = S.dm(dsrc, tx)
                        if v == 0:    # T[al,b,f] = sum_g Y[al,b,g] D_FG[f,g]; Ht[a,b]
                            T = np.einsum("abg,fg->abf", Y, dblk)
                            ht = np.einsum("aif,ajf->ij", cAF, T)
                            tk = S.key(A, B)
                            dims = cAF.shape[0] * vab.shape[1] * cAF.shape[2] * cBG.shape[2]
                        elif v == 1:  # T[al,f,g] = sum_b Y[al,b,g] D_FB[f,b]; Ht[a,g]
                            T = np.einsum("abg,fb->afg", Y, dblk)
                            ht = np.einsum("aif,afg->ig", cAF, T)
                            tk = S.key(A, G)
                            dims = cAF.shape[0] * vab.shape[1] * cAF.shape[2] * cBG.shape[1]
                        elif v == 2:  # T[al,a,b] = sum_g Y[al,b,g] D_AG[a,g]; Ht[f,b]
                            T = np.einsum("abg,ig->aib", Y, dblk)
                            ht = np.einsum("aif,aib->fb", cAF, T)
                            tk = S.key(F, B)
                            dims = cAF.shape[0] * vab.shape[1] * cAF.shape[1] * cBG.shape[2]
                        else:         # T[al,a,g] = sum_b Y[al,b,g] D_AB[a,b]; Ht[f,g]
                            T = np.einsum("abg,ib->aig", Y, dblk)
                            ht = np.einsum("aif,aig->fg", cAF, T)
                            tk = S.key(F, G)
                            dims = cAF.shape[0] * vab.shape[1] * cAF.shape[1] * cBG.shape[1]
                        # S.key translates the target so its first site is in the home cell
                        if s > theta:
                            counts[v] += 1
                            add(sig, tk, -ht)
                            if each is not None:
                                each(tk, -ht)
                        else:
                            add(bound, tk, dims * s)
    return sig, counts, bound


def supercell(wl, ncell: int):
    """Replicate a workload's blocks into an ncell^3 supercell (same values)."""
    import synth
    sysu = wl.system
    cells = list(itertools.product(range(ncell), repeat=3))
    nat = sysu.natoms
    grid = np.concatenate([sysu.grid + np.array(c) * sysu.period for c in cells])
    sysS = synth.System(sysu.name + f"x{ncell}", sysu.unit, sysu.period * ncell, grid,
                        np.tile(sysu.nao, len(cells)), np.tile(sysu.nabf, len(cells)),
                        np.tile(sysu.species, len(cells)))

    def rep(blocks):
        out = {}
        for (x, y, *n), v in blocks.as_dict().items():
            for ci, c1 in enumerate(cells):
                c2p = [c1[k] + n[k] for k in range(3)]
                N = tuple(int(np.floor_divide(c2p[k], ncell)) for k in range(3))
                c2 = tuple(int(c2p[k] - N[k] * ncell) for k in range(3))
                s1 = ci * nat + x
                s2 = cells.index(c2) * nat + y
                out[(s1, s2) + N] = v.copy()
        return synth.pack(out)

    return synth.Workload(wl.name + f"x{ncell}", sysS, rep(wl.C), rep(wl.V), rep(wl.D),
                          wl.cut_C, wl.cut_V, wl.cut_D, wl.seed), cells
