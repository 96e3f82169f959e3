"""The canonical flop count (Algorithm 3, C((VC)D) order) against Table 1 of
the paper, on a cluster with exactly one quadruple (A, B, F, G) whose four
ABF placements all survive."""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def table1():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table1_multiplication_order.txt")):
        if line.startswith("#") or "|" not in line:
            continue
        order, expr = (x.strip() for x in line.split("|"))
        rows[order] = expr
    return rows


def one_quadruple(nphi, nP, seed=3):
    """Atoms A=0, B=1, F=2, G=3 of a cluster; C only on (A,F) and (B,G), V only
    on (A,B), D on the four pairs the four pieces read."""
    s = synth.custom("quad", 1.0, 1000, [[0, 0, 0], [3, 0, 0], [0, 2, 0], [3, 2, 0]],
                     [nphi] * 4, [nP] * 4)
    rng = np.random.default_rng(seed)
    z = (0, 0, 0)
    C = {(0, 2) + z: rng.standard_normal((nP, nphi, nphi)),
         (1, 3) + z: rng.standard_normal((nP, nphi, nphi))}
    V = {(0, 1) + z: rng.standard_normal((nP, nP))}
    D = {(2, 3) + z: rng.standard_normal((nphi, nphi)), (2, 1) + z: rng.standard_normal((nphi, nphi)),
         (0, 3) + z: rng.standard_normal((nphi, nphi)), (0, 1) + z: rng.standard_normal((nphi, nphi))}
    return synth.Workload("quad", s, synth.pack(C), synth.pack(V), synth.pack(D), 0, 0, 0, seed)


@pytest.mark.parametrize("nphi,nP", [(13, 60), (5, 7), (27, 90)])
def test_canonical_count_is_table1_row(nphi, nP):
    wl = one_quadruple(nphi, nP)
    keys, counts, extra = oracle.Oracle.of(wl).keys(0.0, extra=True)
    np.testing.assert_array_equal(counts, [1, 1, 1, 1])
    assert extra["active_abg"] == 1
    macs = eval(table1()["C((VC)D)"], {"nP": nP, "nphi": nphi})
    assert extra["canonical_flops"] == 2 * macs
    # with n_P several times n_phi (the paper's premise) C((VC)D) beats
    # C(V(CD)) and the two n_phi^4 orders
    others = [eval(e, {"nP": nP, "nphi": nphi}) for o, e in table1().items()
              if o not in ("C((VC)D)", "(CV)(CD)")]
    if nP >= 3 * nphi:
        assert all(macs < x for x in others)


class _Tally:
    """Matrix products that count their multiply-adds (m k n each)."""

    def __init__(self):
        self.macs = 0

    def mm(self, x, y):
        assert x.ndim == 2 and y.ndim == 2 and x.shape[1] == y.shape[0]
        self.macs += x.shape[0] * x.shape[1] * y.shape[1]
        return x @ y


def _uneven_quadruple(seed=4):
    """Atoms A=0, B=1, F=2, G=3 with four different sizes (n_phi, n_P)."""
    nphi, nP = [13, 27, 5, 9], [60, 90, 7, 11]
    s = synth.custom("quad4", 1.0, 1000, [[0, 0, 0], [3, 0, 0], [0, 2, 0], [3, 2, 0]], nphi, nP)
    rng = np.random.default_rng(seed)
    z = (0, 0, 0)
    A, B, F, G = 0, 1, 2, 3
    C = {(A, F) + z: rng.standard_normal((nP[A], nphi[A], nphi[F])),
         (B, G) + z: rng.standard_normal((nP[B], nphi[B], nphi[G]))}
    V = {(A, B) + z: rng.standard_normal((nP[A], nP[B]))}
    D = {(F, G) + z: rng.standard_normal((nphi[F], nphi[G])),
         (F, B) + z: rng.standard_normal((nphi[F], nphi[B])),
         (A, G) + z: rng.standard_normal((nphi[A], nphi[G])),
         (A, B) + z: rng.standard_normal((nphi[A], nphi[B]))}
    wl = synth.Workload("quad4", s, synth.pack(C), synth.pack(V), synth.pack(D), 0, 0, 0, seed)
    return wl, nphi, nP, C, V, D


def test_canonical_count_uneven_sizes_by_counted_products():
    """Table 1's C((VC)D) order carried out with explicit matrix products on a
    quadruple whose four atoms all differ in size (13/60, 27/90, 5/7, 9/11):
    the products give the oracle's four Sigma blocks, and the multiply-adds
    they count equal the oracle's canonical count."""
    wl, nphi, nP, C, V, D = _uneven_quadruple()
    A, B, F, G = 0, 1, 2, 3
    na, nb, nf, ng = (nphi[x] for x in (A, B, F, G))
    pA, pB = nP[A], nP[B]
    z = (0, 0, 0)
    cAF, cBG, vAB = C[(A, F) + z], C[(B, G) + z], V[(A, B) + z]
    t = _Tally()
    # Y[al][b][g] = sum_be V[al][be] C_BG[be][b][g]: once per (A, B, G)
    Y = t.mm(vAB, cBG.reshape(pB, nb * ng)).reshape(pA, nb, ng)
    # piece 1 (D_FG -> Sigma_AB): T[al][b][f] = sum_g Y D_FG^T; Ht = sum_{al,f} C_AF T
    T1 = t.mm(Y.reshape(pA * nb, ng), D[(F, G) + z].T).reshape(pA, nb, nf)
    h1 = t.mm(cAF.transpose(1, 0, 2).reshape(na, pA * nf), T1.transpose(0, 2, 1).reshape(pA * nf, nb))
    # piece 2 (D_FB -> Sigma_AG): T[al][f][g] = sum_b D_FB Y[al]; Ht = sum_{al,f} C_AF T
    T2 = np.stack([t.mm(D[(F, B) + z], Y[al]) for al in range(pA)])
    h2 = t.mm(cAF.transpose(1, 0, 2).reshape(na, pA * nf), T2.reshape(pA * nf, ng))
    # piece 3 (D_AG -> Sigma_FB): T[al][a][b] = sum_g D_AG Y[al]^T; Ht = sum_{al,a} C_AF^T T
    T3 = np.stack([t.mm(D[(A, G) + z], Y[al].T) for al in range(pA)])
    h3 = t.mm(cAF.transpose(2, 0, 1).reshape(nf, pA * na), T3.reshape(pA * na, nb))
    # piece 4 (D_AB -> Sigma_FG): T[al][a][g] = sum_b D_AB Y[al]; Ht = sum_{al,a} C_AF^T T
    T4 = np.stack([t.mm(D[(A, B) + z], Y[al]) for al in range(pA)])
    h4 = t.mm(cAF.transpose(2, 0, 1).reshape(nf, pA * na), T4.reshape(pA * na, ng))
    o = oracle.Oracle.of(wl)
    keys, counts, extra = o.keys(0.0, extra=True)
    np.testing.assert_array_equal(counts, [1, 1, 1, 1])
    data, offs = o.blocks(0.0, keys)
    got = oracle.block_dict(keys, data, offs, np.array(nphi))
    for key, h in (((A, B) + z, h1), ((A, G) + z, h2), ((F, B) + z, h3), ((F, G) + z, h4)):
        np.testing.assert_allclose(got[key], -h, rtol=1e-12, atol=1e-12 * np.abs(h).max())
    assert extra["active_abg"] == 1
    assert extra["canonical_flops"] == 2 * t.macs
