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
