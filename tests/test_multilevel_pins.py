"""Pins for the multi-level screening oracle (oracle/multilevel.py; Sec. III.C,
Eq. CS_upper_bounds, Algorithm 4): the Schatten-4 norm against singular
values, the three bounds as true upper bounds on random matrices, the
reduction to the block-screened build at eps = 0, the dropped-mass bound and
monotonicity in eps."""
import numpy as np
import pytest

import refforms
import synth
from oracle import multilevel


def _cell():
    s = synth.custom("pair", 1.0, 5, [[0, 0, 0], [2, 1, 1]], [2, 3], [3, 4])
    return synth.make_workload(s, 3.2, 4.5, 3.2, seed=9)


def test_schatten4_is_the_fourth_root_of_the_sum_of_sigma4():
    rng = np.random.default_rng(0)
    for shape in ((3, 5), (6, 2), (4, 4)):
        m = rng.normal(size=shape)
        sv = np.linalg.svd(m, compute_uv=False)
        assert abs(multilevel.s4(m) - (sv ** 4).sum() ** 0.25) < 1e-12 * sv.max()


def test_the_three_bounds_hold_on_random_matrices():
    """|tr[X^T V Y D^T]| <= L1, L2, L3 (Hoelder with Schatten-4 and Frobenius)."""
    rng = np.random.default_rng(1)
    fro = np.linalg.norm
    for _ in range(200):
        na, nb, k, l = rng.integers(1, 7, 4)
        X, V = rng.normal(size=(na, k)), rng.normal(size=(na, nb))
        Y, D = rng.normal(size=(nb, l)), rng.normal(size=(k, l))
        h = abs(np.trace(X.T @ V @ Y @ D.T))
        l1 = multilevel.s4(X) * multilevel.s4(V) * multilevel.s4(Y) * multilevel.s4(D)
        l2 = multilevel.s4(X) * fro(V @ Y) * multilevel.s4(D)
        l3 = fro(X) * fro(V @ Y @ D.T)
        # each is a bound of its own; they are tested in turn, not nested
        assert h <= l1 * (1 + 1e-12) and h <= l2 * (1 + 1e-12) and h <= l3 * (1 + 1e-12)


def _flat(sig, keys):
    return np.concatenate([np.ravel(sig.get(k, 0.0)) for k in keys])


@pytest.mark.parametrize("theta", [0.0, 1e-2])
def test_eps_zero_is_the_block_screened_build(theta):
    wl = _cell()
    ref, _, _ = refforms.ab_form(wl, theta)
    got, stats = multilevel.build(wl, theta, 0.0)
    assert set(got) == set(ref)
    keys = sorted(ref)
    np.testing.assert_allclose(_flat(got, keys), _flat(ref, keys), rtol=0,
                               atol=1e-12 * np.abs(_flat(ref, keys)).max())
    assert stats[3] > 0


def test_dropped_mass_and_monotone_in_eps():
    """Every element Algorithm 4 drops is below eps in magnitude, so the change
    of any Sigma element is at most eps times the number of dropped elements;
    a larger eps never computes more elements."""
    wl = _cell()
    ref, _ = multilevel.build(wl, 0.0, 0.0)
    keys = sorted(ref)
    base = _flat(ref, keys)
    computed = []
    for eps in (1e-3, 0.05, 0.1, 0.3, 1.0):  # the tiny cell's elements are O(1)
        got, stats = multilevel.build(wl, 0.0, eps)
        dropped = int(stats[:3].sum())
        err = np.abs(_flat(got, keys) - base).max()
        assert err <= eps * max(dropped, 1)
        computed.append(int(stats[3]))
    assert computed == sorted(computed, reverse=True)
    assert computed[-1] < computed[0]
    # all three levels stop some element at eps = 0.1
    _, stats = multilevel.build(wl, 0.0, 0.1)
    assert (stats[:3] > 0).all()


def test_diagonal_eris_match_the_lri_map():
    """Q(A, F) from the oracle equals the largest diagonal of M_A V M_A^T over
    the rows (F, a, f) of the brute-force LRI map."""
    wl = _cell()
    q = multilevel.diag_eri_max(wl)
    S = refforms.Sites(wl)
    for a in range(wl.system.natoms):
        A = (a, (0, 0, 0))
        sites = sorted({A} | set(S.partners(A)))
        abf, c = {}, 0
        for s in sites:
            abf[s] = (c, c + int(S.nabf[s[0]]))
            c += int(S.nabf[s[0]])
        V = np.zeros((c, c))
        for s in sites:
            for t in sites:
                vb = S.v(s, t)
                if vb is not None:
                    V[abf[s][0]:abf[s][1], abf[t][0]:abf[t][1]] = vb
        M, rows = refforms._lri_matrix(S, A, abf)
        diag = np.einsum("ij,jk,ik->i", M, V, M)
        r0 = 0
        for (F, nx, ny) in rows:
            key = S.key(A, F)
            if key in q:
                assert abs(diag[r0:r0 + nx * ny].max() - q[key]) <= 1e-12 * max(1.0, abs(q[key]))
            r0 += nx * ny


def test_eri_screen_limits():
    """eps_eri below every bound keeps every quadruple (the plain build); the
    screen removes more quadruples as eps_eri grows."""
    wl = _cell()
    ref, _ = multilevel.build(wl, 0.0, 0.0)
    got, stats = multilevel.build(wl, 0.0, 0.0, eps_eri=-1.0)
    keys = sorted(ref)
    np.testing.assert_array_equal(_flat(got, keys), _flat(ref, keys))
    assert stats[4] == 0
    removed = [int(multilevel.build(wl, 0.0, 0.0, eps_eri=e)[1][4]) for e in (0.1, 1.0, 5.0, 50.0)]
    assert removed == sorted(removed) and removed[-1] > removed[0]
