"""Pins for the CPU oracle against facts the paper and the mathematics fix.

The paper prints no worked numeric example, so the oracle is pinned by
* brute force: Eq. LRI as a linear map, ERI = M_I V M_J^T (Eq. ERI_split), and
  Sigma = -ERI . D (Eq. HFX_ERIs) on tiny periodic cells;
* a special case that reduces to a library routine: a finite cluster is one
  dense numpy.einsum;
* Algorithm 1 == Algorithm 3: a slow <A,B>-loop form gives the same Sigma,
  key set and surviving-term counts at any theta;
* invariants: Sigma_IJ(R) = Sigma_JI(-R)^T, E_X = 1/2 sum D.Sigma, linearity in
  D and V, quadratic scaling in C, supercell folding (the k-mesh / supercell
  equivalence of Sec. IV), and the Cauchy-Schwarz-style screening bound.
"""
import math

import numpy as np
import pytest

import oracle
import refforms
import synth


def tiny(seed=5):
    s = synth.custom("tiny", 1.0, 4, [[0, 0, 0], [1, 1, 1]], [2, 3], [3, 4])
    return synth.make_workload(s, 3.5, 4.5, 3.5, seed=seed)


def tiny3(seed=6):
    """Three atoms, uneven sizes, a denser neighbourhood."""
    s = synth.custom("tiny3", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    return synth.make_workload(s, 3.2, 4.2, 3.0, seed=seed)


def scaled(wl, which, lam):
    import copy
    w = copy.copy(wl)
    b = getattr(wl, which)
    setattr(w, which, synth.Blocks(b.keys, b.data * lam, b.offs))
    return w


def as_dict(res, nao):
    return oracle.block_dict(res["keys"], res["data"], res["offs"], nao)


@pytest.mark.parametrize("make", [tiny, tiny3])
def test_brute_force_four_centre(make):
    """Theta = 0: oracle == -sum_{KL} (M_I V M_J^T) D_KL to 1e-12 relative."""
    wl = make()
    res = oracle.Oracle.of(wl).build(0.0)
    sig = as_dict(res, wl.system.nao)
    scale = max(np.abs(v).max() for v in sig.values())
    assert scale > 0.1
    for k, v in sig.items():
        b = refforms.brute_sigma(wl, k[0], (k[1], tuple(k[2:])))
        assert np.abs(b - v).max() <= 1e-12 * scale, k
    # sites just outside the key set receive nothing in the brute-force form either
    keys = set(sig)
    for k in list(sig)[:5]:
        for dn in ((3, 0, 0), (0, -3, 0)):
            kk = (k[0], k[1], k[2] + dn[0], k[3] + dn[1], k[4] + dn[2])
            if kk not in keys:
                b = refforms.brute_sigma(wl, kk[0], (kk[1], tuple(kk[2:])))
                assert np.abs(b).max() == 0.0


def test_finite_cluster_einsum():
    """A cluster with no periodic images in reach is a single dense einsum."""
    s = synth.custom("cluster", 1.0, 1000, [[0, 0, 0], [1, 1, 0], [2, 0, 1], [0, 2, 2]],
                     [2, 3, 2, 4], [3, 2, 4, 3])
    wl = synth.make_workload(s, 2.9, 3.5, 2.6, seed=9)
    res = oracle.Oracle.of(wl).build(0.0)
    sig = as_dict(res, s.nao)
    dense, ao = refforms.cluster_sigma(wl)
    scale = np.abs(dense).max()
    seen = np.zeros_like(dense, dtype=bool)
    for (i, j, *n), v in sig.items():
        assert tuple(n) == (0, 0, 0)
        blk = dense[ao[i]:ao[i + 1], ao[j]:ao[j + 1]]
        assert np.abs(blk - v).max() <= 1e-12 * scale
        seen[ao[i]:ao[i + 1], ao[j]:ao[j + 1]] = True
    assert np.all(dense[~seen] == 0.0)


def test_single_atom_onsite_is_one_term():
    """One atom alone: {I,K} = {I} so Sigma = -sum C V C D exactly once
    (a double-counted on-site piece would give 4x)."""
    s = synth.custom("atom", 1.0, 1000, [[0, 0, 0]], [3], [5])
    wl = synth.make_workload(s, 1.0, 1.0, 1.0, seed=3)
    res = oracle.Oracle.of(wl).build(0.0)
    C = wl.C.data.reshape(5, 3, 3)
    V = wl.V.data.reshape(5, 5)
    D = wl.D.data.reshape(3, 3)
    ref = -np.einsum("aik,ab,bjl,kl->ij", C, V, C, D)
    np.testing.assert_allclose(res["data"].reshape(3, 3), ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("make,theta", [(tiny, 0.0), (tiny, 3e-3), (tiny, 1e-2),
                                        (tiny3, 0.0), (tiny3, 2e-2)])
def test_algorithm1_equals_algorithm3(make, theta):
    """The <I,J> loop (oracle) and the <A,B> loop (Algorithm 3) give the same
    Sigma, the same key set and the same surviving terms per variant."""
    wl = make()
    res = oracle.Oracle.of(wl).build(theta)
    sig = as_dict(res, wl.system.nao)
    ab, counts, _ = refforms.ab_form(wl, theta)
    assert set(ab) == set(sig)
    np.testing.assert_array_equal(counts, res["counts"])
    scale = max(np.abs(v).max() for v in sig.values())
    for k in sig:
        assert np.abs(ab[k] - sig[k]).max() <= 1e-12 * scale


@pytest.mark.parametrize("theta", [0.0, 1e-2])
def test_hermiticity(theta):
    """V_AB = V_BA^T and D_KL(R) = D_LK(-R)^T give Sigma_IJ(R) = Sigma_JI(-R)^T,
    and the screen is symmetric, so the key set is closed under the mirror."""
    wl = tiny3()
    res = oracle.Oracle.of(wl).build(theta)
    sig = as_dict(res, wl.system.nao)
    for (i, j, a, b, c), v in sig.items():
        m = (j, i, -a, -b, -c)
        assert m in sig
        assert np.abs(sig[m].T - v).max() <= 1e-13 * max(1.0, np.abs(v).max())


def test_ex_identity():
    wl = tiny3()
    o = oracle.Oracle.of(wl)
    res = o.build(0.0)
    sig = as_dict(res, wl.system.nao)
    D = wl.D.as_dict()
    ex = 0.5 * sum(float(np.sum(D[k].reshape(v.shape) * v)) for k, v in sig.items() if k in D)
    assert math.isclose(ex, res["ex"], rel_tol=1e-13)
    assert res["ex"] != 0.0


def test_linear_in_D_and_V_quadratic_in_C():
    wl = tiny3()
    base = oracle.Oracle.of(wl).build(0.0)
    for which, lam, power in (("D", 2.0, 1), ("V", 3.0, 1), ("C", 1.5, 2)):
        r = oracle.Oracle.of(scaled(wl, which, lam)).build(0.0)
        np.testing.assert_array_equal(r["keys"], base["keys"])
        np.testing.assert_allclose(r["data"], base["data"] * lam ** power, rtol=1e-12,
                                   atol=1e-14 * np.abs(base["data"]).max())


@pytest.mark.parametrize("theta", [0.0, 1e-2])
def test_supercell_folding(theta):
    """A unit cell and its 2x2x2 supercell built from the same blocks give the
    same Sigma on every mapped key (the unit-cell / supercell equivalence);
    block norms are identical, so this holds with screening too."""
    wl = tiny()
    unit = as_dict(oracle.Oracle.of(wl).build(theta), wl.system.nao)
    sup, cells = refforms.supercell(wl, 2)
    big = as_dict(oracle.Oracle.of(sup).build(theta), sup.system.nao)
    nat = wl.system.natoms
    mapped = 0
    for (s1, s2, *N), v in big.items():
        c1, x = divmod(s1, nat)
        c2, y = divmod(s2, nat)
        n = tuple(cells[c2][k] - cells[c1][k] + 2 * N[k] for k in range(3))
        u = unit[(x, y) + n]
        assert np.abs(u - v).max() <= 1e-13 * max(1.0, np.abs(u).max())
        mapped += 1
    assert mapped == 8 * len(unit)


def test_screening_error_bound_and_monotone():
    """|Sigma(theta) - Sigma(0)| <= sum over dropped terms of (pA pB nK nL) S,
    elementwise per block, and the error falls as theta falls."""
    wl = tiny3()
    o = oracle.Oracle.of(wl)
    full = as_dict(o.build(0.0), wl.system.nao)
    errs = []
    for theta in (5e-2, 2e-2, 5e-3):
        scr = as_dict(o.build(theta), wl.system.nao)
        _, _, bound = refforms.ab_form(wl, theta)
        worst = 0.0
        for k, v in full.items():
            d = np.abs(v - scr.get(k, 0.0)).max()
            b = bound.get(k, 0.0)
            assert d <= b * (1 + 1e-12) + 1e-14, (k, d, b)
            worst = max(worst, d)
        errs.append(worst)
    assert errs[0] > errs[1] > errs[2] > 0.0


def test_threshold_is_strict():
    """A term with S exactly equal to theta is dropped (strict '>')."""
    wl = tiny()
    o = oracle.Oracle.of(wl)
    mc = {tuple(k): m for k, m in zip(wl.C.keys.tolist(), o.maxabs("C"))}
    mv = {tuple(k): m for k, m in zip(wl.V.keys.tolist(), o.maxabs("V"))}
    md = {tuple(k): m for k, m in zip(wl.D.keys.tolist(), o.maxabs("D"))}
    # the on-site term: A = F = B = G = atom 0 in the home cell, variant 1
    z = (0, 0, 0, 0, 0)
    s = (mc[z] * mc[z]) * (mv[z] * md[z])
    _, c_at = o.keys(np.nextafter(s, 0.0))
    _, c_above = o.keys(s)
    assert c_at[0] - c_above[0] >= 1
    # values: theta = S drops the term exactly as theta just above S does
    ref = o.blocks(np.nextafter(s, np.inf), [z])[0]
    np.testing.assert_array_equal(o.blocks(s, [z])[0], ref)
    assert np.abs(o.blocks(np.nextafter(s, 0.0), [z])[0] - ref).max() > 0.0


def test_block_maxabs():
    wl = tiny3()
    o = oracle.Oracle.of(wl)
    for which in "CVD":
        b = getattr(wl, which)
        ref = [np.abs(b.data[b.offs[e]:b.offs[e + 1]]).max() for e in range(b.count)]
        np.testing.assert_array_equal(o.maxabs(which), ref)


def test_frozen_screen_for_finite_differences():
    """With the unperturbed block norms frozen, E_X is exactly linear in V and
    quadratic in C, so central differences of any step reproduce each other
    (the property the gradient tests rely on)."""
    wl = tiny3()
    o0 = oracle.Oracle.of(wl)
    norms = {k: o0.maxabs(k) for k in "CVD"}
    theta = 2e-2

    def ex_with(which, idx, delta):
        b = getattr(wl, which)
        d = b.data.copy()
        d[idx] += delta
        w = scaled(wl, which, 1.0)
        setattr(w, which, synth.Blocks(b.keys, d, b.offs))
        o = oracle.Oracle.of(w)
        for k in "CVD":
            o.set_maxabs(k, norms[k])
        return o.build(theta)["ex"]

    for which, idx in (("V", 7), ("C", 11)):
        g1 = (ex_with(which, idx, 1e-3) - ex_with(which, idx, -1e-3)) / 2e-3
        g2 = (ex_with(which, idx, 0.25) - ex_with(which, idx, -0.25)) / 0.5
        assert abs(g1 - g2) <= 1e-9 * max(1.0, abs(g1))
