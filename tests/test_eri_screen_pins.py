"""Pins for the C oracle's Cauchy-Schwarz ERI screen (Sec. III.C, Eq. CS-ERI;
oracle/hfx_oracle.c orc_set_eri), which the GPU screen is checked against.

* Its per-C-block sqrt(max(Q, 0)) equals the numpy restatement in
  oracle/multilevel.py, whose Q is itself pinned to the largest diagonal of
  M V M^T from the brute-force LRI map (test_multilevel_pins.py).
* With the screen on, its Sigma and key set equal multilevel.build at element
  threshold 0 (only the block and ERI screens act) for several eps_eri; a
  negative eps_eri is the plain build; more quadruples go as eps_eri grows."""
import numpy as np
import pytest

import oracle
import synth
from oracle import multilevel


def _pair():
    s = synth.custom("pair", 1.0, 5, [[0, 0, 0], [2, 1, 1]], [2, 3], [3, 4])
    return synth.make_workload(s, 3.2, 4.5, 3.2, seed=9)


def _three():
    s = synth.custom("three", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    return synth.make_workload(s, 3.2, 4.2, 3.0, seed=6)


@pytest.mark.parametrize("make", [_pair, _three])
def test_eri_bounds_match_the_numpy_restatement(make):
    wl = make()
    o = oracle.Oracle.of(wl)
    o.set_eri(0.0)
    got = o.eri_sq()
    q = multilevel.diag_eri_max(wl)
    ref = np.array([np.sqrt(max(q[tuple(int(x) for x in k)], 0.0)) for k in wl.C.keys])
    assert (ref > 0).any()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    o.set_eri(None)
    assert not o.eri_sq().any()


def _flat(sig, keys):
    return np.concatenate([np.ravel(sig.get(tuple(int(x) for x in k), 0.0)) for k in keys])


@pytest.mark.parametrize("make", [_pair, _three])
def test_eri_screened_build_matches_multilevel(make):
    wl = make()
    o = oracle.Oracle.of(wl)
    o.set_eri(0.0)
    sq = o.eri_sq()
    # thresholds halfway between distinct bound products (a threshold equal to
    # a product would let the last rounding bit decide)
    prods = np.unique(np.outer(sq, sq).ravel())
    mids = (prods[1:] + prods[:-1]) / 2
    grid = [0.0] + [float(mids[int(f * (len(mids) - 1))]) for f in (0.25, 0.5, 0.75)]
    sizes = []
    for theta in (0.0, 1e-2):
        for eps in grid:
            o.set_eri(eps)
            got = o.build(theta)
            ref, stats = multilevel.build(wl, theta, 0.0, eps_eri=eps)
            assert {tuple(k) for k in got["keys"].tolist()} == set(ref)
            flat = _flat(ref, got["keys"])
            scale = max(np.abs(flat).max(), 1.0) if flat.size else 1.0
            assert np.abs(got["data"] - flat).max(initial=0.0) <= 1e-12 * scale
            sizes.append(int(got["counts"].sum()))
    # within each theta, fewer terms survive as eps_eri grows, and some go
    for t in range(2):
        run = sizes[4 * t:4 * t + 4]
        assert run == sorted(run, reverse=True) and run[-1] < run[0]


def test_negative_eps_is_the_plain_build():
    wl = _three()
    o = oracle.Oracle.of(wl)
    plain = o.build(1e-3)
    o.set_eri(-1.0)
    got = o.build(1e-3)
    np.testing.assert_array_equal(got["keys"], plain["keys"])
    np.testing.assert_array_equal(got["data"], plain["data"])
