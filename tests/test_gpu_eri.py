"""GPU parity of the Cauchy-Schwarz ERI screen (Sec. III.C, Eq. CS-ERI;
hfx_set_eri_screen) against the CPU oracle with the same screen on:

* exact Sigma key set and surviving-term counts, max |dSigma| <= 1e-10 Ha in
  FP64 and <= 1e-8 Ha in the 6-digit split precision, on the shrunk Si-like
  and two-element cells at thresholds that remove a good share of the terms;
* the number of removed quadruples equals the <A,B>-form oracle's
  (oracle/multilevel.py) on a small cell;
* a negative threshold turns the screen off (bitwise the plain build)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare_full, gpu_build
from oracle import multilevel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def eps_between(sq, q):
    """A threshold at quantile q of the pairwise bound products, halfway in
    the widest relative gap nearby (no product within rounding of it)."""
    p = np.unique(np.outer(sq, sq).ravel())
    p = p[p > 0]
    i0 = int(q * (len(p) - 1))
    lo, hi = max(i0 - 20, 0), min(i0 + 20, len(p) - 1)
    gaps = p[lo + 1:hi + 1] / p[lo:hi]
    j = lo + int(np.argmax(gaps))
    assert gaps.max() > 1 + 1e-6
    return float(np.sqrt(p[j] * p[j + 1]))


def _with_eri(wl, theta, eps, prec, nslices):
    ctx = None
    import paper_2009_12505_gb300 as hfx
    ctx = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    ctx.set_eri_screen(eps)
    return gpu_build(wl, theta, prec, nslices, ctx=ctx)


@pytest.mark.parametrize("make,theta", [(synth.si_shrunk, 0.0), (synth.si_shrunk, 1e-3),
                                        (synth.ab_shrunk, 1e-3)])
@pytest.mark.parametrize("q", [0.3, 0.6])
def test_eri_screen_matches_oracle(make, theta, q):
    wl = make()
    o = oracle.Oracle.of(wl)
    plain_counts = o.keys(theta)[1]
    o.set_eri(0.0)
    eps = eps_between(o.eri_sq(), q)
    o.set_eri(eps)
    ref = o.build(theta)
    assert ref["counts"].sum() < plain_counts.sum()      # the screen removes terms
    for prec, nsl, tol in (("fp64", 0, 1e-10), ("ozaki", 6, 1e-8)):
        _, g = _with_eri(wl, theta, eps, prec, nsl)
        assert g["stats"]["eps_eri"] == eps and g["stats"]["n_eri_removed"] > 0
        err = compare_full(wl, theta, g, ref, tol)
        print(f"{wl.name} theta={theta} eps_eri={eps:.4g} {prec}: "
              f"{ref['counts'].sum()} of {plain_counts.sum()} terms, max|dSigma| = {err:.2e}")


def test_removed_quadruples_match_the_ab_form():
    s = synth.custom("three", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    wl = synth.make_workload(s, 3.2, 4.2, 3.0, seed=6)
    o = oracle.Oracle.of(wl)
    o.set_eri(0.0)
    eps = eps_between(o.eri_sq(), 0.5)
    _, stats = multilevel.build(wl, 0.0, 0.0, eps_eri=eps)
    _, g = _with_eri(wl, 0.0, eps, "fp64", 0)
    assert g["stats"]["n_eri_removed"] == int(stats[4]) > 0


def test_negative_eps_is_the_plain_build():
    wl = synth.si_shrunk()
    _, plain = gpu_build(wl, 1e-3)
    _, off = _with_eri(wl, 1e-3, -1.0, "fp64", 0)
    np.testing.assert_array_equal(plain["keys"], off["keys"])
    np.testing.assert_array_equal(plain["data"], off["data"])
    assert off["stats"]["n_eri_removed"] == 0
