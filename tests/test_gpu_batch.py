"""hfx_build_batch as one merged build: cells of uneven size (13/60 and 27/90
atoms, small clusters) with their own thresholds are built together -- one
screen launch and one launch per persistent kernel per wave for all cells --
and every cell must get exactly (bitwise) the Sigma blocks, fixed-point words
and E_X of its own hfx_build.  One cell is also checked against the oracle,
and the calls that need a cell's own build refuse batch results."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def tiny3(seed):
    s = synth.custom("tiny3", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    return synth.make_workload(s, 3.2, 4.2, 3.0, seed=seed)


def _cells(prec):
    cells = [(synth.si_shrunk(seed=11), 1e-3), (synth.ab_shrunk(seed=12), 1e-5),
             (synth.si_shrunk(seed=21), 0.0), (synth.ab_shrunk(seed=22), 1e-6)]
    if prec == "fp64":
        cells += [(tiny3(6), 2e-2), (tiny3(7), 0.0)]
    return cells


@pytest.mark.parametrize("prec,nsl", [("fp64", 0), ("ozaki", 6)])
def test_batch_bitwise_equals_separate_builds(prec, nsl):
    import paper_2009_12505_gb300 as hfx
    cells = _cells(prec)
    ctxs, sep = [], []
    for wl, th in cells:
        c, g = gpu_build(wl, th, prec, nsl)
        g["fixed"] = c.sigma_fixed()
        sep.append(g)
        ctxs.append(c)
    ex = hfx.build_batch(ctxs, [th for _, th in cells], prec, nsl)
    for c, g, e in zip(ctxs, sep, ex):
        np.testing.assert_array_equal(c.keys(), g["keys"])
        np.testing.assert_array_equal(c.offsets(), g["offs"])
        np.testing.assert_array_equal(c.sigma(), g["data"])
        np.testing.assert_array_equal(c.sigma_fixed(), g["fixed"])
        assert e == g["ex"]
    # one launch of each persistent kernel per wave serves every cell
    st = ctxs[0].stats()
    assert st["n_work_items"] == sum(len(wl.V.keys) for wl, _ in cells)


def test_batch_cell_matches_oracle_and_refuses_grad():
    import paper_2009_12505_gb300 as hfx
    wl_a, wl_b = synth.si_shrunk(seed=11), synth.ab_shrunk(seed=12)
    ctxs = []
    for wl in (wl_a, wl_b):
        c = hfx.Context(wl.system.nao, wl.system.nabf)
        for k in "CVD":
            c.set_blocks(k, getattr(wl, k))
        ctxs.append(c)
    ex = hfx.build_batch(ctxs, [1e-3, 1e-3], "ozaki", 6)
    ref = oracle.Oracle.of(wl_a).build(1e-3)
    np.testing.assert_array_equal(ctxs[0].keys(), ref["keys"])
    assert float(np.abs(ctxs[0].sigma() - ref["data"]).max()) <= 1e-8
    assert abs(ex[0] - ref["ex"]) <= 1e-8 * wl_a.system.natoms
    with pytest.raises(hfx.HfxError) as e:
        ctxs[0].grad(wl_a.C.data.size, wl_a.V.data.size)
    assert e.value.status == 3
    ctxs[0].build(1e-3, "fp64")          # a build of the cell alone
    dC, dV = ctxs[0].grad(wl_a.C.data.size, wl_a.V.data.size)
    assert np.isfinite(dC).all() and np.isfinite(dV).all()


def test_batch_argument_errors():
    import paper_2009_12505_gb300 as hfx
    wl = synth.si_shrunk()
    c = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        c.set_blocks(k, getattr(wl, k))
    with pytest.raises(hfx.HfxError) as e:
        hfx.build_batch([c, c], [1e-3, 1e-3], "fp64")
    assert e.value.status == 1
    with pytest.raises(hfx.HfxError) as e:
        hfx.build_batch([c], [-1.0], "fp64")
    assert e.value.status == 1


def test_batch_reuses_its_merged_system_and_follows_new_d():
    """A second batch of the same cells reuses the merged system; after one
    cell's D values change, the next batch copies them in and still equals a
    build of that cell alone with the new D, bitwise."""
    import paper_2009_12505_gb300 as hfx
    wls = [synth.si_shrunk(seed=11), synth.ab_shrunk(seed=12)]
    thetas = [1e-3, 1e-5]
    ctxs = []
    for wl in wls:
        c = hfx.Context(wl.system.nao, wl.system.nabf)
        for k in "CVD":
            c.set_blocks(k, getattr(wl, k))
        ctxs.append(c)
    hfx.build_batch(ctxs, thetas, "ozaki", 6)
    first = [c.sigma() for c in ctxs]
    ex2 = hfx.build_batch(ctxs, thetas, "ozaki", 6)      # the cached plan
    for c, f in zip(ctxs, first):
        np.testing.assert_array_equal(c.sigma(), f)
    # new D values for cell 1 (same keys; a common scale keeps D Hermitian)
    d_new = synth.Blocks(wls[1].D.keys, wls[1].D.data * 1.5, wls[1].D.offs)
    ctxs[1].set_blocks("D", d_new)
    ex3 = hfx.build_batch(ctxs, thetas, "ozaki", 6)
    wl_new = synth.Workload(wls[1].name, wls[1].system, wls[1].C, wls[1].V, d_new,
                            wls[1].cut_C, wls[1].cut_V, wls[1].cut_D, wls[1].seed)
    _, alone = gpu_build(wl_new, thetas[1], "ozaki", 6)
    np.testing.assert_array_equal(ctxs[1].keys(), alone["keys"])
    np.testing.assert_array_equal(ctxs[1].sigma(), alone["data"])
    assert ex3[1] == alone["ex"] and ex3[0] == ex2[0]
    np.testing.assert_array_equal(ctxs[0].sigma(), first[0])
