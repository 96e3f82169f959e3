"""GPU parity of the FP64 build against the CPU oracle (through the C ABI).

Bar: identical Sigma key set, identical surviving-term counts per variant,
max |dSigma| <= 1e-10 Ha and |dE_X| <= 1e-10 Ha per atom (FP64 mode)."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_common import as_dict, compare_full, gpu_build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def tiny():
    s = synth.custom("tiny", 1.0, 4, [[0, 0, 0], [1, 1, 1]], [2, 3], [3, 4])
    return synth.make_workload(s, 3.5, 4.5, 3.5, seed=5)


def tiny3():
    s = synth.custom("tiny3", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    return synth.make_workload(s, 3.2, 4.2, 3.0, seed=6)


@pytest.mark.parametrize("make,theta", [(tiny, 0.0), (tiny, 3e-3), (tiny3, 0.0), (tiny3, 2e-2)])
def test_tiny_full(make, theta):
    wl = make()
    ref = oracle.Oracle.of(wl).build(theta)
    _, g = gpu_build(wl, theta)
    compare_full(wl, theta, g, ref, TOL)
    assert abs(g["ex"] - ref["ex"]) <= TOL * wl.system.natoms


@pytest.mark.parametrize("theta", [0.0, 1e-2])
@pytest.mark.parametrize("mirror", ["1", "0"])
def test_si_shrunk_full(theta, mirror, monkeypatch):
    """8-atom Si-like cell, full 13/60 blocks, short cutoffs: several tiles,
    ragged 13-wide blocks, all four variants; with and without the mirror
    pieces (Hermitian inputs)."""
    monkeypatch.setenv("HFX_NO_MIRROR", "0" if mirror == "1" else "1")
    wl = synth.si_shrunk()
    ref = oracle.Oracle.of(wl).build(theta)
    _, g = gpu_build(wl, theta)
    assert g["stats"]["mirror"] == int(mirror)
    compare_full(wl, theta, g, ref, TOL)
    assert abs(g["ex"] - ref["ex"]) <= TOL * wl.system.natoms


def test_non_hermitian_input_uses_full_sum():
    """A V block whose mirror is not its transpose disables the mirror
    pieces; the result still equals the oracle's (which needs no symmetry)."""
    wl = synth.ab_shrunk()
    V = dict(wl.V.as_dict())
    k = next(k for k in V if k[0] != k[1])
    V[k] = V[k] * 1.25
    wl2 = synth.Workload("t", wl.system, wl.C, synth.pack(V), wl.D, 0, 0, 0, 0)
    ref = oracle.Oracle.of(wl2).build(1e-3)
    _, g = gpu_build(wl2, 1e-3)
    assert g["stats"]["mirror"] == 0
    compare_full(wl2, 1e-3, g, ref, TOL)


def test_two_element_shrunk_full():
    """Uneven 13/60 and 27/90 atoms."""
    wl = synth.ab_shrunk()
    theta = 1e-3
    ref = oracle.Oracle.of(wl).build(theta)
    _, g = gpu_build(wl, theta)
    compare_full(wl, theta, g, ref, TOL)


def _sample_keys(keys, n, seed):
    rng = np.random.default_rng(seed)
    onsite = [k for k in keys.tolist() if k[0] == k[1] and k[2:] == [0, 0, 0]][:2]
    pick = rng.choice(len(keys), size=min(n, len(keys)), replace=False)
    return np.array(onsite + [keys[p].tolist() for p in sorted(pick)], np.int32)


@pytest.mark.parametrize("theta", [1e-6, 0.0])
def test_si8_full_size_sampled(theta):
    """The 8-atom Si-like cell at full size (123 C / 275 V / 123 D blocks per
    atom): exact key set and counts at any size, values on sampled blocks."""
    wl = synth.si8()
    o = oracle.Oracle.of(wl)
    keys, counts = o.keys(theta)
    _, g = gpu_build(wl, theta)
    np.testing.assert_array_equal(g["keys"], keys)
    np.testing.assert_array_equal(np.array(g["stats"]["survivors"]), counts)
    sample = _sample_keys(keys, 10, 7)
    ref, roffs = o.blocks(theta, sample)
    gd = as_dict(g, wl.system.nao)
    for e, k in enumerate(sample.tolist()):
        blk = gd[tuple(k)].ravel()
        err = np.abs(blk - ref[roffs[e]:roffs[e + 1]]).max()
        assert err <= TOL, (k, err)


def test_deterministic_and_wave_invariant(monkeypatch):
    """Bitwise identical across runs and across wave partitions of the work."""
    wl = synth.si_shrunk()
    _, a = gpu_build(wl, 1e-3)
    _, b = gpu_build(wl, 1e-3)
    np.testing.assert_array_equal(a["data"], b["data"])
    assert a["ex"] == b["ex"]
    monkeypatch.setenv("HFX_SCRATCH_MB", "16")
    _, c = gpu_build(wl, 1e-3)
    assert c["stats"]["n_waves"] > 1
    np.testing.assert_array_equal(a["data"], c["data"])


def test_hermitian():
    wl = synth.ab_shrunk()
    _, g = gpu_build(wl, 1e-4)
    d = as_dict(g, wl.system.nao)
    for (i, j, a, b, c), v in d.items():
        np.testing.assert_allclose(d[(j, i, -a, -b, -c)].T, v, rtol=0, atol=1e-12)


def test_input_paths_agree():
    """Bulk host, bulk device (torch tensor) and per-block sets give one result."""
    import paper_2009_12505_gb300 as hfx
    wl = tiny3()
    _, ref = gpu_build(wl, 0.0)
    c = hfx.Context(wl.system.nao, wl.system.nabf,
                    stream=torch.cuda.current_stream().cuda_stream)
    c.set_blocks("C", wl.C)
    vt = torch.from_numpy(wl.V.data).cuda()
    c.set_many("V", wl.V.keys, vt, wl.V.offs, on_device=True)
    for e, k in enumerate(wl.D.keys.tolist()):
        c.set_block("D", k[0], k[1], k[2:], wl.D.data[wl.D.offs[e]:wl.D.offs[e + 1]])
    ex = c.build(0.0)
    np.testing.assert_array_equal(c.sigma(), ref["data"])
    assert ex == ref["ex"]
    # device output
    out = torch.zeros(int(c.offsets()[-1]), dtype=torch.float64, device="cuda")
    c.sigma(out, on_device=True)
    np.testing.assert_array_equal(out.cpu().numpy(), ref["data"])


def test_replacing_a_block_and_results_staleness():
    import paper_2009_12505_gb300 as hfx
    wl = tiny()
    c, g0 = gpu_build(wl, 0.0)
    k = wl.D.keys[0].tolist()
    c.set_block("D", k[0], k[1], k[2:], 2.0 * wl.D.data[wl.D.offs[0]:wl.D.offs[1]])
    with pytest.raises(hfx.HfxError) as e:
        c.count()
    assert e.value.status == 3  # HFX_E_STATE
    c.build(0.0)
    d = dict(wl.D.as_dict())
    d[tuple(k)] = 2.0 * d[tuple(k)]
    wl2 = synth.Workload("t", wl.system, wl.C, wl.V, synth.pack(d), 0, 0, 0, 0)
    ref = oracle.Oracle.of(wl2).build(0.0)
    np.testing.assert_array_equal(c.keys(), ref["keys"])
    assert np.abs(c.sigma() - ref["data"]).max() <= TOL


def test_error_paths():
    import paper_2009_12505_gb300 as hfx
    wl = tiny()
    c = hfx.Context(wl.system.nao, wl.system.nabf)
    with pytest.raises(hfx.HfxError) as e:
        c.build(0.0)
    assert e.value.status == 3  # nothing set
    with pytest.raises(hfx.HfxError) as e:   # block sizes do not match nao/nabf
        c.set_many("C", wl.C.keys[1:], wl.C.data, wl.C.offs[:-1])
    assert e.value.status == 2
    with pytest.raises(hfx.HfxError) as e:
        c.set_block("C", 0, 0, [0, 0, 0], np.zeros(5))
    assert e.value.status == 2
    with pytest.raises(hfx.HfxError) as e:
        c.set_block("V", 5, 0, [0, 0, 0], np.zeros(12))
    assert e.value.status == 1
    with pytest.raises(hfx.HfxError) as e:   # lattice vector out of range (C ABI check)
        c.set_block("D", 0, 0, [300, 0, 0], np.zeros(4))
    assert e.value.status == 1
    bad = wl.D.data.copy()
    bad[3] = np.nan
    for k in "CV":
        c.set_blocks(k, getattr(wl, k))
    c.set_many("D", wl.D.keys, bad, wl.D.offs)
    with pytest.raises(hfx.HfxError) as e:
        c.build(0.0)
    assert e.value.status == 1
    c.set_blocks("D", wl.D)
    c.build(0.0)
    with pytest.raises(hfx.HfxError) as e:
        c.get(0, 1, [50, 0, 0])
    assert e.value.status == 7
    # a threshold above every S: no surviving term, empty key set, E_X = 0
    assert c.build(1e30) == 0.0
    assert c.count() == 0


@pytest.mark.parametrize("make,theta", [(synth.si_shrunk, 1e-2), (synth.si8, 1e-6)])
def test_flop_accounting_matches_oracle(make, theta):
    """The library's canonical flop count and active (A,B,G) count equal the
    oracle's, which equals Table 1 per quadruple (test_flop_accounting)."""
    wl = make()
    _, _, extra = oracle.Oracle.of(wl).keys(theta, extra=True)
    _, g = gpu_build(wl, theta)
    assert g["stats"]["canonical_flops"] == extra["canonical_flops"]
    assert g["stats"]["n_active_abg"] == extra["active_abg"]
