"""GPU parity on the 512-atom Si-like supercell (4x4x4 diamond, 13 NAOs / 60
ABFs per atom, theta = 1e-6): the benchmark's workload, built through the C
ABI in the 6-digit split precision and in FP64, against the CPU oracle.

* The Sigma key set and the surviving-term counts per piece equal the
  oracle's exactly, in both modes.
* Sampled blocks (on-site and random, around three central atoms spread over
  the cell) are within 1e-8 Ha of the oracle's in split mode and 1e-10 Ha in
  FP64 mode.
* Every block of the split build is within 1e-8 Ha of the FP64 build; |dE_X|
  per atom is printed and bounded by the same bar."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import as_dict, gpu_build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA = 1e-6
TOL_SPLIT, TOL_FP64 = 1e-8, 1e-10


@pytest.fixture(scope="module")
def si512():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.si512()
    o = oracle.Oracle.of(wl)
    keys, counts = o.keys(THETA)
    ctx, split = gpu_build(wl, THETA, "ozaki", 6)
    _, fp64 = gpu_build(wl, THETA, "fp64", 0, ctx=ctx)
    return wl, o, keys, counts, split, fp64


def test_si512_keys_and_counts(si512):
    wl, o, keys, counts, split, fp64 = si512
    for g in (split, fp64):
        np.testing.assert_array_equal(g["keys"], keys)
        np.testing.assert_array_equal(np.array(g["stats"]["survivors"]), counts)


def test_si512_sampled_blocks(si512):
    wl, o, keys, counts, split, fp64 = si512
    rng = np.random.default_rng(512)
    sample = []
    for a in (0, 255, 511):
        mine = np.flatnonzero(keys[:, 0] == a)
        onsite = [int(e) for e in mine if keys[e, 1] == a and not keys[e, 2:].any()]
        sample += onsite + [int(e) for e in rng.choice(mine, 6, replace=False)]
    sample += [int(e) for e in rng.choice(len(keys), 6, replace=False)]
    sel = keys[sorted(set(sample))]
    ref, roffs = o.blocks(THETA, sel)
    ds, df = as_dict(split, wl.system.nao), as_dict(fp64, wl.system.nao)
    es = ef = 0.0
    for e, k in enumerate(sel.tolist()):
        r = ref[roffs[e]:roffs[e + 1]]
        es = max(es, float(np.abs(ds[tuple(k)].ravel() - r).max()))
        ef = max(ef, float(np.abs(df[tuple(k)].ravel() - r).max()))
    print(f"{len(sel)} blocks: split max|dSigma| = {es:.3e}, fp64 max|dSigma| = {ef:.3e}")
    assert es <= TOL_SPLIT, es
    assert ef <= TOL_FP64, ef


def test_si512_split_vs_fp64_every_block(si512):
    wl, o, keys, counts, split, fp64 = si512
    err = float(np.abs(split["data"] - fp64["data"]).max())
    dex = abs(split["ex"] - fp64["ex"]) / wl.system.natoms
    print(f"split vs fp64: max|dSigma| = {err:.3e} Ha, |dE_X| per atom = {dex:.3e} Ha")
    assert err <= TOL_SPLIT, err
    assert dex <= TOL_SPLIT, dex
