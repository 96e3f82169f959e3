"""GPU parity on the second workload, whose tasks are denser for the same
kernels: an 8-atom Si-like cell with full-range Coulomb V out to 50 bohr (the
range Hartree-Fock needs, Sec. IV) and one with a metallic, polynomially
decaying D out to 24 bohr (Sec. III.B).  Full-size cells at theta = 1e-6,
through the C ABI:

* exact Sigma key set and surviving-term counts against the oracle, in the
  6-digit split precision and in FP64;
* sampled blocks within 1e-8 Ha (split) and 1e-10 Ha (FP64) of the oracle;
* every split block within 1e-8 Ha of the FP64 build."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import as_dict, gpu_build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("make", [synth.si8_fullrange, synth.si8_metal])
def test_second_workload(make):
    wl = make()
    o = oracle.Oracle.of(wl)
    keys, counts = o.keys(THETA)
    ctx, split = gpu_build(wl, THETA, "ozaki", 6)
    _, fp64 = gpu_build(wl, THETA, "fp64", 0, ctx=ctx)
    for g in (split, fp64):
        np.testing.assert_array_equal(g["keys"], keys)
        np.testing.assert_array_equal(np.array(g["stats"]["survivors"]), counts)
    rng = np.random.default_rng(7)
    onsite = [e for e in range(len(keys)) if keys[e, 0] == keys[e, 1] and not keys[e, 2:].any()]
    sel = keys[sorted(set(onsite[:2] + [int(e) for e in rng.choice(len(keys), 10, replace=False)]))]
    ref, roffs = o.blocks(THETA, sel)
    ds, df = as_dict(split, wl.system.nao), as_dict(fp64, wl.system.nao)
    es = ef = 0.0
    for e, k in enumerate(sel.tolist()):
        r = ref[roffs[e]:roffs[e + 1]]
        es = max(es, float(np.abs(ds[tuple(k)].ravel() - r).max()))
        ef = max(ef, float(np.abs(df[tuple(k)].ravel() - r).max()))
    every = float(np.abs(split["data"] - fp64["data"]).max())
    print(f"{wl.name}: {split['stats']['canonical_flops'] / 1e12:.2f} TFLOP; sampled split "
          f"{es:.2e}, fp64 {ef:.2e}; split vs fp64 {every:.2e}")
    assert es <= 1e-8 and ef <= 1e-10 and every <= 1e-8, (es, ef, every)
