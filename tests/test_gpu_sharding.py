"""Sharded builds on one GPU as host-emulated ranks: each rank contracts its
LPT-assigned central atoms, the fixed-point accumulators are summed as 64-bit
integers, and Sigma / E_X must be bitwise equal to the unsharded build."""
import numpy as np
import pytest

import synth
from paper_2009_12505_gb300 import sharding

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_build_bitwise(prec, world):
    import paper_2009_12505_gb300 as hfx
    wl = synth.ab_shrunk()
    theta = 1e-3
    ctx = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    ex_full = ctx.build(theta, prec)
    full = ctx.sigma()
    words_full = ctx.sigma_fixed()
    owner = sharding.lpt(sharding.atom_costs(wl.system.natoms, wl.C.keys, wl.V.keys), world)
    total = np.zeros_like(words_full)
    for r in range(world):
        ctx.set_shard(owner, r)
        ctx.build(theta, prec)
        total += ctx.sigma_fixed()
    np.testing.assert_array_equal(total, words_full)
    ex = ctx.set_sigma_fixed(total)
    np.testing.assert_array_equal(ctx.sigma(), full)
    assert ex == ex_full
    ctx.set_shard(None, 0)
