"""The sharded build through the library with two real processes: two gloo
ranks on one GPU, each calling sharding.build_sharded (its own central atoms'
terms by machine scheduling or K-means, then one 64-bit integer all-reduce
of the fixed-point Sigma over gloo), must give Sigma and E_X bitwise equal to
the unsharded build.  The ranks' kernels never wait on one another: each rank
runs its own builds, and the only exchange is the host-side all-reduce."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA = 1e-3


def _rank(rank, world, port, prec, scheme, out):
    import torch
    import torch.distributed as dist

    import paper_2009_12505_gb300 as hfx
    import synth
    from paper_2009_12505_gb300 import sharding
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    torch.cuda.set_device(0)
    wl = synth.ab_shrunk()
    ctx = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    ex = sharding.build_sharded(ctx, wl.C.keys, wl.V.keys, THETA, prec, group=None,
                                scheme=scheme, positions=wl.system.positions)
    np.save(os.path.join(out, f"sigma{rank}.npy"), ctx.sigma())
    np.save(os.path.join(out, f"ex{rank}.npy"), np.array([ex]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec,scheme", [("fp64", "lpt"), ("ozaki", "kmeans")])
def test_two_gloo_ranks_bitwise(tmp_path, prec, scheme):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp

    import paper_2009_12505_gb300 as hfx
    import synth
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx_mp = mp.get_context("spawn")
    procs = [ctx_mp.Process(target=_rank, args=(r, 2, port, prec, scheme, str(tmp_path)))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    wl = synth.ab_shrunk()
    ctx = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    ex = ctx.build(THETA, prec)
    full = ctx.sigma()
    for r in range(2):
        np.testing.assert_array_equal(np.load(os.path.join(tmp_path, f"sigma{r}.npy")), full)
        assert float(np.load(os.path.join(tmp_path, f"ex{r}.npy"))[0]) == ex
