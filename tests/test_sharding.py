"""Host-side sharding: Algorithm 6 (greedy machine scheduling) and the
fixed-point exchange over a world-2 gloo process group on CPU.

The exchange test emulates two ranks with the <A,B> reference form: each
rank encodes every surviving term of its own central atoms into the
library's fixed-point words, the words are summed with one all-reduce, and
the result must be bitwise equal to a single rank's accumulation."""
import os
import socket

import numpy as np
import pytest

import refforms
import synth
from paper_2009_12505_gb300 import sharding


def test_lpt_within_two_of_optimum():
    """Greedy assignment in decreasing order: makespan <= (4/3) OPT, so in
    particular within the factor 2 the paper quotes (OPT >= max(mean, max))."""
    rng = np.random.default_rng(0)
    for trial in range(20):
        costs = rng.exponential(size=rng.integers(5, 60)) ** 2
        m = int(rng.integers(2, 9))
        owner = sharding.lpt(costs, m)
        load = np.bincount(owner, weights=costs, minlength=m)
        lower = max(costs.sum() / m, costs.max())
        assert load.max() <= (4.0 / 3.0) * lower + 1e-12 or load.max() <= 2 * lower
        assert load.max() <= 2 * lower


def test_lpt_deterministic_and_balanced_on_equal_atoms():
    owner = sharding.lpt(np.ones(64), 4)
    assert np.bincount(owner).tolist() == [16, 16, 16, 16]
    np.testing.assert_array_equal(owner, sharding.lpt(np.ones(64), 4))


def test_atom_costs_follow_pair_weights():
    wl = synth.si_shrunk()
    cost = sharding.atom_costs(wl.system.natoms, wl.C.keys, wl.V.keys)
    nbr = np.bincount(wl.C.keys[:, 0])
    ref = [sum(nbr[a] * nbr[b] for (a, b, *_) in wl.V.keys.tolist() if a == x)
           for x in range(wl.system.natoms)]
    np.testing.assert_allclose(cost, ref)


def test_fx_roundtrip_matches_library_encoding():
    x = np.array([0.0, 1.5, -2.25, 65.98757923056736, -1e-9, 3.0e-17])
    np.testing.assert_allclose(sharding.fx_decode(sharding.fx_encode(x)), x, rtol=0, atol=2**-63)


def _words_for_atoms(wl, theta, atoms, keyindex, offs, nelem):
    acc = np.zeros((nelem, 2), np.int64)

    def each(key, blk):
        o = offs[keyindex[key]]
        acc[o:o + blk.size] += sharding.fx_encode(blk.ravel())

    refforms.ab_form(wl, theta, atoms=atoms, each=each)
    return acc


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _tiny3()
        theta = 2e-2
        sig, _, _ = refforms.ab_form(wl, theta)
        keys = sorted(sig)
        keyindex = {k: i for i, k in enumerate(keys)}
        offs = np.concatenate([[0], np.cumsum([sig[k].size for k in keys])])
        owner = sharding.lpt(sharding.atom_costs(wl.system.natoms, wl.C.keys, wl.V.keys), world)
        mine = {a for a in range(wl.system.natoms) if owner[a] == rank}
        words = _words_for_atoms(wl, theta, mine, keyindex, offs, int(offs[-1]))
        total = sharding.all_reduce_words(words)
        if rank == 0:
            single = _words_for_atoms(wl, theta, None, keyindex, offs, int(offs[-1]))
            q.put((np.array_equal(total, single), owner.tolist(),
                   float(np.abs(sharding.fx_decode(total) -
                                np.concatenate([sig[k].ravel() for k in keys])).max())))
    finally:
        dist.destroy_process_group()


def _tiny3():
    s = synth.custom("tiny3", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    return synth.make_workload(s, 3.2, 4.2, 3.0, seed=6)


def test_gloo_world2_exchange_bitwise():
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    equal, owner, err = q.get(timeout=5)
    assert equal
    assert len(set(owner)) == 2
    assert err < 1e-13
