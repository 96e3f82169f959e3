"""Sharding the exchange build over ranks (one GPU per rank).

Pairs <A,B> are distributed by their central atom A (Sec. III.D); atoms
are balanced with the greedy machine-scheduling rule of Algorithm 6: every
pair carries the work estimate |N[A]| |N[B]| (neighbour counts from the C
keys), atoms are taken in decreasing order of their pairs' total and each
goes to the least-loaded rank.

Every rank screens globally and contracts its own atoms' pairs into the
128-bit fixed-point Sigma accumulators; the one exchange step is an
elementwise 64-bit integer sum of those accumulators across ranks, which is
exact and order-independent, so the combined Sigma and E_X are bitwise
identical to a single-rank build.
"""
from __future__ import annotations

import numpy as np


def atom_costs(natoms: int, c_keys, v_keys) -> np.ndarray:
    """Per central atom: sum over its V pairs <A,B> of |N[A]| |N[B]|."""
    c_keys = np.asarray(c_keys).reshape(-1, 5)
    v_keys = np.asarray(v_keys).reshape(-1, 5)
    nbr = np.bincount(c_keys[:, 0], minlength=natoms).astype(np.float64)
    cost = np.zeros(natoms, np.float64)
    np.add.at(cost, v_keys[:, 0], nbr[v_keys[:, 0]] * nbr[v_keys[:, 1]])
    return cost


def lpt(costs, nranks: int) -> np.ndarray:
    """Greedy longest-processing-time assignment (Algorithm 6): returns the
    rank of every item; ties broken by item index, then by rank index."""
    costs = np.asarray(costs, np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = np.zeros(nranks, np.float64)
    owner = np.zeros(len(costs), np.int32)
    for i in order:
        r = int(np.argmin(load))   # first least-loaded rank
        owner[i] = r
        load[r] += costs[i]
    return owner


def fx_encode(x) -> np.ndarray:
    """The library's fixed-point words of FP64 values: (hi, lo) int64 with
    x ~ hi 2^-32 + lo 2^-64."""
    x = np.asarray(x, np.float64)
    s = x * 4294967296.0
    h = np.rint(s)
    r = (s - h) * 4294967296.0
    return np.stack([h.astype(np.int64), np.rint(r).astype(np.int64)], axis=-1)


def fx_decode(words) -> np.ndarray:
    w = np.asarray(words, np.int64)
    return w[..., 0].astype(np.float64) * 2.0 ** -32 + w[..., 1].astype(np.float64) * 2.0 ** -64


def all_reduce_words(words: np.ndarray, group=None) -> np.ndarray:
    """Elementwise int64 sum of fixed-point words over the process group."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(words, np.int64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def build_sharded(ctx, c_keys, v_keys, theta: float, prec="fp64", nslices: int = 0, group=None):
    """Sharded hfx_build on the calling rank: LPT owners, this rank's terms,
    one integer all-reduce, then Sigma and E_X from the summed words.
    Returns E_X (identical on every rank)."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    owner = lpt(atom_costs(len(ctx.nao), c_keys, v_keys), world)
    ctx.set_shard(owner, rank)
    ctx.build(theta, prec, nslices)
    words = all_reduce_words(ctx.sigma_fixed(), group)
    return ctx.set_sigma_fixed(words)
