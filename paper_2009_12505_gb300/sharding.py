"""Sharding the exchange build over ranks (one GPU per rank).

Pairs <A,B> are distributed by their central atom A (Sec. III.D), with one of
the paper's two schemes:
- machine scheduling (Algorithm 6), for balanced time: every pair carries the
  work estimate |N[A]| |N[B]| (neighbour counts from the C keys), atoms are
  taken in decreasing order of their pairs' total and each goes to the
  least-loaded rank;
- K-means (Algorithm 7), for less memory per rank: atoms are clustered by
  position, one cluster per rank, so a rank's F and G neighbourhoods overlap
  and it touches fewer Sigma_FG blocks.
load_ratio (Delta t_max / Delta t_av of Sec. IV) and sigma_fg_footprint (the
Sigma_FG blocks a rank touches) measure the two goals.

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


def kmeans(positions, k: int, max_iter: int = 200):
    """Algorithm 7 (K-means distribution): Lloyd iterations on the atoms'
    Cartesian coordinates.  Each atom joins the category with the nearest
    centre (ties: lowest category), each centre becomes the mean of its atoms,
    until no atom changes category.  Returns (category per atom, centres).

    Where the paper is silent: the centres start at farthest points (atom 0,
    then repeatedly the atom farthest from every chosen centre, ties to the
    lowest index); distances are plain Euclidean in the cell, without periodic
    images, as the algorithm is stated; a category left empty takes the atom
    farthest from its own centre among categories holding more than one."""
    x = np.asarray(positions, np.float64).reshape(-1, 3)
    n = x.shape[0]
    k = max(1, min(int(k), n))
    chosen = [0]
    d2 = ((x - x[0]) ** 2).sum(1)
    for _ in range(1, k):
        i = int(np.argmax(d2))
        chosen.append(i)
        d2 = np.minimum(d2, ((x - x[i]) ** 2).sum(1))
    centres = x[chosen].copy()
    labels = np.full(n, -1, np.int64)
    for _ in range(max_iter):
        dist = ((x[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
        new = np.argmin(dist, axis=1)
        counts = np.bincount(new, minlength=k)
        own = dist[np.arange(n), new]
        for j in range(k):
            if counts[j] == 0:
                # k <= n: some category holds two atoms; take its farthest atom
                cand = np.nonzero(counts[new] > 1)[0]
                far = int(cand[np.argmax(own[cand])])
                counts[new[far]] -= 1
                new[far] = j
                counts[j] = 1
        if np.array_equal(new, labels):
            break
        labels = new
        for j in range(k):
            centres[j] = x[labels == j].mean(0)
    return labels.astype(np.int32), centres


def kmeans_owner(positions, nranks: int) -> np.ndarray:
    """Owner rank of every central atom under the K-means distribution."""
    labels, _ = kmeans(positions, nranks)
    return labels


def load_ratio(owner, costs, nranks: int) -> float:
    """Delta t_max / Delta t_av with the cost model as the time: the largest
    rank load over the mean rank load (1 is perfect balance)."""
    load = np.bincount(np.asarray(owner), weights=np.asarray(costs, np.float64),
                       minlength=nranks)
    return float(load.max() / load.mean())


def sigma_fg_footprint(owner, c_keys, v_keys, nranks: int) -> np.ndarray:
    """Per rank: the number of distinct Sigma_FG blocks (F, G, n) that its
    pairs <A,B> touch, F in N[A] and G in N[B] (the memory of H_FG on a
    process, Sec. III.D).  A pair is a V key (A, B, n_B); a neighbour is a C
    key (A, F, n_F); the block is (F, G, n_B + n_G - n_F)."""
    c_keys = np.asarray(c_keys, np.int64).reshape(-1, 5)
    v_keys = np.asarray(v_keys, np.int64).reshape(-1, 5)
    owner = np.asarray(owner)
    natoms = int(max(c_keys[:, :2].max(), v_keys[:, :2].max())) + 1
    nbr = [c_keys[c_keys[:, 0] == a][:, 1:] for a in range(natoms)]

    out = np.zeros(nranks, np.int64)
    for r in range(nranks):
        parts = []
        for A, B, n1, n2, n3 in v_keys[owner[v_keys[:, 0]] == r].tolist():
            F, G = nbr[A], nbr[B]
            if len(F) == 0 or len(G) == 0:
                continue
            ii = np.repeat(F[:, 0], len(G))
            jj = np.tile(G[:, 0], len(F))
            nn = (np.array([n1, n2, n3])[None, :] + np.tile(G[:, 1:], (len(F), 1)) -
                  np.repeat(F[:, 1:], len(G), axis=0))
            parts.append(np.column_stack([ii, jj, nn]))
        out[r] = len(np.unique(np.concatenate(parts), axis=0)) if parts else 0
    return out


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


def build_sharded(ctx, c_keys, v_keys, theta: float, prec="fp64", nslices: int = 0, group=None,
                  scheme: str = "lpt", positions=None):
    """Sharded hfx_build on the calling rank: owners by machine scheduling
    (scheme "lpt") or K-means on the atom positions ("kmeans"), this rank's
    terms, one integer all-reduce, then Sigma and E_X from the summed words.
    Returns E_X (identical on every rank)."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if scheme == "kmeans":
        if positions is None:
            raise ValueError("the K-means distribution needs the atom positions")
        owner = kmeans_owner(positions, world)
    elif scheme == "lpt":
        owner = lpt(atom_costs(len(ctx.nao), c_keys, v_keys), world)
    else:
        raise ValueError(f"unknown distribution scheme {scheme!r}")
    ctx.set_shard(owner, rank)
    ctx.build(theta, prec, nslices)
    words = all_reduce_words(ctx.sigma_fixed(), group)
    return ctx.set_sigma_fixed(words)
