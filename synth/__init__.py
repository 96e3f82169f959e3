"""Seeded synthetic inputs for the periodic LRI exchange build.

This module is input infrastructure shared by the CPU oracle's tests, the GPU
parity tests and the benchmark. It holds geometry, cutoff-based neighbour
enumeration and random block draws only -- none of the exchange arithmetic.

Data model (Sec. II, Eq. AO and Eq. ABF of the paper): a site is an atom of the
unit cell plus an integer lattice vector n.  Every input is a sparse set of
dense blocks keyed by ``(i, j, n1, n2, n3)``, the block between site
``(i, 0)`` and site ``(j, n)``:

* ``C`` key ``(a, f, n)``: LRI coefficients with the ABFs on ``a``, shape
  ``[nabf(a)][nao(a)][nao(f)]`` (Eq. LRI).
* ``V`` key ``(a, b, n)``: two-centre Coulomb block, shape ``[nabf(a)][nabf(b)]``.
* ``D`` key ``(k, l, n)``: real-space density-matrix block, shape ``[nao(k)][nao(l)]``.

Positions live on an integer grid of spacing ``unit`` (bohr) with period
``period`` grid steps per lattice vector (cubic cells only), so squared
distances are exact integers times ``unit**2`` and inclusive cutoffs that fall
exactly on a neighbour shell (the rocksalt cell at a = 8 bohr) are decided
without rounding.

Random numbers: every block is drawn from its own Philox stream whose 128-bit
key packs ``(seed, kind, i, j, n)``, so any block can be regenerated alone.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

KIND_C, KIND_V, KIND_D = 1, 2, 3


@dataclass
class System:
    """A periodic (or, with a huge period, finite) cubic system on an integer grid."""

    name: str
    unit: float                 # grid spacing in bohr
    period: int                 # lattice vector length in grid steps (cubic cell)
    grid: np.ndarray            # (natoms, 3) int64 grid coordinates inside the cell
    nao: np.ndarray             # (natoms,) int32 NAOs per atom
    nabf: np.ndarray            # (natoms,) int32 ABFs per atom
    species: np.ndarray = field(default=None)

    @property
    def natoms(self) -> int:
        return int(self.grid.shape[0])

    @property
    def lattice(self) -> np.ndarray:
        """Lattice vectors (rows a1, a2, a3) in bohr."""
        return np.eye(3) * (self.unit * self.period)

    @property
    def positions(self) -> np.ndarray:
        return self.grid.astype(np.float64) * self.unit

    def pairs_within(self, cut: float):
        """All (i, j, n) with |tau_j + n L - tau_i| <= cut (inclusive).

        Returns a list of (i, j, (n1, n2, n3), d) sorted by (i, j, n)."""
        out = []
        cut2 = cut * cut
        u2 = self.unit * self.unit
        reach = int(math.ceil(cut / (self.unit * self.period))) + 1
        shifts = np.array(list(itertools.product(range(-reach, reach + 1), repeat=3)),
                          dtype=np.int64)
        g = self.grid
        for i in range(self.natoms):
            dv = (g[:, None, :] - g[i][None, None, :]) + shifts[None, :, :] * self.period
            m = np.einsum("jsk,jsk->js", dv, dv)
            js, ss = np.nonzero(m.astype(np.float64) * u2 <= cut2)
            for j, s in zip(js.tolist(), ss.tolist()):
                n = tuple(int(c) for c in shifts[s])
                out.append((i, j, n, math.sqrt(float(m[j, s]) * u2)))
        out.sort(key=lambda t: (t[0], t[1], t[2]))
        return out


def _cell_sites(ncell: int, basis: list[tuple[int, int, int]], cell_steps: int):
    pts = []
    for c in itertools.product(range(ncell), repeat=3):
        for b in basis:
            pts.append([b[k] + c[k] * cell_steps for k in range(3)])
    return np.array(pts, dtype=np.int64)


def si_diamond(ncell: int = 1, a: float = 10.26, nao: int = 13, nabf: int = 60) -> System:
    """Diamond-cubic Si-like supercell: 8 ncell^3 atoms, grid spacing a/4."""
    fcc = [(0, 0, 0), (0, 2, 2), (2, 0, 2), (2, 2, 0)]
    basis = fcc + [(x + 1, y + 1, z + 1) for (x, y, z) in fcc]
    grid = _cell_sites(ncell, basis, 4)
    n = grid.shape[0]
    return System(f"si{n}", a / 4.0, 4 * ncell, grid,
                  np.full(n, nao, np.int32), np.full(n, nabf, np.int32),
                  np.zeros(n, np.int32))


def two_element_rocksalt(ncell: int = 3, a: float = 8.0, seed: int = 4,
                         sizes=((13, 60), (27, 90))) -> System:
    """Rocksalt-like supercell (grid spacing a/2, 8 sites per cubic cell) whose
    sites carry element A or B, exactly half each, by a seeded permutation."""
    basis = list(itertools.product((0, 1), repeat=3))
    grid = _cell_sites(ncell, basis, 2)
    n = grid.shape[0]
    rng = np.random.Generator(np.random.Philox(key=_pack_key(seed, 0, 0, 0, (0, 0, 0))))
    species = np.zeros(n, np.int32)
    species[rng.permutation(n)[: n // 2]] = 1
    nao = np.array([sizes[s][0] for s in species], np.int32)
    nabf = np.array([sizes[s][1] for s in species], np.int32)
    return System(f"ab{n}", a / 2.0, 2 * ncell, grid, nao, nabf, species)


def custom(name, unit, period, grid, nao, nabf) -> System:
    grid = np.asarray(grid, np.int64).reshape(-1, 3)
    n = grid.shape[0]
    return System(name, float(unit), int(period), grid,
                  np.broadcast_to(np.asarray(nao, np.int32), (n,)).copy(),
                  np.broadcast_to(np.asarray(nabf, np.int32), (n,)).copy(),
                  np.zeros(n, np.int32))


def _pack_key(seed: int, kind: int, i: int, j: int, n) -> int:
    k = seed & 0xFFFFFFFF
    k = (k << 8) | (kind & 0xFF)
    k = (k << 24) | (i & 0xFFFFFF)
    k = (k << 24) | (j & 0xFFFFFF)
    for c in n:
        k = (k << 8) | ((c + 128) & 0xFF)
    return k


def _rng(seed, kind, i, j, n):
    return np.random.Generator(np.random.Philox(key=_pack_key(seed, kind, i, j, n)))


def _canonical(i, j, n) -> bool:
    """Canonical orientation of a symmetric pair (the other is its transpose)."""
    if i != j:
        return i < j
    return tuple(n) >= (0, 0, 0)


@dataclass
class Blocks:
    """A packed sparse block set: keys (nblk, 5) int32, data float64, offs (nblk+1,) int64."""

    keys: np.ndarray
    data: np.ndarray
    offs: np.ndarray

    @property
    def count(self) -> int:
        return int(self.keys.shape[0])

    def as_dict(self):
        return {tuple(int(x) for x in k): self.data[self.offs[b]:self.offs[b + 1]]
                for b, k in enumerate(self.keys)}


def pack(blocks: dict) -> Blocks:
    """Pack {(i, j, n1, n2, n3): ndarray} into a Blocks set sorted by key."""
    items = sorted(blocks.items())
    keys = np.array([k for k, _ in items], np.int32).reshape(-1, 5)
    sizes = [v.size for _, v in items]
    offs = np.zeros(len(items) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    data = np.empty(int(offs[-1]), np.float64)
    for b, (_, v) in enumerate(items):
        data[offs[b]:offs[b + 1]] = np.ravel(v)
    return Blocks(keys, data, offs)


def gen_C(system: System, cut: float, seed: int) -> dict:
    """C(a, f, n) for every pair within ``cut``: N(0,1) exp(-d/2); on-site blocks
    symmetrised in the two AO indices; C(a,f,n) and C(f,a,-n) drawn independently."""
    out = {}
    for i, j, n, d in system.pairs_within(cut):
        shape = (int(system.nabf[i]), int(system.nao[i]), int(system.nao[j]))
        x = _rng(seed, KIND_C, i, j, n).standard_normal(shape)
        if i == j and n == (0, 0, 0):
            x = (x + x.transpose(0, 2, 1)) / math.sqrt(2.0)
        out[(i, j) + tuple(n)] = x * math.exp(-d / 2.0)
    return out


def gen_V(system: System, cut: float, seed: int, mu: float = 0.11) -> dict:
    """V(a, b, n) within ``cut``: N(0,1) erfc(mu d)/max(d,1) off-site, X X^T/nP + I
    on-site; V(b, a, -n) = V(a, b, n)^T."""
    out = {}
    for i, j, n, d in system.pairs_within(cut):
        if not _canonical(i, j, n):
            continue
        g = _rng(seed, KIND_V, i, j, n)
        pa, pb = int(system.nabf[i]), int(system.nabf[j])
        if i == j and n == (0, 0, 0):
            x = g.standard_normal((pa, pa))
            v = x @ x.T / pa + np.eye(pa)
            v = 0.5 * (v + v.T)
        else:
            v = g.standard_normal((pa, pb)) * (math.erfc(mu * d) / max(d, 1.0))
        out[(i, j) + tuple(n)] = v
        out[(j, i) + tuple(-c for c in n)] = v.T.copy()
    return out


def d_envelope(d: float, decay: str = "exp") -> float:
    """Off-site magnitude of D at distance d: exponential for an insulator
    (exp(-d/3)), polynomial for a metal ((1 + d/3)^-2; Sec. III.B: an
    insulator's D decays exponentially, a metal's only polynomially)."""
    if decay == "exp":
        return math.exp(-d / 3.0)
    if decay == "power":
        return (1.0 + d / 3.0) ** -2
    raise ValueError(f"unknown D decay {decay!r}")


def gen_D(system: System, cut: float, seed: int, decay: str = "exp") -> dict:
    """D(k, l, n) within ``cut``: N(0, 0.1) times d_envelope(d, decay); on-site
    (X + X^T)/sqrt2 with X ~ N(0, 0.1^2); D(l, k, -n) = D(k, l, n)^T."""
    out = {}
    for i, j, n, d in system.pairs_within(cut):
        if not _canonical(i, j, n):
            continue
        g = _rng(seed, KIND_D, i, j, n)
        ka, kb = int(system.nao[i]), int(system.nao[j])
        if i == j and n == (0, 0, 0):
            x = 0.1 * g.standard_normal((ka, ka))
            blk = (x + x.T) / math.sqrt(2.0)
        else:
            blk = 0.1 * g.standard_normal((ka, kb)) * d_envelope(d, decay)
        out[(i, j) + tuple(n)] = blk
        out[(j, i) + tuple(-c for c in n)] = blk.T.copy()
    return out


@dataclass
class Workload:
    name: str
    system: System
    C: Blocks
    V: Blocks
    D: Blocks
    cut_C: float
    cut_V: float
    cut_D: float
    seed: int


def make_workload(system: System, cut_C=16.0, cut_V=20.0, cut_D=16.0, seed=1,
                  name=None, mu=0.11, d_decay="exp") -> Workload:
    """mu: range separation of V (erfc(mu d) / d; 0 is the full-range
    Coulomb of Hartree-Fock); d_decay: "exp" (insulator) or "power" (metal)."""
    return Workload(name or system.name, system,
                    pack(gen_C(system, cut_C, seed)),
                    pack(gen_V(system, cut_V, seed, mu=mu)),
                    pack(gen_D(system, cut_D, seed, decay=d_decay)),
                    cut_C, cut_V, cut_D, seed)


# Named workloads with the benchmark shapes: Si-like diamond (13 NAOs, 60 ABFs,
# a = 10.26 bohr) and the two-element rocksalt-like cell (13/60 and 27/90,
# a = 8.0 bohr); C and D within 16 bohr, V within 20 bohr; seed = workload index.
def si8(seed=1):
    return make_workload(si_diamond(1), seed=seed, name="si8")


def si64(seed=2):
    return make_workload(si_diamond(2), seed=seed, name="si64")


def si512(seed=3):
    return make_workload(si_diamond(4), seed=seed, name="si512")


def ab216(seed=4):
    return make_workload(two_element_rocksalt(3, seed=seed), seed=seed, name="ab216")


# The second workload (denser tasks for the same kernels): full-range Coulomb V
# out to R_Q = 50 bohr, as Hartree-Fock or long-range-corrected functionals
# need (Sec. IV), and a metallic D kept out to 24 bohr with polynomial decay.
def si8_fullrange(seed=5):
    return make_workload(si_diamond(1), cut_V=50.0, mu=0.0, seed=seed, name="si8_fullrange")


def si8_metal(seed=6):
    return make_workload(si_diamond(1), cut_D=24.0, d_decay="power", seed=seed,
                         name="si8_metal")


def si_shrunk(ncell=1, cut_C=8.0, cut_V=10.0, cut_D=8.0, seed=11, nao=13, nabf=60):
    """Si-like cell with shortened cutoffs: full block sizes, few neighbours."""
    return make_workload(si_diamond(ncell, nao=nao, nabf=nabf), cut_C, cut_V, cut_D,
                         seed, name=f"si{8 * ncell ** 3}_shrunk")


def ab_shrunk(ncell=1, cut_C=6.0, cut_V=8.0, cut_D=6.0, seed=12):
    """Two-element cell with shortened cutoffs (uneven 13/60 and 27/90 blocks)."""
    return make_workload(two_element_rocksalt(ncell, seed=seed), cut_C, cut_V, cut_D,
                         seed, name=f"ab{8 * ncell ** 3}_shrunk")
