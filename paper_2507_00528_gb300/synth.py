"""Seeded synthetic Sb/Te-like periodic structures and random parameter vectors.

This module only draws inputs: cells, wrapped Cartesian positions, species and
uniform random parameter vectors.  It holds none of the method's arithmetic
(no descriptors, no network, no labels), so that both the FP64 oracle and the
CUDA path can be fed the very same arrays.

The paper trains on an Sb-Te DFT set mixing crystalline, liquid and
disordered phases (Sec. III.A); that set is not available, so the three phase
families below stand in for it:

* rocksalt  -- perturbed rocksalt lattice with vacancies, density 0.033 /A^3,
               Gaussian displacements sigma = 0.1 A;
* liquid    -- random sequential insertion in a cube, density 0.031 /A^3,
               minimum image distance 2.3 A;
* strained  -- a liquid-like packing at 0.033 /A^3 mapped by (I + eps), eps
               symmetric with entries U(-0.05, 0.05): triclinic cells.

Species 0 is Sb, species 1 is Te; each structure holds round(0.4 N) Sb atoms on
random sites.  Positions are wrapped into the cell (fractional coordinates in
[0, 1)), which the neighbour build of both implementations requires.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20250701

__all__ = [
    "Batch",
    "rocksalt",
    "liquid",
    "strained",
    "make_batch",
    "make_config",
    "uniform_params",
    "CONFIGS",
]


@dataclass
class Batch:
    """A packed batch of periodic structures (host numpy arrays).

    struct_off : int32 [S+1]  atom offsets of each structure (CSR)
    pos        : float64 [N,3] Cartesian positions (A), wrapped into the cell
    types      : int32 [N]    species index (0 = Sb, 1 = Te)
    cell       : float64 [S,3,3] cell rows a, b, c (A)
    """

    struct_off: np.ndarray
    pos: np.ndarray
    types: np.ndarray
    cell: np.ndarray

    @property
    def n_struct(self) -> int:
        return int(self.struct_off.shape[0] - 1)

    @property
    def n_atoms(self) -> int:
        return int(self.struct_off[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.struct_off)

    def subset(self, idx) -> "Batch":
        """Batch made of the structures listed in ``idx`` (in that order)."""
        idx = list(idx)
        parts_pos, parts_typ, sizes = [], [], []
        for s in idx:
            a, b = int(self.struct_off[s]), int(self.struct_off[s + 1])
            parts_pos.append(self.pos[a:b])
            parts_typ.append(self.types[a:b])
            sizes.append(b - a)
        off = np.zeros(len(idx) + 1, dtype=np.int32)
        off[1:] = np.cumsum(sizes)
        return Batch(off, np.concatenate(parts_pos).copy(),
                     np.concatenate(parts_typ).astype(np.int32),
                     self.cell[idx].copy())


def _wrap(pos: np.ndarray, cell: np.ndarray) -> np.ndarray:
    frac = pos @ np.linalg.inv(cell)
    frac -= np.floor(frac)
    return frac @ cell


def _species(n: int, rng: np.random.Generator, frac_sb: float = 0.4) -> np.ndarray:
    n_sb = int(round(frac_sb * n))
    t = np.ones(n, dtype=np.int32)
    t[rng.permutation(n)[:n_sb]] = 0
    return t


def rocksalt(n: int, rng: np.random.Generator, rho: float = 0.033,
             sigma: float = 0.1):
    """Perturbed rocksalt cube holding ``n`` atoms (vacancies if needed)."""
    k = max(1, math.ceil((n / 8.0) ** (1.0 / 3.0) - 1e-12))
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5],
                     [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0.5, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k),
                             indexing="ij"), -1).reshape(-1, 3)
    sites = (g[:, None, :] + base[None, :, :]).reshape(-1, 3)
    keep = np.sort(rng.permutation(sites.shape[0])[:n])
    length = (n / rho) ** (1.0 / 3.0)
    a = length / k
    pos = sites[keep] * a + rng.normal(0.0, sigma, size=(n, 3))
    cell = np.eye(3) * length
    return cell, _wrap(pos, cell), _species(n, rng)


def _rsa(n: int, length: float, dmin: float, rng: np.random.Generator,
         max_tries: int = 200000) -> np.ndarray:
    pos = np.empty((n, 3))
    placed = 0
    tries = 0
    d2min = dmin * dmin
    while placed < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(
                f"random packing of {n} atoms (L={length:.2f}, dmin={dmin}) "
                "exceeded the retry cap")
        p = rng.random(3) * length
        if placed:
            d = pos[:placed] - p
            d -= length * np.round(d / length)
            if np.min(np.einsum("ij,ij->i", d, d)) < d2min:
                continue
        pos[placed] = p
        placed += 1
    return pos


def liquid(n: int, rng: np.random.Generator, rho: float = 0.031,
           dmin: float = 2.3):
    """Liquid-like random packing in a cube."""
    length = (n / rho) ** (1.0 / 3.0)
    cell = np.eye(3) * length
    pos = _rsa(n, length, dmin, rng)
    return cell, _wrap(pos, cell), _species(n, rng)


def strained(n: int, rng: np.random.Generator, rho: float = 0.033,
             dmin: float = 2.3, eps_max: float = 0.05):
    """Random packing mapped by a symmetric random strain (triclinic cell)."""
    length = (n / rho) ** (1.0 / 3.0)
    pos = _rsa(n, length, dmin, rng)
    e = rng.uniform(-eps_max, eps_max, size=(3, 3))
    e = np.triu(e) + np.triu(e, 1).T
    m = np.eye(3) + e
    cell = (np.eye(3) * length) @ m
    pos = pos @ m
    return cell, _wrap(pos, cell), _species(n, rng)


_PHASES = (rocksalt, liquid, strained)


def make_batch(sizes, phases, rng: np.random.Generator) -> Batch:
    cells, poss, typs = [], [], []
    for n, ph in zip(sizes, phases):
        c, p, t = _PHASES[ph](int(n), rng)
        cells.append(c)
        poss.append(p)
        typs.append(t)
    off = np.zeros(len(sizes) + 1, dtype=np.int32)
    off[1:] = np.cumsum(sizes)
    return Batch(off, np.concatenate(poss), np.concatenate(typs).astype(np.int32),
                 np.stack(cells))


# Workload shapes (structure counts, size ranges, descriptor hyper-parameters).
CONFIGS = {
    1: dict(n_struct=16, size=(64, 64), mix=False, n_max=(4, 4), basis=(8, 8),
            l_max=4, four_body=False, hidden=30),
    2: dict(n_struct=256, size=(32, 400), mix=True, n_max=(8, 8), basis=(12, 12),
            l_max=4, four_body=True, hidden=50),
    3: dict(n_struct=1000, size=(64, 256), mix=True, n_max=(4, 4), basis=(8, 8),
            l_max=4, four_body=False, hidden=30),
    4: dict(n_struct=4000, size=(100, 300), mix=True, n_max=(8, 8), basis=(12, 12),
            l_max=4, four_body=False, hidden=100),
    5: dict(n_struct=10000, size=(64, 512), mix=True, n_max=(8, 8), basis=(12, 12),
            l_max=4, four_body=True, hidden=100),
}
CUTOFFS = (7.0, 4.0)


def make_config(cfg_id: int, n_struct: int | None = None,
                seed: int | None = None) -> Batch:
    """Structures of workload ``cfg_id`` (optionally only the first ``n_struct``).

    Sizes and phases are drawn first for the whole workload, so a prefix of a
    workload is the same structures whatever ``n_struct`` is.
    """
    c = CONFIGS[cfg_id]
    rng = np.random.default_rng(SEED_BASE + cfg_id if seed is None else seed)
    total = c["n_struct"]
    lo, hi = c["size"]
    sizes = rng.integers(lo, hi + 1, size=total)
    phases = (np.arange(total) % 3) if c["mix"] else np.zeros(total, dtype=int)
    if n_struct is not None:
        sizes, phases = sizes[:n_struct], phases[:n_struct]
    return make_batch(sizes, phases, rng)


def config_chunk(cfg_id: int, chunk: int, chunk_size: int = 256) -> Batch:
    """Structures chunk*chunk_size .. of workload ``cfg_id`` for per-batch
    training steps.  Sizes and phases are those of the whole workload (drawn
    as in make_config); positions come from a generator seeded by (workload,
    chunk), so chunks can be generated independently and in parallel."""
    c = CONFIGS[cfg_id]
    rng = np.random.default_rng(SEED_BASE + cfg_id)
    total = c["n_struct"]
    lo, hi = c["size"]
    sizes = rng.integers(lo, hi + 1, size=total)
    phases = (np.arange(total) % 3) if c["mix"] else np.zeros(total, dtype=int)
    s0, s1 = chunk * chunk_size, min(total, (chunk + 1) * chunk_size)
    if s0 >= s1:
        raise ValueError(f"workload {cfg_id} has no chunk {chunk}")
    return make_batch(sizes[s0:s1], phases[s0:s1], np.random.default_rng([SEED_BASE + cfg_id, chunk]))


def n_chunks(cfg_id: int, chunk_size: int = 256) -> int:
    return (CONFIGS[cfg_id]["n_struct"] + chunk_size - 1) // chunk_size


def uniform_params(n: int, seed: int, lo: float = -0.5, hi: float = 0.5) -> np.ndarray:
    """Parameter vector with entries U(lo, hi), rounded to float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n).astype(np.float32)
