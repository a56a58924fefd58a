"""Molecular dynamics with a trained (or teacher) model: velocity-Verlet NVE
steps through gnep_md_verlet (forward-only inference, Eqs. 1 and 3), for
EOS- and RDF-style sampling of a batch of periodic structures.

Units: A, fs, amu, eV.  Velocities start from a seeded Maxwell-Boltzmann draw
at temperature T with the centre-of-mass velocity of each structure removed.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check
from .gnep import GNEP, DeviceBatch, _ptr, _stream

KB = 8.617333262e-5          # eV / K
ACCEL = 1.602176634e-19 / (1e-10 * 1.66053906660e-27) * 1e-20  # 1 eV / (A amu) in A / fs^2
MASS = {"Sb": 121.760, "Te": 127.60}


class NVE:
    """A batch of structures integrated with a model's forces."""

    def __init__(self, model: GNEP, batch, masses=(MASS["Sb"], MASS["Te"]), temperature=300.0, seed=0):
        self.model = model
        self.batch = batch
        self.nl = model.neighbors(DeviceBatch.from_host(batch))
        types = np.asarray(batch.types)
        m = np.asarray(masses, dtype=np.float64)[types]
        self.mass = m
        self.inv_mass = torch.tensor(1.0 / m, dtype=torch.float64, device="cuda")
        rng = np.random.default_rng(seed)
        v = rng.standard_normal((len(types), 3)) * np.sqrt(ACCEL * KB * temperature / m)[:, None]
        off = np.asarray(batch.struct_off)
        for s in range(len(off) - 1):  # no centre-of-mass drift
            a, b = off[s], off[s + 1]
            v[a:b] -= (m[a:b, None] * v[a:b]).sum(0) / m[a:b].sum()
        self.vel = torch.tensor(v, dtype=torch.float64, device="cuda")
        self.pos = torch.tensor(np.asarray(batch.pos), dtype=torch.float64, device="cuda")
        _, Es, F, _ = model.forward(self.nl)
        self.F = F.contiguous()
        self.E_pot = Es

    def step(self, dt: float, n: int = 1, stream=None):
        L = _lib.load()
        Es = torch.empty(self.batch.n_struct, dtype=torch.float64, device="cuda")
        for _ in range(n):
            check(L.gnep_md_verlet(self.model.h, self.nl.h, _ptr(self.pos), _ptr(self.vel), _ptr(self.inv_mass),
                                   _ptr(self.F), C.c_double(dt), _ptr(Es), _stream(stream)))
        self.E_pot = Es

    def kinetic(self) -> np.ndarray:
        """Kinetic energy per structure (eV)."""
        v = self.vel.cpu().numpy()
        ke = 0.5 * self.mass * (v * v).sum(1) / ACCEL
        off = np.asarray(self.batch.struct_off)
        return np.add.reduceat(ke, off[:-1])

    def total(self) -> np.ndarray:
        return self.E_pot.cpu().numpy() + self.kinetic()

    def momentum(self) -> np.ndarray:
        p = self.mass[:, None] * self.vel.cpu().numpy()
        return np.add.reduceat(p, np.asarray(self.batch.struct_off)[:-1], axis=0)
