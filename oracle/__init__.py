"""FP64 CPU oracle for gradient-optimised NEP training (ctypes binding).

TEST INFRASTRUCTURE ONLY.  The plain, slow reference implementation that the
CUDA path is checked against; only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library: the C source is ``gnep_oracle.c`` and every formula there cites
the paper passage it follows.

Arrays are numpy, FP64 (parameters and scales are promoted from float32 by the
caller when the GPU side is fed the same values).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_long)


class _Cfg(C.Structure):
    _fields_ = [("n_species", C.c_int), ("nq_r", C.c_int), ("nq_a", C.c_int),
                ("k_r", C.c_int), ("k_a", C.c_int), ("l_max", C.c_int),
                ("four_body", C.c_int), ("hidden", C.c_int),
                ("rc_r", C.c_double), ("rc_a", C.c_double)]


class _Batch(C.Structure):
    _fields_ = [("n_struct", C.c_int), ("struct_off", _ip), ("pos", _dp),
                ("type", _ip), ("cell", _dp)]


class _Labels(C.Structure):
    _fields_ = [("energy", _dp), ("force", _dp), ("virial", _dp),
                ("lambda_e", C.c_double), ("lambda_f", C.c_double),
                ("lambda_v", C.c_double), ("lambda_l2", C.c_double),
                ("loss_form", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_num_des.argtypes = [C.POINTER(_Cfg)]
        L.orc_num_params.argtypes = [C.POINTER(_Cfg)]
        L.orc_num_params.restype = C.c_long
        L.orc_clm.restype = _dp
        L.orc_chebyshev.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.orc_cutoff.argtypes = [C.c_double, C.c_double, _dp, _dp]
        L.orc_radial_basis.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp]
        L.orc_blm.argtypes = [_dp, _dp, _dp]
        L.orc_blm_lmax.argtypes = [_dp, C.c_int, _dp, _dp]
        L.orc_clm_quadrature.argtypes = [C.c_int]
        L.orc_clm_quadrature.restype = C.c_double
        L.orc_neighbors.argtypes = [C.POINTER(_Batch), C.c_double, C.c_long, _lp, _ip, _ip]
        L.orc_neighbors.restype = C.c_long
        L.orc_descriptors.argtypes = [C.POINTER(_Cfg), _dp, C.POINTER(_Batch), _dp]
        L.orc_ann.argtypes = [C.POINTER(_Cfg), _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_forward.argtypes = [C.POINTER(_Cfg), _dp, _dp, C.POINTER(_Batch), _dp, _dp, _dp, _dp]
        L.orc_loss.argtypes = [C.POINTER(_Cfg), _dp, _dp, C.POINTER(_Batch), C.POINTER(_Labels), _dp]
        L.orc_loss_grad.argtypes = [C.POINTER(_Cfg), _dp, _dp, C.POINTER(_Batch),
                                    C.POINTER(_Labels), _dp, _dp]
        L.orc_adam.argtypes = [C.c_long, _dp, _dp, _dp, _dp, C.c_long, C.c_double,
                               C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_lr.argtypes = [C.c_double, C.c_double, C.c_long, C.c_long, C.c_long]
        L.orc_lr.restype = C.c_double
        _lib = L
    return _lib


@dataclass
class Cfg:
    """Model hyper-parameters: channels nq = n_max + 1, basis k = basis_size + 1."""
    n_species: int = 2
    nq_r: int = 5
    nq_a: int = 5
    k_r: int = 9
    k_a: int = 9
    l_max: int = 4
    four_body: bool = False
    hidden: int = 30
    rc_r: float = 7.0
    rc_a: float = 4.0

    def c(self) -> _Cfg:
        return _Cfg(self.n_species, self.nq_r, self.nq_a, self.k_r, self.k_a,
                    self.l_max, int(self.four_body), self.hidden, self.rc_r, self.rc_a)

    @property
    def n_des(self) -> int:
        return lib().orc_num_des(C.byref(self.c()))

    @property
    def n_params(self) -> int:
        return int(lib().orc_num_params(C.byref(self.c())))


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_dp)


class _BatchView:
    def __init__(self, b):
        self.off = np.ascontiguousarray(b.struct_off, dtype=np.int32)
        self.pos = _d(b.pos).reshape(-1, 3)
        self.typ = np.ascontiguousarray(b.types, dtype=np.int32)
        self.cell = _d(b.cell).reshape(-1, 9)
        self.c = _Batch(len(self.off) - 1, self.off.ctypes.data_as(_ip),
                        self.pos.ctypes.data_as(_dp), self.typ.ctypes.data_as(_ip),
                        self.cell.ctypes.data_as(_dp))
        self.n_struct = len(self.off) - 1
        self.n_atoms = int(self.off[-1])


def nlm(l_max: int = 4) -> int:
    """(l, m) components for l = 1..l_max."""
    return (l_max + 1) ** 2 - 1


def clm(l_max: int = 4) -> np.ndarray:
    p = lib().orc_clm()
    return np.array([p[i] for i in range(nlm(l_max))])


def clm_quadrature(lm: int) -> float:
    """4 pi / ((2l + 1) int B_lm^2 dOmega) by the oracle's quadrature."""
    return lib().orc_clm_quadrature(lm)


def chebyshev(K: int, xi: float):
    T = np.zeros(K); dT = np.zeros(K)
    lib().orc_chebyshev(K, xi, _p(T), _p(dT))
    return T, dT


def cutoff(rc: float, r: float):
    fc = C.c_double(); fcp = C.c_double()
    lib().orc_cutoff(rc, r, C.byref(fc), C.byref(fcp))
    return fc.value, fcp.value


def radial_basis(K: int, rc: float, r: float):
    f = np.zeros(K); fp = np.zeros(K)
    lib().orc_radial_basis(K, rc, r, _p(f), _p(fp))
    return f, fp


def blm(d, l_max: int = 4):
    """B_lm (B9.1) and their gradients (B9.2) for l = 1..l_max (at most 8)."""
    d = _d(d)
    n = nlm(l_max)
    B = np.zeros(n); dB = np.zeros(3 * n)
    lib().orc_blm_lmax(_p(d), l_max, _p(B), _p(dB))
    return B, dB.reshape(n, 3)


def neighbors(batch, rc: float):
    """Canonical neighbour lists: (off[N+1], j[P] global index, shift[P,3])."""
    bv = _BatchView(batch)
    off = np.zeros(bv.n_atoms + 1, dtype=np.int64)
    n = lib().orc_neighbors(C.byref(bv.c), rc, 0, off.ctypes.data_as(_lp),
                            None, None)
    j = np.zeros(max(n, 1), dtype=np.int32)
    sh = np.zeros((max(n, 1), 3), dtype=np.int32)
    lib().orc_neighbors(C.byref(bv.c), rc, n, off.ctypes.data_as(_lp),
                        j.ctypes.data_as(_ip), sh.ctypes.data_as(_ip))
    return off, j[:n], sh[:n]


def descriptors(cfg: Cfg, params, batch) -> np.ndarray:
    """Unscaled descriptors G [N, n_des] (Eqs. 5-8, 4-body reading)."""
    bv = _BatchView(batch)
    P = _d(params)
    G = np.zeros((bv.n_atoms, cfg.n_des))
    lib().orc_descriptors(C.byref(cfg.c()), _p(P), C.byref(bv.c), _p(G))
    return G


def scale_from_descriptors(G) -> np.ndarray:
    """The fixed input scale read into the method (the paper gives none; raw
    descriptors are O(10) and tanh would saturate): per component v,
    s_v = 1 / (max_v - min_v) over the atoms of a set, and 1 where max = min."""
    G = np.asarray(G, dtype=np.float64)
    span = G.max(axis=0) - G.min(axis=0)
    return np.where(span > 0, 1.0 / np.where(span > 0, span, 1.0), 1.0)


def descriptor_scale(cfg: Cfg, params, batch) -> np.ndarray:
    """Fixed per-component input scale over a set of structures."""
    return scale_from_descriptors(descriptors(cfg, params, batch))


def ann(cfg: Cfg, params, scale, e: int, G):
    P = _d(params); s = _d(scale); g = _d(G)
    E = C.c_double()
    Ep = np.zeros(cfg.n_des); Epp = np.zeros((cfg.n_des, cfg.n_des))
    lib().orc_ann(C.byref(cfg.c()), _p(P), _p(s), e, _p(g), C.byref(E), _p(Ep), _p(Epp))
    return E.value, Ep, Epp


def forward(cfg: Cfg, params, scale, batch):
    """Per-atom energy, per-structure energy, forces, symmetrised total virial."""
    bv = _BatchView(batch)
    P = _d(params); s = _d(scale)
    Ea = np.zeros(bv.n_atoms); Es = np.zeros(bv.n_struct)
    F = np.zeros((bv.n_atoms, 3)); W = np.zeros((bv.n_struct, 6))
    lib().orc_forward(C.byref(cfg.c()), _p(P), _p(s), C.byref(bv.c), _p(Ea), _p(Es),
                      _p(F), _p(W))
    return Ea, Es, F, W


@dataclass
class Labels:
    energy: np.ndarray   # [S] per-atom energy
    force: np.ndarray    # [N,3]
    virial: np.ndarray   # [S,6] per-atom virial
    lambda_e: float = 1.0
    lambda_f: float = 1.0
    lambda_v: float = 0.1
    lambda_l2: float = 0.0
    loss_form: int = 0

    def c(self):
        self._e = _d(self.energy); self._f = _d(self.force); self._v = _d(self.virial)
        return _Labels(_p(self._e), _p(self._f), _p(self._v), self.lambda_e,
                       self.lambda_f, self.lambda_v, self.lambda_l2, self.loss_form)


def teacher_labels(cfg: Cfg, params, scale, batch, **kw) -> Labels:
    """Labels E_s/N_s, F, W_s/N_s produced by a teacher parameter vector."""
    _, Es, F, W = forward(cfg, params, scale, batch)
    ns = np.diff(np.asarray(batch.struct_off)).astype(np.float64)
    return Labels(Es / ns, F, W / ns[:, None], **kw)


def loss(cfg: Cfg, params, scale, batch, y: Labels) -> np.ndarray:
    bv = _BatchView(batch)
    P = _d(params); s = _d(scale)
    t = np.zeros(4)
    yc = y.c()
    lib().orc_loss(C.byref(cfg.c()), _p(P), _p(s), C.byref(bv.c), C.byref(yc), _p(t))
    return t


def loss_grad(cfg: Cfg, params, scale, batch, y: Labels):
    """Loss terms [L, L_e, L_f, L_v] and dL/dtheta by the explicit route."""
    bv = _BatchView(batch)
    P = _d(params); s = _d(scale)
    t = np.zeros(4); g = np.zeros(cfg.n_params)
    yc = y.c()
    lib().orc_loss_grad(C.byref(cfg.c()), _p(P), _p(s), C.byref(bv.c), C.byref(yc),
                        _p(t), _p(g))
    return t, g


def adam(theta, m, v, g, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8,
         weight_decay=0.0):
    """One Adam update in place (float64 arrays)."""
    lib().orc_adam(len(theta), _p(theta), _p(m), _p(v), _p(_d(g)), t, lr, beta1,
                   beta2, eps, weight_decay)


def lr(lr_start: float, lr_stop: float, s: int, n_warmup: int, n_total: int) -> float:
    return lib().orc_lr(lr_start, lr_stop, s, n_warmup, n_total)


# 1 eV / (A amu) in A / fs^2, from the SI values of the electronvolt
# (1.602176634e-19 J) and the atomic mass unit (1.66053906660e-27 kg):
# 1 eV / (1e-10 m x 1 amu) in m / s^2, times 1e10 A/m x 1e-30 s^2/fs^2.
EV_PER_A_AMU_IN_A_PER_FS2 = 1.602176634e-19 / (1e-10 * 1.66053906660e-27) * 1e10 * 1e-30


def wrap(batch, pos) -> np.ndarray:
    """Positions mapped into their cell: fractional f = x H^-1 reduced to
    [0, 1), then x = f H (rows of H are the lattice vectors)."""
    out = np.array(pos, dtype=np.float64)
    off = np.asarray(batch.struct_off)
    for s in range(len(off) - 1):
        H = np.asarray(batch.cell[s], dtype=np.float64).reshape(3, 3)
        f = out[off[s]:off[s + 1]] @ np.linalg.inv(H)
        f -= np.floor(f)
        out[off[s]:off[s + 1]] = f @ H
    return out


def md_verlet(cfg: Cfg, params, scale, batch, vel, inv_mass, dt: float, steps: int):
    """Velocity-Verlet NVE with the model's FP64 forces (the MD use of a
    trained potential, Sec. III): per step, v += dt/2 F/m, x += dt v (then
    wrapped into the cell), F = F(x), v += dt/2 F/m.  Units A, fs, amu, eV.
    Returns the positions, velocities, forces and per-structure potential
    energies after each step."""
    from types import SimpleNamespace
    acc = EV_PER_A_AMU_IN_A_PER_FS2 * np.asarray(inv_mass, dtype=np.float64)[:, None]
    x = np.array(batch.pos, dtype=np.float64)
    v = np.array(vel, dtype=np.float64)
    b = SimpleNamespace(struct_off=batch.struct_off, pos=x, types=batch.types, cell=batch.cell)
    F = forward(cfg, params, scale, b)[2]
    traj = []
    for _ in range(steps):
        v = v + 0.5 * dt * acc * F
        x = wrap(batch, x + dt * v)
        b = SimpleNamespace(struct_off=batch.struct_off, pos=x, types=batch.types, cell=batch.cell)
        _, Es, F, _ = forward(cfg, params, scale, b)
        v = v + 0.5 * dt * acc * F
        traj.append((x.copy(), v.copy(), F.copy(), Es.copy()))
    return traj
