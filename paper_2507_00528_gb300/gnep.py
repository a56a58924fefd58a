"""Python layer over libgnep: torch tensors for device memory, torch streams.

Every computation runs in the library's CUDA kernels; this module only
allocates tensors, passes pointers and wraps the step in a
``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libgnep needs a CUDA device (sm_103a); there is no CPU fallback")


@dataclass
class DeviceBatch:
    """A batch of structures resident on the GPU (inputs of the neighbour build)."""
    struct_off: torch.Tensor  # int32 [S+1]
    pos: torch.Tensor         # float64 [N,3]
    types: torch.Tensor       # int32 [N]
    cell: torch.Tensor        # float64 [S,3,3]

    @staticmethod
    def from_host(b, device="cuda") -> "DeviceBatch":
        return DeviceBatch(torch.as_tensor(np.ascontiguousarray(b.struct_off, dtype=np.int32), device=device),
                           torch.as_tensor(np.ascontiguousarray(b.pos, dtype=np.float64), device=device),
                           torch.as_tensor(np.ascontiguousarray(b.types, dtype=np.int32), device=device),
                           torch.as_tensor(np.ascontiguousarray(b.cell, dtype=np.float64), device=device))

    @property
    def n_struct(self):
        return self.struct_off.numel() - 1

    @property
    def n_atoms(self):
        return self.types.numel()

    def c(self) -> _lib.Batch:
        return _lib.Batch(self.n_struct, self.n_atoms, self.struct_off.data_ptr(), self.pos.data_ptr(),
                          self.types.data_ptr(), self.cell.data_ptr())


def host_batch_struct(b) -> tuple[_lib.Batch, list]:
    """C batch view of host numpy arrays (kept alive by the returned list)."""
    arrs = [np.ascontiguousarray(b.struct_off, dtype=np.int32), np.ascontiguousarray(b.pos, dtype=np.float64),
            np.ascontiguousarray(b.types, dtype=np.int32), np.ascontiguousarray(b.cell, dtype=np.float64)]
    cb = _lib.Batch(len(arrs[0]) - 1, len(arrs[2]), arrs[0].ctypes.data, arrs[1].ctypes.data,
                    arrs[2].ctypes.data, arrs[3].ctypes.data)
    return cb, arrs


@dataclass
class Labels:
    """Labels and loss weights (Eqs. 9-12); tensors on the GPU or in host memory."""
    energy: torch.Tensor  # float64 [S] per-atom energy
    force: torch.Tensor   # float32 [N,3]
    virial: torch.Tensor  # float64 [S,6] per-atom virial
    lambda_e: float = 1.0
    lambda_f: float = 1.0
    lambda_v: float = 0.1
    lambda_l2: float = 0.0
    loss_form: int = _lib.LOSS_MSE

    def c(self) -> _lib.Labels:
        for t, dt in ((self.energy, torch.float64), (self.force, torch.float32), (self.virial, torch.float64)):
            assert t.dtype == dt and t.is_contiguous()
        return _lib.Labels(self.energy.data_ptr(), self.force.data_ptr(), self.virial.data_ptr(),
                           self.lambda_e, self.lambda_f, self.lambda_v, self.lambda_l2, self.loss_form)


class NeighborList:
    """Neighbour lists (Eq. 2) and per-step workspace of one batch."""

    def __init__(self, model: "GNEP", batch, stream=None):
        self.model = model
        L = _lib.load()
        h = C.c_void_p()
        if isinstance(batch, DeviceBatch):
            cb = batch.c()
            check(L.gnep_build_neighbors(model.h, C.byref(cb), C.byref(h), _stream(stream)))
        else:
            cb, keep = host_batch_struct(batch)
            check(L.gnep_build_neighbors(model.h, C.byref(cb), C.byref(h), _stream(stream)))
        self.h = h
        self.n_struct = cb.n_struct
        self.n_atoms = cb.n_atoms
        so = batch.struct_off.cpu().numpy() if isinstance(batch, DeviceBatch) else batch.struct_off
        self.struct_off_host = np.array(so, dtype=np.int64)

    def rebuild(self, batch, stream=None):
        L = _lib.load()
        if isinstance(batch, DeviceBatch):
            cb = batch.c()
            check(L.gnep_rebuild_neighbors(self.model.h, C.byref(cb), self.h, _stream(stream)))
        else:
            cb, keep = host_batch_struct(batch)
            check(L.gnep_rebuild_neighbors(self.model.h, C.byref(cb), self.h, _stream(stream)))

    def info(self):
        a, b = C.c_int64(), C.c_int64()
        check(_lib.load().gnep_nlist_info(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def export(self, which: int):
        """(off [N+1], j [P], shift [P,3]) as int32 numpy arrays."""
        n = self.info()[which]
        off = np.zeros(self.n_atoms + 1, dtype=np.int32)
        j = np.zeros(max(n, 1), dtype=np.int32)
        sh = np.zeros((max(n, 1), 3), dtype=np.int32)
        check(_lib.load().gnep_nlist_export(self.h, which, off.ctypes.data, j.ctypes.data, sh.ctypes.data,
                                            _stream()))
        return off, j[:n], sh[:n]

    TUNING_KEYS = ("desc_tile_atoms", "desc_tile_pairs", "force_tile_atoms", "force_tile_pairs", "cgrad_blocks",
                   "net_blocks", "radial_lanes", "net_tile_atoms", "radial_beside")

    def autotune(self, y: "Labels", reps: int = 3, stream=None) -> dict:
        """Pick the fastest launch shapes of the angular sweeps for this batch
        (times loss + gradient; invalidates graphs captured on this list)."""
        yc = y.c()
        check(_lib.load().gnep_autotune(self.model.h, self.h, C.byref(yc), reps, _stream(stream)))
        return self.tuning()

    def tuning(self) -> dict:
        v = np.zeros(len(self.TUNING_KEYS), dtype=np.int32)
        check(_lib.load().gnep_tuning_get(self.model.h, self.h, v.ctypes.data))
        return dict(zip(self.TUNING_KEYS, v.tolist()))

    def set_tuning(self, values: dict | None = None, stream=None):
        """Set launch shapes (missing or 0 = built-in default) and rebuild the tiles."""
        values = values or {}
        v = np.array([int(values.get(k, 0)) for k in self.TUNING_KEYS], dtype=np.int32)
        check(_lib.load().gnep_tuning_set(self.model.h, self.h, v.ctypes.data, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            _lib.load().gnep_nlist_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GNEP:
    """A NEP model: hyper-parameters (Sec. II.B), parameters and Adam state on the GPU."""

    def __init__(self, n_species=2, rc_radial=7.0, rc_angular=4.0, n_max=(4, 4), basis=(8, 8), l_max=4,
                 four_body=False, hidden=30, seed=0, precision="fp32"):
        _require_cuda()
        L = _lib.load()
        h = C.c_void_p()
        check(L.gnep_create(C.byref(h), n_species, None, rc_radial, rc_angular, n_max[0], n_max[1], basis[0],
                            basis[1], l_max, int(four_body), hidden, seed, _lib.PREC[precision]))
        self.h = h
        self.hyper = dict(n_species=n_species, rc_radial=rc_radial, rc_angular=rc_angular, n_max=tuple(n_max),
                          basis=tuple(basis), l_max=l_max, four_body=four_body, hidden=hidden)
        n = C.c_int64()
        check(L.gnep_num_params(h, C.byref(n)))
        d = C.c_int32()
        check(L.gnep_num_descriptors(h, C.byref(d)))
        self.n_params = n.value
        self.n_des = d.value

    # parameters -------------------------------------------------------------
    def get_params(self) -> torch.Tensor:
        t = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        check(_lib.load().gnep_get_params(self.h, _ptr(t), self.n_params, _stream()))
        return t

    def set_params(self, p):
        t = torch.as_tensor(p, dtype=torch.float32).contiguous()
        t = t.cuda() if not t.is_cuda else t
        check(_lib.load().gnep_set_params(self.h, _ptr(t), self.n_params, _stream()))

    def get_scale(self) -> torch.Tensor:
        t = torch.empty(self.n_des, dtype=torch.float32, device="cuda")
        check(_lib.load().gnep_get_descriptor_scale(self.h, _ptr(t), self.n_des, _stream()))
        return t

    def set_scale(self, s):
        t = torch.as_tensor(s, dtype=torch.float32).contiguous().cuda()
        check(_lib.load().gnep_set_descriptor_scale(self.h, _ptr(t), self.n_des, _stream()))

    def compute_scale(self, nl: NeighborList):
        check(_lib.load().gnep_compute_descriptor_scale(self.h, nl.h, _stream()))

    def set_precision(self, precision: str):
        check(_lib.load().gnep_set_precision(self.h, _lib.PREC[precision]))

    # evaluation -------------------------------------------------------------
    def neighbors(self, batch, stream=None) -> NeighborList:
        return NeighborList(self, batch, stream)

    def descriptors(self, nl: NeighborList) -> torch.Tensor:
        G = torch.empty(nl.n_atoms, self.n_des, dtype=torch.float32, device="cuda")
        check(_lib.load().gnep_descriptors(self.h, nl.h, _ptr(G), _stream()))
        return G

    def forward(self, nl: NeighborList):
        Ea = torch.empty(nl.n_atoms, dtype=torch.float32, device="cuda")
        Es = torch.empty(nl.n_struct, dtype=torch.float64, device="cuda")
        F = torch.empty(nl.n_atoms, 3, dtype=torch.float32, device="cuda")
        W = torch.empty(nl.n_struct, 6, dtype=torch.float64, device="cuda")
        check(_lib.load().gnep_forward(self.h, nl.h, _ptr(Ea), _ptr(Es), _ptr(F), _ptr(W), _stream()))
        return Ea, Es, F, W

    def teacher_labels(self, nl: NeighborList, batch_sizes, **kw) -> Labels:
        """Labels E_s/N_s, F, W_s/N_s produced by this model (a teacher)."""
        _, Es, F, W = self.forward(nl)
        ns = torch.as_tensor(np.asarray(batch_sizes, dtype=np.float64), device="cuda")
        return Labels(Es / ns, F.contiguous(), (W / ns[:, None]).contiguous(), **kw)

    def loss_grad(self, nl: NeighborList, y: Labels, grad=True, stream=None):
        terms = torch.empty(4, dtype=torch.float64, device="cuda")
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda") if grad else None
        yc = y.c()
        check(_lib.load().gnep_loss_grad(self.h, nl.h, C.byref(yc), _ptr(terms), _ptr(g), _stream(stream)))
        return terms, g

    def loss(self, nl: NeighborList, y: Labels, stream=None):
        """Loss terms {L, L_e, L_f, L_v} without the backward pass."""
        terms = torch.empty(4, dtype=torch.float64, device="cuda")
        yc = y.c()
        check(_lib.load().gnep_loss(self.h, nl.h, C.byref(yc), _ptr(terms), _stream(stream)))
        return terms

    def get_grad(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """The model's FP64 gradient (the one adam_step applies)."""
        if out is None:
            out = torch.empty(self.n_params, dtype=torch.float64, device="cuda")
        assert out.dtype == torch.float64 and out.is_contiguous() and out.numel() == self.n_params
        check(_lib.load().gnep_get_grad(self.h, _ptr(out), self.n_params, _stream(stream)))
        return out

    def set_grad(self, g: torch.Tensor, stream=None):
        assert g.dtype == torch.float64 and g.is_contiguous() and g.numel() == self.n_params
        check(_lib.load().gnep_set_grad(self.h, _ptr(g), self.n_params, _stream(stream)))

    # optimiser --------------------------------------------------------------
    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        check(_lib.load().gnep_adam_step(self.h, lr, beta1, beta2, eps, weight_decay, _stream(stream)))

    def adam_step_scheduled(self, lr_start, lr_stop, n_warmup, n_total, beta1=0.9, beta2=0.999, eps=1e-8,
                            weight_decay=0.0, stream=None):
        check(_lib.load().gnep_adam_step_scheduled(self.h, lr_start, lr_stop, n_warmup, n_total, beta1, beta2,
                                                   eps, weight_decay, _stream(stream)))

    def step_count(self) -> int:
        t = C.c_int64()
        check(_lib.load().gnep_get_step(self.h, C.byref(t), _stream()))
        return t.value

    def sync_status(self):
        check(_lib.load().gnep_sync_status(self.h, _stream()))

    def save(self, path: str):
        check(_lib.load().gnep_save(self.h, path.encode()))

    def load(self, path: str):
        check(_lib.load().gnep_load(self.h, path.encode()))

    def close(self):
        if getattr(self, "h", None):
            _lib.load().gnep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lr_schedule(lr_start, lr_stop, s, n_warmup, n_total) -> float:
    """Eq. 17 (host scalar)."""
    return _lib.load().gnep_lr_schedule(lr_start, lr_stop, s, n_warmup, n_total)


class TrainGraph:
    """One captured training step (loss + gradient + scheduled Adam) replayed as
    a CUDA graph; with lists of neighbour lists and labels, that many steps in
    order (for instance an epoch of one-structure batches) in one graph, whose
    `loss` holds the loss terms of each step (shape [n_steps, 4])."""

    def __init__(self, model: GNEP, nl, y, lr_start, lr_stop, n_warmup, n_total,
                 beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        self.stream = stream or torch.cuda.Stream()
        steps = isinstance(nl, (list, tuple))
        nls, ys = (list(nl), list(y)) if steps else ([nl], [y])
        assert len(nls) == len(ys) and len(nls) >= 1
        self.loss = torch.zeros((len(nls), 4) if steps else (4,), dtype=torch.float64, device="cuda")
        self._keep = (model, nls, ys)
        h = C.c_void_p()
        torch.cuda.synchronize()
        if steps:
            self._yc = (_lib.Labels * len(ys))(*[yy.c() for yy in ys])
            self._nlh = (C.c_void_p * len(nls))(*[n.h.value for n in nls])
            check(_lib.load().gnep_graph_create_steps(model.h, self._nlh, self._yc, len(nls), _ptr(self.loss),
                                                      lr_start, lr_stop, n_warmup, n_total, beta1, beta2, eps,
                                                      weight_decay, C.c_void_p(self.stream.cuda_stream),
                                                      C.byref(h)))
        else:
            self._yc = y.c()
            check(_lib.load().gnep_graph_create(model.h, nl.h, C.byref(self._yc), _ptr(self.loss), lr_start,
                                                lr_stop, n_warmup, n_total, beta1, beta2, eps, weight_decay,
                                                C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def launch(self, stream=None):
        """Replay the step on `stream` (default: torch's current stream, so the
        replay is ordered with the caller's subsequent torch operations)."""
        s = stream if stream is not None else torch.cuda.current_stream()
        check(_lib.load().gnep_graph_launch(self.h, C.c_void_p(s.cuda_stream)))

    def kernel_count(self) -> int:
        """Kernels one replay launches."""
        n = C.c_int32()
        check(_lib.load().gnep_graph_kernel_count(self.h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            _lib.load().gnep_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GNEPLoss(torch.autograd.Function):
    """L(theta) of one batch with the library's analytic gradient as backward.

    forward(params, model, nl, labels) loads ``params`` into the model, runs
    gnep_loss_grad and stashes dL/dtheta; backward returns grad_output * dL/dtheta.
    """

    @staticmethod
    def forward(ctx, params, model: GNEP, nl: NeighborList, y: Labels):
        model.set_params(params.detach())
        terms, g = model.loss_grad(nl, y, grad=True)
        ctx.save_for_backward(g)
        return terms[0].to(params.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None
