"""Data-parallel training over structures (one process per GPU).

Structures are independent (Eq. 1 sums over them), so a batch is split by
structure across ranks and each rank runs the whole step on its shard.  The
loss normalisers of Eqs. 10-12 (structure count N_str and atom count N) are
those of the whole batch, and the RMSE form needs the whole-batch MSE before
any gradient is formed.  Both are folded into per-rank loss weights, so each
rank's call of the library computes exactly its share of the whole-batch
gradient; one sum over ranks (all-reduce) then gives the gradient every
replica applies in the same Adam step.

For a shard with S_r structures and N_r atoms of a batch with S and N:
    MSE form:   lambda_e' = lambda_e S_r / S,   lambda_f' = lambda_f N_r / N,
                lambda_v' = lambda_v S_r / S
    RMSE form:  the MSE weights above times 1 / (2 sqrt(L_x)) with L_x the
                whole-batch MSE of term x (zero weight when L_x = 0),
and the L2 term is carried by rank 0 alone.  With these weights the shard's
MSE-form gradient is its exact contribution to the whole-batch gradient.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LOSS_MSE, LOSS_RMSE = 0, 1


def shard_structures(cost, world: int) -> list[np.ndarray]:
    """Split structures over `world` ranks, balancing the summed cost (atoms x
    neighbours, or atoms): largest first to the least-loaded rank, ties to
    the lower rank.  Each shard lists its structures in ascending order."""
    cost = np.asarray(cost, dtype=np.float64)
    load = np.zeros(world)
    owner = np.empty(len(cost), dtype=np.int64)
    for s in sorted(range(len(cost)), key=lambda k: (-cost[k], k)):
        r = int(np.argmin(load))
        owner[s] = r
        load[r] += cost[s]
    return [np.nonzero(owner == r)[0] for r in range(world)]


@dataclass
class Counts:
    n_struct: int
    n_atoms: int


def _f64(v):
    return np.ascontiguousarray(v, dtype=np.float64)


def combine_mse(local_terms, local: Counts, reduce_sum) -> np.ndarray:
    """Whole-batch (Le, Lf, Lv) from each rank's shard MSEs (Eqs. 10-12):
    count-weighted sums over ranks (gnep_shard_mse_partials, then
    gnep_shard_mse_total).  `reduce_sum` sums a float64 vector over ranks (an
    all-reduce)."""
    from . import _lib
    L = _lib.load()
    terms = _f64(np.asarray(local_terms, dtype=np.float64)[:3])
    part = np.zeros(5)
    _lib.check(L.gnep_shard_mse_partials(terms.ctypes.data, local.n_struct, local.n_atoms, part.ctypes.data))
    sums = _f64(reduce_sum(part))
    out = np.zeros(3)
    _lib.check(L.gnep_shard_mse_total(sums.ctypes.data, out.ctypes.data))
    return out


def effective_weights(lam_e, lam_f, lam_v, lam_l2, form, local: Counts, total: Counts, mse_total=None,
                      rank: int = 0):
    """Per-rank MSE-form loss weights (lambda_e', lambda_f', lambda_v', lambda_l2')
    whose gradient is the shard's exact share of the whole-batch gradient
    (gnep_shard_loss_weights)."""
    from . import _lib
    L = _lib.load()
    mse = None if mse_total is None else _f64(mse_total)
    out = np.zeros(4)
    _lib.check(L.gnep_shard_loss_weights(float(lam_e), float(lam_f), float(lam_v), float(lam_l2), int(form),
                                         local.n_struct, local.n_atoms, total.n_struct, total.n_atoms,
                                         None if mse is None else mse.ctypes.data, int(rank), out.ctypes.data))
    return tuple(float(x) for x in out)


def structure_costs(nl) -> np.ndarray:
    """Per-structure cost for shard balancing: atoms x neighbours, i.e. the
    structure's radial plus angular pair count, from a neighbour list built
    over the whole batch (NeighborList of gnep.py)."""
    offR = nl.export(0)[0].astype(np.int64)
    offA = nl.export(1)[0].astype(np.int64)
    soff = np.asarray(nl.struct_off_host, dtype=np.int64)
    return (offR[soff[1:]] - offR[soff[:-1]]) + (offA[soff[1:]] - offA[soff[:-1]])


def total_loss(lam_e, lam_f, lam_v, form, mse_total, l2_term=0.0) -> float:
    """Eq. 9 (or its RMSE form) from the whole-batch MSE terms."""
    f = np.sqrt if form == LOSS_RMSE else (lambda x: x)
    Le, Lf, Lv = mse_total
    return float(lam_e * f(Le) + lam_f * f(Lf) + lam_v * f(Lv) + l2_term)


class DataParallelStep:
    """One training step of a shard on this rank's GPU, with the gradient
    summed over ranks by torch.distributed (NCCL, or gloo through host
    copies) before the Adam update.

    ``model`` is a GNEP, ``nl`` the neighbour list of this rank's shard and
    ``y`` its labels (gnep.Labels with the whole-batch loss weights); ``local``
    and ``total`` are the shard and batch counts."""

    def __init__(self, model, nl, y, local: Counts, total: Counts):
        import torch
        import torch.distributed as dist
        from . import gnep
        self.torch, self.dist, self.gnep = torch, dist, gnep
        self.model, self.nl, self.y = model, nl, y
        self.local, self.total = local, total
        self.rank = dist.get_rank() if dist.is_initialized() else 0
        self.grad = torch.zeros(model.n_params, dtype=torch.float64, device="cuda")

    def _on_host(self):
        """gloo reduces host tensors; NCCL device tensors."""
        return self.dist.is_initialized() and self.dist.get_backend() == "gloo"

    def _reduce(self, v):
        dev = "cpu" if self._on_host() else "cuda"
        t = self.torch.as_tensor(np.asarray(v, dtype=np.float64), dtype=self.torch.float64, device=dev)
        if self.dist.is_initialized():
            self.dist.all_reduce(t)
        return t.cpu().numpy()

    def step(self, lr_start, lr_stop, n_warmup, n_total, want_loss=True):
        """One step; returns the whole-batch loss (Eq. 9, without the L2 term)
        when `want_loss`, else None.  The MSE form makes no host round trip
        unless the loss is asked for; the RMSE form needs one (the whole-batch
        MSE sets the loss weights)."""
        y, gnep = self.y, self.gnep
        mse = None
        if y.loss_form == LOSS_RMSE:
            terms = self.model.loss(self.nl, y)
            mse = combine_mse(terms.cpu().numpy()[1:], self.local, self._reduce)
        le, lf, lv, l2 = effective_weights(y.lambda_e, y.lambda_f, y.lambda_v, y.lambda_l2, y.loss_form,
                                           self.local, self.total, mse, self.rank)
        yr = gnep.Labels(y.energy, y.force, y.virial, le, lf, lv, l2, LOSS_MSE)
        terms, _ = self.model.loss_grad(self.nl, yr, grad=False)
        self.model.get_grad(self.grad)
        if self.dist.is_initialized():
            if self._on_host():
                g = self.grad.cpu()
                self.dist.all_reduce(g)
                self.grad.copy_(g)
            else:
                self.dist.all_reduce(self.grad)
        self.model.set_grad(self.grad)
        self.model.adam_step_scheduled(lr_start, lr_stop, n_warmup, n_total)
        if not want_loss:
            return None
        if mse is None:
            mse = combine_mse(terms.cpu().numpy()[1:], self.local, self._reduce)
        return total_loss(y.lambda_e, y.lambda_f, y.lambda_v, y.loss_form, mse)
