"""Shared set-up of the GPU parity tests: the same seeded inputs for both sides."""
import numpy as np
import torch

import oracle as O
from paper_2507_00528_gb300 import gnep, synth

# Model shapes of the workloads: oracle configuration and library arguments.
SHAPES = {
    "nmax4_basis8_h30": (O.Cfg(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30, four_body=False),
                         dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False)),
    "nmax8_basis12_h50_4b": (O.Cfg(nq_r=9, nq_a=9, k_r=13, k_a=13, hidden=50, four_body=True),
                             dict(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True)),
    "nmax8_basis12_h100": (O.Cfg(nq_r=9, nq_a=9, k_r=13, k_a=13, hidden=100, four_body=False),
                           dict(n_max=(8, 8), basis=(12, 12), hidden=100, four_body=False)),
    "nmax4_basis8_lmax6_h30": (O.Cfg(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30, four_body=False, l_max=6),
                               dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False, l_max=6)),
    "nmax4_basis8_lmax8_4b_h30": (O.Cfg(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30, four_body=True, l_max=8),
                                  dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=True, l_max=8)),
}


class Case:
    """Oracle inputs (FP64 copies of the float32 values the GPU gets) and the GPU model."""

    def __init__(self, shape, batch, seed_p=11, seed_t=12, lambdas=(1.0, 1.0, 0.1, 0.0), loss_form=0,
                 labels=True, model_kw=None, scale_batch=None):
        self.cfg, kw = SHAPES[shape]
        if model_kw:
            kw = dict(kw, **model_kw)
        self.batch = batch
        self.P = synth.uniform_params(self.cfg.n_params, seed_p)
        self.T = synth.uniform_params(self.cfg.n_params, seed_t)
        sb = batch if scale_batch is None else scale_batch
        self.scale = O.descriptor_scale(self.cfg, self.T.astype(np.float64), sb).astype(np.float32)
        self.P64 = self.P.astype(np.float64)
        self.s64 = self.scale.astype(np.float64)
        le, lf, lv, l2 = lambdas
        if labels:
            y = O.teacher_labels(self.cfg, self.T.astype(np.float64), self.s64, batch, lambda_e=le,
                                 lambda_f=lf, lambda_v=lv, lambda_l2=l2, loss_form=loss_form)
            y.force = y.force.astype(np.float32).astype(np.float64)  # the GPU takes float32 forces
            self.y = y
        self.m = gnep.GNEP(**kw)
        self.m.set_params(torch.from_numpy(self.P))
        self.m.set_scale(torch.from_numpy(self.scale))
        self.nl = self.m.neighbors(gnep.DeviceBatch.from_host(batch))

    def gpu_labels(self):
        y = self.y
        return gnep.Labels(torch.tensor(y.energy, device="cuda"),
                           torch.tensor(y.force, dtype=torch.float32, device="cuda").contiguous(),
                           torch.tensor(y.virial, device="cuda").contiguous(),
                           y.lambda_e, y.lambda_f, y.lambda_v, y.lambda_l2, y.loss_form)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def small_cells_batch(seed=3):
    """Mixed phases with cells smaller than 2 r_c (several images of one j)."""
    return synth.make_batch([32, 17, 40, 9], [1, 2, 0, 2], np.random.default_rng(seed))
