"""Tensor-core network modes (TF32 and BF16 operands, FP32 accumulation in
tensor memory) against the FP64 oracle and against the plain FP32 GPU form.

The error bounds are multiples of the operand rounding unit u (2^-11 for
TF32, 2^-8 for BF16; round to nearest).  Each network contraction rounds its
operands once, so energies, forces, virials and the loss carry relative
errors of order u, and the gradient (which also rounds alpha and beta before
the contractions over atoms) of order 2u.  Measured on the cases below:
energies <= 1.3u, forces and virials <= 1.4u, gradients <= 1.7u; the bounds
are those with a factor of about 2 to spare.  The measured errors are printed.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2507_00528_gb300 import gnep, synth

from gpu_common import Case, rel_l2, small_cells_batch

pytestmark = pytest.mark.gpu

U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}
# multiples of u: per-atom energy, force / virial, gradient (relative L2)
K_E, K_F, K_G = 3.0, 3.0, 4.0


def _case(shape, batch, mode, **kw):
    c = Case(shape, batch, **kw)
    c.m.set_precision(mode)
    return c


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("shape,which", [("nmax4_basis8_h30", "cfg1"), ("nmax8_basis12_h50_4b", "small_cells"),
                                         ("nmax8_basis12_h100", "small_cells")])
def test_forward_within_rounding_bound(mode, shape, which):
    b = synth.make_config(1) if which == "cfg1" else small_cells_batch()
    c = _case(shape, b, mode, labels=False)
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    u = U[mode]
    errs = dict(E=rel_l2(Ea, Eao), F=rel_l2(F, Fo), W=rel_l2(W, Wo))
    print(mode, shape, {k: f"{v:.2e}" for k, v in errs.items()}, f"u={u:.2e}")
    assert errs["E"] < K_E * u and errs["F"] < K_F * u and errs["W"] < K_F * u, errs
    # the plain FP32 form on the same inputs differs (the tensor-core path ran)
    c.m.set_precision("fp32")
    Ea32 = c.m.forward(c.nl)[0].double().cpu().numpy()
    assert rel_l2(Ea32, Eao) < 1e-6 and rel_l2(Ea, Ea32) > 0


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("shape,lambdas,form", [("nmax4_basis8_h30", (1.0, 1.0, 0.1, 0.0), 0),
                                                ("nmax8_basis12_h50_4b", (1.0, 1.0, 0.1, 0.0), 0),
                                                ("nmax8_basis12_h100", (1.0, 1.0, 0.1, 0.01), 1)])
def test_gradient_within_rounding_bound(mode, shape, lambdas, form):
    b = synth.make_batch([20, 13], [2, 1], np.random.default_rng(7))
    c = _case(shape, b, mode, lambdas=lambdas, loss_form=form)
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.sync_status()
    ref_terms, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    u = U[mode]
    eg = rel_l2(g.cpu().numpy(), ref_g)
    el = abs(terms.cpu().numpy()[0] - ref_terms[0]) / abs(ref_terms[0])
    print(mode, shape, f"grad {eg:.2e} loss {el:.2e} u={u:.2e}")
    assert eg < K_G * u and el < K_F * u, (eg, el)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_many_tiles_species_switches_and_determinism(mode):
    """12 structures (~2,500 atoms): several 128-atom tiles per species, blocks
    that switch species, ragged last tiles; against the FP32 GPU form, and
    bit-identical on repetition."""
    b = synth.make_config(2, n_struct=12)
    c = Case("nmax8_basis12_h50_4b", b.subset([0]), labels=False)
    nl = c.m.neighbors(gnep.DeviceBatch.from_host(b))
    c.m.compute_scale(nl)
    y = c.m.teacher_labels(nl, b.sizes())
    c.m.set_params(torch.from_numpy(synth.uniform_params(c.cfg.n_params, 5)))
    t32, g32 = c.m.loss_grad(nl, y)
    F32 = c.m.forward(nl)[2].double().cpu().numpy()
    c.m.set_precision(mode)
    t1, g1 = c.m.loss_grad(nl, y)
    t2, g2 = c.m.loss_grad(nl, y)
    c.m.sync_status()
    assert torch.equal(g1, g2) and torch.equal(t1, t2)
    F1 = c.m.forward(nl)[2].double().cpu().numpy()
    u = U[mode]
    eg, ef = rel_l2(g1.cpu().numpy(), g32.cpu().numpy()), rel_l2(F1, F32)
    print(mode, f"grad vs fp32 {eg:.2e} force vs fp32 {ef:.2e}")
    assert eg < K_G * u and ef < K_F * u


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_one_species_only_and_single_atom(mode):
    """A batch whose atoms are all of one species (no tiles for the other) and
    a one-atom structure."""
    rng = np.random.default_rng(21)
    b = synth.make_batch([40, 1], [1, 1], rng)
    b.types[:] = 1
    c = _case("nmax4_basis8_h30", b, mode, scale_batch=synth.make_config(1, n_struct=2))
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.sync_status()
    ref_terms, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    assert rel_l2(g.cpu().numpy(), ref_g) < K_G * U[mode]
    # the network of species 0 saw no atom: its gradient is exactly zero (no L2 term here)
    net_size = c.cfg.n_des * c.cfg.hidden + 2 * c.cfg.hidden + 1
    assert np.all(g.cpu().numpy()[:net_size] == 0) and np.all(ref_g[:net_size] == 0)


def test_precision_switch_rejects_wide_hidden_layer():
    m = gnep.GNEP(n_max=(4, 4), basis=(8, 8), hidden=120)
    with pytest.raises(gnep._lib.GnepError):
        m.set_precision("bf16")
    m.set_precision("fp32")
