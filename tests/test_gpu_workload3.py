"""The differentiation workload at full size: 1,000 structures of 64-256
atoms (about 160k atoms), the RMSE + L2 loss, the step behind
torch.autograd.Function, and 100 Adam steps (Eq. 17 schedule) that move a
random student toward a random teacher.  The gradient through the autograd
Function is the library's analytic gradient; its per-entry agreement with the
FP64 oracle is covered by the parity tests on smaller batches, and central
differences of the FP64 loss pin the oracle itself."""
import numpy as np
import pytest
import torch

from paper_2507_00528_gb300 import gnep, synth

pytestmark = pytest.mark.gpu

SHAPE = dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False)


def test_thousand_structures_autograd_and_training():
    b = synth.make_config(3)
    assert b.n_struct == 1000
    teacher = gnep.GNEP(**SHAPE, seed=101)
    nl = teacher.neighbors(gnep.DeviceBatch.from_host(b))
    teacher.compute_scale(nl)
    y = teacher.teacher_labels(nl, b.sizes(), lambda_e=1.0, lambda_f=1.0, lambda_v=0.1, lambda_l2=1e-4,
                               loss_form=gnep._lib.LOSS_RMSE)
    student = gnep.GNEP(**SHAPE, seed=7)
    student.set_scale(teacher.get_scale())
    p0 = student.get_params().double().clone().requires_grad_(True)
    loss = gnep.GNEPLoss.apply(p0, student, nl, y)
    loss.backward()
    _, g = student.loss_grad(nl, y)
    assert torch.allclose(p0.grad.float(), g)
    assert torch.isfinite(g).all() and g.abs().max() > 0

    steps = 100
    graph = gnep.TrainGraph(student, nl, y, 2e-3, 2e-5, 10, steps)
    losses = []
    for _ in range(steps):
        graph.launch()
        losses.append(graph.loss.cpu().numpy()[0])
    student.sync_status()
    losses = np.array(losses)
    print(f"{b.n_atoms} atoms: loss {losses[0]:.4f} -> {losses[-1]:.4f}")
    assert np.all(np.isfinite(losses))
    w = losses.reshape(10, 10).mean(1)
    assert np.sum(np.diff(w) < 0) >= 8, w
    assert losses[-1] < 0.6 * losses[0]
