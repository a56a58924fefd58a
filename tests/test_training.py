"""Training with the library's own kernels: 300 Adam steps (Eq. 17 schedule)
on the RMSE + L2 loss move a random student toward a random teacher.  On
held-out structures the trained network beats the predictors that have no
network: the best linear fit of per-atom energy on the structure-averaged
descriptors (ridge, fitted on the training energies), and the zero force."""
import numpy as np
import pytest
import torch

from paper_2507_00528_gb300 import gnep, synth

pytestmark = pytest.mark.gpu

SHAPE = dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False)


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(64, 257, size=n)
    return synth.make_batch(sizes, np.arange(n) % 3, rng)


def _energy_rmse(model, nl, y, sizes):
    _, Es, _, _ = model.forward(nl)
    pred = Es.cpu().numpy() / sizes
    return float(np.sqrt(np.mean((pred - y.energy.cpu().numpy()) ** 2)))


def _ridge_baseline(model, nl, y, sizes, nl_test, y_test, sizes_test, alpha=1e-6):
    """Per-atom energy ~ w . mean_i(G_i) + b, fitted on the training set."""
    def feats(nl_, sizes_):
        G = model.descriptors(nl_).double().cpu().numpy()
        off = np.concatenate([[0], np.cumsum(sizes_)]).astype(int)
        X = np.stack([G[off[s]:off[s + 1]].mean(0) for s in range(len(sizes_))])
        return np.hstack([X, np.ones((len(X), 1))])
    X = feats(nl, sizes)
    t = y.energy.cpu().numpy()
    w = np.linalg.solve(X.T @ X + alpha * np.eye(X.shape[1]), X.T @ t)
    Xt = feats(nl_test, sizes_test)
    return float(np.sqrt(np.mean((Xt @ w - y_test.energy.cpu().numpy()) ** 2)))


def test_adam_training_converges_and_beats_no_network_baseline():
    train, test = _batch(24, 3), _batch(8, 4)
    teacher = gnep.GNEP(**SHAPE, seed=101)
    nl_tr = teacher.neighbors(gnep.DeviceBatch.from_host(train))
    nl_te = teacher.neighbors(gnep.DeviceBatch.from_host(test))
    teacher.compute_scale(nl_tr)
    lam = dict(lambda_e=1.0, lambda_f=1.0, lambda_v=0.1, lambda_l2=1e-4, loss_form=gnep._lib.LOSS_RMSE)
    y_tr = teacher.teacher_labels(nl_tr, train.sizes(), **lam)
    y_te = teacher.teacher_labels(nl_te, test.sizes(), **lam)

    student = gnep.GNEP(**SHAPE, seed=7)
    student.set_scale(teacher.get_scale())
    rmse_e0 = _energy_rmse(student, nl_te, y_te, test.sizes())
    _, _, F0, _ = (t.cpu().numpy() for t in student.forward(nl_te))
    ridge = _ridge_baseline(student, nl_tr, y_tr, train.sizes(), nl_te, y_te, test.sizes())

    losses = []
    steps = 300
    g = gnep.TrainGraph(student, nl_tr, y_tr, 5e-3, 5e-5, 10, steps)
    for _ in range(steps):
        g.launch()
        losses.append(g.loss.cpu().numpy()[0])  # ordered after the replay on the current stream
    student.sync_status()
    losses = np.array(losses)
    assert np.all(np.isfinite(losses))
    # converges toward the teacher: window averages fall and the end is far below the start
    w = losses.reshape(10, 30).mean(1)
    assert np.sum(np.diff(w) < 0) >= 8, w
    assert w[-1] < 0.25 * losses[0], (losses[0], w)

    rmse_e = _energy_rmse(student, nl_te, y_te, test.sizes())
    _, _, F1, _ = (t.cpu().numpy() for t in student.forward(nl_te))
    Fte = y_te.force.cpu().numpy()
    rmse_f0 = np.sqrt(np.mean((F0 - Fte) ** 2))
    rmse_f1 = np.sqrt(np.mean((F1 - Fte) ** 2))
    rmse_f_zero = np.sqrt(np.mean(Fte ** 2))
    print(f"energy RMSE test: untrained {rmse_e0:.4g}, ridge on descriptors {ridge:.4g}, trained {rmse_e:.4g}; "
          f"force RMSE: zero {rmse_f_zero:.4g}, untrained {rmse_f0:.4g}, trained {rmse_f1:.4g}; "
          f"loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    assert rmse_e < 0.5 * ridge, (rmse_e, ridge)
    assert rmse_f1 < 0.3 * rmse_f_zero and rmse_f1 < 0.3 * rmse_f0, (rmse_f1, rmse_f_zero, rmse_f0)
