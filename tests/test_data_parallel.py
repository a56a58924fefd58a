"""Data-parallel decomposition of one training step over ranks (gloo, CPU).

Each of two ranks holds a shard of the structures, forms its loss weights
from the whole-batch counts (and, for the RMSE form, the whole-batch MSE
gathered by an all-reduce), computes its shard's MSE-form gradient with the
FP64 oracle and all-reduces it.  The summed gradient and the loss must equal
the oracle's whole-batch values: the host logic the GPU data-parallel step
runs between its kernels is checked without a GPU.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2507_00528_gb300 import data_parallel as dp
from paper_2507_00528_gb300 import synth

CFG = dict(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30, four_body=False)


@pytest.fixture(scope="module", autouse=True)
def _library():
    """The shard-weight arithmetic lives in libgnep (host-side entry points)."""
    from paper_2507_00528_gb300 import build
    build.build()


def _problem(form):
    rng = np.random.default_rng(44)
    b = synth.make_batch([9, 14, 6, 11, 8], [0, 1, 2, 1, 0], rng)
    cfg = O.Cfg(**CFG)
    T = synth.uniform_params(cfg.n_params, 12).astype(np.float64)
    P = synth.uniform_params(cfg.n_params, 11).astype(np.float64)
    s = O.descriptor_scale(cfg, T, b)
    y = O.teacher_labels(cfg, T, s, b, lambda_e=0.7, lambda_f=1.3, lambda_v=0.4, lambda_l2=0.02, loss_form=form)
    return b, cfg, P, s, y


def _sub_labels(y, b, idx, **kw):
    rows = np.concatenate([np.arange(b.struct_off[i], b.struct_off[i + 1]) for i in idx])
    fields = dict(lambda_e=y.lambda_e, lambda_f=y.lambda_f, lambda_v=y.lambda_v, lambda_l2=y.lambda_l2,
                  loss_form=y.loss_form)
    fields.update(kw)
    return O.Labels(y.energy[idx], y.force[rows], y.virial[idx], **fields)


def _worker(rank, world, port, form, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, cfg, P, s, y = _problem(form)
        shards = dp.shard_structures(b.sizes(), world)
        idx = shards[rank]
        sub = b.subset(idx)
        local = dp.Counts(len(idx), int(sub.n_atoms))
        total = dp.Counts(b.n_struct, int(b.n_atoms))

        def reduce_sum(v):
            t = torch.as_tensor(np.asarray(v, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        mse = None
        if form == dp.LOSS_RMSE:
            t = O.loss(cfg, P, s, sub, _sub_labels(y, b, idx))
            mse = dp.combine_mse(t[1:], local, reduce_sum)
        le, lf, lv, l2 = dp.effective_weights(y.lambda_e, y.lambda_f, y.lambda_v, y.lambda_l2, form, local, total,
                                              mse, rank)
        yr = _sub_labels(y, b, idx, lambda_e=le, lambda_f=lf, lambda_v=lv, lambda_l2=l2, loss_form=dp.LOSS_MSE)
        t, g = O.loss_grad(cfg, P, s, sub, yr)
        g = reduce_sum(g)
        if mse is None:
            mse = dp.combine_mse(t[1:], local, reduce_sum)
        if rank == 0:
            l2_term = y.lambda_l2 * float(np.sum(P * P)) / cfg.n_params
            L = dp.total_loss(y.lambda_e, y.lambda_f, y.lambda_v, form, mse, l2_term)
            np.savez(out, g=g, L=L, mse=mse)
    finally:
        dist.destroy_process_group()


def _port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("form", [dp.LOSS_MSE, dp.LOSS_RMSE])
def test_two_rank_gradient_equals_whole_batch(form):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r0.npz")
        mp.spawn(_worker, args=(2, _port(), form, out), nprocs=2, join=True)
        r = np.load(out)
        b, cfg, P, s, y = _problem(form)
        t, g = O.loss_grad(cfg, P, s, b, y)
        np.testing.assert_allclose(r["mse"], t[1:], rtol=1e-12)
        assert abs(float(r["L"]) - t[0]) <= 1e-12 * abs(t[0])
        assert np.linalg.norm(r["g"] - g) <= 1e-11 * np.linalg.norm(g)


def test_shards_are_balanced_disjoint_and_deterministic():
    rng = np.random.default_rng(5)
    cost = rng.integers(32, 401, size=256)
    for world in (1, 2, 3, 8):
        sh = dp.shard_structures(cost, world)
        allidx = np.sort(np.concatenate(sh))
        np.testing.assert_array_equal(allidx, np.arange(256))
        loads = np.array([cost[s].sum() for s in sh])
        assert loads.max() - loads.min() <= cost.max()  # greedy bound
        sh2 = dp.shard_structures(cost, world)
        assert all(np.array_equal(a, c) for a, c in zip(sh, sh2))


def test_effective_weights_single_rank_is_identity():
    w = dp.effective_weights(0.5, 2.0, 0.3, 0.05, dp.LOSS_MSE, dp.Counts(7, 90), dp.Counts(7, 90))
    assert w == (0.5, 2.0, 0.3, 0.05)
    w = dp.effective_weights(1.0, 1.0, 1.0, 0.0, dp.LOSS_RMSE, dp.Counts(3, 30), dp.Counts(6, 90),
                             mse_total=[4.0, 0.0, 0.25], rank=1)
    assert w == pytest.approx((0.5 * 0.25, 0.0, 0.5 * 1.0, 0.0))


def test_shard_entry_points_by_hand():
    """gnep_shard_mse_partials / gnep_shard_mse_total on hand values: two
    shards (2 structures, 30 atoms; 1 structure, 10 atoms) with MSEs
    (4, 1, 9) and (1, 4, 0) combine to the count-weighted means of Eqs. 10-12."""
    a = dp.combine_mse([4.0, 1.0, 9.0], dp.Counts(2, 30), lambda v: v + np.array([1.0 * 1, 4.0 * 30, 0.0, 1, 10]))
    np.testing.assert_allclose(a, [(4.0 * 2 + 1.0) / 3, (1.0 * 90 + 4.0 * 30) / 120, 9.0 * 12 / 18], rtol=1e-15)
    w = dp.effective_weights(2.0, 3.0, 0.5, 0.1, dp.LOSS_MSE, dp.Counts(1, 10), dp.Counts(4, 50), rank=2)
    assert w == pytest.approx((0.5, 0.6, 0.125, 0.0), rel=1e-15)
    with pytest.raises(Exception):
        dp.effective_weights(1.0, 1.0, 1.0, 0.0, dp.LOSS_RMSE, dp.Counts(1, 10), dp.Counts(4, 50))
