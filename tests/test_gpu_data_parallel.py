"""The data-parallel step on the GPU: two gloo ranks, one process each, share
the one GPU (their kernels never wait on each other; the gradient is summed
over ranks on the host).  Each rank runs DataParallelStep on its shard of the
structures (balanced by radial plus angular pairs) with the shard loss
weights of the C ABI; the summed gradient, the whole-batch loss and the
updated parameters must equal the single-process whole-batch step, and both
replicas must hold the same parameters afterwards."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2507_00528_gb300 import data_parallel as dp
from paper_2507_00528_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPE = dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False)
CFG = dict(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30, four_body=False)
LR = (1e-3, 1e-5, 2, 10)


def _problem(form):
    b = synth.make_batch([40, 21, 33, 17, 28, 12], [0, 1, 2, 1, 0, 2], np.random.default_rng(45))
    cfg = O.Cfg(**CFG)
    T = synth.uniform_params(cfg.n_params, 12)
    P = synth.uniform_params(cfg.n_params, 11)
    s = O.descriptor_scale(cfg, T.astype(np.float64), b).astype(np.float32)
    y = O.teacher_labels(cfg, T.astype(np.float64), s.astype(np.float64), b, lambda_e=0.7, lambda_f=1.3,
                         lambda_v=0.4, lambda_l2=0.02, loss_form=form)
    return b, P, s, y


def _labels(y, b, idx, torch, gnep):
    rows = np.concatenate([np.arange(b.struct_off[i], b.struct_off[i + 1]) for i in idx])
    return gnep.Labels(torch.tensor(y.energy[idx], device="cuda"),
                       torch.tensor(y.force[rows], dtype=torch.float32, device="cuda").contiguous(),
                       torch.tensor(y.virial[idx], device="cuda").contiguous(),
                       y.lambda_e, y.lambda_f, y.lambda_v, y.lambda_l2, y.loss_form)


def _model(P, s, torch, gnep):
    m = gnep.GNEP(**SHAPE)
    m.set_params(torch.from_numpy(P))
    m.set_scale(torch.from_numpy(s))
    return m


def _worker(rank, world, port, form, shards, out):
    import torch
    import torch.distributed as dist
    from paper_2507_00528_gb300 import gnep
    torch.cuda.set_device(0)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, P, s, y = _problem(form)
        idx = shards[rank]
        sub = b.subset(idx)
        m = _model(P, s, torch, gnep)
        nl = m.neighbors(gnep.DeviceBatch.from_host(sub))
        step = dp.DataParallelStep(m, nl, _labels(y, b, idx, torch, gnep), dp.Counts(len(idx), int(sub.n_atoms)),
                                   dp.Counts(b.n_struct, int(b.n_atoms)))
        L = step.step(*LR)
        m.sync_status()
        np.savez(out.format(rank), g=m.get_grad().cpu().numpy(), p=m.get_params().cpu().numpy(), L=L)
    finally:
        dist.destroy_process_group()


def _port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("form", [dp.LOSS_MSE, dp.LOSS_RMSE])
def test_two_ranks_on_one_gpu_equal_the_whole_batch_step(form):
    import torch
    import torch.multiprocessing as mp
    from paper_2507_00528_gb300 import gnep
    b, P, s, y = _problem(form)
    m = _model(P, s, torch, gnep)
    nl = m.neighbors(gnep.DeviceBatch.from_host(b))
    shards = dp.shard_structures(dp.structure_costs(nl), 2)
    assert all(len(sh) > 0 for sh in shards)
    terms, _ = m.loss_grad(nl, _labels(y, b, np.arange(b.n_struct), torch, gnep), grad=False)
    g_ref = m.get_grad().cpu().numpy()
    m.adam_step_scheduled(*LR)
    p_ref = m.get_params().cpu().numpy()
    m.sync_status()
    l2 = y.lambda_l2 * float(np.sum(P.astype(np.float64) ** 2)) / len(P)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r{}.npz")
        mp.spawn(_worker, args=(2, _port(), form, shards, out), nprocs=2, join=True)
        r0, r1 = np.load(out.format(0)), np.load(out.format(1))
    np.testing.assert_array_equal(r0["g"], r1["g"])
    np.testing.assert_array_equal(r0["p"], r1["p"])
    assert np.linalg.norm(r0["g"] - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
    L_ref = float(terms.cpu().numpy()[0])
    assert abs(float(r0["L"]) + l2 - L_ref) <= 1e-6 * abs(L_ref)
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()  # Adam's sign of tiny entries follows rounding
    np.testing.assert_allclose(r0["p"][big], p_ref[big], rtol=0, atol=1e-6)
