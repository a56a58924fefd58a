"""Two neighbour lists used alternately, as a training loop that prepares the
next batch while the current one trains: a rebuild on a second stream while a
loss + gradient evaluation runs on the first must leave both results exactly as
when the same calls run one after another (the kernels are deterministic)."""
import numpy as np
import pytest
import torch

from paper_2507_00528_gb300 import gnep, synth

pytestmark = pytest.mark.gpu

SHAPE = dict(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True)


def _moved(b, seed):
    """The same structures with every atom displaced (up to 0.2 A) and wrapped."""
    rng = np.random.default_rng(seed)
    pos = b.pos + rng.uniform(-0.2, 0.2, b.pos.shape)
    out = []
    for s in range(b.n_struct):
        a0, a1 = b.struct_off[s], b.struct_off[s + 1]
        H = b.cell[s]
        f = pos[a0:a1] @ np.linalg.inv(H)
        out.append((f - np.floor(f)) @ H)
    return synth.Batch(b.struct_off.copy(), np.concatenate(out), b.types.copy(), b.cell.copy())


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rebuild_beside_training_step(precision):
    a = synth.make_config(2, n_struct=24)
    bb = _moved(a, 5)
    m = gnep.GNEP(**SHAPE, seed=11, precision=precision)
    nl_a = m.neighbors(gnep.DeviceBatch.from_host(a))
    m.compute_scale(nl_a)
    nl_b_ref = m.neighbors(gnep.DeviceBatch.from_host(bb))
    y_a = m.teacher_labels(nl_a, a.sizes())
    y_b = m.teacher_labels(nl_b_ref, bb.sizes())
    m.set_params(torch.from_numpy(synth.uniform_params(m.n_params, 7)))
    # one after another
    ta, ga = m.loss_grad(nl_a, y_a)
    tb, gb = m.loss_grad(nl_b_ref, y_b)
    torch.cuda.synchronize()
    ta, ga, tb, gb = (x.cpu().clone() for x in (ta, ga, tb, gb))
    # the second list starts on batch a and is rebuilt for batch b while batch a trains
    nl_b = m.neighbors(gnep.DeviceBatch.from_host(a))
    s_train, s_load = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        ta2, ga2 = m.loss_grad(nl_a, y_a, stream=s_train)
        nl_b.rebuild(bb, stream=s_load)
        s_train.wait_stream(s_load)
        tb2, gb2 = m.loss_grad(nl_b, y_b, stream=s_train)
        s_train.synchronize()
        m.sync_status()
        assert torch.equal(ta2.cpu(), ta) and torch.equal(ga2.cpu(), ga)
        assert torch.equal(tb2.cpu(), tb) and torch.equal(gb2.cpu(), gb)
        nl_b.rebuild(a, stream=s_load)  # back to batch a for the next round
        s_load.synchronize()
    for w in (0, 1):
        for x, y in zip(nl_b.export(w), nl_a.export(w)):
            np.testing.assert_array_equal(x, y)


def test_calls_on_other_streams_wait_for_a_rebuild():
    """A rebuild returns with its compaction, reverse entries and tile upload
    still queued on its stream; calls that read the list on other streams (a
    loss + gradient, a list export on the default stream) must see the new
    lists without any wait by the caller."""
    a = synth.make_config(2, n_struct=24)
    bb = _moved(a, 6)
    m = gnep.GNEP(**SHAPE, seed=12, precision="fp32")
    nl = m.neighbors(gnep.DeviceBatch.from_host(a))
    m.compute_scale(nl)
    ref = m.neighbors(gnep.DeviceBatch.from_host(bb))
    y = m.teacher_labels(ref, bb.sizes())
    t_ref, g_ref = m.loss_grad(ref, y)
    torch.cuda.synchronize()
    t_ref, g_ref = t_ref.cpu().clone(), g_ref.cpu().clone()
    lists_ref = [ref.export(w) for w in (0, 1)]
    s_load, s_use = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        nl.rebuild(bb, stream=s_load)
        t, g = m.loss_grad(nl, y, stream=s_use)
        for w in (0, 1):
            for x, z in zip(nl.export(w), lists_ref[w]):
                np.testing.assert_array_equal(x, z)
        s_use.synchronize()
        assert torch.equal(t.cpu(), t_ref) and torch.equal(g.cpu(), g_ref)
        nl.rebuild(a, stream=s_load)  # and back, for the next round
        s_load.synchronize()
    m.sync_status()
