"""Autotuned and hand-set launch shapes of the angular sweeps: parity with the
FP64 oracle holds under any tiling, the tuner keeps values in range, and a
graph captured before retuning refuses to launch."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2507_00528_gb300 import gnep, synth

from gpu_common import Case, rel_l2

pytestmark = pytest.mark.gpu


def test_small_tiles_match_oracle():
    b = synth.make_batch([20, 13, 9], [2, 1, 0], np.random.default_rng(17))
    c = Case("nmax8_basis12_h50_4b", b)
    y = c.gpu_labels()
    _, g_default = c.m.loss_grad(c.nl, y)
    c.nl.set_tuning(dict(desc_tile_atoms=3, desc_tile_pairs=16, force_tile_atoms=2, force_tile_pairs=8,
                         cgrad_blocks=2))
    t = c.nl.tuning()
    assert t["desc_tile_pairs"] == 16 and t["force_tile_atoms"] == 2 and t["cgrad_blocks"] == 2
    terms, g = c.m.loss_grad(c.nl, y)
    c.m.sync_status()
    _, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    assert rel_l2(g.cpu().numpy(), ref_g) < 1e-4
    assert rel_l2(g.cpu().numpy(), g_default.cpu().numpy()) < 1e-5
    c.nl.set_tuning(None)  # back to the defaults
    assert c.nl.tuning()["desc_tile_pairs"] > 16


def test_autotune_in_range_and_invalidates_graphs():
    b = synth.make_config(2, n_struct=12)
    c = Case("nmax8_basis12_h50_4b", b.subset([0]), labels=False)
    nl = c.m.neighbors(gnep.DeviceBatch.from_host(b))
    c.m.compute_scale(nl)
    y = c.m.teacher_labels(nl, b.sizes())
    c.m.set_params(torch.from_numpy(synth.uniform_params(c.cfg.n_params, 5)))
    _, g0 = c.m.loss_grad(nl, y)
    g = gnep.TrainGraph(c.m, nl, y, 1e-3, 1e-5, 2, 10)
    before = nl.tuning()
    after = nl.autotune(y, reps=2)
    print("tuning", before, "->", after)
    assert 1 <= after["desc_tile_atoms"] <= before["desc_tile_atoms"]
    assert 1 <= after["force_tile_atoms"] <= before["force_tile_atoms"]
    assert after["desc_tile_pairs"] >= 1 and after["force_tile_pairs"] >= 1
    assert 1 <= after["cgrad_blocks"] <= 608
    assert after["radial_lanes"] in (4, 8, 16) and after["net_tile_atoms"] in (32, 128)
    assert after["radial_beside"] in (1, 2)
    _, g1 = c.m.loss_grad(nl, y)
    c.m.sync_status()
    assert rel_l2(g1.cpu().numpy(), g0.cpu().numpy()) < 1e-5
    with pytest.raises(gnep._lib.GnepError):
        g.launch()
    g2 = gnep.TrainGraph(c.m, nl, y, 1e-3, 1e-5, 2, 10)
    g2.launch()
    torch.cuda.synchronize()
    c.m.sync_status()


def test_launch_shape_values_are_checked():
    b = synth.make_batch([20, 13], [2, 1], np.random.default_rng(5))
    c = Case("nmax4_basis8_h30", b, labels=False)
    t = c.nl.tuning()
    # a 33-atom batch takes the small-batch shapes
    assert t["radial_lanes"] == 16 and t["net_tile_atoms"] == 32 and t["radial_beside"] == 2, t
    for bad in (dict(radial_lanes=5), dict(radial_lanes=32), dict(net_tile_atoms=64), dict(cgrad_blocks=10 ** 6),
                dict(radial_beside=3)):
        with pytest.raises(gnep._lib.GnepError):
            c.nl.set_tuning(bad)
    c.nl.set_tuning(dict(radial_lanes=8, net_tile_atoms=128, radial_beside=1))
    t = c.nl.tuning()
    assert t["radial_lanes"] == 8 and t["net_tile_atoms"] == 128 and t["radial_beside"] == 1
