"""Parity with the FP64 oracle at the benchmark model shape (n_max 8/8, basis
12/12, l_max 4 with the 4-body term, 50 hidden neurons) on a batch that spans
several network tiles of each species.

The batch is the smallest structures of the 256-structure workload, at least
420 atoms: more than 128 atoms of each species, so that each species spans at
least two 128-atom tiles and several 32-atom tiles.  Running the network
kernels with the default, one and three persistent blocks puts several tiles,
and a species switch, inside one block, and gives the gradient assembly one or
many block partials to combine.  The FP32 network runs with each tile size
(32 atoms on the CUDA cores, 128 atoms on the tensor cores) and the
radial sweeps with 4, 8 and 16 lanes per atom, in turn with the angular
sweeps or beside them on a second stream.  Checked against the oracle:
the loss terms and gradient (Eqs. 9-16, D1.18-D1.21) in the FP32 form at the
FP32 tolerances and in the TF32 and BF16 network modes within four rounding
units of their operand format; the descriptor scale computed on the GPU; and
Adam (refs 21-22, Eq. 17) on every entry, fed the gradient the GPU used.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2507_00528_gb300 import gnep, synth

from gpu_common import Case, rel_l2

pytestmark = pytest.mark.gpu

G_TOL = 1e-4
UNIT = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def _batch():
    b = synth.make_config(2)
    sizes = b.sizes()
    idx, tot = [], 0
    for s in np.argsort(sizes, kind="stable"):
        idx.append(int(s))
        tot += int(sizes[s])
        if tot >= 420:
            break
    return b.subset(sorted(idx))


@pytest.fixture(scope="module")
def case():
    b = _batch()
    c = Case("nmax8_basis12_h50_4b", b, lambdas=(1.0, 1.0, 0.1, 0.0))
    c.ref_terms, c.ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    return c


def _grad(c, mode, net_blocks, net_tile_atoms=0, radial_lanes=0, radial_beside=0):
    c.m.set_precision(mode)
    c.m.set_params(torch.from_numpy(c.P))
    c.nl.set_tuning(dict(net_blocks=net_blocks, net_tile_atoms=net_tile_atoms, radial_lanes=radial_lanes,
                         radial_beside=radial_beside))
    t = c.nl.tuning()
    assert net_tile_atoms in (0, t["net_tile_atoms"]) and radial_lanes in (0, t["radial_lanes"]), t
    assert radial_beside in (0, t["radial_beside"]), t
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.sync_status()
    return terms.cpu().numpy(), g.double().cpu().numpy()


def test_batch_spans_several_tiles_per_species(case):
    counts = np.bincount(case.batch.types, minlength=2)
    assert case.batch.n_atoms >= 420 and counts.min() > 128, counts


@pytest.mark.parametrize("net_blocks,net_tile_atoms,radial_lanes,radial_beside",
                         [(0, 0, 0, 0), (1, 32, 4, 1), (3, 32, 8, 2), (0, 128, 16, 1), (1, 128, 4, 2),
                          (3, 128, 0, 0)])
def test_fp32_gradient_matches_oracle(case, net_blocks, net_tile_atoms, radial_lanes, radial_beside):
    terms, g = _grad(case, "fp32", net_blocks, net_tile_atoms, radial_lanes, radial_beside)
    np.testing.assert_allclose(terms, case.ref_terms, rtol=2e-5, atol=1e-12)
    ref = case.ref_g
    assert rel_l2(g, ref) < G_TOL, rel_l2(g, ref)
    bad = np.nonzero(np.abs(g - ref) > G_TOL * (np.abs(ref) + np.abs(ref).max()))[0]
    assert bad.size == 0, (bad[:10], g[bad[:10]], ref[bad[:10]])


def test_radial_sweeps_beside_the_angular_ones_change_no_bit(case, tmp_path):
    """The radial sweeps on the second stream run the same kernels on the same
    data as in turn: the loss terms, the gradient and two graph-replayed
    training steps (from the same saved model and Adam state) agree bit for
    bit."""
    ck = str(tmp_path / "start.ckpt")
    case.m.save(ck)
    out = {}
    for beside in (1, 2):
        case.m.load(ck)
        terms, g = _grad(case, "fp32", 0, radial_beside=beside)
        gr = gnep.TrainGraph(case.m, case.nl, case.gpu_labels(), 1e-3, 1e-5, 2, 10)
        gr.launch()
        gr.launch()
        torch.cuda.synchronize()
        gr.close()
        case.m.sync_status()
        out[beside] = (terms, g, case.m.get_params().cpu().numpy())
    case.m.load(ck)
    case.nl.set_tuning(None)
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("net_blocks", [0, 1])
def test_tensor_core_network_gradient_within_four_units(case, mode, net_blocks):
    u = UNIT[mode]
    terms, g = _grad(case, mode, net_blocks)
    np.testing.assert_allclose(terms, case.ref_terms, rtol=3 * u, atol=1e-12)
    assert rel_l2(g, case.ref_g) < 4 * u, rel_l2(g, case.ref_g)


def test_descriptor_scale_matches_oracle(case):
    m = gnep.GNEP(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True)
    m.set_params(torch.from_numpy(case.T))
    nl = m.neighbors(gnep.DeviceBatch.from_host(case.batch))
    m.compute_scale(nl)
    s = m.get_scale().double().cpu().numpy()
    np.testing.assert_allclose(s, case.scale.astype(np.float64), rtol=2e-5)


def test_adam_every_entry_with_the_gpu_gradient(case):
    """Adam in FP32 on the device against the FP64 update from the same FP32
    parameters and the same (FP64) gradient, on every entry, small gradients
    included: within 1.5 units in the last place of the parameter plus 1e-5 of
    the learning rate (the FP32 rounding of the update and of the sum)."""
    _grad(case, "fp32", 0)
    g = case.m.get_grad().cpu().numpy()
    lr1, lr2 = 1e-3, O.lr(1e-3, 1e-5, 1, 2, 10)
    case.m.adam_step(lr1, weight_decay=0.01)
    p1 = case.m.get_params().double().cpu().numpy()
    th = case.P64.copy()
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    O.adam(th, mm, vv, g, 1, lr1, weight_decay=0.01)
    tol = 1.5 * np.spacing(np.abs(th).astype(np.float32)).astype(np.float64) + 1e-5 * lr1
    assert np.all(np.abs(p1 - th) <= tol), np.abs(p1 - th).max()
    # a second update from the device's own state, with the Eq. 17 rate at s = 1
    case.m.adam_step_scheduled(1e-3, 1e-5, 2, 10)
    p2 = case.m.get_params().double().cpu().numpy()
    th2 = p1.copy()
    m_dev = mm.astype(np.float32).astype(np.float64)  # the device keeps FP32 moments
    v_dev = vv.astype(np.float32).astype(np.float64)
    O.adam(th2, m_dev, v_dev, g, 2, lr2)
    tol2 = 1.5 * np.spacing(np.abs(th2).astype(np.float32)).astype(np.float64) + 1e-5 * lr2
    assert np.all(np.abs(p2 - th2) <= tol2), np.abs(p2 - th2).max()
    assert case.m.step_count() == 2
