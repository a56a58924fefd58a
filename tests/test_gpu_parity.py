"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: neighbour lists bit-exact; per-atom energies 1e-6 relative (L2 over
atoms); forces and virials 1e-5 relative RMS; parameter gradients 1e-4 relative
(L2) and per entry |g - g_ref| <= 1e-4 (|g_ref| + max|g_ref|).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2507_00528_gb300 import gnep, synth

from gpu_common import Case, rel_l2, small_cells_batch

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, G_TOL = 1e-6, 1e-5, 1e-4


def check_grad(g, ref):
    g = np.asarray(g, dtype=np.float64)
    assert rel_l2(g, ref) < G_TOL, rel_l2(g, ref)
    bound = G_TOL * (np.abs(ref) + np.abs(ref).max())
    bad = np.nonzero(np.abs(g - ref) > bound)[0]
    assert bad.size == 0, (bad[:10], g[bad[:10]], ref[bad[:10]])


# ------------------------------------------------------------------ Eq. 2

@pytest.mark.parametrize("which_batch", ["cfg1", "small_cells", "cfg2_prefix"])
def test_neighbor_lists_bit_exact(which_batch):
    b = {"cfg1": lambda: synth.make_config(1), "small_cells": small_cells_batch,
         "cfg2_prefix": lambda: synth.make_config(2, n_struct=12)}[which_batch]()
    c = Case("nmax4_basis8_h30", b, labels=False)
    for which, rc in ((0, 7.0), (1, 4.0)):
        off, j, sh = c.nl.export(which)
        ooff, oj, osh = O.neighbors(b, rc)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(j, oj)
        np.testing.assert_array_equal(sh, osh)


# ------------------------------------------------------------ Eqs. 5-8

@pytest.mark.parametrize("shape", ["nmax4_basis8_h30", "nmax8_basis12_h50_4b"])
def test_descriptors(shape):
    b = small_cells_batch() if shape != "nmax4_basis8_h30" else synth.make_config(1, n_struct=4)
    c = Case(shape, b, labels=False)
    G = c.m.descriptors(c.nl).double().cpu().numpy()
    Go = O.descriptors(c.cfg, c.P64, b)
    for v in range(Go.shape[1]):
        assert rel_l2(G[:, v], Go[:, v]) < 2e-6, (v, rel_l2(G[:, v], Go[:, v]))


# ------------------------------------------------------------ Eqs. 1, 3, 4

@pytest.mark.parametrize("shape,which_batch", [("nmax4_basis8_h30", "cfg1"),
                                               ("nmax8_basis12_h50_4b", "small_cells"),
                                               ("nmax8_basis12_h100", "small_cells")])
def test_forward_energy_force_virial(shape, which_batch):
    b = synth.make_config(1) if which_batch == "cfg1" else small_cells_batch()
    c = Case(shape, b, labels=False)
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Ea, Eao) < E_TOL
    assert rel_l2(Es, Eso) < E_TOL
    assert rel_l2(F, Fo) < F_TOL
    assert rel_l2(W, Wo) < F_TOL
    for s in range(b.n_struct):  # Newton's third law per structure
        f = F[b.struct_off[s]:b.struct_off[s + 1]]
        assert np.abs(f.sum(0)).max() < 1e-4 * np.abs(f).max()


# ------------------------------------------------------------ Eqs. 9-16

@pytest.mark.parametrize("shape,which_batch,lambdas,form", [
    ("nmax4_basis8_h30", "cfg1", (1.0, 1.0, 0.1, 0.0), 0),
    ("nmax4_basis8_h30", "cfg1_2", (0.5, 2.0, 0.3, 0.05), 1),
    ("nmax4_basis8_h30", "small_cells", (1.0, 1.0, 1.0, 0.0), 0),
    ("nmax8_basis12_h50_4b", "tiny_mixed", (1.0, 1.0, 0.1, 0.0), 0),
    ("nmax8_basis12_h50_4b", "tiny_mixed", (0.0, 0.0, 1.0, 0.0), 0),
    ("nmax8_basis12_h100", "tiny_mixed", (1.0, 1.0, 0.1, 0.01), 1),
])
def test_loss_and_gradient(shape, which_batch, lambdas, form):
    b = {"cfg1": lambda: synth.make_config(1),
         "cfg1_2": lambda: synth.make_config(1, n_struct=2),
         "small_cells": small_cells_batch,
         "tiny_mixed": lambda: synth.make_batch([20, 13], [2, 1], np.random.default_rng(7))}[which_batch]()
    c = Case(shape, b, lambdas=lambdas, loss_form=form)
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.sync_status()
    ref_terms, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    np.testing.assert_allclose(terms.cpu().numpy(), ref_terms, rtol=2e-5, atol=1e-12)
    check_grad(g.cpu().numpy(), ref_g)


@pytest.mark.parametrize("shape,which_batch,form", [
    ("nmax4_basis8_h30", "cfg1_2", 1),
    ("nmax8_basis12_h50_4b", "tiny_mixed", 0),
    ("nmax8_basis12_h100", "tiny_mixed", 1),
])
def test_loss_and_gradient_large_batch_kernels(shape, which_batch, form):
    """The kernels that large batches take, forced on small ones: 128-atom
    network tiles (tensor-core forward; tensor-core backward up to 64 hidden
    units, the two-thread CUDA-core backward at 100) and four radial lanes."""
    b = {"cfg1_2": lambda: synth.make_config(1, n_struct=2),
         "tiny_mixed": lambda: synth.make_batch([20, 13], [2, 1], np.random.default_rng(7))}[which_batch]()
    c = Case(shape, b, lambdas=(1.0, 1.0, 0.1, 0.0), loss_form=form)
    c.nl.set_tuning(dict(net_tile_atoms=128, radial_lanes=4))
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.sync_status()
    ref_terms, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    np.testing.assert_allclose(terms.cpu().numpy(), ref_terms, rtol=2e-5, atol=1e-12)
    check_grad(g.cpu().numpy(), ref_g)


def test_adam_step_matches_oracle():
    b = synth.make_config(1, n_struct=2)
    c = Case("nmax4_basis8_h30", b)
    _, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.adam_step(1e-3, weight_decay=0.01)
    c.m.adam_step_scheduled(1e-3, 1e-5, 2, 10)  # second update, Eq. 17 at s = 1
    p_gpu = c.m.get_params().double().cpu().numpy()
    _, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    th = c.P64.copy(); mm = np.zeros_like(th); vv = np.zeros_like(th)
    O.adam(th, mm, vv, ref_g, 1, 1e-3, weight_decay=0.01)
    O.adam(th, mm, vv, ref_g, 2, O.lr(1e-3, 1e-5, 1, 2, 10))
    keep = np.abs(ref_g) > 1e-4 * np.abs(ref_g).max()
    np.testing.assert_allclose(p_gpu[keep], th[keep], rtol=0, atol=2e-6)
    assert c.m.step_count() == 2


def test_full_config2_sampled_structures():
    """The full 256-structure batch in one launch; sampled structures vs the oracle."""
    b = synth.make_config(2)
    c = Case("nmax8_basis12_h50_4b", b.subset([0]), labels=False)
    nl = c.m.neighbors(gnep.DeviceBatch.from_host(b))
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(nl))
    sizes = b.sizes()
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), 2, 100]
    for s in picks:
        sb = b.subset([s])
        _, eso, fo, wo = O.forward(c.cfg, c.P64, c.s64, sb)
        a0, a1 = b.struct_off[s], b.struct_off[s + 1]
        assert abs(Es[s] - eso[0]) <= E_TOL * abs(eso[0]) + 1e-9
        assert rel_l2(F[a0:a1], fo) < F_TOL
        assert rel_l2(W[s], wo[0]) < F_TOL


# ------------------------------------------------------------ edge cases

def test_single_atom_self_images_and_isolated_atom():
    """One atom in a 3 A cell (only self images), one isolated atom, a dimer."""
    pos = np.array([[0.3, 0.4, 0.5], [15.0, 15.0, 15.0], [10.0, 10.0, 10.0], [12.6, 10.4, 9.1]])
    cells = np.stack([np.diag([3.0, 3.2, 3.4]), np.eye(3) * 30.0, np.eye(3) * 30.0])
    b = synth.Batch(np.array([0, 1, 2, 4], dtype=np.int32), pos, np.array([1, 0, 0, 1], dtype=np.int32), cells)
    # the input scale comes from a training-like set, not from these four atoms
    c = Case("nmax8_basis12_h50_4b", b, lambdas=(1.0, 1.0, 1.0, 0.0), scale_batch=small_cells_batch())
    for which, rc in ((0, 7.0), (1, 4.0)):
        off, j, sh = c.nl.export(which)
        ooff, oj, osh = O.neighbors(b, rc)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(j, oj)
        np.testing.assert_array_equal(sh, osh)
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Ea, Eao) < E_TOL
    assert np.abs(F[1]).max() == 0.0
    # forces here are cancellation residuals of O(1) pair terms: absolute bound
    assert np.abs(F - Fo).max() < 1e-5 and rel_l2(W, Wo) < F_TOL
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    ref_terms, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    check_grad(g.cpu().numpy(), ref_g)


def test_rejects_unwrapped_positions_and_bad_batches():
    b = synth.make_config(1, n_struct=1)
    m = gnep.GNEP()
    bad = synth.Batch(b.struct_off, b.pos + np.array([100.0, 0, 0]), b.types, b.cell)
    with pytest.raises(gnep._lib.GnepError, match="INVALID_ARG"):
        m.neighbors(gnep.DeviceBatch.from_host(bad))
    bad_t = synth.Batch(b.struct_off, b.pos, b.types + 5, b.cell)
    with pytest.raises(gnep._lib.GnepError, match="INVALID_ARG"):
        m.neighbors(gnep.DeviceBatch.from_host(bad_t))
    bad_off = synth.Batch(np.array([0, 70], dtype=np.int32), b.pos, b.types, b.cell)
    with pytest.raises(gnep._lib.GnepError, match="INVALID_ARG"):
        m.neighbors(bad_off)
    empty = synth.Batch(np.array([0, 0, 64], dtype=np.int32), b.pos, b.types, np.concatenate([b.cell, b.cell]))
    with pytest.raises(gnep._lib.GnepError, match="INVALID_ARG"):
        m.neighbors(empty)
    m.sync_status()  # the model is still usable
    nl = m.neighbors(b)  # host arrays are accepted too
    assert nl.info()[0] > 0


def test_nonfinite_loss_skips_update():
    b = synth.make_config(1, n_struct=1)
    c = Case("nmax4_basis8_h30", b)
    y = c.gpu_labels()
    y.energy[0] = float("nan")
    p0 = c.m.get_params().clone()
    terms, _ = c.m.loss_grad(c.nl, y)
    c.m.adam_step(1e-3)
    with pytest.raises(gnep._lib.GnepError, match="NONFINITE"):
        c.m.sync_status()
    assert torch.equal(c.m.get_params(), p0)
    assert c.m.step_count() == 0
    c.m.sync_status()  # flag cleared
    # the captured step (gradient, loss copy and update in one kernel) skips
    # its update too, and still reports the loss
    g = gnep.TrainGraph(c.m, c.nl, y, 1e-3, 1e-5, 2, 10)
    g.launch()
    torch.cuda.synchronize()
    with pytest.raises(gnep._lib.GnepError, match="NONFINITE"):
        c.m.sync_status()
    assert torch.equal(c.m.get_params(), p0)
    assert c.m.step_count() == 0
    assert torch.isnan(g.loss[0]).item() and torch.equal(g.loss[2:].cpu(), terms[2:].cpu())
    g.close()
    c.m.sync_status()


def test_step_is_deterministic_and_graph_replay_matches():
    b = small_cells_batch()
    c1 = Case("nmax4_basis8_h30", b)
    c2 = Case("nmax4_basis8_h30", b)
    y1, y2 = c1.gpu_labels(), c2.gpu_labels()
    t_a, g_a = c1.m.loss_grad(c1.nl, y1)
    t_b, g_b = c1.m.loss_grad(c1.nl, y1)
    assert torch.equal(g_a, g_b) and torch.equal(t_a, t_b)
    # eager steps on c1, graph replays on c2, same schedule
    for _ in range(3):
        t_last, _ = c1.m.loss_grad(c1.nl, y1, grad=False)
        c1.m.adam_step_scheduled(1e-3, 1e-5, 2, 10)
    g = gnep.TrainGraph(c2.m, c2.nl, y2, 1e-3, 1e-5, 2, 10)
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    assert torch.equal(c1.m.get_params(), c2.m.get_params())
    assert torch.equal(c1.m.get_grad(), c2.m.get_grad())  # the graph's gradient is kept for the API too
    assert torch.equal(g.loss, t_last)  # the loss terms of the third step, before its update
    assert c2.m.step_count() == 3
    # eleven sweep, network and loss kernels, and the gradient with the update
    assert g.kernel_count() == 12


def test_checkpoint_roundtrip_and_corruption(tmp_path):
    b = synth.make_config(1, n_struct=1)
    c = Case("nmax4_basis8_h30", b)
    y = c.gpu_labels()
    c.m.loss_grad(c.nl, y, grad=False)
    c.m.adam_step(1e-3)
    path = str(tmp_path / "m.ckpt")
    c.m.save(path)
    # continue two steps; then reload and redo them: identical trajectory
    traj = []
    for _ in range(2):
        t, _ = c.m.loss_grad(c.nl, y, grad=False)
        c.m.adam_step(1e-3)
        traj.append(t.cpu().numpy().copy())
    p_end = c.m.get_params().clone()
    c.m.load(path)
    assert c.m.step_count() == 1
    for k in range(2):
        t, _ = c.m.loss_grad(c.nl, y, grad=False)
        c.m.adam_step(1e-3)
        np.testing.assert_array_equal(t.cpu().numpy(), traj[k])
    assert torch.equal(c.m.get_params(), p_end)
    raw = bytearray(open(path, "rb").read())
    raw[200] ^= 0x40
    open(path, "wb").write(bytes(raw))
    with pytest.raises(gnep._lib.GnepError, match="CHECKPOINT_CORRUPT"):
        c.m.load(path)
    assert torch.equal(c.m.get_params(), p_end)


def test_autograd_function_and_gpu_finite_differences():
    b = synth.make_config(1, n_struct=2)
    c = Case("nmax4_basis8_h30", b, lambdas=(1.0, 1.0, 0.1, 0.0))
    y = c.gpu_labels()
    p = torch.from_numpy(c.P).cuda().double().requires_grad_(True)
    loss = gnep.GNEPLoss.apply(p, c.m, c.nl, y)
    loss.backward()
    _, g = c.m.loss_grad(c.nl, y)
    assert torch.allclose(p.grad.float(), g)
    # central differences of the GPU loss itself (FP32 forward, loose tolerance)
    rng = np.random.default_rng(0)
    gh = g.double().cpu().numpy()
    idx = np.argsort(-np.abs(gh))[:8].tolist() + rng.choice(len(gh), 4, replace=False).tolist()
    h = 3e-3
    for k in idx:
        pp = torch.from_numpy(c.P).clone()
        pp[k] += h
        c.m.set_params(pp)
        lp = c.m.loss_grad(c.nl, y, grad=False)[0][0].item()
        pp[k] -= 2 * h
        c.m.set_params(pp)
        lm = c.m.loss_grad(c.nl, y, grad=False)[0][0].item()
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gh[k]) <= 2e-2 * (abs(gh[k]) + 1e-2 * np.abs(gh).max()), (k, fd, gh[k])


@pytest.mark.parametrize("loss_form", [0, 1])
def test_directional_derivatives_match_finite_differences(loss_form):
    """The GPU gradient against central differences of the GPU loss along
    random directions of all parameters at once (the network weights and both
    coefficient sets move together), at the benchmark model shape, in the MSE
    and RMSE forms (Eqs. 9-12).  A step of at most 3e-3 per parameter moves the
    loss far more than its FP32 rounding, and the cubic term of the central
    difference stays far below the 2e-3 relative tolerance."""
    b = synth.make_config(1, n_struct=3)
    c = Case("nmax8_basis12_h50_4b", b, lambdas=(1.0, 1.0, 0.1, 0.0), loss_form=loss_form)
    y = c.gpu_labels()
    _, g = c.m.loss_grad(c.nl, y)
    gh = g.double().cpu().numpy()
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(len(gh))
        d = 3e-3 * v / np.abs(v).max()
        pp = torch.from_numpy((c.P.astype(np.float64) + d).astype(np.float32))
        pm = torch.from_numpy((c.P.astype(np.float64) - d).astype(np.float32))
        dp = pp.double().numpy() - pm.double().numpy()  # the step actually taken, after FP32 rounding
        c.m.set_params(pp)
        lp = c.m.loss(c.nl, y)[0].item()
        c.m.set_params(pm)
        lm = c.m.loss(c.nl, y)[0].item()
        fd = lp - lm
        an = float(gh @ dp)
        assert abs(fd - an) <= 2e-3 * abs(an), (fd, an)
    c.m.set_params(torch.from_numpy(c.P))


def test_skewed_cells_many_images_and_largest_structure():
    """A strongly sheared triclinic cell, a two-atom cell far below both
    cut-offs (dozens of images of each atom in both lists), and one structure
    of the largest size of the 10,000-structure workload (512 atoms)."""
    rng = np.random.default_rng(31)
    # shear: a = (9, 0, 0), b = (5.5, 8, 0), c = (-4, 3.5, 8.5)
    H = np.array([[9.0, 0.0, 0.0], [5.5, 8.0, 0.0], [-4.0, 3.5, 8.5]])
    f = rng.random((24, 3))
    sk_pos = f @ H
    tiny = np.array([[0.2, 0.3, 0.1], [1.9, 1.6, 1.7]])
    tiny_H = np.diag([3.4, 3.3, 3.6])
    big = synth.make_batch([512], [1], np.random.default_rng(32))
    pos = np.concatenate([sk_pos, tiny, big.pos])
    types = np.concatenate([rng.integers(0, 2, 24), [0, 1], big.types]).astype(np.int32)
    cells = np.stack([H, tiny_H, big.cell[0]])
    b = synth.Batch(np.array([0, 24, 26, 538], dtype=np.int32), pos, types, cells)
    c = Case("nmax8_basis12_h50_4b", b.subset([0, 1]), labels=False)
    nl = c.m.neighbors(gnep.DeviceBatch.from_host(b))
    for which, rc in ((0, 7.0), (1, 4.0)):
        off, j, sh = nl.export(which)
        ooff, oj, osh = O.neighbors(b, rc)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(j, oj)
        np.testing.assert_array_equal(sh, osh)
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(nl))
    small = b.subset([0, 1])  # the oracle on the two small cells; the 512-atom one sampled by structure sums
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, small)
    assert rel_l2(Ea[:26], Eao) < E_TOL
    assert rel_l2(F[:26], Fo) < F_TOL and rel_l2(W[:2], Wo) < F_TOL
    _, eso, fo, wo = O.forward(c.cfg, c.P64, c.s64, b.subset([2]))
    assert abs(Es[2] - eso[0]) <= E_TOL * abs(eso[0])
    assert rel_l2(F[26:], fo) < F_TOL and rel_l2(W[2], wo[0]) < F_TOL


def test_binned_search_large_structures_bit_exact():
    """Structures above 1024 atoms take the binned pair search, the others the
    all-pairs one, in the same build: a 1500-atom rocksalt cell, a 1300-atom
    strained (triclinic) cell and a 40-atom cell.  Both lists equal the
    oracle's (Eq. 2) entry for entry, and so do the forces of the large cells."""
    b = synth.make_batch([1500, 40, 1300], [0, 2, 2], np.random.default_rng(41))
    c = Case("nmax4_basis8_h30", b.subset([1]), labels=False)
    nl = c.m.neighbors(gnep.DeviceBatch.from_host(b))
    for which, rc in ((0, 7.0), (1, 4.0)):
        off, j, sh = nl.export(which)
        ooff, oj, osh = O.neighbors(b, rc)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(j, oj)
        np.testing.assert_array_equal(sh, osh)
    _, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(nl))
    _, eso, fo, wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Es, eso) < E_TOL
    assert rel_l2(F, fo) < F_TOL and rel_l2(W, wo) < F_TOL


@pytest.mark.parametrize("dense", [False, True])
def test_binned_search_sheared_and_elongated_cells_bit_exact(dense):
    """The binned pair search on cells that stress its bounds: a 1200-atom
    cell under a strong shear (the extended bins follow the fractional bounds
    along each cell direction, not Cartesian boxes) and a 1100-atom cell
    elongated along c (many bins along c, two along a and b, the bin count
    reduced to the atom count).  At the workload density the lists come from
    the slots; at 3.5 times that density (about 170 radial neighbours) the
    slots overflow and the binned search's counts place the entries of the
    writing pass.  Both lists equal the oracle's (Eq. 2) entry for entry."""
    rng = np.random.default_rng(43)
    n1, n2 = 1200, 1100
    shear = np.array([[22.0, 0.0, 0.0], [9.5, 21.0, 0.0], [-7.0, 6.5, 22.5]])
    rho = 0.115 if dense else 0.033
    H1 = shear * (n1 / rho / abs(np.linalg.det(shear))) ** (1.0 / 3.0)
    H2 = np.diag([10.4, 10.1, n2 / rho / (10.4 * 10.1)])
    f1, f2 = rng.random((n1, 3)), rng.random((n2, 3))
    pos = np.concatenate([f1 @ H1, f2 @ H2])
    types = rng.integers(0, 2, n1 + n2).astype(np.int32)
    b = synth.Batch(np.array([0, n1, n1 + n2], dtype=np.int32), pos, types, np.stack([H1, H2]))
    c = Case("nmax4_basis8_h30", b.subset([0]), labels=False)
    nl = c.m.neighbors(gnep.DeviceBatch.from_host(b))
    for which, rc in ((0, 7.0), (1, 4.0)):
        off, j, sh = nl.export(which)
        ooff, oj, osh = O.neighbors(b, rc)
        if which == 0:
            assert (np.diff(ooff).max() > 96) == dense
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(j, oj)
        np.testing.assert_array_equal(sh, osh)


def test_dense_image_lattice_overflows_the_slots():
    """A one-atom cubic cell of 2.3 A holds about 118 images within the radial
    cut-off, more than the 96 per-atom slots of the one-pass search: the lists
    are then written by the counting pass's fill fallback, and must still equal
    the oracle's (Eq. 2), with energies and forces to match."""
    cells = np.stack([np.eye(3) * 2.3, np.diag([3.4, 3.3, 3.6])])
    pos = np.array([[0.4, 0.7, 1.1], [0.2, 0.3, 0.1], [1.9, 1.6, 1.7]])
    b = synth.Batch(np.array([0, 1, 3], dtype=np.int32), pos, np.array([1, 0, 1], dtype=np.int32), cells)
    c = Case("nmax4_basis8_h30", b, labels=False)
    for which, rc in ((0, 7.0), (1, 4.0)):
        off, j, sh = c.nl.export(which)
        ooff, oj, osh = O.neighbors(b, rc)
        assert which == 1 or off[1] - off[0] > 96
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(j, oj)
        np.testing.assert_array_equal(sh, osh)
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Ea, Eao) < E_TOL
    assert rel_l2(W, Wo) < F_TOL
    assert np.abs(F - Fo).max() <= F_TOL * max(np.abs(Fo).max(), 1.0)


def test_atoms_without_angular_neighbours():
    """A sparse cell whose atoms lie 5.5-6.5 A apart: radial neighbours (r_c 7 A)
    but no angular ones (r_c 4 A).  Their S, q_nl and q4 are zero, and the
    sweeps that walk angular pairs per atom still write them (Eqs. 5-8), next to
    an ordinary structure in the same tiles; energies, forces and the gradient
    match the oracle."""
    rng = np.random.default_rng(41)
    H = np.diag([12.0, 12.0, 12.0])
    sparse = np.array([[1.0, 1.0, 1.0], [7.0, 1.5, 1.2], [1.3, 7.2, 1.1], [6.6, 6.9, 6.8]])
    dense = synth.make_batch([30], [1], rng)
    pos = np.concatenate([sparse, dense.pos])
    types = np.concatenate([[0, 1, 1, 0], dense.types]).astype(np.int32)
    b = synth.Batch(np.array([0, 4, 34], dtype=np.int32), pos, types, np.stack([H, dense.cell[0]]))
    c = Case("nmax8_basis12_h50_4b", b)
    off, _, _ = c.nl.export(1)
    assert np.all(np.diff(off)[:4] == 0) and off[-1] > 0
    G = c.m.descriptors(c.nl).double().cpu().numpy()
    Go = O.descriptors(c.cfg, c.P64, b)
    assert np.all(G[:4, c.cfg.nq_r:] == 0.0)
    assert rel_l2(G, Go) < 2e-6
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Ea, Eao) < E_TOL and rel_l2(F, Fo) < F_TOL and rel_l2(W, Wo) < F_TOL
    y = c.gpu_labels()
    _, g = c.m.loss_grad(c.nl, y)
    _, ref = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    check_grad(g.cpu().numpy(), ref)


@pytest.mark.parametrize("loss_form,lambda_l2", [(0, 0.0), (1, 1e-3)])
def test_step_sequence_graph_matches_single_steps(loss_form, lambda_l2):
    """Four training steps over three one-structure batches (the first batch
    twice) captured as one graph give, bit for bit, the parameters, the
    update count and each step's loss terms of the eager step pairs, in the
    MSE form and in the RMSE form with the L2 term; a second launch continues
    the same way, and a retuned list refuses the launch."""
    kw = dict(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True)
    b = synth.make_config(2, n_struct=6)
    teacher = gnep.GNEP(**kw, seed=12)
    teacher.compute_scale(teacher.neighbors(gnep.DeviceBatch.from_host(b)))
    subs = [b.subset([k]) for k in (0, 3, 5)]
    ys = [teacher.teacher_labels(teacher.neighbors(gnep.DeviceBatch.from_host(s)), s.sizes(), lambda_e=1.0,
                                 lambda_f=1.0, lambda_v=0.1, lambda_l2=lambda_l2, loss_form=loss_form)
          for s in subs]
    seq = [0, 1, 2, 0]

    def student():
        m = gnep.GNEP(**kw, seed=11)
        m.set_scale(teacher.get_scale())
        return m, [m.neighbors(gnep.DeviceBatch.from_host(s)) for s in subs]

    ma, nla = student()
    mb, nlb = student()
    g = gnep.TrainGraph(mb, [nlb[k] for k in seq], [ys[k] for k in seq], 1e-3, 1e-5, 2, 10)
    assert g.kernel_count() == (12 + loss_form) * len(seq)  # the RMSE form adds the residual-weight kernel
    for rep in range(2):
        terms = []
        for k in seq:
            t, _ = ma.loss_grad(nla[k], ys[k], grad=False)
            ma.adam_step_scheduled(1e-3, 1e-5, 2, 10)
            terms.append(t.clone())
        g.launch()
        torch.cuda.synchronize()
        ma.sync_status()
        mb.sync_status()
        assert torch.equal(ma.get_params(), mb.get_params()), rep
        assert torch.equal(g.loss, torch.stack(terms)), rep
        assert mb.step_count() == len(seq) * (rep + 1)
    nlb[1].set_tuning(None)
    with pytest.raises(gnep._lib.GnepError, match="INVALID_ARG"):
        g.launch()
    g.close()
