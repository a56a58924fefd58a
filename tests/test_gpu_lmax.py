"""Angular degree above 4 (App. B, B5-B8; Eq. 7 with l = 1..l_max): parity of
the CUDA path with the FP64 oracle at l_max 6 (3-body) and l_max 8 (with the
4-body term).  The GPU takes the recurrence basis of real solid harmonics for
l >= 5 and the oracle the printed forms of App. B with the addition-theorem
C_lm; q_nl agrees because both satisfy the addition theorem.  Tolerances as
in test_gpu_parity: descriptors 2e-6 per column, energies 1e-6, forces and
virials 1e-5, gradient 1e-4 (relative L2 and per entry)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2507_00528_gb300 import _lib, gnep, synth

from gpu_common import Case, rel_l2, small_cells_batch

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, G_TOL = 1e-6, 1e-5, 1e-4
SHAPES = ["nmax4_basis8_lmax6_h30", "nmax4_basis8_lmax8_4b_h30"]


def _check_grad(g, ref):
    g = np.asarray(g, dtype=np.float64)
    assert rel_l2(g, ref) < G_TOL, rel_l2(g, ref)
    bad = np.nonzero(np.abs(g - ref) > G_TOL * (np.abs(ref) + np.abs(ref).max()))[0]
    assert bad.size == 0, (bad[:10], g[bad[:10]], ref[bad[:10]])


@pytest.mark.parametrize("shape", SHAPES)
def test_descriptors(shape):
    b = small_cells_batch()
    c = Case(shape, b, labels=False)
    G = c.m.descriptors(c.nl).double().cpu().numpy()
    Go = O.descriptors(c.cfg, c.P64, b)
    assert G.shape == Go.shape
    for v in range(Go.shape[1]):
        assert rel_l2(G[:, v], Go[:, v]) < 2e-6, (v, rel_l2(G[:, v], Go[:, v]))


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_energy_force_virial(shape):
    b = small_cells_batch()
    c = Case(shape, b, labels=False)
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Ea, Eao) < E_TOL
    assert rel_l2(Es, Eso) < E_TOL
    assert rel_l2(F, Fo) < F_TOL
    assert rel_l2(W, Wo) < F_TOL


@pytest.mark.parametrize("shape,lambdas,form", [
    ("nmax4_basis8_lmax6_h30", (1.0, 1.0, 0.1, 0.0), 0),
    ("nmax4_basis8_lmax8_4b_h30", (1.0, 1.0, 0.1, 0.0), 0),
    ("nmax4_basis8_lmax8_4b_h30", (0.5, 2.0, 0.3, 0.05), 1),
])
@pytest.mark.parametrize("net_tile_atoms,radial_lanes", [(0, 0), (128, 4)])
def test_loss_and_gradient(shape, lambdas, form, net_tile_atoms, radial_lanes):
    """With the small-batch defaults (32-atom CUDA-core network tiles, 16
    radial lanes) and with the large-batch kernels forced (128-atom
    tensor-core network tiles, 4 radial lanes)."""
    b = synth.make_batch([20, 13, 17], [2, 1, 0], np.random.default_rng(7))
    c = Case(shape, b, lambdas=lambdas, loss_form=form)
    c.nl.set_tuning(dict(net_tile_atoms=net_tile_atoms, radial_lanes=radial_lanes))
    terms, g = c.m.loss_grad(c.nl, c.gpu_labels())
    c.m.sync_status()
    ref_terms, ref_g = O.loss_grad(c.cfg, c.P64, c.s64, b, c.y)
    np.testing.assert_allclose(terms.cpu().numpy(), ref_terms, rtol=2e-5, atol=1e-12)
    _check_grad(g.cpu().numpy(), ref_g)


def test_atoms_without_angular_neighbours_and_noalloc():
    """A sparse cell (radial but no angular neighbours) beside an ordinary
    structure at l_max 8: zero angular columns, energies and forces against the
    oracle, and the allocation-free descriptors equal the workspace ones."""
    rng = np.random.default_rng(41)
    H = np.diag([12.0, 12.0, 12.0])
    sparse = np.array([[1.0, 1.0, 1.0], [7.0, 1.5, 1.2], [1.3, 7.2, 1.1], [6.6, 6.9, 6.8]])
    dense = synth.make_batch([30], [1], rng)
    b = synth.Batch(np.array([0, 4, 34], dtype=np.int32), np.concatenate([sparse, dense.pos]),
                    np.concatenate([[0, 1, 1, 0], dense.types]).astype(np.int32), np.stack([H, dense.cell[0]]))
    c = Case("nmax4_basis8_lmax8_4b_h30", b, labels=False, scale_batch=small_cells_batch())
    G = c.m.descriptors(c.nl).double().cpu().numpy()
    assert np.all(G[:4, c.cfg.nq_r:] == 0.0)
    assert rel_l2(G, O.descriptors(c.cfg, c.P64, b)) < 2e-6
    Ea, Es, F, W = (t.double().cpu().numpy() for t in c.m.forward(c.nl))
    Eao, Eso, Fo, Wo = O.forward(c.cfg, c.P64, c.s64, b)
    assert rel_l2(Ea, Eao) < E_TOL and rel_l2(F, Fo) < F_TOL and rel_l2(W, Wo) < F_TOL
    L = _lib.load()
    Gn = torch.full((c.nl.n_atoms, c.m.n_des), float("nan"), dtype=torch.float32, device="cuda")
    rc = L.gnep_descriptors_noalloc(c.m.h, c.nl.h, C.c_void_p(Gn.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.gnep_last_error()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Gn.cpu().numpy(), G.astype(np.float32))


def test_tensor_core_modes_are_refused_above_l4():
    m = gnep.GNEP(n_max=(4, 4), basis=(8, 8), hidden=30, l_max=6)
    with pytest.raises(_lib.GnepError):
        m.set_precision("bf16")
