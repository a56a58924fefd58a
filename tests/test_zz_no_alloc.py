"""gnep_descriptors_noalloc: descriptors without any device allocation.

Some callers must not allocate device memory when they need descriptors: hosts
whose device memory is reserved up front by another allocator or a fixed pool,
and per-step hooks of simulation engines that forbid allocation in their hot
loop (cudaMalloc and cudaFree may synchronise the device).  This entry point
serves them from a fixed scratch array inside the library.  This file checks it
through the C ABI against gnep_descriptors on two calls in a row, after a call
of another shape has left different values in the scratch, on atoms without
angular neighbours, and that batches beyond the scratch size are refused.  It is
named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2507_00528_gb300 import _lib, gnep, synth

pytestmark = pytest.mark.gpu

TOL = 2e-6  # per descriptor column, relative L2 (the descriptor parity bound)


def _rel_cols(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    num = np.linalg.norm(a - b, axis=0)
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return num / den


def _noalloc(L, m, nl, G):
    stream = torch.cuda.current_stream()
    rc = L.gnep_descriptors_noalloc(m.h, nl.h, C.c_void_p(G.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0, L.gnep_last_error()
    torch.cuda.synchronize()


def _fill_scratch_with_another_shape(L):
    """A larger batch of another model shape: its basis sums and S rows leave
    other values at other places of the shared scratch."""
    m = gnep.GNEP(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True, seed=9)
    nl = m.neighbors(gnep.DeviceBatch.from_host(synth.make_config(2, n_struct=30)))
    assert nl.n_atoms * (2 * 13 + 24 * 9) <= 1 << 21
    G = torch.empty(nl.n_atoms, m.n_des, dtype=torch.float32, device="cuda")
    _noalloc(L, m, nl, G)


@pytest.mark.parametrize("kw,batch_fn", [
    (dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False), lambda: synth.make_config(1)),
    (dict(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True), lambda: synth.make_config(2, n_struct=20)),
])
def test_noalloc_descriptors_match_workspace_path(kw, batch_fn):
    L = _lib.load()
    _fill_scratch_with_another_shape(L)
    m = gnep.GNEP(**kw, seed=5)
    nl = m.neighbors(gnep.DeviceBatch.from_host(batch_fn()))
    ref = m.descriptors(nl)
    for _ in range(2):  # two calls in a row share and reuse the scratch array
        G = torch.full_like(ref, float("nan"))
        _noalloc(L, m, nl, G)
        assert torch.isfinite(G).all()
        assert np.all(_rel_cols(G.cpu().numpy(), ref.cpu().numpy()) < TOL)


def test_noalloc_atoms_without_angular_neighbours():
    """A sparse cell (atoms 5.5-6.5 A apart: radial neighbours, no angular ones)
    beside an ordinary structure: the angular columns of the sparse atoms come
    out exactly zero over a NaN-filled output, after stale scratch."""
    L = _lib.load()
    _fill_scratch_with_another_shape(L)
    rng = np.random.default_rng(41)
    H = np.diag([12.0, 12.0, 12.0])
    sparse = np.array([[1.0, 1.0, 1.0], [7.0, 1.5, 1.2], [1.3, 7.2, 1.1], [6.6, 6.9, 6.8]])
    dense = synth.make_batch([30], [1], rng)
    pos = np.concatenate([sparse, dense.pos])
    types = np.concatenate([[0, 1, 1, 0], dense.types]).astype(np.int32)
    b = synth.Batch(np.array([0, 4, 34], dtype=np.int32), pos, types, np.stack([H, dense.cell[0]]))
    m = gnep.GNEP(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True, seed=5)
    nl = m.neighbors(gnep.DeviceBatch.from_host(b))
    ref = m.descriptors(nl).cpu().numpy()
    for _ in range(2):
        G = torch.full((nl.n_atoms, m.n_des), float("nan"), dtype=torch.float32, device="cuda")
        _noalloc(L, m, nl, G)
        g = G.cpu().numpy()
        assert np.all(g[:4, 9:] == 0.0)
        assert np.all(np.isfinite(g))
        assert np.all(_rel_cols(g, ref) < TOL)


def test_noalloc_refuses_batches_beyond_the_scratch():
    L = _lib.load()
    m = gnep.GNEP(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True)
    nl = m.neighbors(gnep.DeviceBatch.from_host(synth.make_config(2)))  # 57k atoms, ~14M floats
    G = torch.empty(nl.n_atoms, m.n_des, dtype=torch.float32, device="cuda")
    rc = L.gnep_descriptors_noalloc(m.h, nl.h, C.c_void_p(G.data_ptr()), None)
    assert rc == -1
    assert b"too large" in L.gnep_last_error()
    host = np.zeros((4, m.n_des), dtype=np.float32)
    assert L.gnep_descriptors_noalloc(m.h, nl.h, C.c_void_p(host.ctypes.data), None) == -1
