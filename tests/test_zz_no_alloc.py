"""gnep_descriptors_noalloc: descriptors without any device allocation.

Callers that cannot allocate device memory when they need descriptors (code
running while a stream is captured into a CUDA graph, hosts whose device memory
is owned by another allocator or a fixed pool, allocation-free per-step hooks of
simulation engines) use this entry point; it works in a fixed scratch array
inside the library.  This file checks it through the C ABI against
gnep_descriptors on two calls in a row, and that batches beyond the scratch
size are refused.  It is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2507_00528_gb300 import _lib, gnep, synth

pytestmark = pytest.mark.gpu


def _rel_cols(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    num = np.linalg.norm(a - b, axis=0)
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return num / den


@pytest.mark.parametrize("kw,batch_fn", [
    (dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False), lambda: synth.make_config(1)),
    (dict(n_max=(8, 8), basis=(12, 12), hidden=50, four_body=True), lambda: synth.make_config(2, n_struct=20)),
])
def test_noalloc_descriptors_match_workspace_path(kw, batch_fn):
    L = _lib.load()
    m = gnep.GNEP(**kw, seed=5)
    nl = m.neighbors(gnep.DeviceBatch.from_host(batch_fn()))
    ref = m.descriptors(nl)
    stream = torch.cuda.current_stream()
    for _ in range(2):  # two calls in a row share and reuse the scratch array
        G = torch.full_like(ref, float("nan"))
        rc = L.gnep_descriptors_noalloc(m.h, nl.h, C.c_void_p(G.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0, L.gnep_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(G).all()
        assert np.all(_rel_cols(G.cpu().numpy(), ref.cpu().numpy()) < 2e-6)


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
    m.sync_status()
