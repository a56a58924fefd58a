"""Failure detection without a fault: a bounded device wait is made to run out
(an mbarrier that nothing arrives on, 1 ms limit).  The kernel gives up,
waits once more within the limit, frees its tensor memory and raises TIMEOUT
in the model's device flag; gnep_sync_status reports it once and clears it,
and the context keeps working."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2507_00528_gb300 import _lib, gnep, synth

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_survives():
    L = _lib.load()
    m = gnep.GNEP(n_max=(4, 4), basis=(8, 8), hidden=30)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.gnep_selftest_wait_timeout(m.h, 10, stream) == -1  # limit below 1 us is refused
    for _ in range(2):
        assert L.gnep_selftest_wait_timeout(m.h, 1_000_000, stream) == 0
        with pytest.raises(_lib.GnepError) as e:
            m.sync_status()
        assert e.value.code == -6
        m.sync_status()  # reported once, then cleared
    # the same context still computes: descriptors against the oracle
    b = synth.make_batch([20, 16], [0, 1], np.random.default_rng(8))
    nl = m.neighbors(gnep.DeviceBatch.from_host(b))
    G = m.descriptors(nl).double().cpu().numpy()
    cfg = O.Cfg(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30)
    Go = O.descriptors(cfg, m.get_params().double().cpu().numpy(), b)
    assert rel_l2(G, Go) < 2e-6
