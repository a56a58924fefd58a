"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/gnep.h; host-side argument validation."""
import ctypes as C
import os
import re

import pytest

from paper_2507_00528_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared():
    hdr = open(os.path.join(ROOT, "include", "gnep.h")).read()
    return set(re.findall(r"^(?:int|double|const char \*)\s*(gnep_\w+)\(", hdr, re.M))


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(_lib.EXPORTS)


def test_abi_version(lib):
    assert lib.gnep_abi_version() == 5


def test_lr_schedule_matches_oracle(lib, oracle):
    """Eq. 17 host scalar against the oracle's."""
    for s in [0, 3, 10, 11, 57, 99, 100, 150]:
        assert lib.gnep_lr_schedule(2e-3, 1e-5, s, 10, 100) == pytest.approx(
            oracle.lr(2e-3, 1e-5, s, 10, 100), rel=1e-15, abs=1e-18)


def test_create_rejects_bad_arguments(lib):
    h = C.c_void_p()
    # rc_angular > rc_radial
    rc = lib.gnep_create(C.byref(h), 2, None, 4.0, 7.0, 4, 4, 8, 8, 4, 0, 30, 0, 0)
    assert rc == -1 and not h.value
    # hidden out of range
    rc = lib.gnep_create(C.byref(h), 2, None, 7.0, 4.0, 4, 4, 8, 8, 4, 0, 1000, 0, 0)
    assert rc == -1
    # shape without a compiled kernel
    rc = lib.gnep_create(C.byref(h), 3, None, 7.0, 4.0, 4, 4, 8, 8, 4, 0, 30, 0, 0)
    assert rc == -8
    assert b"kernel" in lib.gnep_last_error()
    assert lib.gnep_create(None, 2, None, 7.0, 4.0, 4, 4, 8, 8, 4, 0, 30, 0, 0) == -1


def test_null_handles_are_rejected(lib):
    assert lib.gnep_destroy(None) == 0
    assert lib.gnep_nlist_destroy(None) == 0
    assert lib.gnep_graph_destroy(None) == 0
    n = C.c_int64()
    assert lib.gnep_num_params(None, C.byref(n)) == -1
    assert lib.gnep_sync_status(None, None) == -1
    assert lib.gnep_graph_launch(None, None) == -1
