"""The product path has no CPU fallback: with the CUDA library absent, loading
it and constructing a model raise instead of computing anything."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
from paper_2507_00528_gb300 import build, _lib
build.LIB = "/nonexistent/libgnep.so"
try:
    _lib.load()
    print("LOADED")
except RuntimeError as e:
    assert "no CPU fallback" in str(e), e
    print("LOUD-LOAD")
from paper_2507_00528_gb300 import gnep
try:
    gnep.GNEP(n_max=(4, 4), basis=(8, 8), hidden=30)
    print("CONSTRUCTED")
except RuntimeError as e:
    assert "no CPU fallback" in str(e), e
    print("LOUD-MODEL")
"""


def test_missing_library_raises_instead_of_computing():
    p = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.split() == ["LOUD-LOAD", "LOUD-MODEL"], p.stdout
