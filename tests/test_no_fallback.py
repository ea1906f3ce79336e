"""The product path has no CPU fallback and never touches the oracle (no GPU needed): a missing
library and a missing GPU both raise, and importing the package loads nothing from oracle/."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_raises(monkeypatch):
    from paper_1810_12707_gb300 import mhd
    monkeypatch.setattr(mhd, "_lib", None)  # as in a fresh process: nothing loaded yet
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mhd.load_library(os.path.join(ROOT, "does-not-exist", "libmhd_gb300.so"))


def test_no_gpu_raises_instead_of_falling_back():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    for allocator in ("torch", "cuda"):
        with pytest.raises((RuntimeError, mhd.MhdError)):
            mhd.mhd_init(16, [(1e-3, 1e-3, 1.0)], allocator=allocator)


def test_package_does_not_load_the_oracle():
    code = ("import sys; import paper_1810_12707_gb300.mhd, paper_1810_12707_gb300.inputs, "
            "paper_1810_12707_gb300.serving, paper_1810_12707_gb300.build_lib; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "False"
