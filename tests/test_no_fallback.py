"""The library has no CPU fallback and never touches the oracle.

  * Importing the package does not import anything under oracle/, and no source file of the
    package names it.
  * Without a GPU, every solver entry point raises instead of computing on the host.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1602_05033_gb300")


def test_package_import_does_not_load_the_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_1602_05033_gb300; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().splitlines()[-1] == "False"


def test_package_sources_do_not_name_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f), encoding="utf-8").read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_entry_points_fail_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np

    import workloads as wl
    from paper_1602_05033_gb300 import Batch, ExtendedKrylov, Solver

    A = wl.laplacian_2d(8)
    C = wl.rhs(64, 2, 0)
    for make in (lambda: Solver(A, C), lambda: Batch([(A, C)]), lambda: ExtendedKrylov(A, C, grid=(8, 8))):
        with pytest.raises(RuntimeError):
            make()
    assert np.isfinite(C).all()
