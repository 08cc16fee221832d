"""The table-driven exponential of the LavaMD pair loop (csrc/fast_exp.cuh,
Tang's method): a checker compiled from tests/cuda/exp_check.cu compares it
with CUDA's exp on 2^28 grid points of [-700, 700] (at most 2 units in the last
place apart) and with the host's long-double expl on 2^20 random points (at
most 4e-16 relative error), and checks its exact cases and its range test."""
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_16877_gb300", "csrc")


def test_table_driven_exp_accuracy():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import build
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "exp_check")
        subprocess.run([build.nvcc(), *build.ARCH, "-O3", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "cuda", "exp_check.cu")], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "range test mismatches 0" in r.stdout
