"""The precision conversions that the iACT and quality kernels run on the
integer pipes (csrc/convert.cuh) give the same bits as the hardware
conversions: a checker compiled from tests/cuda/convert_check.cu runs every
single-precision input through float_to_double and 5 x 2^30 doubles (random
bits, the single range, ties, the subnormal range and its ties) through
double_to_float_rn."""
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2308_16877_gb300", "csrc")


def test_conversions_bit_exact():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16877_gb300 import build
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "convert_check")
        subprocess.run([build.nvcc(), *build.ARCH, "-O3", "-I", CSRC, "-o", exe,
                        os.path.join(HERE, "cuda", "convert_check.cu")], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("mismatches 0") == 6
