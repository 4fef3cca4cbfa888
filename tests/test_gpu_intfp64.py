"""The weight build's reciprocal, quotient and square root on the integer pipes
(csrc/intfp64.cuh) equal the library's correctly rounded FP64 reciprocal, quotient
and square root bit for bit: a probe kernel compiled from the same header, on 1.2e8
seeded operands per routine in four families (uniform significands; significands
next to 1 and 2; exponents across the whole normal range, where the routines hand
over to the library; powers of two, zeros, subnormals and exact squares)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2502_12878_gb300", "csrc")


def test_integer_pipe_fp64_routines_match_library(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "intfp64_probe"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false",
                    "-I", CSRC, os.path.join(HERE, "intfp64_probe.cu"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lines = [l.split() for l in out.strip().splitlines()]
    assert len(lines) == 12, out
    for f in lines:
        assert int(f[4]) > 1e7 and int(f[6]) == 0, out
