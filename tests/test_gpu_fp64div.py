"""The weight build's back-substitution quotient (Markstein's method from the pivot's
reciprocal, csrc/fp64div.cuh) equals the library's correctly rounded quotient bit for
bit: a probe kernel compiled from the same header, on 2.4e8 seeded operand pairs in three
operand families (uniform mantissas, mantissas next to 1 and 2, exponents outside the
fast path's range)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2502_12878_gb300", "csrc")


def test_quotient_matches_library(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "fp64div_probe"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false",
                    "-I", CSRC, os.path.join(HERE, "fp64div_probe.cu"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lines = [l.split() for l in out.strip().splitlines()]
    assert len(lines) == 3
    for f in lines:
        assert int(f[3]) > 1e7 and int(f[5]) == 0, out
