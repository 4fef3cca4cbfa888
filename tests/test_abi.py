"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares (no compute calls: this runs on CPU-only hosts)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2502_12878_gb300 import build
    return build.build()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"RBFFD_API\s+[\w\s\*]*?\b(rbffd_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = _declared()
    for core in ["rbffd_nodes", "rbffd_knn", "rbffd_weights", "rbffd_apply",
                 "rbffd_solve_explicit"]:
        assert core in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header(built):
    import paper_2502_12878_gb300 as rb
    assert set(rb.EXPORTED) <= set(_declared())
    assert rb.lib().rbffd_version() >= 100


def test_invalid_arguments_rejected_without_gpu(built):
    """Argument checks run before any device work, so they answer on a CPU host."""
    import paper_2502_12878_gb300 as rb
    L = rb.lib()
    n = ctypes.c_int64(0)
    assert L.rbffd_nodes(4, 0, 10, 0.3, 1, None, None, 0, ctypes.byref(n), None) == rb.RBFFD_ERR_ARG
    assert b"dimension" in L.rbffd_last_error()
    assert L.rbffd_nodes(2, 0, 10, 0.7, 1, None, None, 0, ctypes.byref(n), None) == rb.RBFFD_ERR_ARG
    assert L.rbffd_knn(None, 10, 2, None, 5, 3, None, None) == rb.RBFFD_ERR_ARG
    assert L.rbffd_apply(None, None, 5, 3, None, None, None) == rb.RBFFD_ERR_ARG


def test_oracle_and_library_share_no_code():
    """The oracle's sources include nothing from the CUDA library and vice versa."""
    osrc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "csrc" not in osrc and "rbffd.h" not in osrc
    for f in glob.glob(os.path.join(ROOT, "paper_2502_12878_gb300", "**", "*"), recursive=True):
        if os.path.isfile(f) and f.endswith((".cu", ".cuh", ".py")):
            txt = open(f).read()
            assert "import oracle" not in txt and "oracle/" not in txt, f


def test_noalloc_binding_rejects_a_short_output_before_any_call():
    """rbffd_knn_noalloc writes one row of idx per centre: a caller's buffer with
    too few rows, or of the wrong rank, is refused in the binding (no launch)."""
    torch = pytest.importorskip("torch")
    import paper_2502_12878_gb300 as rb
    xyz = torch.zeros((2, 100), dtype=torch.float64)
    centres = torch.arange(10, dtype=torch.int32)
    for bad in (torch.zeros((9, 12), dtype=torch.int32),        # one row short
                torch.zeros((10, 129), dtype=torch.int32),      # n above 128
                torch.zeros(120, dtype=torch.int32)):           # not [nc, n]
        with pytest.raises(ValueError):
            rb.rbffd_knn_noalloc(xyz, centres, bad)
    # right shape, but host tensors: refused too (never copied to the device)
    with pytest.raises(ValueError, match="CUDA"):
        rb.rbffd_knn_noalloc(xyz, centres, torch.zeros((10, 12), dtype=torch.int32))
