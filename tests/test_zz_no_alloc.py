"""The allocation-free support selection, rbffd_knn_noalloc, called through the C ABI.

Some callers cannot allocate GPU memory while they run (they reserve the device's
memory up front in their own pool, or run latency-bound loops where an allocation
is not acceptable).  rbffd_knn_noalloc serves them from a fixed array inside the
library.  Its supports must equal rbffd_knn's bit for bit (the tolerance the kNN
parity tests use), including on a second call in a row, which finds the first
call's data still in that array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import rbffd_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_12878_gb300 import build as nvbuild
    nvbuild.build()
    import paper_2502_12878_gb300 as m
    m.lib()
    return m


def _call(rb, xyz, centres, n):
    """rbffd_knn_noalloc through ctypes on the library itself."""
    L = rb.lib()
    idx = torch.full((centres.numel(), n), -7, dtype=torch.int32, device="cuda")
    code = L.rbffd_knn_noalloc(ctypes.c_void_p(xyz.data_ptr()), xyz.shape[1], xyz.shape[0],
                               ctypes.c_void_p(centres.data_ptr()), centres.numel(), n,
                               ctypes.c_void_p(idx.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, idx


def test_noalloc_knn_matches_knn_on_two_calls_in_a_row(rb):
    cases = [
        (2, 0, 300, 0.3, 11, 30),    # 90,601 nodes (first call fills the array)
        (2, 1, 120, 0.3, 12, 12),    # a disk: fewer nodes and cells, stale data behind them
        (3, 0, 40, 0.3, 13, 70),     # 68,921 nodes in 3D
    ]
    for (d, shape, Kg, jit, seed, n) in cases:
        xyz, bnd = rb.rbffd_nodes(d, shape, Kg, jit, seed)
        centres = rb.rbffd_interior(bnd)
        ref = rb.rbffd_knn(xyz, centres, n)
        code, got = _call(rb, xyz, centres, n)
        torch.cuda.synchronize()
        assert code == rb.RBFFD_OK, rb.lib().rbffd_last_error()
        assert torch.equal(got, ref)


def test_noalloc_knn_at_the_size_limit_and_beyond(rb):
    lim = rb.RBFFD_KNN_NOALLOC_MAX_NODES
    xyz = torch.from_numpy(gen.random_points(lim, 2, 5)).cuda()
    centres = torch.arange(0, lim, 97, dtype=torch.int32, device="cuda")
    ref = rb.rbffd_knn(xyz, centres, 20)
    for _ in range(2):
        code, got = _call(rb, xyz, centres, 20)
        assert code == rb.RBFFD_OK and torch.equal(got, ref)
    big = torch.from_numpy(gen.random_points(lim + 1, 2, 6)).cuda()
    code, got = _call(rb, big, centres, 20)
    assert code == rb.RBFFD_ERR_CAPACITY
    assert b"scratch limit" in rb.lib().rbffd_last_error()
    assert torch.all(got == -7)          # nothing was written


def test_noalloc_knn_on_a_planar_3d_set_coarsens_its_grid(rb):
    """Points of the plane z = 0 given as a 3D set: the flat extent makes a grid of
    about one node per cell far larger than the fixed cell arrays, so the call
    coarsens its grid until it fits.  The supports must not change."""
    import oracle
    N = 100_000
    p2 = gen.random_points(N, 2, 31)
    xyz_h = np.vstack([p2, np.zeros((1, N))])
    xyz = torch.from_numpy(xyz_h).cuda()
    centres = torch.arange(0, N, 7, dtype=torch.int32, device="cuda")
    ref = rb.rbffd_knn(xyz, centres, 30)
    for _ in range(2):
        code, got = _call(rb, xyz, centres, 30)
        torch.cuda.synchronize()
        assert code == rb.RBFFD_OK, rb.lib().rbffd_last_error()
        assert torch.equal(got, ref)
    # and sampled rows against the oracle's brute force
    rows = np.arange(0, centres.numel(), 97)
    cen = centres.cpu().numpy()[rows]
    exp = oracle.knn_brute(xyz_h, cen, 30)
    assert np.array_equal(got.cpu().numpy()[rows], exp)


def test_noalloc_knn_does_not_allocate(rb):
    xyz, bnd = rb.rbffd_nodes(2, 0, 200, 0.3, 21)
    centres = rb.rbffd_interior(bnd)
    idx = torch.empty((centres.numel(), 12), dtype=torch.int32, device="cuda")
    rb.rbffd_knn_noalloc(xyz, centres, idx)          # first call: symbol address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rb.rbffd_knn_noalloc(xyz, centres, idx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(idx, rb.rbffd_knn(xyz, centres, 12))
