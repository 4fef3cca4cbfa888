"""Poisson-disc node placement on the GPU against the oracle's sequential walk.

The GPU walks one generation at a time (candidates tested in parallel, the
conflicts among a generation's candidates resolved in key order); the node
list must equal the oracle's first-in first-out walk bit for bit: same
count, same coordinates, same order, same boundary flags.  Also: the error
paths, and the explicit solve on a Poisson-disc node set against the oracle.
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


def H(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("shape,Kg,seed,K,zeta", [
    (0, 40, 1, 15, 1 - 1e-10),
    (0, 123, 2, 15, 1 - 1e-10),
    (1, 60, 3, 15, 1 - 1e-10),
    (1, 151, 4, 15, 1 - 1e-10),
    (0, 90, 5, 9, 1 - 1e-10),
    (0, 90, 6, 24, 0.8),
    (1, 2, 7, 15, 1 - 1e-10),          # tiny: the disk boundary alone nearly fills it
])
def test_pds_bit_exact(rb, orc, shape, Kg, seed, K, zeta):
    xyz, bnd, rounds = rb.rbffd_nodes_pds(shape, Kg, seed, K=K, zeta=zeta)
    oxyz, obnd = orc.nodes_pds(shape, Kg, seed, K=K, zeta=zeta)
    assert xyz.shape == oxyz.shape
    assert np.array_equal(H(xyz), oxyz) and np.array_equal(H(bnd), obnd)
    assert rounds >= 1


def test_pds_full_size_bit_exact(rb, orc):
    """h = 1e-3 on the unit square: 873,547 nodes, several hundred generations."""
    xyz, bnd, rounds = rb.rbffd_nodes_pds(0, 1000, 2)
    oxyz, obnd = orc.nodes_pds(0, 1000, 2)
    assert np.array_equal(H(xyz), oxyz) and np.array_equal(H(bnd), obnd)
    assert 300 < rounds < 2000


def test_pds_errors(rb):
    L = rb.lib()
    n, r = ctypes.c_int64(0), (ctypes.c_int64 * 2)()
    buf = torch.empty((2, 10), dtype=torch.float64, device="cuda")
    b = torch.empty(10, dtype=torch.uint8, device="cuda")
    s = rb._stream("cuda")
    code = L.rbffd_nodes_pds(2, 0, 20, 15, 1 - 1e-10, 1, rb._ptr(buf), rb._ptr(b), 10,
                             ctypes.byref(n), r, s)
    assert code == rb.RBFFD_ERR_CAPACITY and n.value > 10
    for args in ((4, 0, 20, 15, 0.9), (3, 1, 20, 50, 0.9), (2, 2, 20, 15, 0.9),
                 (2, 0, 20, 0, 0.9), (2, 0, 20, 65, 0.9), (3, 0, 20, 257, 0.9),
                 (2, 0, 20, 15, 0.0), (2, 0, 1, 15, 0.9), (3, 0, 1001, 50, 0.9)):
        code = L.rbffd_nodes_pds(*args, 1, rb._ptr(buf), rb._ptr(b), 10, ctypes.byref(n),
                                 r, s)
        assert code == rb.RBFFD_ERR_ARG


def test_solve_on_pds_nodes(rb, orc):
    """Supports, weights and 300 explicit steps on a Poisson-disc node set (m=4)."""
    Kg, m, seed = 50, 4, 9
    n = gen.stencil_size(2, m)
    xyz, bnd, _ = rb.rbffd_nodes_pds(0, Kg, seed)
    oxyz, obnd = orc.nodes_pds(0, Kg, seed)
    inter = rb.rbffd_interior(bnd)
    ointer = gen.interior_ids(obnd)
    idx = rb.rbffd_knn(xyz, inter, n)
    oidx = orc.knn_kdtree(oxyz, ointer, n)
    assert np.array_equal(H(idx), oidx)
    w, st = rb.rbffd_weights(xyz, idx, m)
    ow, ost = orc.weights(oxyz, oidx, m)
    assert np.all(ost == 0) and np.array_equal(H(st), ost)
    assert np.all(np.abs(H(w) - ow) <= 1e-12 * np.abs(ow).max(axis=1, keepdims=True))
    f = gen.source(oxyz, ointer)
    u0 = gen.start_iterate(oxyz, obnd)
    dt = 0.9 * orc.stable_dt(ow, oidx, ointer, oxyz.shape[1], gen.random_vector(len(ointer), 3),
                             200)
    ou, osteps, ores, _ = orc.solve_explicit(ow, oidx, ointer, f, u0, dt, 300, 0.0)
    plan = rb.Plan(xyz, bnd, inter, idx, w)
    u = torch.from_numpy(u0).cuda()
    code, steps, res = plan.solve_explicit(torch.from_numpy(f).cuda(), u, dt, 300, 0.0)
    assert steps == osteps == 300
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    plan.destroy()


# ---------------------------------------------------------------- 3D (unit cube)
@pytest.mark.parametrize("Kg,seed,K,zeta", [
    (6, 1, 50, 1 - 1e-10),
    (13, 2, 50, 1 - 1e-10),
    (25, 3, 50, 1 - 1e-10),
    (20, 4, 20, 1 - 1e-10),
    (18, 5, 80, 0.85),
])
def test_pds3_bit_exact(rb, orc, Kg, seed, K, zeta):
    xyz, bnd, rounds = rb.rbffd_nodes_pds(0, Kg, seed, K=K, zeta=zeta, d=3)
    oxyz, obnd = orc.nodes_pds3(Kg, seed, K=K, zeta=zeta)
    assert xyz.shape == oxyz.shape
    assert np.array_equal(H(xyz), oxyz) and np.array_equal(H(bnd), obnd)


def test_pds3_larger_bit_exact(rb, orc):
    """h = 1/70 in the unit cube: about 290,000 nodes."""
    xyz, bnd, rounds = rb.rbffd_nodes_pds(0, 70, 6, d=3)
    oxyz, obnd = orc.nodes_pds3(70, 6)
    assert np.array_equal(H(xyz), oxyz) and np.array_equal(H(bnd), obnd)
    assert rounds > 20


def test_pds3_capacity(rb):
    L = rb.lib()
    n, r = ctypes.c_int64(0), (ctypes.c_int64 * 2)()
    buf = torch.empty((3, 10), dtype=torch.float64, device="cuda")
    b = torch.empty(10, dtype=torch.uint8, device="cuda")
    code = L.rbffd_nodes_pds(3, 0, 8, 50, 1 - 1e-10, 1, rb._ptr(buf), rb._ptr(b), 10,
                             ctypes.byref(n), r, rb._stream("cuda"))
    assert code == rb.RBFFD_ERR_CAPACITY and n.value > 10


def test_supports_weights_on_pds3_nodes(rb, orc):
    """Supports and weights on a 3D Poisson-disc set (m = 2, n = 20) against the oracle."""
    Kg, m, seed = 12, 2, 7
    n = gen.stencil_size(3, m)
    xyz, bnd, _ = rb.rbffd_nodes_pds(0, Kg, seed, d=3)
    oxyz, obnd = orc.nodes_pds3(Kg, seed)
    inter = rb.rbffd_interior(bnd)
    ointer = gen.interior_ids(obnd)
    idx = rb.rbffd_knn(xyz, inter, n)
    oidx = orc.knn_kdtree(oxyz, ointer, n)
    assert np.array_equal(H(idx), oidx)
    w, st = rb.rbffd_weights(xyz, idx, m)
    ow, ost = orc.weights(oxyz, oidx, m)
    assert np.array_equal(H(st), ost)
    ok = ost == 0
    assert ok.mean() > 0.99
    assert np.all(np.abs(H(w)[ok] - ow[ok]) <= 1e-12 * np.abs(ow[ok]).max(axis=1, keepdims=True))


def test_convergence_order_on_pds_nodes(rb):
    """The whole GPU path on Poisson-disc squares (h = 1/20, 1/40, 1/80, m = 4),
    iterated to max|r| < 1e-10: the max error against u = sin(pi x) sin(pi y) falls
    at an observed order of at least m - 1 = 3 (the local truncation order)."""
    hs, errs = [], []
    for Kg in (20, 40, 80):
        xyz, bnd, _ = rb.rbffd_nodes_pds(0, Kg, 11)
        n = gen.stencil_size(2, 4)
        inter = rb.rbffd_interior(bnd)
        idx = rb.rbffd_knn(xyz, inter, n)
        w, st = rb.rbffd_weights(xyz, idx, 4)
        xh, bh, ih = H(xyz), H(bnd), H(inter)
        f = torch.from_numpy(gen.source(xh, ih)).cuda()
        u = torch.from_numpy(gen.start_iterate(xh, bh)).cuda()
        ua = torch.from_numpy(gen.exact_solution(xh)).cuda()
        plan = rb.Plan(xyz, bnd, inter, idx, w)
        dt, rho = plan.stable_dt(torch.from_numpy(gen.random_vector(len(ih), 3)).cuda(), 200)
        code, steps, res = plan.solve_explicit(f, u, 0.9 * dt, 2_000_000, 1e-10)
        assert code == rb.RBFFD_OK
        emax, _ = rb.rbffd_error(u, ua)
        hs.append(1.0 / Kg)
        errs.append(emax)
        plan.destroy()
    assert errs[0] > errs[1] > errs[2]
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert order >= 3.0, (errs, order)
