"""Parity at the workloads' full sizes, on outputs the oracle can compute one by one.

* 2D square, 1,002,001 nodes, m = 4 (the benchmark's configuration, Morton plan,
  graph launch mode): all node coordinates; supports and weights of 2,000 sampled
  rows against the oracle's brute-force supports and its weights; one explicit step
  from a seeded iterate on the sampled rows.
* 3D cube, 8,120,601 nodes, m = 4 (n = 70, s = 105): supports and weights of 300
  sampled rows.
* 2D square, 10,201 nodes, m = 2: the whole solve (tolerance 1e-10 or 20,000
  steps) against the oracle's.
"""
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


def test_square_1M_m4_sampled(rb, orc):
    d, Kg, m, seed = 2, 1000, 4, 2
    n = gen.stencil_size(d, m)
    xyz, bnd = rb.rbffd_nodes(d, 0, Kg, 0.3, seed)
    oxyz, obnd = orc.nodes(d, 0, Kg, 0.3, seed)
    assert np.array_equal(H(xyz), oxyz) and np.array_equal(H(bnd), obnd)
    inter = rb.rbffd_interior(bnd)
    ointer = gen.interior_ids(obnd)
    assert np.array_equal(H(inter), ointer)
    idx = rb.rbffd_knn(xyz, inter, n)
    w, st = rb.rbffd_weights(xyz, idx, m)
    rows = np.sort(np.random.default_rng(11).choice(len(ointer), 2000, replace=False))
    oidx = orc.knn_brute(oxyz, ointer[rows], n)
    assert np.array_equal(H(idx)[rows], oidx)
    ow, ost = orc.weights(oxyz, oidx, m)
    assert np.all(ost == 0)
    wr = H(w)[rows]
    assert np.all(np.abs(wr - ow) <= 1e-12 * np.abs(ow).max(axis=1, keepdims=True))
    # one explicit step from a seeded iterate, checked on the sampled rows
    plan = rb.Plan(xyz, bnd, inter, idx, w)
    u0 = gen.random_vector(len(oxyz[0]), 3, "uniform")
    f = gen.source(oxyz, ointer)
    dt = 3.7e-8
    u = torch.from_numpy(u0).cuda()
    plan.solve_explicit(torch.from_numpy(f).cuda(), u, dt, 1, 0.0)
    Lu = orc.apply(ow, oidx, u0)
    ref = u0[ointer[rows]] + dt * (Lu - f[rows])
    scale = np.abs(u0[ointer[rows]]) + dt * np.abs(ow * u0[oidx]).sum(axis=1)
    got = H(u)[ointer[rows]]
    assert np.all(np.abs(got - ref) <= 1e-12 * scale)
    plan.destroy()


def test_cube_8M_m4_sampled(rb, orc):
    d, Kg, m, seed = 3, 200, 4, 3
    n = gen.stencil_size(d, m)
    xyz, bnd = rb.rbffd_nodes(d, 0, Kg, 0.3, seed)
    oxyz, obnd = orc.nodes(d, 0, Kg, 0.3, seed)
    assert np.array_equal(H(xyz), oxyz)
    ointer = gen.interior_ids(obnd)
    rows = np.sort(np.random.default_rng(12).choice(len(ointer), 300, replace=False))
    centres = torch.from_numpy(ointer[rows]).cuda()
    idx = rb.rbffd_knn(xyz, centres, n)
    oidx = orc.knn_brute(oxyz, ointer[rows], n)
    assert np.array_equal(H(idx), oidx)
    w, st = rb.rbffd_weights(xyz, idx, m)
    ow, ost = orc.weights(oxyz, oidx, m)
    assert np.array_equal(H(st), ost)
    assert np.all(np.abs(H(w) - ow) <= 1e-12 * np.abs(ow).max(axis=1, keepdims=True))


def test_square_10k_full_solve(rb, orc):
    from oracle_problem import build
    p = build(orc, 2, 100, 2, seed=1)
    dt = 0.9 * orc.stable_dt(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, 7), 200)
    ou, osteps, ores, ost = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 20000, 1e-10)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for flags in (0, 16):
        plan = rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w), flags)
        u = T(p.u0)
        code, steps, res = plan.solve_explicit(T(p.f), u, dt, 20000, 1e-10)
        assert steps == osteps and res == ores
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
        plan.destroy()
    # the error against the closed form that the solve reaches (Eq. 8 and max)
    mx, mean = rb.rbffd_error(T(ou), T(p.ua))
    assert mean == pytest.approx(orc.mean_abs_error(ou, p.ua), rel=1e-13)
