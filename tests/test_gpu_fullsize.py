"""Parity at the workloads' full sizes, on outputs the oracle can compute one by one.

* 2D square, 1,002,001 nodes, m = 4 (the benchmark's configuration, Morton plan,
  graph launch mode): all node coordinates; supports and weights of 2,000 sampled
  rows against the oracle's brute-force supports and its weights; one explicit step
  from a seeded iterate on the sampled rows.
* the same configuration, every row: 50 FP64 sweeps and one defect correction of
  50 FP32 inner steps from a seeded iterate, on a plan of the oracle's supports and
  weights (the plan mixes 16-bit and 32-bit index slices, as the benchmark's does).
* 3D cube, 8,120,601 nodes, m = 4 (n = 70, s = 105): supports and weights of 300
  sampled rows; one explicit step of the full GPU-built plan on 2,000 sampled rows.
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


def test_square_1M_m4_all_rows(rb, orc):
    """Every row of the benchmark's problem: K = 50 FP64 sweeps and one defect
    correction of K_in = 50 FP32 inner steps, from a seeded iterate, against the
    oracle's iterations (Eq. 6), max |du| <= 1e-12 max |u|."""
    d, Kg, m, seed = 2, 1000, 4, 2
    n = gen.stencil_size(d, m)
    oxyz, obnd = orc.nodes(d, 0, Kg, 0.3, seed)
    ointer = gen.interior_ids(obnd)
    oidx = orc.knn_kdtree(oxyz, ointer, n)
    ow, ost = orc.weights(oxyz, oidx, m)
    assert np.all(ost == 0)
    f = gen.source(oxyz, ointer)
    u0 = gen.random_vector(oxyz.shape[1], 5, "uniform")
    dt = 3.7e-8
    K = 50
    ou, osteps, ores, _ = orc.solve_explicit(ow, oidx, ointer, f, u0, dt, K, 0.0)
    # defect correction: one outer pass of 50 FP32 inner steps
    du, oo, oi, ores_dc, _ = orc.solve_dc(ow, oidx, ointer, f, u0, dt, 0.0, 1, K, 0.0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # graph-replayed steps, and the split persistent launch (each SM's share of
    # rows ordered inner rows first, its iterate in shared memory)
    for flags in (rb.RBFFD_LAUNCH_GRAPH, rb.RBFFD_LAUNCH_SPLIT):
        plan = rb.Plan(T(oxyz), T(obnd), T(ointer), T(oidx), T(ow), rb.RBFFD_ORDER_MORTON | flags)
        lay = plan.layout()
        assert 0 < lay["rows16"] < len(ointer)          # both kinds of slice run
        u = T(u0)
        code, steps, res = plan.solve_explicit(T(f), u, dt, K, 0.0)
        assert steps == osteps == K
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
        assert res == pytest.approx(ores, rel=1e-12)
        u = T(u0)
        code, outer, inner, res_dc = plan.solve_dc(T(f), u, dt, 0.0, 1, K, 0.0)
        assert (outer, inner) == (oo, oi) == (1, K)
        assert np.max(np.abs(H(u) - du)) <= 1e-12 * np.max(np.abs(du))
        assert res_dc == pytest.approx(ores_dc, rel=1e-12)
        if flags == rb.RBFFD_LAUNCH_SPLIT:
            shape = plan.stats()[3]
            assert shape[1] == -2 and shape[3] == -2
        plan.destroy()


def test_cube_8M_m4_one_step_sampled(rb, orc):
    """The 3D workload's whole GPU pipeline (nodes, supports, weights of all
    7,880,599 rows, Morton plan with 16-bit and 32-bit slices), one explicit step
    from a seeded iterate, checked on 2,000 sampled rows against the oracle's
    brute-force supports, its weights and its stencil sums."""
    d, Kg, m, seed = 3, 200, 4, 3
    n = gen.stencil_size(d, m)
    xyz, bnd = rb.rbffd_nodes(d, 0, Kg, 0.3, seed)
    inter = rb.rbffd_interior(bnd)
    idx = rb.rbffd_knn(xyz, inter, n)
    w, st = rb.rbffd_weights(xyz, idx, m)
    plan = rb.Plan(xyz, bnd, inter, idx, w, rb.RBFFD_ORDER_MORTON)
    lay = plan.layout()
    assert 0 < lay["rows16"] < inter.numel()
    del idx, w
    oxyz, obnd = orc.nodes(d, 0, Kg, 0.3, seed)
    ointer = gen.interior_ids(obnd)
    assert np.array_equal(H(inter), ointer)
    u0 = gen.random_vector(oxyz.shape[1], 6, "uniform")
    f = gen.source(oxyz, ointer)
    dt = 1e-6
    u = torch.from_numpy(u0).cuda()
    plan.solve_explicit(torch.from_numpy(f).cuda(), u, dt, 1, 0.0)
    rows = np.sort(np.random.default_rng(13).choice(len(ointer), 2000, replace=False))
    oidx = orc.knn_brute(oxyz, ointer[rows], n)
    ow, ost = orc.weights(oxyz, oidx, m)
    assert np.all(ost == 0)
    Lu = orc.apply(ow, oidx, u0)
    ref = u0[ointer[rows]] + dt * (Lu - f[rows])
    scale = np.abs(u0[ointer[rows]]) + dt * np.abs(ow * u0[oidx]).sum(axis=1)
    got = H(u)[ointer[rows]]
    assert np.all(np.abs(got - ref) <= 1e-12 * scale)
    # boundary values are held
    b = np.nonzero(obnd)[0][::101]
    assert np.array_equal(H(u)[b], u0[b])
    plan.destroy()
