"""GPU path vs the CPU oracle, element by element, through the C ABI.

Tolerances (fixed here, stated per check):
* node coordinates, interior lists, support indices: bit-exact;
* weights: per stencil max_j |dw_j| <= 1e-12 max_j |w_j|;
* stencil application: |d(Lu)_i| <= 1e-12 max(|Lu_i|, sum_j |w_ij u_j|);
* K-step FP64 sweep (K <= 1000): max |du| <= 1e-12 max |u|, same step count;
* FP32 defect correction: same outer/inner counts, max |du| <= 1e-12 max|u|;
* stability estimate: relative 1e-9 on rho;
* adjoint: max |dg| <= 1e-12 max |g| per gradient.
The kernels follow the oracle's operation order, so most of these are met
with equality; the tolerances leave room only for reduction order.
"""
import numpy as np
import pytest

import rbffd_inputs as gen
from oracle_problem import build

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


DEV = "cuda"


def T(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def H(t):
    return t.cpu().numpy()


# ------------------------------------------------------------------ nodes
@pytest.mark.parametrize("d,shape,Kg,seed", [(2, 0, 37, 1), (3, 0, 11, 2), (2, 1, 45, 3),
                                             (1, 0, 50, 4), (2, 0, 2, 5)])
def test_nodes_bit_exact(rb, orc, d, shape, Kg, seed):
    xyz, bnd = rb.rbffd_nodes(d, shape, Kg, 0.3, seed)
    oxyz, obnd = orc.nodes(d, shape, Kg, 0.3, seed)
    assert np.array_equal(H(xyz), oxyz)
    assert np.array_equal(H(bnd), obnd)
    inter = rb.rbffd_interior(bnd)
    assert np.array_equal(H(inter), gen.interior_ids(obnd))


def test_nodes_capacity_error(rb):
    import ctypes
    L = rb.lib()
    n = ctypes.c_int64(0)
    buf = torch.empty(10, dtype=torch.float64, device=DEV)
    b = torch.empty(10, dtype=torch.uint8, device=DEV)
    code = L.rbffd_nodes(2, 0, 20, 0.3, 1, rb._ptr(buf), rb._ptr(b), 5, ctypes.byref(n), None)
    assert code == rb.RBFFD_ERR_CAPACITY and n.value == 21 * 21


# ------------------------------------------------------------------ kNN
def _knn_case(orc, case):
    if case == "jit2_n12":
        xyz, bnd = orc.nodes(2, 0, 60, 0.3, 11)
        return xyz, gen.interior_ids(bnd), 12
    if case == "jit2_n30":
        xyz, bnd = orc.nodes(2, 0, 45, 0.3, 12)
        return xyz, gen.interior_ids(bnd), 30
    if case == "jit2_n56_all":
        xyz, bnd = orc.nodes(2, 0, 30, 0.3, 13)
        return xyz, np.arange(xyz.shape[1], dtype=np.int32), 56
    if case == "jit3_n70":
        xyz, bnd = orc.nodes(3, 0, 12, 0.3, 14)
        return xyz, gen.interior_ids(bnd), 70
    if case == "grid2_ties":
        xyz = gen.grid_points(23, 2)
        return xyz, np.arange(xyz.shape[1], dtype=np.int32), 30
    if case == "grid3_ties":
        xyz = gen.grid_points(9, 3)
        return xyz, np.arange(xyz.shape[1], dtype=np.int32), 35
    if case == "random2_clustered":
        rng = np.random.default_rng(5)
        a = rng.uniform(0, 1, (2, 2000))
        b = rng.normal(0.3, 0.002, (2, 600))      # dense cluster: many nodes per cell
        xyz = np.concatenate([a, b], axis=1)
        return xyz, rng.choice(xyz.shape[1], 500, replace=False).astype(np.int32), 40
    if case == "disk_n56":
        xyz, bnd = orc.nodes(2, 1, 50, 0.3, 15)
        return xyz, gen.interior_ids(bnd), 56
    if case == "tiny_n_eq_N":
        xyz = gen.random_points(9, 2, 3)
        return xyz, np.arange(9, dtype=np.int32), 9
    if case == "max_n128":
        xyz = gen.random_points(3000, 2, 4)
        return xyz, np.arange(0, 3000, 7, dtype=np.int32), 128
    if case == "line1d":
        xyz, bnd = orc.nodes(1, 0, 400, 0.3, 16)
        return xyz, gen.interior_ids(bnd), 7
    raise KeyError(case)


KNN_CASES = ["jit2_n12", "jit2_n30", "jit2_n56_all", "jit3_n70", "grid2_ties", "grid3_ties",
             "random2_clustered", "disk_n56", "tiny_n_eq_N", "max_n128", "line1d"]


@pytest.mark.parametrize("case", KNN_CASES)
def test_knn_bit_exact(rb, orc, case):
    xyz, centres, n = _knn_case(orc, case)
    ref = orc.knn_kdtree(xyz, centres, n)
    got = H(rb.rbffd_knn(T(xyz), T(centres), n))
    assert np.array_equal(got, ref)


def test_knn_empty_centres(rb):
    xyz = T(gen.random_points(50, 2, 1))
    idx = rb.rbffd_knn(xyz, torch.empty(0, dtype=torch.int32, device=DEV), 5)
    assert idx.shape == (0, 5)


# ------------------------------------------------------------------ weights
@pytest.mark.parametrize("d,m,Kg,nplus", [(2, 2, 40, 0), (2, 4, 35, 0), (2, 6, 30, 0),
                                          (3, 4, 10, 0), (2, 2, 30, 1), (3, 2, 10, 3),
                                          (2, 4, 30, 9), (1, 4, 200, 0)])
def test_weights_parity(rb, orc, d, m, Kg, nplus):
    xyz, bnd = orc.nodes(d, 0, Kg, 0.3, 21 + m)
    inter = gen.interior_ids(bnd)
    n = gen.stencil_size(d, m) + nplus
    idx = orc.knn_kdtree(xyz, inter, n)
    ow, ost = orc.weights(xyz, idx, m)
    w, st = rb.rbffd_weights(T(xyz), T(idx), m)
    w, st = H(w), H(st)
    assert np.array_equal(st, ost)
    scale = np.abs(ow).max(axis=1, keepdims=True)
    assert np.all(np.abs(w - ow) <= 1e-12 * scale)
    # the operation order is the oracle's, so nearly every row is bit-identical
    assert np.mean(np.all(w == ow, axis=1)) > 0.99


def test_weights_max_system(rb, orc):
    # s = n + M = 128 (largest supported): d=2, m=7 (M=36), n=92
    xyz, bnd = orc.nodes(2, 0, 30, 0.3, 8)
    inter = gen.interior_ids(bnd)[::37]
    idx = orc.knn_kdtree(xyz, inter, 92)
    ow, ost = orc.weights(xyz, idx, 7)
    w, st = rb.rbffd_weights(T(xyz), T(idx), 7)
    assert np.array_equal(H(st), ost)
    ok = ost == 0
    scale = np.abs(ow[ok]).max(axis=1, keepdims=True)
    assert np.all(np.abs(H(w)[ok] - ow[ok]) <= 1e-12 * scale)


def test_weights_singular_status(rb, orc):
    pts = np.array([[0.0, 0.1, 0.1, 0.0, 0.2, -0.1, 0.05, 0.3],
                    [0.0, 0.0, 0.0, 0.1, 0.1, 0.2, -0.1, 0.3]])
    idx = np.array([[0, 1, 2, 3, 4, 5, 6], [7, 0, 3, 4, 5, 6, 1]], np.int32)
    ow, ost = orc.weights(pts, idx, 2)
    w, st = rb.rbffd_weights(T(pts), T(idx), 2, check=False)
    assert list(H(st)) == list(ost) == [1, 0]
    assert np.all(H(w)[0] == 0)
    with pytest.raises(rb.RbffdError) as ei:
        rb.rbffd_weights(T(pts), T(idx), 2)
    assert ei.value.code == rb.RBFFD_ERR_SINGULAR


@pytest.mark.parametrize("d,m,Kg", [(2, 2, 20), (2, 4, 20), (2, 6, 18), (3, 4, 8)])
def test_weights_singular_rows_every_team_size(rb, orc, d, m, Kg):
    """A duplicated support node makes its stencil singular, for every team shape:
    half-warp teams (s = 18), one warp (s = 45), pivot warp + four update warps
    (s = 84, 105).  Status and weights match the oracle row by row; the singular rows
    sit next to regular ones (same warp or block)."""
    xyz, bnd = orc.nodes(d, 0, Kg, 0.3, 40 + m)
    inter = gen.interior_ids(bnd)
    n = gen.stencil_size(d, m)
    idx = orc.knn_kdtree(xyz, inter, n)
    for r in (0, 3, 17, len(inter) - 1):
        idx[r, 2] = idx[r, 1]
    ow, ost = orc.weights(xyz, idx, m)
    w, st = rb.rbffd_weights(T(xyz), T(idx), m, check=False)
    w, st = H(w), H(st)
    assert np.array_equal(st, ost)
    assert all(ost[r] == 1 for r in (0, 3, 17, len(inter) - 1))
    assert np.all(w[ost != 0] == 0)
    ok = ost == 0
    scale = np.abs(ow[ok]).max(axis=1, keepdims=True)
    assert np.all(np.abs(w[ok] - ow[ok]) <= 1e-12 * scale)


# ------------------------------------------------------------------ apply
def test_apply_parity(rb, orc):
    p = build(orc, 2, 50, 4, seed=31)
    u = gen.random_vector(p.N, 3)
    ref = orc.apply(p.w, p.idx, u)
    got = H(rb.rbffd_apply(T(p.w), T(p.idx), T(u)))
    bound = 1e-12 * np.maximum(np.abs(ref), np.abs(p.w * u[p.idx]).sum(axis=1))
    assert np.all(np.abs(got - ref) <= bound)


# ------------------------------------------------------------------ sweep
def _plan(rb, p, flags=0, seed=0):
    return rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w), flags, seed)


def _dt(orc, p):
    return 0.9 * orc.stable_dt(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, 77), 200)


SWEEP_CASES = [
    (2, 40, 2, 0, "morton_graph"),
    (2, 33, 4, 16, "morton_persistent"),
    (2, 30, 6, 1, "input_graph"),
    (2, 29, 4, 2 | 16, "random_persistent"),
    (3, 9, 4, 0, "cube_m4"),
    (2, 35, 4, 64, "morton_auto"),
    (2, 37, 6, 128, "morton_resident"),
    (2, 31, 2, 2 | 128, "random_resident"),
    (3, 10, 4, 128, "cube_resident"),
    (2, 34, 4, 32 | 128, "resident_int32_planes"),
    (2, 37, 4, 2048, "morton_resident_far"),
    (2, 31, 2, 2 | 2048, "random_resident_far"),
    (3, 10, 4, 2048, "cube_resident_far"),
    (2, 90, 4, 2048, "morton_resident_far_every_sm"),
]


@pytest.mark.parametrize("d,Kg,m,flags,name", SWEEP_CASES)
def test_sweep_parity_fixed_steps(rb, orc, d, Kg, m, flags, name):
    p = build(orc, d, Kg, m, seed=41)
    dt = _dt(orc, p)
    K = 300
    ou, os_, ores, ost = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
    plan = _plan(rb, p, flags, seed=9)
    u = T(p.u0)
    code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
    assert code == rb.RBFFD_NOT_CONVERGED and steps == os_ == K
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    assert res == pytest.approx(ores, rel=1e-12)
    plan.destroy()


# every stencil size with a kernel of its own (n fixed at compile time), in both
# launch modes: 2D m = 1 for n = 6 (= 2M), m = 2 for n = 12..57, 3D m = 4 for 70, 71
NN_CASES = [(2, 1, 6)] + [(2, 2, n) for n in (12, 13, 16, 20, 24, 30, 31, 40, 48, 56, 57)] + \
           [(3, 4, 70), (3, 4, 71)]


@pytest.mark.parametrize("d,m,n", NN_CASES)
def test_sweep_parity_every_compiled_stencil_size(rb, orc, d, m, n):
    """FP64 sweeps (graph, persistent and resident-with-far-lists launches) and a
    defect correction with FP32 inner sweeps, at each stencil size that has a
    specialised kernel; 529 interior rows in 2D (16 full slices and a ragged one),
    512 in 3D."""
    p = build(orc, d, 24 if d == 2 else 9, m, seed=48, n=n)
    dt = _dt(orc, p)
    K = 100
    ou, os_, ores, _ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
    for flags in (0, 16, 2048):
        plan = _plan(rb, p, flags)
        u = T(p.u0)
        code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
        assert steps == os_ == K
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou)), (n, flags)
        assert res == pytest.approx(ores, rel=1e-12)
        plan.destroy()
    args = (dt, 1e-7, 3, 400, 1e-3)
    du, oo, oi, _, ost = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, *args)
    plan = _plan(rb, p)
    u = T(p.u0)
    code, outer, inner, res = plan.solve_dc(T(p.f), u, *args)
    assert (outer, inner) == (oo, oi)
    assert np.max(np.abs(H(u) - du)) <= 1e-12 * np.max(np.abs(du))
    plan.destroy()


@pytest.mark.parametrize("d,m,n", NN_CASES)
def test_split_launch_every_compiled_stencil_size(rb, orc, d, m, n):
    """The split persistent launch at each stencil size that has a kernel of its
    own, in each block size it is compiled with (512; 1024 from n = 12 on), and at
    n = 30 also with int32 neighbour indices only: 50 FP64 sweeps and a defect
    correction (FP32 inner sweeps) against the oracle, on plans of at least two
    slices per SM (11,881 interior rows in 2D, 12,167 in 3D)."""
    p = build(orc, d, 110 if d == 2 else 24, m, seed=57, n=n)
    G = torch.cuda.get_device_properties(0).multi_processor_count
    assert (p.NI + 31) // 32 >= 2 * G
    dt = _dt(orc, p)
    K = 50
    ou, os_, ores, _ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
    args = (dt, 1e-7, 2, 60, 1e-3)
    du, oo, oi, _, _ = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, *args)
    shapes = [(th, 0) for th in ((512,) if n < 12 else (512, 1024))]
    if n == 30:   # and with int32 neighbour indices only
        shapes += [(512, rb.RBFFD_PACK_IDX32), (1024, rb.RBFFD_PACK_IDX32)]
    for threads, pack in shapes:
        plan = _plan(rb, p, rb.RBFFD_LAUNCH_SPLIT | pack)
        plan.set_block(threads)
        u = T(p.u0)
        code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
        assert steps == os_ == K
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou)), (n, threads)
        assert res == pytest.approx(ores, rel=1e-12)
        u2 = T(p.u0)
        code, outer, inner, res = plan.solve_dc(T(p.f), u2, *args)
        assert (outer, inner) == (oo, oi)
        assert np.max(np.abs(H(u2) - du)) <= 1e-12 * np.max(np.abs(du)), (n, threads)
        shape = plan.stats()[3]
        assert shape[1] == shape[3] == -2 and shape[0] == shape[2] == threads // 512
        plan.destroy()


def test_plan_set_block_rejects_other_sizes(rb, orc):
    p = build(orc, 2, 20, 2, seed=58)
    plan = _plan(rb, p, rb.RBFFD_LAUNCH_AUTO)
    for bad in (-1, 256, 768, 2048):
        with pytest.raises(rb.RbffdError) as ei:
            plan.set_block(bad)
        assert ei.value.code == rb.RBFFD_ERR_ARG
    plan.set_block(0)
    plan.destroy()


def test_sweep_stop_rule_matches(rb, orc):
    p = build(orc, 2, 24, 2, seed=42)
    dt = _dt(orc, p)
    # a tolerance the oracle reaches after a few hundred steps
    ou, os_, ores, ost = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 5000, 1.0)
    assert ost == 0 and 1 < os_ < 5000
    for flags in (0, 16, 128, 2048):
        plan = _plan(rb, p, flags)
        u = T(p.u0)
        code, steps, res = plan.solve_explicit(T(p.f), u, dt, 5000, 1.0)
        assert code == rb.RBFFD_OK and steps == os_ and res == ores
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
        plan.destroy()


def test_sweep_ragged_small_and_generic_n(rb, orc):
    # NI = 9 (one partial slice), n = 7 (generic-n kernel path)
    p = build(orc, 2, 4, 1, seed=43, n=7)
    dt = _dt(orc, p)
    for flags in (0, 16):
        ou, os_, _, _ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 50, 0.0)
        plan = _plan(rb, p, flags)
        u = T(p.u0)
        plan.solve_explicit(T(p.f), u, dt, 50, 0.0)
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * max(np.max(np.abs(ou)), 1e-300)
        plan.destroy()


def test_sweep_zero_steps_and_errors(rb, orc):
    p = build(orc, 2, 12, 2, seed=44)
    plan = _plan(rb, p)
    u = T(p.u0)
    code, steps, _ = plan.solve_explicit(T(p.f), u, 1e-5, 0, 0.0)
    assert steps == 0 and np.array_equal(H(u), p.u0)
    # non-finite source -> RBFFD_ERR_NONFINITE after one step (host-made failure)
    f = p.f.copy()
    f[5] = np.inf
    with pytest.raises(rb.RbffdError) as ei:
        plan.solve_explicit(T(f), T(p.u0), 1e-5, 100, 0.0)
    assert ei.value.code == rb.RBFFD_ERR_NONFINITE
    # dt far above the stability bound -> RBFFD_ERR_DIVERGED, both launch modes
    for flags in (0, 16):
        pl = _plan(rb, p, flags)
        with pytest.raises(rb.RbffdError) as ei:
            pl.solve_explicit(T(p.f), T(p.u0), 50 * _dt(orc, p), 5000, 0.0)
        assert ei.value.code == rb.RBFFD_ERR_DIVERGED
        pl.destroy()
    with pytest.raises(rb.RbffdError):
        plan.solve_explicit(T(p.f), T(p.u0), -1.0, 10, 0.0)
    plan.destroy()


def test_launch_modes_same_bits(rb, orc):
    """Graph (tuned, with and without programmatic dependent launches), persistent,
    resident and autotuned launch modes: the same FP64 iterate and the same
    defect-corrected iterate bit for bit; the reported shape says which mode ran
    (0 blocks per SM = persistent, -1 = resident, + 16 = programmatic launches)."""
    p = build(orc, 2, 30, 4, seed=47)
    dt = _dt(orc, p)
    outs = []
    for flags in (0, 16, 64, 128, 256, 512, 2048):
        plan = _plan(rb, p, flags)
        u = T(p.u0)
        plan.solve_explicit(T(p.f), u, dt, 500, 0.0)
        u2 = T(p.u0)
        plan.solve_dc(T(p.f), u2, dt, 0.0, 2, 200, 0.0)
        shape = plan.stats()[3]
        if flags == 0:
            assert shape[1] > 0 and shape[3] > 0
        if flags == 16:
            assert shape[1] == 0 and shape[3] == 0
        if flags == 128:
            assert shape[1] == -1 and shape[3] == -1
        if flags == 256:
            assert shape[1] > 16 and shape[3] > 16
        if flags == 512:
            assert 0 < shape[1] <= 4 and 0 < shape[3] <= 4
        if flags == 2048:
            assert shape[1] == -1 and shape[3] == -1 and shape[0] >= 4 and shape[2] >= 4
        outs.append((H(u), H(u2)))
        plan.destroy()
    for a, b in outs[1:]:
        assert np.array_equal(a, outs[0][0]) and np.array_equal(b, outs[0][1])


def test_plan_rejects_bad_interior(rb, orc):
    p = build(orc, 2, 10, 2, seed=45)
    bad = p.interior.copy()
    bad[3] = np.nonzero(p.is_bnd)[0][0]       # a boundary node in the interior list
    with pytest.raises(rb.RbffdError):
        rb.Plan(T(p.xyz), T(p.is_bnd), T(bad), T(p.idx), T(p.w))


def test_orderings_are_permutations(rb, orc):
    p = build(orc, 2, 20, 2, seed=46)
    for flags in (0, 1, 2):
        plan = _plan(rb, p, flags, seed=3)
        perm = H(plan.perm())
        assert np.array_equal(np.sort(perm), np.arange(p.N))
        assert np.all(p.is_bnd[perm[: p.NI]] == 0)
        plan.destroy()


# ------------------------------------------------------------------ stable dt
def test_stable_dt_parity(rb, orc):
    p = build(orc, 2, 30, 4, seed=51)
    v0 = gen.random_vector(p.NI, 5)
    rho = orc.power_rho(p.w, p.idx, p.interior, p.N, v0, 200)
    plan = _plan(rb, p)
    dt, rho_g = plan.stable_dt(T(v0), 200, 1.05)
    assert rho_g == pytest.approx(rho, rel=1e-9)
    assert dt == pytest.approx(2.0 / (1.05 * rho), rel=1e-9)
    plan.destroy()


# ------------------------------------------------------------------ defect correction
def test_dc_parity(rb, orc):
    p = build(orc, 2, 20, 4, seed=61)
    dt = _dt(orc, p)
    args = (dt, 1e-8, 30, 3000, 1e-3)
    ou, oo, oi, ores, ost = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, *args)
    for flags in (0, 128, 32 | 128, 2048):  # graph; resident (16-bit, int32 planes; far lists)
        plan = _plan(rb, p, flags)
        u = T(p.u0)
        code, outer, inner, res = plan.solve_dc(T(p.f), u, *args)
        assert (outer, inner) == (oo, oi)
        assert code == (rb.RBFFD_OK if ost == 0 else rb.RBFFD_NOT_CONVERGED)
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
        plan.destroy()


# ------------------------------------------------------------------ adjoint
def test_adjoint_parity(rb, orc):
    p = build(orc, 2, 25, 4, seed=71)
    dt = _dt(orc, p)
    K = 200
    dLdu = np.zeros(p.N)
    sens = gen.sensors(p.NI, 40, 2)
    dLdu[p.interior[sens]] = gen.random_vector(40, 3)
    gf, gg, l0 = orc.adjoint(p.w, p.idx, p.interior, p.N, dLdu, K, dt)
    # reverse steps as plain and as programmatic dependent launches
    for flags in (rb.RBFFD_LAUNCH_NO_PDL, rb.RBFFD_LAUNCH_PDL):
        plan = _plan(rb, p, flags)
        plan.transpose()
        plan.transpose()                  # a second call keeps the built transpose
        g_f, g_g, g_l0 = plan.adjoint(T(dLdu), K, dt)
        for a, b in ((H(g_f), gf), (H(g_g), gg), (H(g_l0), l0)):
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
        plan.destroy()


def test_adjoint_with_boundary_sensors(rb, orc):
    """A loss that also observes boundary nodes: dL/dg gets the direct term inside
    the library (rbffd_adjoint through the C ABI), against the oracle and against
    central differences of the GPU forward solve (the loss is quadratic in f, g)."""
    import ctypes
    p = build(orc, 2, 22, 4, seed=74)
    dt = _dt(orc, p)
    K = 80
    bnd = np.nonzero(p.is_bnd)[0]
    sens = gen.sensors(p.NI, 30, 7)
    bsens = bnd[::4]
    g = p.u0[bnd] + 0.1 * gen.random_vector(len(bnd), 8)
    uobs = p.ua[p.interior][sens]
    bobs = gen.random_vector(len(bsens), 9)
    plan = _plan(rb, p)

    def forward(f, gb):
        u = p.u0.copy()
        u[bnd] = gb
        u = T(u)
        plan.solve_explicit(T(f), u, dt, K, 0.0)
        return H(u)

    def loss(f, gb):
        u = forward(f, gb)
        return np.sum((u[p.interior][sens] - uobs) ** 2) + np.sum((u[bsens] - bobs) ** 2)

    uK = forward(p.f, g)
    dLdu = np.zeros(p.N)
    dLdu[p.interior[sens]] = 2 * (uK[p.interior][sens] - uobs)
    dLdu[bsens] = 2 * (uK[bsens] - bobs)
    gf, gg, l0 = orc.adjoint(p.w, p.idx, p.interior, p.N, dLdu, K, dt)
    L = rb.lib()
    d_dLdu = T(dLdu)
    g_f = torch.empty(p.NI, dtype=torch.float64, device=DEV)
    g_g = torch.empty(p.N, dtype=torch.float64, device=DEV)
    code = L.rbffd_adjoint(plan.handle, rb._ptr(d_dLdu), K, dt, rb._ptr(g_f), rb._ptr(g_g),
                           None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == rb.RBFFD_OK
    torch.cuda.synchronize()
    for a, b in ((H(g_f), gf), (H(g_g), gg)):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    assert np.all(H(g_g)[p.interior] == 0)
    rng = np.random.default_rng(3)
    for _ in range(4):
        vf = rng.standard_normal(p.NI)
        vg = rng.standard_normal(len(bnd))
        eps = 1e-3
        fd = (loss(p.f + eps * vf, g + eps * vg) - loss(p.f - eps * vf, g - eps * vg)) / (2 * eps)
        an = H(g_f) @ vf + H(g_g)[bnd] @ vg
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12)
    plan.destroy()


# ------------------------------------------------------------------ whole pipeline on GPU
def test_pipeline_gpu_vs_oracle(rb, orc):
    d, Kg, m, seed = 2, 64, 4, 81
    n = gen.stencil_size(d, m)
    xyz, bnd = rb.rbffd_nodes(d, 0, Kg, 0.3, seed)
    inter = rb.rbffd_interior(bnd)
    idx = rb.rbffd_knn(xyz, inter, n)
    w, st = rb.rbffd_weights(xyz, idx, m)
    p = build(orc, d, Kg, m, seed=seed)
    assert np.array_equal(H(idx), p.idx)
    scale = np.abs(p.w).max(axis=1, keepdims=True)
    assert np.all(np.abs(H(w) - p.w) <= 1e-12 * scale)
    dt = _dt(orc, p)
    plan = rb.Plan(xyz, bnd, inter, idx, w)
    u = T(p.u0)
    plan.solve_explicit(T(p.f), u, dt, 400, 0.0)
    ou, *_ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 400, 0.0)
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    plan.destroy()


# ------------------------------------------------------------------ error metric (Eq. 8)
def test_error_metric(rb, orc):
    p = build(orc, 2, 30, 4, seed=91)
    u = p.u0 + gen.random_vector(p.N, 4) * 1e-3
    mx, mean = rb.rbffd_error(T(u), T(p.ua))
    assert mx == np.max(np.abs(u - p.ua))
    assert mean == pytest.approx(orc.mean_abs_error(u, p.ua), rel=1e-13)


# ------------------------------------------------------------------ weight gradient, autograd
def test_adjoint_w_parity_and_checkpoint_invariance(rb, orc):
    p = build(orc, 2, 18, 4, seed=72)
    dt = _dt(orc, p)
    K = 60
    lamK = np.zeros(p.N)
    lamK[p.interior[gen.sensors(p.NI, 20, 3)]] = gen.random_vector(20, 4)
    lamK[np.nonzero(p.is_bnd)[0][::5]] = gen.random_vector(len(np.nonzero(p.is_bnd)[0][::5]), 5)
    gw, gf, gg, l0 = orc.adjoint_w(p.w, p.idx, p.interior, p.f, p.u0, lamK, K, dt)
    plan = _plan(rb, p)
    results = []
    for every in (1, 7, K):
        # checkpoints of the forward run, every `every` steps
        u = T(p.u0)
        ck = []
        done = 0
        while done < K:
            ck.append(u.clone())
            s = min(every, K - done)
            plan.solve_explicit(T(p.f), u, dt, s, 0.0)
            done += s
        res = plan.adjoint_w(T(p.f), torch.stack(ck), every, T(lamK), K, dt)
        results.append(res)
        for a, b in zip(res, (gw, gf, gg, l0)):
            assert np.max(np.abs(H(a) - b)) <= 1e-12 * np.max(np.abs(b))
    # the replayed iterates are the forward's: checkpoint spacing changes nothing
    for r in results[1:]:
        for a, b in zip(r, results[0]):
            assert torch.equal(a, b)
    plan.destroy()


def test_autograd_function_matches_oracle(rb, orc):
    p = build(orc, 2, 16, 2, seed=73)
    dt = _dt(orc, p)
    K = 45
    sens = gen.sensors(p.NI, 15, 6)
    uobs = p.ua[p.interior][sens]
    solver = rb.ExplicitSolver(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), K, dt)
    bnd = np.nonzero(p.is_bnd)[0]
    f = T(p.f).requires_grad_(True)
    g = T(p.u0[bnd]).requires_grad_(True)
    w = T(p.w).requires_grad_(True)
    uK = solver(f, g, w)
    bsens = bnd[::3]                 # boundary nodes observed too (u^K = g there)
    bobs = gen.random_vector(len(bsens), 11)
    loss = ((uK[T(p.interior).long()[T(sens).long()]] - T(uobs)) ** 2).sum() + \
        ((uK[T(bsens).long()] - T(bobs)) ** 2).sum()
    loss.backward()
    # oracle: forward, dL/du^K, then the weight-aware adjoint
    ou, *_ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
    assert np.max(np.abs(H(uK.detach()) - ou)) <= 1e-12 * np.max(np.abs(ou))
    lamK = np.zeros(p.N)
    lamK[p.interior[sens]] = 2 * (ou[p.interior][sens] - uobs)
    lamK[bsens] = 2 * (ou[bsens] - bobs)
    gw, gf, gg, _ = orc.adjoint_w(p.w, p.idx, p.interior, p.f, p.u0, lamK, K, dt)
    for a, b in ((f.grad, gf), (g.grad, gg[bnd]), (w.grad, gw)):
        assert np.max(np.abs(H(a) - b)) <= 1e-12 * np.max(np.abs(b))


# ------------------------------------------------------------------ bounded waits
def test_persistent_barrier_wait_runs_out(rb, orc):
    """The persistent launch's grid barrier is a bounded wait.  With one arrival
    withheld (a failure injected on the host: the barrier waits for a block that
    does not exist) every block gives up after the 20 ms limit, the solve returns
    RBFFD_ERR_TIMEOUT and the context stays usable: the same plan then solves
    normally, bit-identical to the oracle."""
    import time
    p = build(orc, 2, 30, 4, seed=49)
    dt = _dt(orc, p)
    plan = _plan(rb, p, rb.RBFFD_LAUNCH_PERSISTENT)
    plan.solve_explicit(T(p.f), T(p.u0), dt, 5, 0.0)          # tunes, no waits run out
    plan.set_wait(20.0, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with pytest.raises(rb.RbffdError) as ei:
        plan.solve_explicit(T(p.f), T(p.u0), dt, 100, 0.0)
    el = time.perf_counter() - t0
    assert ei.value.code == rb.RBFFD_ERR_TIMEOUT
    assert el < 5.0                                           # gave up, did not hang
    # FP32 inner steps of defect correction: the same barrier, the same outcome
    with pytest.raises(rb.RbffdError) as ei:
        plan.solve_dc(T(p.f), T(p.u0), dt, 0.0, 1, 50, 0.0)
    assert ei.value.code == rb.RBFFD_ERR_TIMEOUT
    plan.set_wait(0.0, 0)
    ou, *_ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 100, 0.0)
    u = T(p.u0)
    code, steps, res = plan.solve_explicit(T(p.f), u, dt, 100, 0.0)
    assert steps == 100
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    plan.destroy()
    # the resident launch's barrier (with or without far lists) is the same bounded wait
    for flags in (rb.RBFFD_LAUNCH_RESIDENT, rb.RBFFD_LAUNCH_FAR):
        plan = _plan(rb, p, flags)
        plan.solve_explicit(T(p.f), T(p.u0), dt, 5, 0.0)
        plan.set_wait(20.0, 1)
        with pytest.raises(rb.RbffdError) as ei:
            plan.solve_explicit(T(p.f), T(p.u0), dt, 100, 0.0)
        assert ei.value.code == rb.RBFFD_ERR_TIMEOUT
        plan.set_wait(0.0, 0)
        u = T(p.u0)
        plan.solve_explicit(T(p.f), u, dt, 100, 0.0)
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
        plan.destroy()
    # the split launch (a plan of at least two slices per SM): the same bounded
    # wait, while its other warps compute the inner slices
    q = build(orc, 2, 110, 4, seed=53)
    dtq = _dt(orc, q)
    qu, *_ = orc.solve_explicit(q.w, q.idx, q.interior, q.f, q.u0, dtq, 100, 0.0)
    plan = _plan(rb, q, rb.RBFFD_LAUNCH_SPLIT)
    plan.solve_explicit(T(q.f), T(q.u0), dtq, 5, 0.0)
    plan.set_wait(20.0, 1)
    for solve in (lambda: plan.solve_explicit(T(q.f), T(q.u0), dtq, 100, 0.0),
                  lambda: plan.solve_dc(T(q.f), T(q.u0), dtq, 0.0, 1, 50, 0.0)):
        with pytest.raises(rb.RbffdError) as ei:
            solve()
        assert ei.value.code == rb.RBFFD_ERR_TIMEOUT
    plan.set_wait(0.0, 0)
    u = T(q.u0)
    plan.solve_explicit(T(q.f), u, dtq, 100, 0.0)
    assert np.max(np.abs(H(u) - qu)) <= 1e-12 * np.max(np.abs(qu))
    assert plan.stats()[3][1] == -2
    plan.destroy()


def test_resident_launch_refuses_a_plan_too_large(rb):
    """The resident launch keeps a plan's stencils in shared memory; 158,404 rows of 30
    FP64 entries (about 313 KB per SM) do not fit, and a plan that asks for it gets
    RBFFD_ERR_CAPACITY from its first solve (nothing launched)."""
    xyz, bnd = rb.rbffd_nodes(2, 0, 399, 0.3, 3)
    inter = rb.rbffd_interior(bnd)
    idx = rb.rbffd_knn(xyz, inter, 30)
    w, st = rb.rbffd_weights(xyz, idx, 4)
    plan = rb.Plan(xyz, bnd, inter, idx, w, rb.RBFFD_LAUNCH_RESIDENT)
    f = torch.zeros(inter.numel(), dtype=torch.float64, device=DEV)
    with pytest.raises(rb.RbffdError) as ei:
        plan.solve_explicit(f, torch.zeros(xyz.shape[1], dtype=torch.float64, device=DEV),
                            1e-9, 10, 0.0)
    assert ei.value.code == rb.RBFFD_ERR_CAPACITY
    plan.destroy()


def test_graph_replays_launch_exactly_the_steps_asked(rb, orc):
    """Graph mode replays 32-launch chunks and then one graph per set bit of the
    remainder, so a run of K steps launches K step kernels (no early-exit tail)
    besides the solve's fixed few (gathers of f and u, scatter of u)."""
    p = build(orc, 2, 20, 2, seed=50)
    dt = _dt(orc, p)
    plan = _plan(rb, p)
    extra = set()
    for K in (1, 31, 32, 33, 200, 77):
        ou, *_ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
        u = T(p.u0)
        code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
        ms, loop_steps, launches, shape = plan.stats()
        assert steps == loop_steps == K
        assert shape[1] != 0                     # the default plan replays graphs
        extra.add(launches - K)
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    assert len(extra) == 1 and 0 <= extra.pop() <= 4
    plan.destroy()


@pytest.mark.parametrize("halo", [-1, 0, 64, 1 << 20])
def test_resident_halo_windows_same_bits(rb, orc, halo):
    """The resident launch with its halo window fixed: none, the block's own rows, a
    reach of 64 slots, and the whole iterate - FP64 sweeps and a defect correction,
    equal to the oracle, the same bits whatever the window."""
    p = build(orc, 2, 41, 4, seed=51)
    dt = _dt(orc, p)
    ou, *_ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 150, 0.0)
    du, oo, oi, _, _ = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, dt, 1e-7, 3, 300, 1e-3)
    plan = _plan(rb, p, rb.RBFFD_LAUNCH_RESIDENT)
    plan.set_resident_halo(halo)
    u = T(p.u0)
    plan.solve_explicit(T(p.f), u, dt, 150, 0.0)
    assert plan.stats()[3][1] == -1
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    u2 = T(p.u0)
    code, outer, inner, res = plan.solve_dc(T(p.f), u2, dt, 1e-7, 3, 300, 1e-3)
    assert (outer, inner) == (oo, oi)
    assert np.max(np.abs(H(u2) - du)) <= 1e-12 * np.max(np.abs(du))
    plan.destroy()


def _share_inner_flags(p, perm, G):
    """Per resident share (block b of G owns slices [nsl b / G, nsl (b+1) / G)):
    for each of its rows, whether every neighbour is a row of the same share."""
    NI = p.NI
    slot = np.empty(p.N, np.int64)
    slot[perm] = np.arange(p.N)
    row_of_node = np.full(p.N, -1, np.int64)
    row_of_node[p.interior] = np.arange(NI)
    cols = slot[p.idx[row_of_node[perm[:NI]]]]        # [slot][j] neighbour slots
    nsl = (NI + 31) // 32
    out = []
    for b in range(G):
        r0, r1 = nsl * b // G * 32, min(nsl * (b + 1) // G * 32, NI)
        c = cols[r0:r1]
        out.append(np.all((c >= r0) & (c < r1), axis=1))
    return out


@pytest.mark.parametrize("Kg", [200, 300])
def test_resident_shares_inner_rows_first(rb, orc, Kg):
    """Morton plans that may take the resident or split launch put, in each SM's
    share of the rows, the rows whose stencils stay inside the share first (each
    group in Morton order); those launches compute these slices while they wait
    at the step barrier.  40k- and 90k-node squares: the order's invariant (the
    same set of inner rows as plain Morton order, now leading each share), then
    300 FP64 sweeps and a defect correction in the resident launches (window and
    L2, far lists), the split launch and the autotuner's pick, against the
    oracle."""
    p = build(orc, 2, Kg, 4, seed=67)
    G = torch.cuda.get_device_properties(0).multi_processor_count
    dt = _dt(orc, p)
    K = 300
    ou, os_, ores, ost = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
    args = (dt, 1e-7, 3, 400, 1e-3)
    du, oo, oi, _, _ = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, *args)
    plain = _plan(rb, p, rb.RBFFD_LAUNCH_GRAPH)
    pperm = H(plain.perm())
    ref = _share_inner_flags(p, pperm, G)
    plain.destroy()
    # the expected order: per share, plain Morton order's inner rows, then the others
    nsl = (p.NI + 31) // 32
    expect = pperm.copy()
    for b, fl in enumerate(ref):
        r0, r1 = nsl * b // G * 32, min(nsl * (b + 1) // G * 32, p.NI)
        seg = pperm[r0:r1]
        expect[r0:r1] = np.concatenate([seg[fl], seg[~fl]])
    for flags, kind in ((rb.RBFFD_LAUNCH_RESIDENT, -1), (rb.RBFFD_LAUNCH_FAR, -1),
                        (rb.RBFFD_LAUNCH_SPLIT, -2), (rb.RBFFD_LAUNCH_AUTO, None)):
        plan = _plan(rb, p, flags)
        perm = H(plan.perm())
        assert np.array_equal(perm, expect)              # stable: each group in Morton order
        flags_b = _share_inner_flags(p, perm, G)
        for a, b in zip(ref, flags_b):
            assert a.sum() == b.sum()                       # the same inner rows
            assert np.all(np.diff(b.astype(np.int8)) <= 0)  # inner rows lead the share
        assert sum(b.sum() for b in flags_b) > 32 * G       # whole inner slices exist
        u = T(p.u0)
        code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
        assert code == rb.RBFFD_NOT_CONVERGED and steps == os_ == K
        assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
        assert res == pytest.approx(ores, rel=1e-12)
        u2 = T(p.u0)
        code, outer, inner, res = plan.solve_dc(T(p.f), u2, *args)
        assert (outer, inner) == (oo, oi)
        assert np.max(np.abs(H(u2) - du)) <= 1e-12 * np.max(np.abs(du))
        if kind is not None:
            shape = plan.stats()[3]
            assert shape[1] == kind and shape[3] == kind   # resident / split, both sweeps
        plan.destroy()
