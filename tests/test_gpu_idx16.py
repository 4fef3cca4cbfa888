"""Compact 16-bit neighbour codes of the packed sweep layout, through the C ABI.

A plan stores each 32-row slice's neighbour slots as 16-bit codes against up
to four window bases of 2^14 slots (the default), or as 32-bit slots
(RBFFD_PACK_IDX32, and any slice the four windows cannot cover).  The codes
name the same neighbours, so both layouts give the same iterates bit for bit,
and both match the oracle within the sweep tolerance (max |du| <= 1e-12 max|u|).

Cases: one window (N < 2^14); two to four windows (seeded random node order
with 2^15 < N < 2^16, so every slice spans the whole slot range); the 32-bit
fallback (random order with N = 160,801: no slice fits in four windows); and
the 1,002,001-node Morton plan, where both kinds of slice occur in one launch.
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


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


def _plan(rb, p, flags, seed=5):
    return rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w), flags, seed)


def _dt(orc, p):
    return 0.9 * orc.stable_dt(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, 77), 200)


def _layout_bytes(p, rows16, nslices, compact):
    idx = 2 * p.n * rows16 + 4 * p.n * (p.NI - rows16) + (16 * nslices if compact else 0)
    return p.NI * (8 * p.n + 24) + idx, p.NI * (4 * p.n + 12) + idx


CASES = [
    (40, 2, 0, "one_window"),
    (220, 2, 2, "random_multi_window"),
    (400, 2, 2, "random_int32_fallback"),
]


@pytest.mark.parametrize("Kg,m,order,name", CASES)
def test_codes_match_int32_and_oracle(rb, orc, Kg, m, order, name):
    p = build(orc, 2, Kg, m, seed=81)
    dt = _dt(orc, p)
    K = 100
    ou, osteps, ores, _ = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, K, 0.0)
    for launch in (0, 16):
        res = {}
        for pack in (0, rb.RBFFD_PACK_IDX32):
            plan = _plan(rb, p, order | launch | pack)
            L = plan.layout()
            nsl = (p.NI + 31) // 32
            assert L["nslices"] == nsl
            if pack:
                assert L["rows16"] == 0
            elif name == "random_int32_fallback":
                assert L["rows16"] < 0.01 * p.NI
            else:
                assert L["rows16"] == p.NI      # N < 2^16: four windows always suffice
            b64, b32 = _layout_bytes(p, L["rows16"], nsl, not pack)
            assert L["bytes64"] == b64 and L["bytes32"] == b32
            u = T(p.u0)
            code, steps, r = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
            assert steps == osteps == K
            res[pack] = (H(u), r)
            plan.destroy()
        u16, r16 = res[0]
        u32, r32 = res[rb.RBFFD_PACK_IDX32]
        assert np.array_equal(u16, u32) and r16 == r32
        assert np.max(np.abs(u16 - ou)) <= 1e-12 * np.max(np.abs(ou))
        assert r16 == pytest.approx(ores, rel=1e-12)


def test_codes_fp32_defect_correction(rb, orc):
    p = build(orc, 2, 220, 2, seed=82)
    dt = _dt(orc, p)
    args = (dt, 1e-6, 6, 2000, 1e-3)
    ou, oo, oi, ores, ost = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, *args)
    out = {}
    for pack in (0, rb.RBFFD_PACK_IDX32):
        plan = _plan(rb, p, 2 | pack)
        u = T(p.u0)
        code, outer, inner, res = plan.solve_dc(T(p.f), u, *args)
        assert (outer, inner) == (oo, oi)
        out[pack] = H(u)
        plan.destroy()
    assert np.array_equal(out[0], out[rb.RBFFD_PACK_IDX32])
    assert np.max(np.abs(out[0] - ou)) <= 1e-12 * np.max(np.abs(ou))


def test_codes_square_1M_mixed_slices(rb, orc):
    """The 1,002,001-node m=4 Morton plan: compact and int32 slices in one launch.
    Five steps from a seeded iterate, bit-equal to the int32 layout, and the
    first step on 2,000 sampled rows against the oracle's stencil sums."""
    d, Kg, m, seed = 2, 1000, 4, 2
    n = gen.stencil_size(d, m)
    xyz, bnd = rb.rbffd_nodes(d, 0, Kg, 0.3, seed)
    inter = rb.rbffd_interior(bnd)
    idx = rb.rbffd_knn(xyz, inter, n)
    w, st = rb.rbffd_weights(xyz, idx, m)
    NI = inter.numel()
    u0 = gen.random_vector(xyz.shape[1], 4, "uniform")
    f = gen.random_vector(NI, 5)
    dt = 3.7e-8
    out = {}
    for pack in (0, rb.RBFFD_PACK_IDX32):
        plan = rb.Plan(xyz, bnd, inter, idx, w, rb.RBFFD_ORDER_MORTON | pack)
        L = plan.layout()
        if not pack:
            assert 0.98 * NI < L["rows16"] < NI
        u = T(u0)
        plan.solve_explicit(T(f), u, dt, 5, 0.0)
        u1 = T(u0)
        plan.solve_explicit(T(f), u1, dt, 1, 0.0)
        out[pack] = (H(u), H(u1))
        plan.destroy()
    assert np.array_equal(out[0][0], out[rb.RBFFD_PACK_IDX32][0])
    # graph steps as programmatic dependent launches (each warp prefetching its
    # first slice before the wait), and as plain launches: the same bits
    for launch in (rb.RBFFD_LAUNCH_PDL, rb.RBFFD_LAUNCH_NO_PDL):
        plan = rb.Plan(xyz, bnd, inter, idx, w, rb.RBFFD_ORDER_MORTON | launch)
        u = T(u0)
        plan.solve_explicit(T(f), u, dt, 5, 0.0)
        shape = plan.stats()[3]
        assert (shape[1] > 16) == (launch == rb.RBFFD_LAUNCH_PDL)
        assert np.array_equal(H(u), out[0][0])
        plan.destroy()
    # one step on sampled rows against the oracle's own stencil sums
    oxyz, obnd = orc.nodes(d, 0, Kg, 0.3, seed)
    ointer = gen.interior_ids(obnd)
    rows = np.sort(np.random.default_rng(13).choice(NI, 2000, replace=False))
    oidx = orc.knn_brute(oxyz, ointer[rows], n)
    ow, _ = orc.weights(oxyz, oidx, m)
    Lu = orc.apply(ow, oidx, u0)
    ref = u0[ointer[rows]] + dt * (Lu - f[rows])
    scale = np.abs(u0[ointer[rows]]) + dt * np.abs(ow * u0[oidx]).sum(axis=1)
    got = out[0][1][ointer[rows]]
    assert np.all(np.abs(got - ref) <= 1e-12 * scale)


@pytest.mark.parametrize("Kg,m,order,name", CASES)
def test_transpose_codes_match_int32_and_oracle(rb, orc, Kg, m, order, name):
    """The reverse step reads the transpose's 16-bit row codes where a slice's rows
    fit in four windows and int32 rows elsewhere: gradients bit-equal to the int32
    transpose (RBFFD_PACK_IDX32) and within 1e-12 of the oracle's adjoint."""
    p = build(orc, 2, Kg, m, seed=83)
    dt = _dt(orc, p)
    K = 60
    dLdu = np.zeros(p.N)
    sens = gen.sensors(p.NI, min(200, p.NI // 4), 3)
    dLdu[p.interior[sens]] = gen.random_vector(len(sens), 4)
    gf, gg, l0 = orc.adjoint(p.w, p.idx, p.interior, p.N, dLdu, K, dt)
    out = {}
    for pack in (0, rb.RBFFD_PACK_IDX32):
        plan = _plan(rb, p, order | pack)
        plan.transpose()
        L = plan.transpose_layout()
        assert L["slices"] == (p.NI + 31) // 32
        assert L["entries"] >= p.NI * p.n       # every stored entry plus the padding
        if pack:
            assert L["cols16"] == 0
        elif name == "random_int32_fallback":
            assert L["cols16"] < 0.01 * p.NI
        elif name == "one_window":
            assert L["cols16"] == p.NI
        else:
            assert L["cols16"] > 0.5 * p.NI
        e16 = L["entries"] if L["cols16"] == p.NI else None
        if e16 is not None:
            assert L["bytes"] == 10 * e16 + 28 * L["slices"] + 32 * p.NI
        if pack:
            assert L["bytes"] == 12 * L["entries"] + 12 * L["slices"] + 32 * p.NI
        out[pack] = tuple(H(t) for t in plan.adjoint(T(dLdu), K, dt))
        plan.destroy()
    for a, b in zip(out[0], out[rb.RBFFD_PACK_IDX32]):
        assert np.array_equal(a, b)
    for a, b in zip(out[0], (gf, gg, l0)):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_transpose_codes_square_1M(rb):
    """The 1,002,001-node m=4 Morton plan's transpose: compact and int32 slices in
    one reverse step; ten reverse steps bit-equal to the int32 transpose."""
    d, Kg, m, seed = 2, 1000, 4, 2
    n = gen.stencil_size(d, m)
    xyz, bnd = rb.rbffd_nodes(d, 0, Kg, 0.3, seed)
    inter = rb.rbffd_interior(bnd)
    idx = rb.rbffd_knn(xyz, inter, n)
    w, st = rb.rbffd_weights(xyz, idx, m)
    NI, N = inter.numel(), xyz.shape[1]
    dLdu = T(gen.random_vector(N, 6))
    out = {}
    for pack in (0, rb.RBFFD_PACK_IDX32):
        plan = rb.Plan(xyz, bnd, inter, idx, w, rb.RBFFD_ORDER_MORTON | pack)
        plan.transpose()
        L = plan.transpose_layout()
        if not pack:
            assert 0.98 * NI < L["cols16"] <= NI
        out[pack] = tuple(H(t) for t in plan.adjoint(dLdu, 10, 3.7e-8))
        plan.destroy()
    for a, b in zip(out[0], out[rb.RBFFD_PACK_IDX32]):
        assert np.array_equal(a, b)
