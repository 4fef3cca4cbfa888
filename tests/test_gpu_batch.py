"""Batched persistent solve (many uneven domains in one launch) vs the CPU oracle,
domain by domain: same iterates (<= 1e-12 max|u|) and the same stop decisions."""
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


def _domains(orc):
    specs = [(0, 14, 2), (1, 20, 4), (0, 25, 6), (1, 30, 2), (0, 9, 4), (1, 24, 6), (0, 40, 4)]
    out = []
    for k, (shape, Kg, m) in enumerate(specs):
        p = build(orc, 2, Kg, m, seed=100 + k, shape=shape)
        dt = 0.9 * orc.stable_dt(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, k), 200)
        out.append((p, dt))
    return out


@pytest.mark.parametrize("bps", [1, 3])
def test_batch_matches_oracle_per_domain(rb, orc, bps):
    doms = _domains(orc)
    plans = [rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w)) for p, _ in doms]
    batch = rb.Batch(plans, blocks_per_sm=bps)
    # uneven caps and tolerances: some domains stop on the tolerance, others on the cap
    caps = [300, 500, 250, 400, 700, 350, 450]
    tols = [0.0, 5.0, 0.0, 2.0, 0.0, 0.0, 1.0]
    fs = [T(p.f) for p, _ in doms]
    us = [T(p.u0) for p, _ in doms]
    code, steps, res, status = batch.solve(fs, us, [dt for _, dt in doms], caps, tols)
    for i, (p, dt) in enumerate(doms):
        ou, os_, ores, ost = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, caps[i],
                                                tols[i])
        assert steps[i] == os_
        assert status[i] == (rb.RBFFD_OK if ost == 0 else rb.RBFFD_NOT_CONVERGED)
        assert res[i] == pytest.approx(ores, rel=1e-12)
        got = us[i].cpu().numpy()
        assert np.max(np.abs(got - ou)) <= 1e-12 * np.max(np.abs(ou))
    # replay: the captured graph runs again with the same tables
    us2 = [T(p.u0) for p, _ in doms]
    code2, steps2, _, _ = batch.solve(fs, us2, [dt for _, dt in doms], caps, tols)
    assert steps2 == steps
    for a, b in zip(us, us2):
        assert torch.equal(a, b)
    batch.destroy()
    for pl in plans:
        pl.destroy()


def test_batch_autotune_and_errors(rb, orc):
    doms = _domains(orc)[:3]
    plans = [rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w)) for p, _ in doms]
    batch = rb.Batch(plans)
    fs = [T(p.f) for p, _ in doms]
    us = [T(p.u0) for p, _ in doms]
    best = batch.tune(fs, us, [dt for _, dt in doms], probe_steps=50)
    ms, shape = batch.stats()
    assert (shape[0], shape[1], shape[4]) == best and ms > 0
    # every block size gives the same iterates; bad shapes are refused
    ref = None
    for th in (256, 512, 768, 1024):
        batch.set_shape(1, 1, th)
        uu = [T(p.u0) for p, _ in doms]
        batch.solve(fs, uu, [dt for _, dt in doms], [80] * 3, [0.0] * 3)
        if ref is None:
            ref = [H(u) for u in uu]
        else:
            assert all(np.array_equal(H(u), r) for u, r in zip(uu, ref))
    for bad in ((2, 1, 1024), (2, 1, 768), (3, 1, 512), (1, 1, 128)):
        with pytest.raises(rb.RbffdError):
            batch.set_shape(*bad)
    batch.set_shape(*best)
    # a non-finite source in one domain stops that domain only
    f_bad = [t.clone() for t in fs]
    f_bad[1][3] = float("nan")
    us = [T(p.u0) for p, _ in doms]
    with pytest.raises(rb.RbffdError):
        batch.solve(f_bad, us, [dt for _, dt in doms], [100] * 3, [0.0] * 3)
    us = [T(p.u0) for p, _ in doms]
    import ctypes
    L = rb.lib()
    nd = 3
    fa = (ctypes.c_void_p * nd)(*[t.data_ptr() for t in f_bad])
    ua = (ctypes.c_void_p * nd)(*[t.data_ptr() for t in us])
    dta = (ctypes.c_double * nd)(*[dt for _, dt in doms])
    ma = (ctypes.c_int64 * nd)(100, 100, 100)
    ta = (ctypes.c_double * nd)(0.0, 0.0, 0.0)
    steps = (ctypes.c_int64 * nd)()
    st = (ctypes.c_int * nd)()
    code = L.rbffd_solve_batch(batch._h, fa, ua, dta, ma, ta, steps, None, st, None)
    assert code == rb.RBFFD_ERR_NONFINITE
    assert list(st) == [rb.RBFFD_NOT_CONVERGED, rb.RBFFD_ERR_NONFINITE, rb.RBFFD_NOT_CONVERGED]
    assert list(steps) == [100, 1, 100]
    batch.destroy()
    for pl in plans:
        pl.destroy()


def test_weights_batch_equals_per_domain(rb, orc):
    """rbffd_weights_batch (all domains in two launches) = rbffd_weights per domain, bit
    for bit, and = the oracle within 1e-12 per stencil; mixed orders, shapes, a 3D set,
    a domain with no stencils, and a singular stencil reported for its own domain only."""
    specs = [(2, 0, 30, 2), (2, 1, 40, 4), (2, 0, 25, 6), (3, 0, 8, 4), (2, 1, 22, 2),
             (2, 0, 12, 6)]
    xyzs, idxs, ms, ohs = [], [], [], []
    for i, (d, shape, Kg, m) in enumerate(specs):
        xyz, bnd = rb.rbffd_nodes(d, shape, Kg, 0.3, 20 + i)
        inter = rb.rbffd_interior(bnd)
        n = gen.stencil_size(d, m)
        xyzs.append(xyz)
        idxs.append(rb.rbffd_knn(xyz, inter, n))
        ms.append(m)
    # an empty call
    xyzs.append(xyzs[0])
    idxs.append(idxs[0][:0])
    ms.append(2)
    out = rb.rbffd_weights_batch(xyzs, idxs, ms)
    for (w, st), xyz, idx, m in zip(out, xyzs, idxs, ms):
        if idx.shape[0] == 0:
            assert w.shape[0] == 0
            continue
        w1, st1 = rb.rbffd_weights(xyz, idx, m)
        assert torch.equal(w, w1) and torch.equal(st, st1)
        rows = np.arange(0, idx.shape[0], max(1, idx.shape[0] // 40))
        ow, ost = orc.weights(H(xyz), H(idx)[rows], m)
        assert np.all(ost == 0)
        assert np.all(np.abs(H(w)[rows] - ow) <= 1e-12 * np.abs(ow).max(axis=1, keepdims=True))
    # duplicate nodes make one stencil singular: only its domain reports it
    xyz_bad = xyzs[0].clone()
    idx_bad = idxs[0].clone()
    idx_bad[5, 1] = idx_bad[5, 0]
    res = rb.rbffd_weights_batch([xyzs[1], xyz_bad], [idxs[1], idx_bad], [4, 2], check=False)
    assert int((res[0][1] != 0).sum()) == 0
    assert int(res[1][1][5]) == 1 and int((res[1][1] != 0).sum()) == 1
    with pytest.raises(rb.RbffdError):
        rb.rbffd_weights_batch([xyz_bad], [idx_bad], [2])
