"""Mixed-boundary variant (Sec. II-C, text after Eq. 5) on the GPU vs the oracle:
half-cube nodes, interior-only supports of the Neumann nodes, normal-derivative
weights, and the explicit iteration with the Neumann update before each step."""
import numpy as np
import pytest

import rbffd_inputs as gen
from oracle_problem import build_mixed

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


@pytest.mark.parametrize("d,Kg", [(2, 25), (3, 7)])
def test_half_cube_nodes_and_neumann_stencils(rb, orc, d, Kg):
    m = 2
    xyz, bnd = rb.rbffd_nodes(d, 2, Kg, 0.3, 17)
    oxyz, obnd = orc.nodes(d, 2, Kg, 0.3, 17)
    assert np.array_equal(H(xyz), oxyz) and np.array_equal(H(bnd), obnd)
    nnode, normals = gen.neumann_nodes(oxyz, obnd)
    nn = gen.stencil_size(d, m)
    cand = (obnd == 0).astype(np.uint8)
    idx = rb.rbffd_knn_masked(xyz, T(cand), T(nnode), nn)
    oidx = orc.knn_kdtree(oxyz, nnode, nn, cand=cand)
    assert np.array_equal(H(idx), oidx)
    w, st = rb.rbffd_weights_dir(xyz, idx, m, T(normals))
    ow, ost = orc.weights_dir(oxyz, oidx, m, normals)
    assert np.array_equal(H(st), ost)
    assert np.all(np.abs(H(w) - ow) <= 1e-12 * np.abs(ow).max(axis=1, keepdims=True))


def test_mixed_solve_matches_oracle(rb, orc):
    mp = build_mixed(orc, 2, 20, 4, seed=7)
    p = mp.base
    plan = rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w))
    plan.set_neumann(T(mp.nnode), T(mp.nidx), T(mp.nw), T(mp.g))
    dt_g, rho = plan.stable_dt(T(gen.random_vector(p.NI, 3)), 400)
    dt = 0.9 * dt_g
    K = 400
    ou, os_, ores, ost = orc.solve_mixed(p.w, p.idx, p.interior, p.f, mp.nnode, mp.nidx, mp.nw,
                                         mp.g, p.u0, dt, K, 0.0)
    assert ost == 1 and np.all(np.isfinite(ou))
    u = T(p.u0)
    code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
    assert steps == os_ == K
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    assert res == pytest.approx(ores, rel=1e-12)
    # with a tolerance: same stop step
    ou2, os2, _, ost2 = orc.solve_mixed(p.w, p.idx, p.interior, p.f, mp.nnode, mp.nidx, mp.nw,
                                        mp.g, p.u0, dt, 20000, 1.0)
    u2 = T(p.u0)
    code2, steps2, _ = plan.solve_explicit(T(p.f), u2, dt, 20000, 1.0)
    assert steps2 == os2 and np.max(np.abs(H(u2) - ou2)) <= 1e-12 * np.max(np.abs(ou2))
    # the explicit-Euler bound the power iteration gives is stable for the coupled operator
    from test_oracle_mixed import _effective_operator
    lam = np.linalg.eigvals(_effective_operator(mp))
    assert np.max(np.abs(1 + dt * lam)) <= 1.0
    with pytest.raises(rb.RbffdError):
        plan.solve_dc(T(p.f), T(p.u0), dt, 0.0, 1, 10, 0.0)
    plan.destroy()


def test_mixed_solve_auto_launch_after_retune(rb, orc):
    """RBFFD_LAUNCH_AUTO: a solve before the Neumann nodes exist may tune the plan to the
    persistent launch; setting Neumann nodes tunes again, and the FP64 sweep must then
    replay graphs (only they run the Neumann update) and match the oracle."""
    mp = build_mixed(orc, 2, 20, 4, seed=8)
    p = mp.base
    plan = rb.Plan(T(p.xyz), T(p.is_bnd), T(p.interior), T(p.idx), T(p.w),
                   rb.RBFFD_LAUNCH_AUTO)
    plan.solve_explicit(T(p.f), T(p.u0), 1e-7, 64, 0.0)
    plan.set_neumann(T(mp.nnode), T(mp.nidx), T(mp.nw), T(mp.g))
    dt = 0.9 * plan.stable_dt(T(gen.random_vector(p.NI, 3)), 400)[0]
    K = 300
    ou, os_, ores, ost = orc.solve_mixed(p.w, p.idx, p.interior, p.f, mp.nnode, mp.nidx, mp.nw,
                                         mp.g, p.u0, dt, K, 0.0)
    u = T(p.u0)
    code, steps, res = plan.solve_explicit(T(p.f), u, dt, K, 0.0)
    assert steps == os_ == K
    assert np.max(np.abs(H(u) - ou)) <= 1e-12 * np.max(np.abs(ou))
    assert plan.stats()[3][1] > 0      # the FP64 sweep replays graphs
    plan.destroy()
