"""Pins for the oracle's explicit iteration (Eq. 6), its stop rule, the
stability estimate, FP32 defect correction, the adjoint and the error metric.

Fixed by the mathematics rather than by the oracle's code:
* the iteration's limit is the discrete solution W_II u = f - W_IB g (numpy LAPACK),
* the start error -u*, close to the slowest mode sin(pi x) sin(pi y), decays
  by (1 - dt d pi^2) per step,
* the discrete solution converges to the closed form at order >= m - 1,
* the power-iteration radius equals numpy's largest |eigenvalue|,
* the loss is quadratic in (f, g), so central differences are exact up to
  rounding and a dense reverse sweep in numpy gives the same gradient.
"""
import math

import numpy as np
import pytest

import rbffd_inputs as gen
from oracle_problem import build, dt_guideline, dt_stable


def _fixed_point(p):
    WII, WIB, bnd = p.dense()
    return np.linalg.solve(WII, p.f - WIB @ p.u0[bnd])


@pytest.mark.parametrize("m", [2, 4])
def test_iteration_reaches_discrete_solution(orc, m):
    p = build(orc, 2, 14, m, seed=3)
    ustar = _fixed_point(p)
    dt = dt_stable(orc, p)
    u, steps, res, st = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 200000, 1e-10)
    assert st == 0 and res < 1e-10
    assert np.max(np.abs(u[p.interior] - ustar)) < 1e-9
    assert np.array_equal(u[p.is_bnd == 1], p.u0[p.is_bnd == 1])   # Dirichlet held


def test_slowest_mode_decay_rate(orc):
    p = build(orc, 2, 30, 4, seed=4)
    ustar = _fixed_point(p)
    dt = dt_stable(orc, p)
    errs = []
    u = p.u0
    for k in range(3):
        u, steps, res, st = orc.solve_explicit(p.w, p.idx, p.interior, p.f, u, dt, 2000, 0.0)
        errs.append(np.max(np.abs(u[p.interior] - ustar)))
    rate = (errs[2] / errs[1]) ** (1.0 / 2000)
    expect = 1.0 - dt * 2 * np.pi ** 2
    assert abs(np.log(rate) / np.log(expect) - 1.0) < 0.02


def test_stop_rule_and_step_count(orc):
    p = build(orc, 2, 10, 2, seed=5)
    dt = dt_stable(orc, p)
    u1, s1, r1, st1 = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 7, 0.0)
    assert (s1, st1) == (7, 1)
    # residual of u^0 is max|W u^0 - f|; a tolerance just above it stops after one step
    R0 = np.max(np.abs(orc.apply(p.w, p.idx, p.u0) - p.f))
    u2, s2, r2, st2 = orc.solve_explicit(p.w, p.idx, p.interior, p.f, p.u0, dt, 100, R0 * 1.0001)
    assert (s2, st2) == (1, 0) and r2 == R0
    # that one step is u + dt (W u - f)
    ref = p.u0.copy()
    ref[p.interior] = p.u0[p.interior] + dt * (orc.apply(p.w, p.idx, p.u0) - p.f)
    np.testing.assert_allclose(u2, ref, rtol=0, atol=1e-15)


def test_nonfinite_source_stops(orc):
    p = build(orc, 2, 10, 2, seed=5)
    f = p.f.copy()
    f[3] = np.nan
    u, s, r, st = orc.solve_explicit(p.w, p.idx, p.interior, f, p.u0, dt_stable(orc, p), 50, 0.0)
    assert st == 2 and s == 1


@pytest.mark.slow
@pytest.mark.parametrize("m,min_slope", [(2, 0.7), (4, 2.7), (6, 4.7)])
def test_convergence_order(orc, m, min_slope):
    errs, hs = [], []
    for Kg in (24, 48, 96):
        p = build(orc, 2, Kg, m, seed=6)
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        NI = p.NI
        rows = np.repeat(np.arange(NI), p.n)
        W = sp.csr_matrix((p.w.ravel(), (rows, p.idx.ravel())), shape=(NI, p.N))
        WII = W[:, p.interior]
        bnd = np.nonzero(p.is_bnd)[0]
        rhs = p.f - W[:, bnd] @ p.u0[bnd]
        u = spl.spsolve(WII.tocsc(), rhs)
        errs.append(np.max(np.abs(u - p.ua[p.interior])))
        hs.append(p.h)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert slope >= min_slope, (slope, errs)
    # higher order is more accurate at the finest spacing (Sec. III-D)
    assert errs[-1] < {2: 1e-3, 4: 1e-6, 6: 1e-8}[m]


def test_power_rho_matches_eigenvalues(orc):
    p = build(orc, 2, 12, 4, seed=8)
    WII, _, _ = p.dense()
    lam = np.linalg.eigvals(WII)
    rho_ref = np.max(np.abs(lam))
    rho = orc.power_rho(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, 1), 3000)
    assert abs(rho / rho_ref - 1) < 1e-3
    # the eigenvalues sit in the left half plane (explicit step can be stable)
    assert np.max(lam.real) < 0


def test_stable_dt_is_stable_and_bounds_are_sharp(orc):
    p = build(orc, 2, 16, 4, seed=9)
    dt = orc.stable_dt(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, 2), 400)
    WII, _, _ = p.dense()
    amp = np.max(np.abs(1 + dt * np.linalg.eigvals(WII)))
    assert amp <= 1.0
    # on jittered nodes rho(W_II) h^2 ~ 32, four times the 5-point stencil's 8, so the
    # paper's alpha = 0.3 of the Eq. 7 guideline would already be unstable here
    assert dt < 0.3 * p.h ** 2 / (2 * p.d)
    amp_paper = np.max(np.abs(1 + dt_guideline(p, 0.3) * np.linalg.eigvals(WII)))
    assert amp_paper > 1.0


def test_defect_correction_reaches_fp64_solution(orc):
    p = build(orc, 2, 14, 4, seed=10)
    ustar = _fixed_point(p)
    dt = dt_stable(orc, p)
    u, outer, inner, res, st = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, dt, 1e-9,
                                            60, 20000, 1e-3)
    assert st == 0 and res < 1e-9
    assert np.max(np.abs(u[p.interior] - ustar)) < 1e-10
    assert outer >= 2          # the FP32 inner loop alone cannot get there


def test_adjoint_matches_dense_reverse_sweep_and_fd(orc):
    p = build(orc, 2, 9, 2, seed=11)
    WII, WIB, bnd = p.dense()
    dt, K = dt_stable(orc, p), 40
    g = p.u0[bnd]
    sens = gen.sensors(p.NI, 10, 3)
    uobs = p.ua[p.interior][sens]

    def forward(f, gb):
        uI = np.zeros(p.NI)
        for _ in range(K):
            uI = uI + dt * (WII @ uI + WIB @ gb - f)
        return uI

    def loss(f, gb):
        return np.sum((forward(f, gb)[sens] - uobs) ** 2)

    uK = forward(p.f, g)
    lamK = np.zeros(p.NI)
    lamK[sens] = 2 * (uK[sens] - uobs)
    dLdu = np.zeros(p.N)
    dLdu[p.interior] = lamK
    gf, gg, l0 = orc.adjoint(p.w, p.idx, p.interior, p.N, dLdu, K, dt)
    # dense reverse sweep
    lam, S = lamK.copy(), np.zeros(p.NI)
    for _ in range(K):
        S += lam
        lam = lam + dt * (WII.T @ lam)
    np.testing.assert_allclose(gf, -dt * S, rtol=1e-12, atol=1e-14 * np.abs(S).max() * dt)
    np.testing.assert_allclose(gg[bnd], dt * (WIB.T @ S), rtol=1e-10,
                               atol=1e-13 * np.abs(gg).max())
    assert np.all(gg[p.interior] == 0)
    np.testing.assert_allclose(l0, lam, rtol=1e-12, atol=1e-15)
    # central differences along seeded directions (exact for a quadratic)
    rng = np.random.default_rng(0)
    for _ in range(5):
        vf = rng.standard_normal(p.NI)
        vg = rng.standard_normal(len(bnd))
        eps = 1e-3
        fd = (loss(p.f + eps * vf, g + eps * vg) - loss(p.f - eps * vf, g - eps * vg)) / (2 * eps)
        an = gf @ vf + gg[bnd] @ vg
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12)


def test_mean_abs_error_definition(orc):
    # Eq. 8 on a hand-made vector
    assert orc.mean_abs_error([1.0, 2.0, 3.0], [1.0, 1.5, 4.0]) == pytest.approx(0.5)


def test_weight_gradient_matches_dense_reverse_sweep_and_fd(orc):
    """dL/dw from a dense numpy reverse sweep over stored iterates, and central
    differences of the loss along random weight perturbations (O(eps^2) exact)."""
    p = build(orc, 2, 8, 2, seed=12)
    WII, WIB, bnd = p.dense()
    dt, K = dt_stable(orc, p), 30
    sens = gen.sensors(p.NI, 8, 4)
    uobs = p.ua[p.interior][sens]
    rows = np.repeat(np.arange(p.NI), p.n)

    def forward(w):
        u = p.u0.copy()
        U = []
        for _ in range(K):
            U.append(u.copy())
            Lu = np.zeros(p.NI)
            np.add.at(Lu, rows, (w * u[p.idx]).ravel())
            u = u.copy()
            u[p.interior] = u[p.interior] + dt * (Lu - p.f)
        return u, U

    def loss(w):
        u, _ = forward(w)
        return np.sum((u[p.interior][sens] - uobs) ** 2)

    uK, U = forward(p.w)
    lamK = np.zeros(p.NI)
    lamK[sens] = 2 * (uK[p.interior][sens] - uobs)
    dLdu = np.zeros(p.N)
    dLdu[p.interior] = lamK
    gw, gf, gg, l0 = orc.adjoint_w(p.w, p.idx, p.interior, p.f, p.u0, dLdu, K, dt)
    # dense reverse sweep
    lam = lamK.copy()
    ref = np.zeros_like(p.w)
    for k in range(K - 1, -1, -1):
        ref += dt * lam[:, None] * U[k][p.idx]
        lam = lam + dt * (WII.T @ lam)
    np.testing.assert_allclose(gw, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())
    # the f/g gradients and lambda^0 equal the f/g-only adjoint's
    gf2, gg2, l02 = orc.adjoint(p.w, p.idx, p.interior, p.N, dLdu, K, dt)
    assert np.array_equal(gf, gf2) and np.array_equal(gg, gg2) and np.array_equal(l0, l02)
    rng = np.random.default_rng(1)
    for _ in range(4):
        v = rng.standard_normal(p.w.shape) * np.abs(p.w)
        eps = 1e-6
        fd = (loss(p.w + eps * v) - loss(p.w - eps * v)) / (2 * eps)
        an = np.sum(gw * v)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12)


def test_defect_correction_inner_loop_stalls_at_the_fp32_floor(orc):
    """The inner iteration runs in FP32: with no inner stop (rho_in = 0) it stalls
    where each increment fmaf(dt32, rho_i, e_i) rounds back to e_i, i.e. at
    |rho_i| <= ulp(e_i) / (2 dt32), a fraction of eps32 * max_i sum_j |w_ij e_j|.
    An inner loop that silently ran in FP64 would keep falling ~1e8 times lower."""
    p = build(orc, 2, 20, 4, seed=10)
    dt = dt_stable(orc, p)
    eps32 = float(np.finfo(np.float32).eps)
    runs = [orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, dt, 0.0, 1, K, 0.0, inner_res=True)
            for K in (20000, 30000)]
    (u1, o1, i1, D1, s1, rin1), (u2, o2, i2, D2, s2, rin2) = runs
    assert (o1, i1, o2, i2) == (1, 20000, 1, 30000)
    # stalled: 10,000 further FP32 steps change nothing
    assert np.array_equal(u1, u2) and rin1 == rin2
    e = (u1 - p.u0)[p.interior]                 # u0 = 0 inside: e exactly, as stored
    assert np.array_equal(e.astype(np.float32).astype(np.float64), e)
    ea = np.zeros(p.N)
    ea[p.interior] = e
    scale = np.max(np.sum(np.abs(p.w * ea[p.idx]), axis=1))
    assert 0.01 * eps32 * scale <= rin1 <= 2.0 * eps32 * scale, rin1 / (eps32 * scale)
    # the stall bound itself: no row's increment survives rounding
    dt32 = float(np.float32(dt))
    spacing = np.spacing(np.abs(e).astype(np.float32)).astype(np.float64)
    assert rin1 <= np.max(spacing) / (2 * dt32) * 1.001
    # the FP64 defect after this one correction sits at the same FP32 level
    assert 0.01 * eps32 * scale <= D1 <= 4.0 * eps32 * scale


@pytest.mark.parametrize("rho_in", [1e-2, 1e-3])
def test_defect_correction_inner_step_count_follows_slowest_mode(orc, rho_in):
    """From e = 0 the inner residual is rho^k = (I + dt W_II)^k d.  Here u0 = 0 and
    g = 0, so d = -f = 2 pi^2 u^a, the slowest mode: max|rho^k| = (1 - dt lam_1)^k D
    with lam_1 the smallest |eigenvalue| of W_II (numpy).  The rule 'stop after step
    k once max|rho^k| < rho_in D' then takes ceil(ln rho_in / ln(1 - dt lam_1)) + 1
    steps; an absolute rule (max|rho| < rho_in) would take ~ln(D)/ln(1/rho_in) more."""
    p = build(orc, 2, 20, 4, seed=10)
    dt = dt_stable(orc, p)
    WII, _, _ = p.dense()
    lam1 = np.min(np.abs(np.linalg.eigvals(WII).real))
    assert abs(lam1 / (2 * np.pi ** 2) - 1) < 1e-3
    u, outer, inner, D, st = orc.solve_dc(p.w, p.idx, p.interior, p.f, p.u0, dt, 0.0, 1,
                                          10 ** 6, rho_in)
    predicted = math.ceil(math.log(rho_in) / math.log(1 - dt * lam1)) + 1
    assert outer == 1 and abs(inner / predicted - 1) < 0.01, (inner, predicted)


def test_defect_correction_inner_arithmetic_is_binary32(orc):
    """A hand-worked case of the inner step in IEEE binary32.  Interior nodes 0, 1,
    boundary node 2 (g = 0), u0 = 0, f = (1, 1), dt = 2^-4, so d = -f = (-1, -1)
    and D = 1.  Step 1 from e = 0: rho = d32, e^1 = fl(dt32 * -1) = (-2^-4, -2^-4).
    Step 2, row 0 (w = -16, -2^-21 on nodes 0, 1): the products 1 and 2^-25 are
    exact, but 1 + 2^-25 rounds to 1 in binary32 (half an ulp is 2^-24), so
    rho_0 = 1 + d32_0 = 0 and e_0 stays -2^-4.  Accumulated in binary64, rho_0
    would be 2^-25 and e_0 = -2^-4 + 2^-29 (a binary32 ulp of 2^-4 is 2^-27)."""
    w = np.array([[-16.0, -2.0 ** -21, 0.0], [-16.0, 0.0, 0.0]])
    idx = np.array([[0, 1, 2], [1, 0, 2]], dtype=np.int32)
    interior = np.array([0, 1], dtype=np.int32)
    f = np.array([1.0, 1.0])
    u0 = np.zeros(3)
    u, outer, inner, D, st, rin = orc.solve_dc(w, idx, interior, f, u0, 2.0 ** -4, 0.0, 1, 2,
                                               0.0, inner_res=True)
    assert (outer, inner) == (1, 2)
    assert u[0] == -2.0 ** -4 and u[1] == -2.0 ** -4 and u[2] == 0.0
    assert rin == 0.0
    # the FP64 defect of the corrected iterate: row 0 is 1 + 2^-25 - 1 exactly
    D_next = orc.solve_dc(w, idx, interior, f, u, 2.0 ** -4, 0.0, 0, 1, 0.0)[3]
    assert D_next == 2.0 ** -25


def test_adjoint_loss_on_boundary_nodes_too(orc):
    """A misfit that also observes boundary nodes: u^K_b = g_b there, so dL/dg_b gets
    the loss's direct derivative on top of the reverse sweep's dt (W_IB^T S)_b.  The
    loss is quadratic in (f, g): central differences are exact up to rounding."""
    p = build(orc, 2, 9, 2, seed=14)
    WII, WIB, bnd = p.dense()
    dt, K = dt_stable(orc, p), 30
    sens = gen.sensors(p.NI, 8, 5)
    bsens = bnd[::3]                      # every third boundary node observed
    uobs = p.ua[p.interior][sens]
    bobs = gen.random_vector(len(bsens), 9)

    def forward(f, gb):
        u = np.zeros(p.N)
        u[bnd] = gb
        uI = np.zeros(p.NI)
        for _ in range(K):
            uI = uI + dt * (WII @ uI + WIB @ gb - f)
        u[p.interior] = uI
        return u

    def loss(f, gb):
        u = forward(f, gb)
        return np.sum((u[p.interior][sens] - uobs) ** 2) + np.sum((u[bsens] - bobs) ** 2)

    g = p.u0[bnd] + 0.1 * gen.random_vector(len(bnd), 10)
    uK = forward(p.f, g)
    dLdu = np.zeros(p.N)
    dLdu[p.interior[sens]] = 2 * (uK[p.interior][sens] - uobs)
    dLdu[bsens] = 2 * (uK[bsens] - bobs)
    gf, gg, l0 = orc.adjoint(p.w, p.idx, p.interior, p.N, dLdu, K, dt)
    # without the direct term the boundary gradient would miss 2 (g_b - obs_b)
    assert np.max(np.abs(dLdu[bsens])) > 1e-3
    rng = np.random.default_rng(2)
    for _ in range(5):
        vf = rng.standard_normal(p.NI)
        vg = rng.standard_normal(len(bnd))
        eps = 1e-3
        fd = (loss(p.f + eps * vf, g + eps * vg) - loss(p.f - eps * vf, g - eps * vg)) / (2 * eps)
        an = gf @ vf + gg[bnd] @ vg
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12)
    assert np.all(gg[p.interior] == 0)
