"""Pins for the mixed-boundary variant of the test problem (Sec. II-C, text after
Eq. 5): the half cube [0, 1/2]^d with u = 0 on the faces at 0 and du/dn = 0 on the
faces at 1/2, Neumann node values set from the previous iterate before each step."""
import numpy as np
import pytest

import rbffd_inputs as gen
from oracle_problem import build_mixed
from test_oracle_weights import _monomial_values


@pytest.mark.parametrize("d,Kg", [(2, 9), (3, 5)])
def test_half_cube_layout(orc, d, Kg):
    xyz, bnd = orc.nodes(d, 2, Kg, 0.3, 3)
    h = 0.5 / Kg
    gi = np.stack(np.meshgrid(*([np.arange(Kg + 1)] * d), indexing="ij")).reshape(d, -1)
    lo = np.any(gi == 0, axis=0)
    hi = np.any(gi == Kg, axis=0)
    assert np.array_equal(bnd == 1, lo) and np.array_equal(bnd == 2, hi & ~lo)
    far = gi == Kg
    assert np.all(xyz[far] == 0.5)
    assert np.all(np.abs(xyz[:, bnd == 0] - gi[:, bnd == 0] * h) <= 0.3 * h * (1 + 1e-12))
    ids, nrm = gen.neumann_nodes(xyz, bnd)
    assert np.allclose(np.linalg.norm(nrm, axis=1), 1.0)


def test_one_sided_derivative_textbook(orc):
    # right boundary node, normal +x, n = M = 3 (m = 2): [3/2, -2, 1/2] / h
    h = 0.01
    pts = np.array([[0.5, 0.5 - h, 0.5 - 2 * h]])
    w, st = orc.weights_dir(pts, np.arange(3, dtype=np.int32)[None, :], 2, np.array([[1.0]]))
    np.testing.assert_allclose(w[0], np.array([1.5, -2.0, 0.5]) / h, rtol=1e-12)


@pytest.mark.parametrize("d,m", [(2, 2), (2, 4), (3, 2)])
def test_directional_derivative_reproduces_polynomials(orc, d, m):
    mp = build_mixed(orc, d, {2: 14, 3: 6}[d], m, seed=4)
    xyz = mp.base.xyz
    ex = [e for deg in range(m + 1) for e in np.ndindex(*([deg + 1] * d)) if sum(e) == deg]
    for b in range(len(mp.nnode)):
        pts = xyz[:, mp.nidx[b]] - 0.2
        xc = xyz[:, mp.nnode[b]] - 0.2
        vals = _monomial_values(pts, ex)
        grad = np.zeros((len(ex), d))
        for k, e in enumerate(ex):
            for a in range(d):
                if e[a] >= 1:
                    t = e[a] * xc[a] ** (e[a] - 1)
                    for c in range(d):
                        if c != a:
                            t *= xc[c] ** e[c]
                    grad[k, a] = t
        exact = grad @ mp.normals[b]
        got = vals @ mp.nw[b]
        scale = np.abs(vals * mp.nw[b]).sum(axis=1)
        assert np.all(np.abs(got - exact) <= 1e-9 * np.maximum(scale, 1.0))


def _coupled_solution(mp):
    """Interior Laplacian rows = f, Neumann rows = g, Dirichlet values fixed (LAPACK)."""
    p = mp.base
    unk = np.concatenate([p.interior, mp.nnode])
    pos = -np.ones(p.N, np.int64)
    pos[unk] = np.arange(len(unk))
    A = np.zeros((len(unk), len(unk)))
    b = np.zeros(len(unk))
    fixed = p.u0
    for r in range(p.NI):
        b[r] = p.f[r]
        for j in range(p.n):
            c = p.idx[r, j]
            if pos[c] >= 0:
                A[r, pos[c]] += p.w[r, j]
            else:
                b[r] -= p.w[r, j] * fixed[c]
    for q in range(len(mp.nnode)):
        r = p.NI + q
        b[r] = mp.g[q]
        for j in range(mp.nidx.shape[1]):
            c = mp.nidx[q, j]
            if pos[c] >= 0:
                A[r, pos[c]] += mp.nw[q, j]
            else:
                b[r] -= mp.nw[q, j] * fixed[c]
    x = np.linalg.solve(A, b)
    u = fixed.copy()
    u[unk] = x
    return u


def _effective_operator(mp):
    """Interior operator with the Neumann values eliminated: u_N = B u_I + c."""
    p = mp.base
    NI, NN = p.NI, len(mp.nnode)
    pos = -np.ones(p.N, np.int64)
    pos[p.interior] = np.arange(NI)
    pos[mp.nnode] = NI + np.arange(NN)
    B = np.zeros((NN, NI))
    for q in range(NN):
        for j in range(1, mp.nidx.shape[1]):
            c = mp.nidx[q, j]
            assert pos[c] < NI          # Neumann supports hold interior nodes only
            if pos[c] >= 0:
                B[q, pos[c]] -= mp.nw[q, j] / mp.nw[q, 0]
    W = np.zeros((NI, NI + NN))
    for r in range(NI):
        for j in range(p.n):
            c = p.idx[r, j]
            if pos[c] >= 0:
                W[r, pos[c]] += p.w[r, j]
    return W[:, :NI] + W[:, NI:] @ B


def test_mixed_operator_is_stable_for_small_dt(orc):
    lam = np.linalg.eigvals(_effective_operator(build_mixed(orc, 2, 10, 2, seed=5)))
    assert lam.real.max() < 0
    # the slowest mode of -Laplace on the half square with these conditions: 2 pi^2
    assert abs(-lam.real.max() / (2 * np.pi ** 2) - 1) < 0.02


def test_mixed_iteration_reaches_coupled_solution(orc):
    mp = build_mixed(orc, 2, 10, 2, seed=5)
    p = mp.base
    ustar = _coupled_solution(mp)
    lam = np.linalg.eigvals(_effective_operator(mp))
    dt = 0.9 * np.min(-2 * lam.real / np.abs(lam) ** 2)   # explicit-Euler bound
    u, steps, res, st = orc.solve_mixed(p.w, p.idx, p.interior, p.f, mp.nnode, mp.nidx, mp.nw,
                                        mp.g, p.u0, dt, 400000, 1e-10)
    assert st == 0
    assert np.max(np.abs(u - ustar)) < 1e-8
    # the Neumann condition holds at the limit
    nres = (mp.nw * u[mp.nidx]).sum(axis=1) - mp.g
    assert np.max(np.abs(nres)) < 1e-6


@pytest.mark.slow
def test_mixed_discrete_solution_converges(orc):
    errs, hs = [], []
    for Kg in (10, 20, 40):
        mp = build_mixed(orc, 2, Kg, 4, seed=6)
        u = _coupled_solution(mp)
        errs.append(np.max(np.abs(u - mp.base.ua)))
        hs.append(0.5 / Kg)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert slope > 2.5 and errs[-1] < 1e-5, (slope, errs)
