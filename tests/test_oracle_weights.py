"""Pins for the oracle's RBF-FD weight build (Eq. 2-3, phi(r) = r^3, monomials <= m).

Each check is fixed by the mathematics, not by the oracle's own code:
* closed forms of the saddle-point system for symmetric m = 1 stencils in
  d = 1, 2, 3 (derived by hand from Eq. 2-3; they pin the r^3 block A and the
  right-hand side Laplacian(r^3) = 3(d+1) r),
* the textbook finite-difference stencils that the case n = M reduces to,
* exact reproduction of the Laplacian of every monomial of degree <= m
  (the constraint rows P^T w = L p),
* the Vandermonde special case n = M against numpy's LAPACK solve,
* translation invariance and the 1/scale^2 law,
* agreement with numpy's LAPACK solve of the same saddle system.
"""
import math

import numpy as np
import pytest

import rbffd_inputs as gen


def _w(orc, pts, m, idx=None):
    xyz = np.asarray(pts, np.float64)
    if xyz.ndim == 1:
        xyz = xyz[None, :]
    if idx is None:
        idx = np.arange(xyz.shape[1], dtype=np.int32)[None, :]
    w, st = orc.weights(xyz, np.asarray(idx, np.int32), m)
    assert np.all(st == 0)
    return w


@pytest.mark.parametrize("h", [1.0, 0.01, 3e-4])
def test_closed_form_1d_m1(orc, h):
    # centre 0, then -h, +h: w = [-3, 3/2, 3/2] / h^2 (symmetry + Eq. 2 rows)
    w = _w(orc, [0.0, -h, h], 1)[0]
    np.testing.assert_allclose(w, np.array([-3.0, 1.5, 1.5]) / h ** 2, rtol=1e-13)


@pytest.mark.parametrize("h", [1.0, 0.02])
def test_closed_form_2d_m1_plus(orc, h):
    # plus-shaped stencil: arm weight a = 9 / (4 sqrt 2 h^2), centre -4a
    pts = np.array([[0, 0], [-h, 0], [h, 0], [0, -h], [0, h]], np.float64).T
    w = _w(orc, pts, 1)[0]
    a = 9.0 / (4.0 * math.sqrt(2.0) * h ** 2)
    np.testing.assert_allclose(w, [-4 * a, a, a, a, a], rtol=1e-13)


@pytest.mark.parametrize("h", [1.0, 0.05])
def test_closed_form_3d_m1_plus(orc, h):
    # 3D cross: a = 12 / ((8 sqrt 2 - 4) h^2), centre -6a
    pts = [[0, 0, 0]]
    for ax in range(3):
        for sg in (-1, 1):
            p = [0.0, 0.0, 0.0]
            p[ax] = sg * h
            pts.append(p)
    w = _w(orc, np.array(pts).T, 1)[0]
    a = 12.0 / ((8.0 * math.sqrt(2.0) - 4.0) * h ** 2)
    np.testing.assert_allclose(w, [-6 * a] + [a] * 6, rtol=1e-13)


def test_textbook_fd_1d(orc):
    h = 0.1
    w = _w(orc, [0.0, -h, h], 2)[0]           # n = M = 3
    np.testing.assert_allclose(w, np.array([-2.0, 1.0, 1.0]) / h ** 2, rtol=1e-13)
    w = _w(orc, [0.0, -h, h, -2 * h, 2 * h], 4)[0]   # n = M = 5
    np.testing.assert_allclose(w, np.array([-30.0, 16, 16, -1, -1]) / (12 * h ** 2),
                               rtol=1e-12)


def _monomial_values(pts, ex):
    out = np.ones((len(ex), pts.shape[1]))
    for k, e in enumerate(ex):
        for a in range(pts.shape[0]):
            out[k] *= pts[a] ** e[a]
    return out


def _monomial_laplacian_at(xc, ex):
    """Laplacian of x^e at xc, by differentiating the monomial by hand."""
    out = np.zeros(len(ex))
    for k, e in enumerate(ex):
        tot = 0.0
        for a in range(len(e)):
            if e[a] >= 2:
                term = e[a] * (e[a] - 1) * xc[a] ** (e[a] - 2)
                for b in range(len(e)):
                    if b != a:
                        term *= xc[b] ** e[b]
                tot += term
        out[k] = tot
    return out


@pytest.mark.parametrize("d,m", [(2, 2), (2, 4), (2, 6), (3, 2), (3, 4)])
def test_polynomial_reproduction(orc, d, m):
    Kg = {2: 24, 3: 9}[d]
    xyz, bnd = orc.nodes(d, 0, Kg, 0.3, 21)
    n = gen.stencil_size(d, m)
    inner = gen.interior_ids(bnd)
    rows = inner[np.random.default_rng(1).choice(len(inner), 40, replace=False)]
    idx = orc.knn_brute(xyz, rows, n)
    w, st = orc.weights(xyz, idx, m)
    assert np.all(st == 0)
    # every monomial of total degree <= m, in shifted coordinates about a fixed point
    ex = [e for deg in range(m + 1) for e in np.ndindex(*([deg + 1] * d)) if sum(e) == deg]
    for r, c in enumerate(rows):
        pts = xyz[:, idx[r]] - 0.37
        vals = _monomial_values(pts, ex)
        lap = _monomial_laplacian_at(xyz[:, c] - 0.37, ex)
        got = vals @ w[r]
        scale = np.abs(vals * w[r]).sum(axis=1)
        assert np.all(np.abs(got - lap) <= 1e-9 * np.maximum(scale, 1.0))
    # constant -> zero row sum
    assert np.all(np.abs(w.sum(axis=1)) <= 1e-10 * np.abs(w).sum(axis=1))


def test_vandermonde_special_case(orc):
    # n = M: the monomial block alone fixes w: P^T w = L p
    rng = np.random.default_rng(3)
    for d, m in [(2, 2), (2, 3), (3, 2)]:
        M = gen.num_monomials(d, m)
        pts = rng.uniform(-1, 1, (d, M)) * 0.1
        pts[:, 0] = 0.0
        w = _w(orc, pts, m)[0]
        ex = orc.monomials(d, m)
        V = _monomial_values(pts, ex)
        rhs = _monomial_laplacian_at(np.zeros(d), ex)
        np.testing.assert_allclose(w, np.linalg.solve(V, rhs), rtol=1e-9, atol=1e-9 * np.abs(w).max())


def test_translation_and_scale(orc):
    rng = np.random.default_rng(7)
    d, m, n = 2, 4, 30
    pts = rng.uniform(-1, 1, (d, n)) * 0.05
    pts[:, 0] = 0.0
    w0 = _w(orc, pts, m)[0]
    w1 = _w(orc, pts + np.array([[0.3], [0.8]]), m)[0]
    np.testing.assert_allclose(w1, w0, rtol=1e-10, atol=1e-10 * np.abs(w0).max())
    w2 = _w(orc, pts * 4.0, m)[0]
    np.testing.assert_allclose(w2 * 16.0, w0, rtol=1e-10, atol=1e-10 * np.abs(w0).max())


@pytest.mark.parametrize("d,m", [(2, 2), (2, 4), (3, 4)])
def test_against_lapack_saddle_solve(orc, d, m):
    """The saddle system assembled from its definition, solved by numpy (LAPACK)."""
    xyz, bnd = orc.nodes(d, 0, {2: 20, 3: 8}[d], 0.3, 13)
    n = gen.stencil_size(d, m)
    rows = gen.interior_ids(bnd)[:12]
    idx = orc.knn_brute(xyz, rows, n)
    w, st = orc.weights(xyz, idx, m)
    ex = orc.monomials(d, m)
    M = len(ex)
    for r, c in enumerate(rows):
        X = xyz[:, idx[r]] - xyz[:, [c]]
        D = np.sqrt(((X[:, :, None] - X[:, None, :]) ** 2).sum(0))
        A = D ** 3
        P = _monomial_values(X, ex).T
        S = np.block([[A, P], [P.T, np.zeros((M, M))]])
        rhs = np.concatenate([3 * (d + 1) * np.sqrt((X ** 2).sum(0)),
                              _monomial_laplacian_at(np.zeros(d), ex)])
        ref = np.linalg.solve(S, rhs)[:n]
        np.testing.assert_allclose(w[r], ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


def test_singular_stencil_reports_status(orc):
    # two coincident support nodes make A and P rank deficient
    pts = np.array([[0.0, 0.1, 0.1, 0.0, 0.2, -0.1, 0.05],
                    [0.0, 0.0, 0.0, 0.1, 0.1, 0.2, -0.1]])
    w, st = orc.weights(pts, np.arange(7, dtype=np.int32)[None, :], 2)
    assert st[0] == 1 and np.all(w == 0)
