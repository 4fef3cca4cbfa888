"""Pins for the oracle's Poisson-disc node placement (CPU only).

The method (Sec. II-C, last paragraph): the boundary nodes are the seeds; the
node list is walked first in, first out; each node proposes K candidates at
distance h (a fixed set of K directions, rotated by a random angle per node);
a candidate inside the domain is appended when no node in the list is closer
than zeta h.  Every check below uses numpy/scipy arithmetic of its own
(atan2, cos, sin, kd-tree), not the oracle's routines:

* closed-form seeds (square: boundary grid points; disk: equispaced angles);
* separation: every interior node is at least zeta h from every other node;
* construction: each interior node lies at distance h from an earlier node
  (its parent), in a direction 2 pi (U_parent + j / K) for an integer j, the
  parents are non-decreasing along the list (first-in first-out order), the
  children of one parent appear with increasing j, and every j in 0..K-1 occurs;
* saturation: every candidate of every node is outside the domain or within
  zeta h of a node (the stopping condition);
* the packing bound of Oler for points at mutual distance >= zeta h in the
  unit square;
* grid-accelerated proximity test == brute force over all nodes.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

ZETA = 1.0 - 1e-10
K = 15


def _u01(orc, seed, c):
    return (orc.sm64_at(seed, c) >> 11) * (1.0 / 9007199254740992.0)


@pytest.mark.parametrize("shape,Kg,seed", [(0, 30, 1), (0, 57, 2), (1, 40, 3), (1, 64, 4)])
def test_pds_grid_equals_brute_force(orc, shape, Kg, seed):
    a = orc.nodes_pds(shape, Kg, seed)
    b = orc.nodes_pds(shape, Kg, seed, brute=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_pds_seeds_closed_form(orc):
    Kg = 25
    xyz, bnd = orc.nodes_pds(0, Kg, 5)
    h = 1.0 / Kg
    ij = [(i, j) for i in range(Kg + 1) for j in range(Kg + 1)
          if i in (0, Kg) or j in (0, Kg)]
    nb = len(ij)
    assert np.all(bnd[:nb] == 1) and np.all(bnd[nb:] == 0)
    assert np.array_equal(xyz[:, :nb], np.array(ij, dtype=np.float64).T * h)
    xyz, bnd = orc.nodes_pds(1, 40, 6)
    nb = int(round(math.pi * 40))
    assert np.all(bnd[:nb] == 1) and np.all(bnd[nb:] == 0)
    ang = 2 * np.pi * np.arange(nb) / nb
    assert np.max(np.abs(xyz[0, :nb] - (0.5 + 0.5 * np.cos(ang)))) < 4e-16
    assert np.max(np.abs(xyz[1, :nb] - (0.5 + 0.5 * np.sin(ang)))) < 4e-16


def _inside(shape, p, tol):
    x, y = p
    if shape == 0:
        return (x > tol) & (x < 1 - tol) & (y > tol) & (y < 1 - tol)
    return (x - 0.5) ** 2 + (y - 0.5) ** 2 < (0.5 - tol) ** 2


def _outside(shape, p, tol):
    x, y = p
    if shape == 0:
        return (x < -tol) | (x > 1 + tol) | (y < -tol) | (y > 1 + tol)
    return (x - 0.5) ** 2 + (y - 0.5) ** 2 > (0.5 + tol) ** 2


@pytest.mark.parametrize("shape,Kg,seed", [(0, 45, 7), (1, 50, 8)])
def test_pds_separation_construction_saturation(orc, shape, Kg, seed):
    h = 1.0 / Kg
    xyz, bnd = orc.nodes_pds(shape, Kg, seed)
    N = xyz.shape[1]
    P = xyz.T
    tree = cKDTree(P)
    nb = int(bnd.sum())
    inner = np.arange(nb, N)
    assert np.all(_inside(shape, xyz[:, inner], 0.0))
    # separation
    d, _ = tree.query(P[inner], k=2)
    assert d[:, 1].min() >= ZETA * h * (1 - 1e-12)
    # construction: the parent is the lowest-index node at distance h
    parents, dirs = [], []
    for i in inner:
        cand = tree.query_ball_point(P[i], h * (1 + 1e-9))
        at_h = [q for q in cand if abs(np.hypot(*(P[i] - P[q])) - h) <= 1e-9 * h]
        assert at_h, f"node {i} has no node at distance h"
        p = min(at_h)
        assert p < i
        parents.append(p)
        v = (P[i] - P[p]) / h
        turns = (math.atan2(v[1], v[0]) / (2 * math.pi) - _u01(orc, seed, p)) * K
        assert abs(turns - round(turns)) < 1e-8
        dirs.append(int(round(turns)) % K)
    parents, dirs = np.array(parents), np.array(dirs)
    assert np.all(np.diff(parents) >= 0)            # first in, first out
    same = np.diff(parents) == 0
    assert np.all(np.diff(dirs)[same] > 0)          # a parent's candidates in order j
    assert set(dirs.tolist()) == set(range(K))
    # saturation: every candidate of every node is blocked or outside
    U = np.array([_u01(orc, seed, p) for p in range(N)])
    for j in range(K):
        ang = 2 * np.pi * (U + j / K)
        C = P + h * np.stack([np.cos(ang), np.sin(ang)], axis=1)
        dist, _ = tree.query(C)
        blocked = dist < ZETA * h * (1 + 1e-9)
        out = _outside(shape, C.T, 1e-12)
        edge = ~_inside(shape, C.T, 1e-12) & ~out      # on the boundary within rounding
        assert np.all(blocked | out | edge)


def test_pds_oler_packing_bound(orc):
    # points at mutual distance >= d in a convex region of area A and perimeter L:
    # N <= 2/sqrt(3) A / d^2 + L / (2 d) + 1  (Oler's inequality)
    for Kg in (40, 120):
        h = 1.0 / Kg
        xyz, bnd = orc.nodes_pds(0, Kg, 9)
        d = ZETA * h
        assert xyz.shape[1] <= 2 / math.sqrt(3) / d ** 2 + 4 / (2 * d) + 1
        # and the fill is dense: well above half the hexagonal packing count
        assert xyz.shape[1] > 0.5 * 2 / math.sqrt(3) / h ** 2


def test_pds_parameters_change_the_set(orc):
    a = orc.nodes_pds(0, 30, 1)[0]
    b = orc.nodes_pds(0, 30, 2)[0]
    c = orc.nodes_pds(0, 30, 1, K=9)[0]
    assert not np.array_equal(a, b) and not np.array_equal(a[:, :200], c[:, :200])
    with pytest.raises(ValueError):
        orc.nodes_pds(2, 30, 1)


# ---------------------------------------------------------------- 3D (unit cube)
K3 = 50


def _rotation(orc, seed, p):
    """Shoemake's uniform rotation from the (3p..3p+2)-th draws, in numpy arithmetic."""
    u1, u2, u3 = (_u01(orc, seed, 3 * p + i) for i in range(3))
    s1, s2 = math.sqrt(1 - u1), math.sqrt(u1)
    x, y = s1 * math.sin(2 * math.pi * u2), s1 * math.cos(2 * math.pi * u2)
    z, w = s2 * math.sin(2 * math.pi * u3), s2 * math.cos(2 * math.pi * u3)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _fibonacci(K):
    j = np.arange(K)
    z = 1 - (2 * j + 1) / K
    rho = np.sqrt(1 - z * z)
    phi = j * math.pi * (3 - math.sqrt(5))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


@pytest.mark.parametrize("Kg,seed", [(6, 1), (9, 2)])
def test_pds3_grid_equals_brute_force(orc, Kg, seed):
    a = orc.nodes_pds3(Kg, seed)
    b = orc.nodes_pds3(Kg, seed, brute=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_pds3_seeds_separation_construction_saturation(orc):
    Kg, seed = 14, 3
    h = 1.0 / Kg
    xyz, bnd = orc.nodes_pds3(Kg, seed)
    P = xyz.T
    N = len(P)
    ijk = [(i, j, k) for i in range(Kg + 1) for j in range(Kg + 1) for k in range(Kg + 1)
           if Kg in (i, j, k) or 0 in (i, j, k)]
    nb = len(ijk)
    assert np.all(bnd[:nb] == 1) and np.all(bnd[nb:] == 0)
    assert np.array_equal(P[:nb], np.array(ijk, dtype=np.float64) * h)
    inner = np.arange(nb, N)
    assert np.all((P[inner] > 0) & (P[inner] < 1))
    tree = cKDTree(P)
    d, _ = tree.query(P[inner], k=2)
    assert d[:, 1].min() >= ZETA * h * (1 - 1e-12)
    E = _fibonacci(K3)
    parents, dirs = [], []
    for i in inner:
        cand = tree.query_ball_point(P[i], h * (1 + 1e-9))
        at_h = [q for q in cand if abs(np.linalg.norm(P[i] - P[q]) - h) <= 1e-9 * h]
        assert at_h
        p = min(at_h)
        assert p < i
        v = (P[i] - P[p]) / h
        err = np.linalg.norm(_rotation(orc, seed, p) @ E.T - v[:, None], axis=0)
        j = int(np.argmin(err))
        assert err[j] < 1e-9
        parents.append(p)
        dirs.append(j)
    parents, dirs = np.array(parents), np.array(dirs)
    assert np.all(np.diff(parents) >= 0)
    same = np.diff(parents) == 0
    assert np.all(np.diff(dirs)[same] > 0)
    assert set(dirs.tolist()) == set(range(K3))
    # saturation
    for p in range(N):
        C = P[p] + h * (_rotation(orc, seed, p) @ E.T).T
        dist, _ = tree.query(C)
        inside = np.all((C > 1e-12) & (C < 1 - 1e-12), axis=1)
        assert np.all(~inside | (dist < ZETA * h * (1 + 1e-9)))


def test_pds3_kepler_bound(orc):
    # mutual distance >= d inside the unit cube: the periodic extension with period 1 + d
    # is a packing of balls of diameter d, so N (pi/6) d^3 <= (pi/sqrt 18)(1 + d)^3 (Hales)
    for Kg in (8, 20):
        h = 1.0 / Kg
        xyz, _ = orc.nodes_pds3(Kg, 4)
        d = ZETA * h
        assert xyz.shape[1] <= math.sqrt(2) * (1 + d) ** 3 / d ** 3
        assert xyz.shape[1] > 0.5 / h ** 3
