"""Builds a full test problem with the CPU oracle only (nodes, supports, weights,
source, start iterate).  Used by the oracle pin tests and as the expected side
of the GPU parity tests; nothing here comes from the CUDA path."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import rbffd_inputs as gen


@dataclass
class Problem:
    d: int
    Kg: int
    m: int
    n: int
    xyz: np.ndarray
    is_bnd: np.ndarray
    interior: np.ndarray
    idx: np.ndarray
    w: np.ndarray
    f: np.ndarray
    u0: np.ndarray
    ua: np.ndarray

    @property
    def N(self):
        return self.xyz.shape[1]

    @property
    def NI(self):
        return len(self.interior)

    @property
    def h(self):
        return 1.0 / self.Kg

    def dense(self):
        """W split into interior/interior and interior/boundary dense blocks."""
        N, NI = self.N, self.NI
        W = np.zeros((NI, N))
        for j in range(self.n):
            np.add.at(W, (np.arange(NI), self.idx[:, j]), self.w[:, j])
        bnd = np.nonzero(self.is_bnd)[0]
        return W[:, self.interior], W[:, bnd], bnd


def build(orc, d=2, Kg=20, m=2, seed=1, shape=0, n=None, jitter=0.3) -> Problem:
    xyz, is_bnd = orc.nodes(d, shape, Kg, jitter, seed)
    interior = gen.interior_ids(is_bnd)
    n = n or gen.stencil_size(d, m)
    idx = orc.knn_kdtree(xyz, interior, n)
    w, st = orc.weights(xyz, idx, m)
    assert np.all(st == 0), "singular stencil in test problem"
    f = gen.source(xyz, interior)
    u0 = gen.start_iterate(xyz, is_bnd)
    ua = gen.exact_solution(xyz)
    return Problem(d, Kg, m, n, xyz, is_bnd, interior, idx, w, f, u0, ua)


def dt_guideline(p: Problem, alpha=0.3) -> float:
    """Eq. 7 (cfl): dt = alpha * h^2 / (2 d)."""
    return alpha * p.h ** 2 / (2 * p.d)


def dt_stable(orc, p: Problem, frac=0.9, seed=12345) -> float:
    """frac x the explicit-Euler bound 2/rho(W_II), rho from 200 power iterations x 1.05."""
    return frac * orc.stable_dt(p.w, p.idx, p.interior, p.N, gen.random_vector(p.NI, seed), 200)


@dataclass
class MixedProblem:
    base: Problem
    nnode: np.ndarray      # Neumann node ids
    normals: np.ndarray
    nidx: np.ndarray       # their supports
    nw: np.ndarray         # their normal-derivative weights
    g: np.ndarray          # Neumann data (du/dn = 0 on the faces at 1/2)


def build_mixed(orc, d=2, Kg=12, m=2, seed=1, n=None, nn=None) -> MixedProblem:
    """The mixed-boundary variant of Sec. II-C on the half cube [0, 1/2]^d."""
    xyz, is_bnd = orc.nodes(d, 2, Kg, 0.3, seed)
    interior = gen.interior_ids(is_bnd)
    n = n or gen.stencil_size(d, m)
    nn = nn or n
    idx = orc.knn_kdtree(xyz, interior, n)
    w, st = orc.weights(xyz, idx, m)
    assert np.all(st == 0)
    nnode, normals = gen.neumann_nodes(xyz, is_bnd)
    # a Neumann node's support: itself and its nearest interior nodes (its value is
    # set from interior values of the previous step, Sec. II-C)
    nidx = orc.knn_kdtree(xyz, nnode, nn, cand=(is_bnd == 0).astype(np.uint8))
    nw, st2 = orc.weights_dir(xyz, nidx, m, normals)
    assert np.all(st2 == 0)
    f = gen.source(xyz, interior)
    u0 = gen.start_iterate(xyz, is_bnd)
    ua = gen.exact_solution(xyz)
    base = Problem(d, Kg, m, n, xyz, is_bnd, interior, idx, w, f, u0, ua)
    return MixedProblem(base, nnode, normals, nidx, nw, np.zeros(len(nnode)))
