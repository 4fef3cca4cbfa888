"""Seeded synthetic inputs for the RBF-FD explicit Poisson path.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds none of the method's arithmetic (no support
selection, no weights, no explicit step): only the test problem of Sec. II-C
(Eq. 4-5: u = prod_i sin(pi x_i), f = -pi^2 d u, Dirichlet data on the
boundary) evaluated at given node coordinates, seeded random vectors and
point clouds, sensor draws, and the named workloads.

The node sets themselves come from the method's own generator (``rbffd_nodes``
on the GPU, ``oracle.nodes`` on the CPU): both implement the same jittered grid
from the published SplitMix64 definition and are compared bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def exact_solution(xyz: np.ndarray) -> np.ndarray:
    """u^a(x) = prod_i sin(pi x_i) at every node (Sec. II-C, Eq. 5)."""
    xyz = np.asarray(xyz, np.float64)
    u = np.ones(xyz.shape[1], np.float64)
    for a in range(xyz.shape[0]):
        u = u * np.sin(np.pi * xyz[a])
    return u


def source(xyz: np.ndarray, interior: np.ndarray) -> np.ndarray:
    """f = Laplacian u^a = -pi^2 d u^a at the interior nodes, in interior-row order."""
    d = xyz.shape[0]
    return (-(np.pi ** 2) * d) * exact_solution(xyz)[np.asarray(interior)]


def start_iterate(xyz: np.ndarray, is_bnd: np.ndarray) -> np.ndarray:
    """u^0: Dirichlet data g = u^a on Dirichlet nodes (code 1), 0 elsewhere (interior
    nodes, and Neumann nodes, code 2, whose values the solver sets)."""
    u = exact_solution(xyz)
    u[np.asarray(is_bnd) != 1] = 0.0
    return u


def neumann_nodes(xyz: np.ndarray, is_bnd: np.ndarray):
    """Neumann nodes (boundary code 2) of the half cube [0, 1/2]^d and their outward unit
    normals: the normal of a face x_a = 1/2 is +e_a; nodes on several such faces take the
    normalised sum.  Returns (node ids ascending, normals [NN, d])."""
    ids = np.nonzero(np.asarray(is_bnd) == 2)[0].astype(np.int32)
    on = (np.asarray(xyz)[:, ids] == 0.5).T.astype(np.float64)
    return ids, on / np.sqrt(on.sum(axis=1, keepdims=True))


def interior_ids(is_bnd: np.ndarray) -> np.ndarray:
    """Interior node indices in ascending order (the row order of stencils)."""
    return np.nonzero(np.asarray(is_bnd) == 0)[0].astype(np.int32)


def random_vector(n: int, seed: int, dist: str = "normal") -> np.ndarray:
    rng = np.random.default_rng(seed)
    if dist == "normal":
        return rng.standard_normal(n)
    return rng.uniform(-1.0, 1.0, n)


def random_points(N: int, d: int, seed: int) -> np.ndarray:
    """Uniform points in the unit d-cube, SoA [d, N]."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, (d, N))


def grid_points(k: int, d: int) -> np.ndarray:
    """Exact k^d grid on [0,1]^d with spacing 1/(k-1), SoA; full of distance ties."""
    ax = np.arange(k, dtype=np.float64) / (k - 1)
    mesh = np.meshgrid(*([ax] * d), indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh])


def sensors(NI: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct interior rows drawn by a seeded shuffle, ascending."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.permutation(NI)[:count]).astype(np.int32)


def num_monomials(d: int, m: int) -> int:
    """M = C(m + d, d) (Sec. II, text after Eq. 3)."""
    return math.comb(m + d, d)


def stencil_size(d: int, m: int) -> int:
    """n = 2M, the support size the workloads use (the paper's rule is 2M + 1)."""
    return 2 * num_monomials(d, m)


@dataclass
class Workload:
    name: str
    d: int
    Kg: int
    m: int
    seed: int
    shape: int = 0           # 0 unit square/cube, 1 disk
    jitter: float = 0.3
    n: int = 0               # 0 -> 2M
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        if self.n == 0:
            self.n = stencil_size(self.d, self.m)

    @property
    def h(self) -> float:
        return 1.0 / self.Kg


# The workloads of the performance study (sizes as quoted with the metric):
WORKLOADS = {
    "square10k_m2": Workload("2D unit square, 10,201 jittered nodes, m=2 (n=12)", 2, 100, 2, 1),
    "square1M_m2": Workload("2D unit square, 1,002,001 jittered nodes, m=2 (n=12)", 2, 1000, 2, 2),
    "square1M_m4": Workload("2D unit square, 1,002,001 jittered nodes, m=4 (n=30)", 2, 1000, 4, 2),
    "square1M_m6": Workload("2D unit square, 1,002,001 jittered nodes, m=6 (n=56)", 2, 1000, 6, 2),
    "cube8M_m4": Workload("3D unit cube, 8,120,601 jittered nodes, m=4 (n=70)", 3, 200, 4, 3),
}


def batched_domains(count: int = 256, seed: int = 4, lo: float = 5e3, hi: float = 2e5):
    """Per-domain (shape, Kg, m, seed) for the batched workload.

    Shape ~ Bernoulli(1/2) between the unit square and the disk of radius 1/2;
    target node count log-uniform in [lo, hi]; m uniform in {2, 4, 6}.
    The square takes Kg = round(sqrt(N)) - 1; the disk takes the Kg whose grid
    spacing gives pi R^2 / h^2 ~ N.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        shape = int(rng.integers(0, 2))
        Nt = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        m = int(rng.choice([2, 4, 6]))
        if shape == 0:
            Kg = max(4, int(round(math.sqrt(Nt))) - 1)
        else:
            h = math.sqrt(math.pi * 0.25 / Nt)
            Kg = max(8, int(round(1.0 / h)))
        out.append((shape, Kg, m, seed * 100003 + k))
    return out
