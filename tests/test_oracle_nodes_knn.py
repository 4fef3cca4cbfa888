"""Pins for the oracle's node generator and support selection (CPU only).

Node sets: the jittered-grid stand-in for the Poisson-disc sampler of Sec. II-C.
Supports: the n nearest nodes with the centre included (Sec. II, text after
Eq. 1); equal distances are ordered by node index.
"""
import os

import numpy as np
import pytest

import rbffd_inputs as gen

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_published_vector(orc):
    vals = [int(l) for l in open(os.path.join(HERE, "golden", "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [orc.sm64_at(1234567, c) for c in range(5)] == vals


@pytest.mark.parametrize("d,Kg", [(1, 17), (2, 23), (3, 9)])
def test_cube_nodes_layout(orc, d, Kg):
    xyz, bnd = orc.nodes(d, 0, Kg, 0.3, 11)
    h = 1.0 / Kg
    assert xyz.shape == (d, (Kg + 1) ** d)
    # generator index of every node, last axis fastest
    gi = np.stack(np.meshgrid(*([np.arange(Kg + 1)] * d), indexing="ij")).reshape(d, -1)
    on_face = np.any((gi == 0) | (gi == Kg), axis=0)
    assert np.array_equal(bnd.astype(bool), on_face)
    # boundary nodes sit on the grid; interior nodes within +-0.3h of it
    assert np.array_equal(xyz[:, on_face], gi[:, on_face] * h)
    off = np.abs(xyz[:, ~on_face] - gi[:, ~on_face] * h)
    assert off.max() <= 0.3 * h * (1 + 1e-12)
    assert off.max() > 0.25 * h          # the jitter is actually there
    # interior jitter is spread over the whole amplitude, mean ~ 0
    sgn = (xyz[:, ~on_face] - gi[:, ~on_face] * h) / (0.3 * h)
    assert abs(sgn.mean()) < 0.1


def test_node_separation_and_reproducibility(orc):
    from scipy.spatial import cKDTree
    xyz, bnd = orc.nodes(2, 0, 60, 0.3, 5)
    dmin = cKDTree(xyz.T).query(xyz.T, k=2)[0][:, 1].min()
    assert dmin >= 0.4 / 60 * (1 - 1e-12)
    xyz2, _ = orc.nodes(2, 0, 60, 0.3, 5)
    assert np.array_equal(xyz, xyz2)
    xyz3, _ = orc.nodes(2, 0, 60, 0.3, 6)
    assert not np.array_equal(xyz, xyz3)


def test_disk_nodes(orc):
    Kg = 40
    h = 1.0 / Kg
    xyz, bnd = orc.nodes(2, 1, Kg, 0.3, 3)
    nb = int(round(np.pi / h))
    assert bnd.sum() == nb and np.all(bnd[-nb:] == 1) and np.all(bnd[:-nb] == 0)
    r = np.hypot(xyz[0] - 0.5, xyz[1] - 0.5)
    assert np.all(r[:-nb] < 0.5 - 0.5 * h)
    # boundary nodes: on the circle, at equispaced angles 2 pi k / nb
    assert np.max(np.abs(r[-nb:] - 0.5)) < 4e-16
    ang = np.arctan2(xyz[1, -nb:] - 0.5, xyz[0, -nb:] - 0.5) % (2 * np.pi)
    assert np.max(np.abs(ang - 2 * np.pi * np.arange(nb) / nb)) < 1e-14
    # interior count close to the disk area over h^2
    ni = len(r) - nb
    assert abs(ni - np.pi * (0.5 - 0.5 * h) ** 2 / h ** 2) < 4 * np.sqrt(ni) + 2 * np.pi / h


def _knn_by_sort(xyz, centres, n):
    """Independent reference: full lexicographic sort of (d2, j) with numpy."""
    out = []
    for c in centres:
        d2 = None
        for a in range(xyz.shape[0]):
            t = xyz[a] - xyz[a, c]
            d2 = t * t if d2 is None else d2 + t * t
        order = np.lexsort((np.arange(xyz.shape[1]), d2))
        out.append(order[:n])
    return np.array(out, np.int32)


@pytest.mark.parametrize("case", ["random2", "random3", "grid2", "grid3", "jit2"])
def test_knn_brute_vs_sort_and_kdtree(orc, case):
    if case == "random2":
        xyz, n = gen.random_points(700, 2, 1), 12
    elif case == "random3":
        xyz, n = gen.random_points(600, 3, 2), 35
    elif case == "grid2":
        xyz, n = gen.grid_points(17, 2), 30       # every distance repeats: ties everywhere
    elif case == "grid3":
        xyz, n = gen.grid_points(8, 3), 70
    else:
        xyz, _ = orc.nodes(2, 0, 25, 0.3, 9)      # exact-grid boundary rows tie
        n = 56
    N = xyz.shape[1]
    centres = np.arange(N, dtype=np.int32)
    ref = _knn_by_sort(xyz, centres, n)
    b = orc.knn_brute(xyz, centres, n)
    k = orc.knn_kdtree(xyz, centres, n)
    assert np.array_equal(b, ref)
    assert np.array_equal(k, ref)
    assert np.array_equal(b[:, 0], centres)      # the centre is its own first neighbour


def test_knn_kdtree_large_sampled(orc):
    xyz, bnd = orc.nodes(2, 0, 300, 0.3, 4)
    centres = np.random.default_rng(0).choice(xyz.shape[1], 300, replace=False).astype(np.int32)
    assert np.array_equal(orc.knn_kdtree(xyz, centres, 30), orc.knn_brute(xyz, centres, 30))


def test_knn_candidate_mask(orc):
    """Masked supports: the centre plus the nearest candidates only, all three ways."""
    xyz, bnd = orc.nodes(2, 2, 20, 0.3, 8)
    cand = (bnd == 0).astype(np.uint8)
    centres = np.nonzero(bnd == 2)[0].astype(np.int32)
    n = 12
    b = orc.knn_brute(xyz, centres, n, cand=cand)
    k = orc.knn_kdtree(xyz, centres, n, cand=cand)
    ref = []
    for c in centres:
        t0 = xyz[0] - xyz[0, c]
        t1 = xyz[1] - xyz[1, c]
        d2 = t0 * t0 + t1 * t1
        ok = (cand == 1) | (np.arange(xyz.shape[1]) == c)
        ids = np.nonzero(ok)[0]
        ref.append(ids[np.lexsort((ids, d2[ids]))][:n])
    assert np.array_equal(b, np.array(ref)) and np.array_equal(k, b)
    assert np.all(b[:, 0] == centres) and np.all(bnd[b[:, 1:]] == 0)
