"""Plain CPU oracle for the RBF-FD explicit Poisson path (arXiv 2502.12878).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2502_12878_gb300``) never loads it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``,
OpenMP over the per-node loops); this module compiles it with gcc and wraps
each routine for numpy arrays.  What each routine follows in the paper:

* ``nodes``            jittered-grid stand-in for the Poisson-disc sampler of
                       Sec. II-C (test problem paragraph on node sampling)
* ``knn_brute``        support = the n nearest nodes, centre included (Sec. II,
                       text after Eq. 1); ties go to the lower node index
* ``knn_kdtree``       same result through a kd-tree, pinned to ``knn_brute``
* ``weights``          RBF-FD augmented system, Eq. 2-3, phi(r) = r^3 with
                       monomials up to order m (Sec. II text after Eq. 3)
* ``weights_dir``      the same system for a directional (normal) derivative
* ``apply``            Eq. 1
* ``solve_mixed``      Eq. 6 with Neumann nodes (mixed-boundary variant, Sec. II-C)
* ``solve_explicit``   Eq. 6 (jacobi_step), time step per Eq. 7 (cfl)
* ``solve_dc``         Eq. 6 in FP32 on the correction inside FP64 defect
                       correction (precision split not in the paper)
* ``adjoint``          transpose of Eq. 6 for a sensor misfit (not in the paper)
* ``adjoint_w``        the same plus the gradient with respect to the weights
* ``power_rho``        spectral radius of the interior operator, from which the
                       stability bound that Eq. 7 only approximates is taken
* ``mean_abs_error``   Eq. 8 (error)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    u64 = ctypes.c_uint64
    sig = {
        "sm64_at": (u64, [u64, u64]),
        "oracle_nodes": (i64, [i32, i32, i32, f64, u64, P, P, i64]),
        "oracle_nodes_pds": (i64, [i32, i32, i32, f64, u64, i32, P, P, i64]),
        "oracle_nodes_pds_cap": (i64, [i32, f64]),
        "oracle_nodes_pds3": (i64, [i32, i32, f64, u64, i32, P, P, i64]),
        "oracle_nodes_pds3_cap": (i64, [i32, f64]),
        "oracle_knn_brute": (i32, [P, i64, i32, P, i64, i32, P]),
        "oracle_knn_kdtree": (i32, [P, i64, i32, P, i64, i32, P]),
        "oracle_knn_brute_masked": (i32, [P, i64, i32, P, P, i64, i32, P]),
        "oracle_knn_kdtree_masked": (i32, [P, i64, i32, P, P, i64, i32, P]),
        "oracle_num_monomials": (i32, [i32, i32]),
        "oracle_monomials": (i32, [i32, i32, P]),
        "oracle_weights": (i64, [P, i64, i32, P, i64, i32, i32, P, P]),
        "oracle_apply": (None, [P, P, i64, i32, P, P]),
        "oracle_solve_explicit": (i32, [P, P, P, i64, i64, i32, P, P, f64, i64, f64, P, P]),
        "oracle_solve_dc": (i32, [P, P, P, i64, i64, i32, P, P, f64, f64, i64, i64, f64,
                                  P, P, P, P]),
        "oracle_adjoint": (i32, [P, P, P, i64, i64, i32, P, i64, f64, P, P, P]),
        "oracle_adjoint_w": (i32, [P, P, P, i64, i64, i32, P, P, P, i64, f64, P, P, P, P]),
        "oracle_power_rho": (f64, [P, P, P, i64, i64, i32, P, i32]),
        "oracle_weights_dir": (i64, [P, i64, i32, P, i64, i32, i32, P, P, P]),
        "oracle_solve_mixed": (i32, [P, P, P, i64, i64, i32, P, P, P, P, i64, i32, P, P, f64,
                                     i64, f64, P, P]),
        "oracle_gepp_dense": (i32, [i32, P, P, P]),
        "oracle_num_threads": (i32, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def sm64_at(seed: int, counter: int) -> int:
    """The counter-th output of SplitMix64 seeded with ``seed``."""
    return int(_load().sm64_at(seed, counter))


def nodes(d: int, shape: int, Kg: int, jitter_frac: float, seed: int):
    """Jittered-grid node set.  Returns (xyz [d, N] float64, is_bnd [N] uint8)."""
    lib = _load()
    z = np.zeros(1, np.float64)
    b = np.zeros(1, np.uint8)
    N = lib.oracle_nodes(d, shape, Kg, jitter_frac, seed, _p(z), _p(b), 0)
    if N < 0:
        raise ValueError("oracle_nodes: bad arguments")
    xyz = np.zeros((d, N), np.float64)
    is_bnd = np.zeros(N, np.uint8)
    N2 = lib.oracle_nodes(d, shape, Kg, jitter_frac, seed, _p(xyz), _p(is_bnd), N)
    assert N2 == N
    return xyz, is_bnd


PDS_K = 15
PDS_ZETA = 1.0 - 1e-10


def nodes_pds(shape: int, Kg: int, seed: int, K: int = PDS_K, zeta: float = PDS_ZETA,
              brute: bool = False):
    """Poisson-disc node set in 2D (unit square or disk), spacing 1/Kg, boundary
    seeds first.  Returns (xyz [2, N] float64, is_bnd [N] uint8)."""
    lib = _load()
    cap = lib.oracle_nodes_pds_cap(Kg, zeta)
    if cap < 0:
        raise ValueError("oracle_nodes_pds: bad arguments")
    xyz = np.zeros((2, cap), np.float64)
    is_bnd = np.zeros(cap, np.uint8)
    N = lib.oracle_nodes_pds(shape, Kg, K, zeta, seed, 1 if brute else 0, _p(xyz), _p(is_bnd),
                             cap)
    if N < 0:
        raise ValueError(f"oracle_nodes_pds failed ({N})")
    return np.ascontiguousarray(xyz[:, :N]), is_bnd[:N].copy()


PDS3_K = 50


def nodes_pds3(Kg: int, seed: int, K: int = PDS3_K, zeta: float = PDS_ZETA, brute: bool = False):
    """Poisson-disc node set in the unit cube, spacing 1/Kg, boundary seeds first.
    Returns (xyz [3, N] float64, is_bnd [N] uint8)."""
    lib = _load()
    cap = lib.oracle_nodes_pds3_cap(Kg, zeta)
    if cap < 0:
        raise ValueError("oracle_nodes_pds3: bad arguments")
    xyz = np.zeros((3, cap), np.float64)
    is_bnd = np.zeros(cap, np.uint8)
    N = lib.oracle_nodes_pds3(Kg, K, zeta, seed, 1 if brute else 0, _p(xyz), _p(is_bnd), cap)
    if N < 0:
        raise ValueError(f"oracle_nodes_pds3 failed ({N})")
    return np.ascontiguousarray(xyz[:, :N]), is_bnd[:N].copy()


def _knn(fn, xyz, centres, n):
    xyz = _c(xyz, np.float64)
    d, N = xyz.shape
    centres = _c(centres, np.int32)
    idx = np.zeros((len(centres), n), np.int32)
    st = fn(_p(xyz), N, d, _p(centres), len(centres), n, _p(idx))
    if st != 0:
        raise ValueError(f"oracle knn failed ({st})")
    return idx


def _knn_masked(fn, xyz, cand, centres, n):
    xyz = _c(xyz, np.float64)
    d, N = xyz.shape
    cand = _c(cand, np.uint8)
    centres = _c(centres, np.int32)
    idx = np.zeros((len(centres), n), np.int32)
    st = fn(_p(xyz), N, d, _p(cand), _p(centres), len(centres), n, _p(idx))
    if st != 0:
        raise ValueError(f"oracle knn failed ({st})")
    return idx


def knn_brute(xyz, centres, n, cand=None):
    """n nearest nodes of every centre by the key (d^2, index), centre first.
    With ``cand`` only nodes with cand != 0 (and the centre) are candidates."""
    if cand is not None:
        return _knn_masked(_load().oracle_knn_brute_masked, xyz, cand, centres, n)
    return _knn(_load().oracle_knn_brute, xyz, centres, n)


def knn_kdtree(xyz, centres, n, cand=None):
    if cand is not None:
        return _knn_masked(_load().oracle_knn_kdtree_masked, xyz, cand, centres, n)
    return _knn(_load().oracle_knn_kdtree, xyz, centres, n)


def monomials(d: int, m: int) -> np.ndarray:
    lib = _load()
    M = lib.oracle_num_monomials(d, m)
    ex = np.zeros((M, 3), np.int32)
    lib.oracle_monomials(d, m, _p(ex))
    return ex[:, :d]


def weights(xyz, idx, m: int):
    """RBF-FD Laplacian weights for each support row of ``idx``.

    Returns (w [rows, n] float64, status [rows] int8; 0 ok, 1 singular)."""
    xyz = _c(xyz, np.float64)
    d, N = xyz.shape
    idx = _c(idx, np.int32)
    rows, n = idx.shape
    w = np.zeros((rows, n), np.float64)
    st = np.zeros(rows, np.int8)
    _load().oracle_weights(_p(xyz), N, d, _p(idx), rows, n, m, _p(w), _p(st))
    return w, st


def weights_dir(xyz, idx, m: int, dirs):
    """RBF-FD weights of the derivative along the unit vectors dirs [rows, d]."""
    xyz = _c(xyz, np.float64)
    d, N = xyz.shape
    idx = _c(idx, np.int32)
    dirs = _c(dirs, np.float64)
    rows, n = idx.shape
    w = np.zeros((rows, n), np.float64)
    st = np.zeros(rows, np.int8)
    _load().oracle_weights_dir(_p(xyz), N, d, _p(idx), rows, n, m, _p(dirs), _p(w), _p(st))
    return w, st


def solve_mixed(w, idx, interior, f, nnode, nidx, nw, g, u0, dt, max_steps, tol):
    """Eq. 6 with Neumann nodes updated from the previous iterate before each step.

    Returns (u, steps, final max-residual, status)."""
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    interior = _c(interior, np.int32)
    f = _c(f, np.float64)
    nnode = _c(nnode, np.int32)
    nidx = _c(nidx, np.int32)
    nw = _c(nw, np.float64)
    g = _c(g, np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    rows, n = idx.shape
    NN, nn = nidx.shape
    steps = ctypes.c_int64(0)
    res = ctypes.c_double(0.0)
    st = _load().oracle_solve_mixed(_p(w), _p(idx), _p(interior), len(u), rows, n, _p(f),
                                    _p(nnode), _p(nidx), _p(nw), NN, nn, _p(g), _p(u), dt,
                                    max_steps, tol, ctypes.byref(steps), ctypes.byref(res))
    return u, int(steps.value), float(res.value), int(st)


def apply(w, idx, u):
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    u = _c(u, np.float64)
    rows, n = idx.shape
    Lu = np.zeros(rows, np.float64)
    _load().oracle_apply(_p(w), _p(idx), rows, n, _p(u), _p(Lu))
    return Lu


def solve_explicit(w, idx, interior, f, u0, dt, max_steps, tol):
    """Run Eq. 6 from u0.  Returns (u, steps, final max-residual, status)."""
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    interior = _c(interior, np.int32)
    f = _c(f, np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    rows, n = idx.shape
    steps = ctypes.c_int64(0)
    res = ctypes.c_double(0.0)
    st = _load().oracle_solve_explicit(_p(w), _p(idx), _p(interior), len(u), rows, n, _p(f),
                                       _p(u), dt, max_steps, tol, ctypes.byref(steps),
                                       ctypes.byref(res))
    return u, int(steps.value), float(res.value), int(st)


def solve_dc(w, idx, interior, f, u0, dt, tol, max_outer, K_in, rho_in, inner_res=False):
    """FP64 defect correction with an FP32 inner explicit iteration.

    Returns (u, outer corrections, inner steps in total, final defect, status), and
    with ``inner_res`` also max|rho| of the last inner step taken."""
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    interior = _c(interior, np.int32)
    f = _c(f, np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    rows, n = idx.shape
    outer = ctypes.c_int64(0)
    inner = ctypes.c_int64(0)
    res = ctypes.c_double(0.0)
    res_in = ctypes.c_double(0.0)
    st = _load().oracle_solve_dc(_p(w), _p(idx), _p(interior), len(u), rows, n, _p(f), _p(u),
                                 dt, tol, max_outer, K_in, rho_in, ctypes.byref(outer),
                                 ctypes.byref(inner), ctypes.byref(res), ctypes.byref(res_in))
    out = (u, int(outer.value), int(inner.value), float(res.value), int(st))
    return out + (float(res_in.value),) if inner_res else out


def adjoint(w, idx, interior, N, dLdu, K, dt):
    """Backward pass of K explicit steps from dLdu = dL/du^K [N] (node order; the
    boundary entries add directly to dL/dg).  Returns (grad_f [NI], grad_g [N], lam0 [NI])."""
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    interior = _c(interior, np.int32)
    lamK = _c(dLdu, np.float64)
    if lamK.shape != (N,):
        raise ValueError("dLdu must have one entry per node")
    rows, n = idx.shape
    gf = np.zeros(rows, np.float64)
    gg = np.zeros(N, np.float64)
    l0 = np.zeros(rows, np.float64)
    st = _load().oracle_adjoint(_p(w), _p(idx), _p(interior), N, rows, n, _p(lamK), K, dt,
                                _p(gf), _p(gg), _p(l0))
    if st != 0:
        raise RuntimeError("oracle_adjoint failed")
    return gf, gg, l0


def adjoint_w(w, idx, interior, f, u0, dLdu, K, dt):
    """Backward pass including the weight gradient, from dLdu = dL/du^K [N].

    Returns (grad_w [NI, n], grad_f [NI], grad_g [N], lam0 [NI])."""
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    interior = _c(interior, np.int32)
    f = _c(f, np.float64)
    u0 = _c(u0, np.float64)
    lamK = _c(dLdu, np.float64)
    rows, n = idx.shape
    N = len(u0)
    if lamK.shape != (N,):
        raise ValueError("dLdu must have one entry per node")
    gw = np.zeros((rows, n), np.float64)
    gf = np.zeros(rows, np.float64)
    gg = np.zeros(N, np.float64)
    l0 = np.zeros(rows, np.float64)
    st = _load().oracle_adjoint_w(_p(w), _p(idx), _p(interior), N, rows, n, _p(f), _p(u0),
                                  _p(lamK), K, dt, _p(gw), _p(gf), _p(gg), _p(l0))
    if st != 0:
        raise RuntimeError("oracle_adjoint_w failed")
    return gw, gf, gg, l0


def power_rho(w, idx, interior, N, v0, iters=200):
    """Power-iteration estimate of the spectral radius of W restricted to interior rows/cols."""
    w = _c(w, np.float64)
    idx = _c(idx, np.int32)
    interior = _c(interior, np.int32)
    v = np.array(v0, dtype=np.float64, copy=True)
    rows, n = idx.shape
    return float(_load().oracle_power_rho(_p(w), _p(idx), _p(interior), N, rows, n, _p(v),
                                          iters))


def gepp_dense(A, b):
    A = _c(A, np.float64)
    b = _c(b, np.float64)
    s = A.shape[0]
    x = np.zeros(s, np.float64)
    st = _load().oracle_gepp_dense(s, _p(A), _p(b), _p(x))
    if st != 0:
        raise ValueError("singular")
    return x


def mean_abs_error(u, ua):
    """Eq. 8: (1/N) sum |u_i - u^a_i| over all nodes."""
    return float(np.mean(np.abs(np.asarray(u) - np.asarray(ua))))


def stable_dt(w, idx, interior, N, v0, iters=200, safety=1.05):
    """Explicit-Euler bound 2/rho for the interior operator, rho inflated by ``safety``."""
    rho = power_rho(w, idx, interior, N, v0, iters)
    return 2.0 / (safety * rho)
