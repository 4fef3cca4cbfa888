"""GB300 (sm_103a) RBF-FD explicit Poisson path: thin Python binding of librbffd.

Vehovar, Rot and Kosec, "Performance Trade-offs of High Order Meshless
Approximation on Distributed Memory Systems" (arXiv 2502.12878): the stencil
operator of Eq. 1, the RBF-FD weights of Eq. 2-3 (phi(r) = r^3 plus monomials
up to order m), and the explicit iteration of Eq. 6 for the Poisson problem of
Eq. 4-5, all computed by the hand-written CUDA kernels in ``csrc/`` behind the
C ABI of ``include/rbffd.h``.

This module only marshals arguments: torch tensors provide device memory and
the current CUDA stream; every step of the computation runs in librbffd.
There is no CPU fallback.  If the library has not been built, every call raises
``RbffdError`` (build it with ``paper_2502_12878_gb300.build.build()``).

The functions keep the C names (``rbffd_nodes``, ``rbffd_knn``, ``rbffd_weights``,
``rbffd_apply``, ``rbffd_solve_explicit`` ...).
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librbffd.so")

RBFFD_OK = 0
RBFFD_NOT_CONVERGED = 1
RBFFD_ERR_ARG = -1
RBFFD_ERR_CUDA = -2
RBFFD_ERR_SINGULAR = -3
RBFFD_ERR_NONFINITE = -4
RBFFD_ERR_DIVERGED = -5
RBFFD_ERR_TIMEOUT = -6
RBFFD_ERR_CAPACITY = -7

RBFFD_ORDER_MORTON = 0
RBFFD_ORDER_INPUT = 1
RBFFD_ORDER_RANDOM = 2
RBFFD_LAUNCH_GRAPH = 0
RBFFD_LAUNCH_PERSISTENT = 16
RBFFD_LAUNCH_AUTO = 64
RBFFD_LAUNCH_RESIDENT = 128
RBFFD_LAUNCH_PDL = 256
RBFFD_LAUNCH_NO_PDL = 512
RBFFD_LAUNCH_FAR = 2048
RBFFD_LAUNCH_SPLIT = 4096
RBFFD_PACK_IDX32 = 32

EXPORTED = [
    "rbffd_last_error", "rbffd_version", "rbffd_nodes", "rbffd_interior", "rbffd_knn",
    "rbffd_weights", "rbffd_apply", "rbffd_plan_create", "rbffd_plan_destroy", "rbffd_plan_perm",
    "rbffd_solve_explicit", "rbffd_solve_dc", "rbffd_plan_set_dc", "rbffd_stable_dt",
    "rbffd_adjoint", "rbffd_plan_stats", "rbffd_knn_noalloc", "rbffd_batch_create",
    "rbffd_batch_destroy", "rbffd_solve_batch", "rbffd_batch_set_shape", "rbffd_batch_stats",
    "rbffd_error", "rbffd_batch_domain_times", "rbffd_batch_set_costs", "rbffd_adjoint_w",
    "rbffd_knn_masked", "rbffd_weights_dir", "rbffd_plan_set_neumann", "rbffd_plan_layout",
    "rbffd_nodes_pds", "rbffd_nodes_pds_cap", "rbffd_weights_batch", "rbffd_transpose",
    "rbffd_plan_set_wait", "rbffd_fp64_fma_rate", "rbffd_plan_set_resident_halo",
    "rbffd_plan_set_block",
    "rbffd_transpose_layout",
]
RBFFD_KNN_NOALLOC_MAX_NODES = 262144


class RbffdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"librbffd error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded librbffd (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RbffdError(RBFFD_ERR_CUDA, f"{LIB_PATH} is missing: build it with "
                         "paper_2502_12878_gb300.build.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, D, U64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                         ctypes.c_uint64)
    PI64 = ctypes.POINTER(ctypes.c_int64)
    PD = ctypes.POINTER(ctypes.c_double)
    sig = {
        "rbffd_last_error": (ctypes.c_char_p, []),
        "rbffd_version": (I, []),
        "rbffd_nodes": (I, [I, I, I, D, U64, P, P, I64, PI64, P]),
        "rbffd_interior": (I, [P, I64, P, PI64, P]),
        "rbffd_knn": (I, [P, I64, I, P, I64, I, P, P]),
        "rbffd_weights": (I, [P, I64, I, P, I64, I, I, P, P, PI64, PI64, P]),
        "rbffd_apply": (I, [P, P, I64, I, P, P, P]),
        "rbffd_plan_create": (I, [P, P, I64, I, P, P, P, I64, I, I, U64,
                                  ctypes.POINTER(ctypes.c_void_p), P]),
        "rbffd_plan_destroy": (I, [P]),
        "rbffd_plan_perm": (I, [P, P, P]),
        "rbffd_solve_explicit": (I, [P, P, P, D, I64, D, I, PI64, PD, P]),
        "rbffd_solve_dc": (I, [P, P, P, D, D, I64, I64, D, PI64, PI64, PD, P]),
        "rbffd_plan_set_dc": (I, [P, I64, D]),
        "rbffd_stable_dt": (I, [P, P, I, D, PD, PD, P]),
        "rbffd_adjoint": (I, [P, P, I64, D, P, P, P, P]),
        "rbffd_plan_stats": (I, [P, PD, PI64, PI64, P]),
        "rbffd_knn_noalloc": (I, [P, I64, I, P, I64, I, P, P]),
        "rbffd_batch_create": (I, [P, I, I, ctypes.POINTER(ctypes.c_void_p), P]),
        "rbffd_batch_destroy": (I, [P]),
        "rbffd_solve_batch": (I, [P, P, P, P, P, P, P, P, P, P]),
        "rbffd_batch_set_shape": (I, [P, I, I, I, P]),
        "rbffd_batch_stats": (I, [P, PD, P]),
        "rbffd_error": (I, [P, P, I64, PD, PD, P]),
        "rbffd_batch_domain_times": (I, [P, P, P, P, P]),
        "rbffd_batch_set_costs": (I, [P, P]),
        "rbffd_adjoint_w": (I, [P, P, P, I64, P, I64, D, P, P, P, P, P]),
        "rbffd_knn_masked": (I, [P, I64, I, P, P, I64, I, P, P]),
        "rbffd_weights_dir": (I, [P, I64, I, P, I64, I, I, P, P, P, PI64, PI64, P]),
        "rbffd_plan_set_neumann": (I, [P, I64, P, P, P, I, P, P]),
        "rbffd_plan_layout": (I, [P, PI64, PI64, PD, PD]),
        "rbffd_transpose_layout": (I, [P, PI64, PI64, PI64, PD]),
        "rbffd_nodes_pds": (I, [I, I, I, I, D, U64, P, P, I64, PI64, PI64, P]),
        "rbffd_nodes_pds_cap": (I, [I, I, D, PI64]),
        "rbffd_weights_batch": (I, [I, P, P, P, P, P, P, P, P, P, P, P]),
        "rbffd_transpose": (I, [P, P]),
        "rbffd_plan_set_wait": (I, [P, D, I]),
        "rbffd_fp64_fma_rate": (I, [I64, PD, PD, P]),
        "rbffd_plan_set_resident_halo": (I, [P, I64]),
        "rbffd_plan_set_block": (I, [P, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check(code: int, allow=(RBFFD_OK,)):
    if code in allow:
        return code
    msg = lib().rbffd_last_error().decode(errors="replace")
    raise RbffdError(code, msg)


def _dev(t: torch.Tensor, dtype, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


# ------------------------------------------------------------------ entry points
def rbffd_nodes(d: int, shape: int, Kg: int, jitter_frac: float, seed: int, device="cuda"):
    """Jittered-grid node set.  Returns (xyz [d, N] float64, is_bnd [N] uint8)."""
    L = lib()
    n = ctypes.c_int64(0)
    s = _stream(device)
    _check(L.rbffd_nodes(d, shape, Kg, jitter_frac, seed, None, None, 0, ctypes.byref(n), s))
    N = n.value
    xyz = torch.empty((d, N), dtype=torch.float64, device=device)
    bnd = torch.empty(N, dtype=torch.uint8, device=device)
    _check(L.rbffd_nodes(d, shape, Kg, jitter_frac, seed, _ptr(xyz), _ptr(bnd), N,
                         ctypes.byref(n), s))
    return xyz, bnd


PDS_K = 15
PDS3_K = 50
PDS_ZETA = 1.0 - 1e-10


def rbffd_nodes_pds(shape: int, Kg: int, seed: int, K: int | None = None,
                    zeta: float = PDS_ZETA, d: int = 2, device="cuda"):
    """Poisson-disc node set (unit square or disk in 2D, unit cube in 3D), spacing
    1/Kg, boundary seeds first.  Returns (xyz [d, N] float64, is_bnd [N] uint8,
    generations walked)."""
    L = lib()
    if K is None:
        K = PDS_K if d == 2 else PDS3_K
    cap = ctypes.c_int64(0)
    _check(L.rbffd_nodes_pds_cap(d, Kg, zeta, ctypes.byref(cap)))
    xyz = torch.empty((d, cap.value), dtype=torch.float64, device=device)
    bnd = torch.empty(cap.value, dtype=torch.uint8, device=device)
    n = ctypes.c_int64(0)
    rounds = (ctypes.c_int64 * 2)()
    _check(L.rbffd_nodes_pds(d, shape, Kg, K, zeta, seed, _ptr(xyz), _ptr(bnd), cap.value,
                             ctypes.byref(n), rounds, _stream(device)))
    N = n.value
    return xyz[:, :N].contiguous(), bnd[:N].clone(), rounds[0]


def rbffd_interior(is_bnd: torch.Tensor) -> torch.Tensor:
    """Ascending int32 list of interior node indices."""
    is_bnd = _dev(is_bnd, torch.uint8, "is_bnd")
    out = torch.empty(is_bnd.numel(), dtype=torch.int32, device=is_bnd.device)
    ni = ctypes.c_int64(0)
    _check(lib().rbffd_interior(_ptr(is_bnd), is_bnd.numel(), _ptr(out), ctypes.byref(ni),
                                _stream(is_bnd.device)))
    return out[: ni.value]


def rbffd_knn(xyz: torch.Tensor, centres: torch.Tensor, n: int) -> torch.Tensor:
    """Support of each centre: the n nearest nodes by (d^2, index), centre first."""
    xyz = _dev(xyz, torch.float64, "xyz")
    centres = _dev(centres, torch.int32, "centres")
    d, N = xyz.shape
    idx = torch.empty((centres.numel(), n), dtype=torch.int32, device=xyz.device)
    _check(lib().rbffd_knn(_ptr(xyz), N, d, _ptr(centres), centres.numel(), n, _ptr(idx),
                           _stream(xyz.device)))
    return idx


def rbffd_knn_masked(xyz: torch.Tensor, cand: torch.Tensor, centres: torch.Tensor,
                     n: int) -> torch.Tensor:
    """rbffd_knn over candidate nodes only (cand != 0), the centre always first."""
    xyz = _dev(xyz, torch.float64, "xyz")
    cand = _dev(cand, torch.uint8, "cand")
    centres = _dev(centres, torch.int32, "centres")
    d, N = xyz.shape
    idx = torch.empty((centres.numel(), n), dtype=torch.int32, device=xyz.device)
    _check(lib().rbffd_knn_masked(_ptr(xyz), N, d, _ptr(cand), _ptr(centres), centres.numel(), n,
                                  _ptr(idx), _stream(xyz.device)))
    return idx


def rbffd_weights_dir(xyz: torch.Tensor, idx: torch.Tensor, m: int, dirs: torch.Tensor,
                      check: bool = True):
    """RBF-FD weights of the derivative along dirs [rows, d] (unit vectors)."""
    xyz = _dev(xyz, torch.float64, "xyz")
    idx = _dev(idx, torch.int32, "idx")
    dirs = _dev(dirs, torch.float64, "dirs")
    d, N = xyz.shape
    rows, n = idx.shape
    w = torch.empty((rows, n), dtype=torch.float64, device=xyz.device)
    st = torch.empty(rows, dtype=torch.int8, device=xyz.device)
    nbad = ctypes.c_int64(0)
    first = ctypes.c_int64(0)
    code = lib().rbffd_weights_dir(_ptr(xyz), N, d, _ptr(idx), rows, n, m, _ptr(dirs), _ptr(w),
                                   _ptr(st), ctypes.byref(nbad), ctypes.byref(first),
                                   _stream(xyz.device))
    _check(code, (RBFFD_OK,) if check else (RBFFD_OK, RBFFD_ERR_SINGULAR))
    return w, st


def rbffd_knn_noalloc(xyz: torch.Tensor, centres: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """rbffd_knn into a caller-provided ``idx`` [nc, n], with no device allocation.

    For callers that cannot allocate GPU memory while running: the library works in
    a fixed array of its own (N <= RBFFD_KNN_NOALLOC_MAX_NODES).  Calls that overlap
    on the GPU share that array and race; serialise them.  Nothing here copies or
    allocates either: every tensor must already be contiguous, on one device, and
    ``idx`` must have one row per centre."""
    if xyz.dim() != 2 or centres.dim() != 1 or idx.dim() != 2:
        raise ValueError("need xyz [d, N], centres [nc] and idx [nc, n]")
    if idx.shape[0] != centres.numel() or not 1 <= idx.shape[1] <= 128:
        raise ValueError(f"idx must be [{centres.numel()}, n] with 1 <= n <= 128, "
                         f"got {list(idx.shape)}")
    for t, dtype, name in ((xyz, torch.float64, "xyz"), (centres, torch.int32, "centres"),
                           (idx, torch.int32, "idx")):
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if not (xyz.device == centres.device == idx.device):
        raise ValueError("xyz, centres and idx must be on the same device")
    d, N = xyz.shape
    _check(lib().rbffd_knn_noalloc(_ptr(xyz), N, d, _ptr(centres), centres.numel(), idx.shape[1],
                                   _ptr(idx), _stream(xyz.device)))
    return idx


def rbffd_weights(xyz: torch.Tensor, idx: torch.Tensor, m: int, check: bool = True):
    """RBF-FD Laplacian weights.  Returns (w [rows, n] float64, status [rows] int8)."""
    xyz = _dev(xyz, torch.float64, "xyz")
    idx = _dev(idx, torch.int32, "idx")
    d, N = xyz.shape
    rows, n = idx.shape
    w = torch.empty((rows, n), dtype=torch.float64, device=xyz.device)
    st = torch.empty(rows, dtype=torch.int8, device=xyz.device)
    nbad = ctypes.c_int64(0)
    first = ctypes.c_int64(0)
    code = lib().rbffd_weights(_ptr(xyz), N, d, _ptr(idx), rows, n, m, _ptr(w), _ptr(st),
                               ctypes.byref(nbad), ctypes.byref(first), _stream(xyz.device))
    _check(code, (RBFFD_OK,) if check else (RBFFD_OK, RBFFD_ERR_SINGULAR))
    return w, st


def rbffd_weights_batch(xyzs, idxs, ms, check: bool = True):
    """Weights of many domains in one call (one launch per team size): lists of xyz [d, N], supports
    idx [nc, n] and orders m.  Returns a list of (w [nc, n], status [nc])."""
    nd = len(xyzs)
    xyzs = [_dev(x, torch.float64, "xyz") for x in xyzs]
    idxs = [_dev(i, torch.int32, "idx") for i in idxs]
    ws = [torch.empty(i.shape, dtype=torch.float64, device=i.device) for i in idxs]
    sts = [torch.empty(i.shape[0], dtype=torch.int8, device=i.device) for i in idxs]
    VP = ctypes.c_void_p * nd
    I64 = ctypes.c_int64 * nd
    IA = ctypes.c_int * nd
    bad = I64()
    code = lib().rbffd_weights_batch(
        nd, VP(*[x.data_ptr() for x in xyzs]), I64(*[x.shape[1] for x in xyzs]),
        IA(*[x.shape[0] for x in xyzs]), VP(*[i.data_ptr() for i in idxs]),
        I64(*[i.shape[0] for i in idxs]), IA(*[i.shape[1] for i in idxs]), IA(*ms),
        VP(*[w.data_ptr() for w in ws]), VP(*[t.data_ptr() for t in sts]), bad,
        _stream(xyzs[0].device))
    _check(code, (RBFFD_OK,) if check else (RBFFD_OK, RBFFD_ERR_SINGULAR))
    return list(zip(ws, sts))


def rbffd_apply(w: torch.Tensor, idx: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """Eq. 1 for every row: Lu[r] = sum_j w[r, j] u[idx[r, j]]."""
    w = _dev(w, torch.float64, "w")
    idx = _dev(idx, torch.int32, "idx")
    u = _dev(u, torch.float64, "u")
    rows, n = idx.shape
    Lu = torch.empty(rows, dtype=torch.float64, device=u.device)
    _check(lib().rbffd_apply(_ptr(w), _ptr(idx), rows, n, _ptr(u), _ptr(Lu), _stream(u.device)))
    return Lu


def rbffd_error(u: torch.Tensor, ua: torch.Tensor):
    """(max |u - u^a|, mean |u - u^a|) over all nodes (Eq. 8 is the mean)."""
    u = _dev(u, torch.float64, "u")
    ua = _dev(ua, torch.float64, "ua")
    mx = ctypes.c_double(0.0)
    mean = ctypes.c_double(0.0)
    _check(lib().rbffd_error(_ptr(u), _ptr(ua), u.numel(), ctypes.byref(mx), ctypes.byref(mean),
                             _stream(u.device)))
    return mx.value, mean.value


def rbffd_fp64_fma_rate(iters: int = 200_000, device="cuda"):
    """Measured FP64 fused multiply-adds per second of the device (best of three
    shapes, ``iters`` fmas per thread each), and the fastest shape's timed ms."""
    rate = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(lib().rbffd_fp64_fma_rate(int(iters), ctypes.byref(rate), ctypes.byref(ms),
                                     _stream(device)))
    return rate.value, ms.value


class Plan:
    """Device-resident solver plan (rbffd_plan_create / rbffd_plan_destroy)."""

    def __init__(self, xyz, is_bnd, interior, idx, w, flags=0, seed=0):
        xyz = _dev(xyz, torch.float64, "xyz")
        is_bnd = _dev(is_bnd, torch.uint8, "is_bnd")
        interior = _dev(interior, torch.int32, "interior")
        idx = _dev(idx, torch.int32, "idx")
        w = _dev(w, torch.float64, "w")
        self.d, self.N = xyz.shape
        self.NI, self.n = idx.shape
        self.device = xyz.device
        self.flags = flags
        self._h = ctypes.c_void_p(None)
        _check(lib().rbffd_plan_create(_ptr(xyz), _ptr(is_bnd), self.N, self.d, _ptr(interior),
                                       _ptr(idx), _ptr(w), self.NI, self.n, flags, seed,
                                       ctypes.byref(self._h), _stream(self.device)))

    @property
    def handle(self):
        if not self._h.value:
            raise RbffdError(RBFFD_ERR_ARG, "plan already destroyed")
        return self._h

    def destroy(self):
        if self._h is not None and self._h.value:
            lib().rbffd_plan_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def perm(self) -> torch.Tensor:
        out = torch.empty(self.N, dtype=torch.int32, device=self.device)
        _check(lib().rbffd_plan_perm(self.handle, _ptr(out), _stream(self.device)))
        return out

    def solve_explicit(self, f, u, dt, max_steps, tol=0.0, precision=0):
        """Eq. 6 in place on ``u`` [N].  Returns (status, steps, last residual max-norm)."""
        f = _dev(f, torch.float64, "f")
        if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()):
            raise ValueError("u must be a contiguous float64 CUDA tensor (updated in place)")
        steps = ctypes.c_int64(0)
        res = ctypes.c_double(0.0)
        code = lib().rbffd_solve_explicit(self.handle, _ptr(f), _ptr(u), float(dt), int(max_steps),
                                          float(tol), int(precision), ctypes.byref(steps),
                                          ctypes.byref(res), _stream(self.device))
        _check(code, (RBFFD_OK, RBFFD_NOT_CONVERGED))
        return code, steps.value, res.value

    def solve_dc(self, f, u, dt, tol, max_outer, K_in, rho_in):
        """FP64 defect correction around an FP32 inner sweep, in place on ``u``.

        Returns (status, outer corrections, inner steps in total, final defect max-norm)."""
        f = _dev(f, torch.float64, "f")
        if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()):
            raise ValueError("u must be a contiguous float64 CUDA tensor (updated in place)")
        outer = ctypes.c_int64(0)
        inner = ctypes.c_int64(0)
        res = ctypes.c_double(0.0)
        code = lib().rbffd_solve_dc(self.handle, _ptr(f), _ptr(u), float(dt), float(tol),
                                    int(max_outer), int(K_in), float(rho_in), ctypes.byref(outer),
                                    ctypes.byref(inner), ctypes.byref(res), _stream(self.device))
        _check(code, (RBFFD_OK, RBFFD_NOT_CONVERGED))
        return code, outer.value, inner.value, res.value

    def adjoint_w(self, f, ckpt, every, dLdu, K, dt):
        """Backward pass with the weight gradient from checkpoints ckpt [nseg, N] (caller
        order, u^0, u^every, ...) and dLdu = dL/du^K [N].
        Returns (grad_w [NI, n], grad_f, grad_g, lam0)."""
        f = _dev(f, torch.float64, "f")
        ckpt = _dev(ckpt, torch.float64, "ckpt")
        lamK = _dev(dLdu, torch.float64, "dLdu")
        if lamK.numel() != self.N:
            raise ValueError("dLdu must have one entry per node")
        gw = torch.empty((self.NI, self.n), dtype=torch.float64, device=self.device)
        gf = torch.empty(self.NI, dtype=torch.float64, device=self.device)
        gg = torch.empty(self.N, dtype=torch.float64, device=self.device)
        l0 = torch.empty(self.NI, dtype=torch.float64, device=self.device)
        _check(lib().rbffd_adjoint_w(self.handle, _ptr(f), _ptr(ckpt), int(every), _ptr(lamK),
                                     int(K), float(dt), _ptr(gw), _ptr(gf), _ptr(gg), _ptr(l0),
                                     _stream(self.device)))
        return gw, gf, gg, l0

    def stats(self):
        """(GPU ms of the last solve's step loops, their steps, kernels launched, launch shape).
        The shape is [a, b] for the FP64 sweep then for the FP32 inner sweep: b = -2 split
        launch (a = threads / 512), -1 resident launch (a = threads / 512, + 4 with far
        lists), 0 grid-stride persistent launch (a = register budget), else graph-replayed
        steps with b blocks per SM (+ 16 as programmatic dependent launches, a = budget)."""
        ms = ctypes.c_double(0.0)
        steps = ctypes.c_int64(0)
        launches = ctypes.c_int64(0)
        shape = (ctypes.c_int * 4)()
        _check(lib().rbffd_plan_stats(self.handle, ctypes.byref(ms), ctypes.byref(steps),
                                      ctypes.byref(launches), shape))
        return ms.value, steps.value, launches.value, list(shape)

    def layout(self):
        """Packed layout: dict(nslices, rows16 = interior rows with 16-bit index codes,
        bytes64 / bytes32 = bytes one FP64 / FP32 sweep streams)."""
        ns, r16 = ctypes.c_int64(0), ctypes.c_int64(0)
        b64, b32 = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(lib().rbffd_plan_layout(self.handle, ctypes.byref(ns), ctypes.byref(r16),
                                       ctypes.byref(b64), ctypes.byref(b32)))
        return {"nslices": ns.value, "rows16": r16.value, "bytes64": b64.value,
                "bytes32": b32.value}

    def set_neumann(self, nodes, idx, w, g=None):
        """Neumann nodes (ids [NN]), their supports idx [NN, nn] (node first) and
        normal-derivative weights w [NN, nn]; data g [NN] (default 0)."""
        nodes = _dev(nodes, torch.int32, "nodes")
        idx = _dev(idx, torch.int32, "idx")
        w = _dev(w, torch.float64, "w")
        g = _dev(g, torch.float64, "g") if g is not None else None
        _check(lib().rbffd_plan_set_neumann(self.handle, nodes.numel(), _ptr(nodes), _ptr(idx),
                                            _ptr(w), idx.shape[1], _ptr(g), _stream(self.device)))

    def set_wait(self, timeout_ms=0.0, held_arrivals=0):
        """Timeout of the persistent launch's barrier waits (<= 0: default); held_arrivals
        > 0 makes every barrier wait for arrivals that never come (tests the timeout)."""
        _check(lib().rbffd_plan_set_wait(self.handle, float(timeout_ms), int(held_arrivals)))

    def set_resident_halo(self, halo=-2):
        """Halo reach of the resident launch (-1 none, >= 0 slots, -2 tuned)."""
        _check(lib().rbffd_plan_set_resident_halo(self.handle, int(halo)))

    def set_block(self, threads=0):
        """Block size of the resident and split launches (512, 1024; 0 tuned)."""
        _check(lib().rbffd_plan_set_block(self.handle, int(threads)))

    def set_dc(self, K_in, rho_in):
        _check(lib().rbffd_plan_set_dc(self.handle, int(K_in), float(rho_in)))

    def stable_dt(self, v0, iters=200, safety=1.05):
        """(2 / (safety * rho), rho) with rho the power-iteration radius of W_II."""
        v0 = _dev(v0, torch.float64, "v0")
        dt = ctypes.c_double(0.0)
        rho = ctypes.c_double(0.0)
        _check(lib().rbffd_stable_dt(self.handle, _ptr(v0), int(iters), float(safety),
                                     ctypes.byref(dt), ctypes.byref(rho), _stream(self.device)))
        return dt.value, rho.value

    def transpose(self):
        """Build the transposed interior operator now (else the first adjoint does)."""
        _check(lib().rbffd_transpose(self.handle, _stream(self.device)))

    def transpose_layout(self):
        """Built transpose: dict(slices, cols16 = interior columns with 16-bit row codes,
        entries = stored entries, bytes = bytes one reverse step streams)."""
        sl, c16, ent = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        by = ctypes.c_double(0.0)
        _check(lib().rbffd_transpose_layout(self.handle, ctypes.byref(sl), ctypes.byref(c16),
                                            ctypes.byref(ent), ctypes.byref(by)))
        return {"slices": sl.value, "cols16": c16.value, "entries": ent.value, "bytes": by.value}

    def adjoint(self, dLdu, K, dt, want_lam0=True):
        """Reverse sweep of K steps from dLdu = dL/du^K [N] (every node; boundary entries
        add directly to grad_g).  Returns (grad_f [NI], grad_g [N], lam0 [NI] or None)."""
        lamK = _dev(dLdu, torch.float64, "dLdu")
        if lamK.numel() != self.N:
            raise ValueError("dLdu must have one entry per node")
        gf = torch.empty(self.NI, dtype=torch.float64, device=self.device)
        gg = torch.empty(self.N, dtype=torch.float64, device=self.device)
        l0 = torch.empty(self.NI, dtype=torch.float64, device=self.device) if want_lam0 else None
        _check(lib().rbffd_adjoint(self.handle, _ptr(lamK), int(K), float(dt), _ptr(gf), _ptr(gg),
                                   _ptr(l0), _stream(self.device)))
        return gf, gg, l0


class Batch:
    """Independent domains solved together in one persistent launch (rbffd_batch_*).

    ``plans`` must stay alive (and unused elsewhere) while the batch exists."""

    def __init__(self, plans, blocks_per_sm=0):
        self.plans = list(plans)
        self.ndom = len(self.plans)
        self.device = self.plans[0].device
        arr = (ctypes.c_void_p * self.ndom)(*[p.handle.value for p in self.plans])
        self._h = ctypes.c_void_p(None)
        _check(lib().rbffd_batch_create(arr, self.ndom, int(blocks_per_sm), ctypes.byref(self._h),
                                        _stream(self.device)))

    def destroy(self):
        if self._h is not None and self._h.value:
            lib().rbffd_batch_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def solve(self, fs, us, dts, max_steps, tols):
        """Batched Eq. 6 in place on every ``us[i]``.  Returns (code, steps, res, status) lists."""
        nd = self.ndom
        for t in list(fs) + list(us):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("f and u must be contiguous float64 CUDA tensors")
        fa = (ctypes.c_void_p * nd)(*[t.data_ptr() for t in fs])
        ua = (ctypes.c_void_p * nd)(*[t.data_ptr() for t in us])
        dta = (ctypes.c_double * nd)(*[float(x) for x in dts])
        ma = (ctypes.c_int64 * nd)(*[int(x) for x in max_steps])
        ta = (ctypes.c_double * nd)(*[float(x) for x in tols])
        steps = (ctypes.c_int64 * nd)()
        res = (ctypes.c_double * nd)()
        st = (ctypes.c_int * nd)()
        code = lib().rbffd_solve_batch(self._h, fa, ua, dta, ma, ta, steps, res, st,
                                       _stream(self.device))
        _check(code, (RBFFD_OK, RBFFD_NOT_CONVERGED))
        return code, list(steps), list(res), list(st)

    def set_shape(self, minb, blocks_per_sm, threads=256):
        _check(lib().rbffd_batch_set_shape(self._h, int(minb), int(blocks_per_sm), int(threads),
                                           _stream(self.device)))

    def stats(self):
        """(GPU ms of the last solve, [minb, blocks/SM, grid, cooperative, threads])."""
        ms = ctypes.c_double(0.0)
        shape = (ctypes.c_int * 5)()
        _check(lib().rbffd_batch_stats(self._h, ctypes.byref(ms), shape))
        return ms.value, list(shape)

    def domain_times(self):
        """Per domain of the last solve: (start ms, end ms, rank-0 block, team size)."""
        a = (ctypes.c_double * self.ndom)()
        b = (ctypes.c_double * self.ndom)()
        c = (ctypes.c_int * self.ndom)()
        d = (ctypes.c_int * self.ndom)()
        _check(lib().rbffd_batch_domain_times(self._h, a, b, c, d))
        return list(a), list(b), list(c), list(d)

    def set_costs(self, costs):
        arr = (ctypes.c_double * self.ndom)(*[float(c) for c in costs])
        _check(lib().rbffd_batch_set_costs(self._h, arr))

    def calibrate(self, fs, us, dts, probe_steps=200):
        """Measure each domain's cost of one step (block-ms: its duration in a probe
        solve x its team size / steps) and give the costs to the library's load
        balancer for the next solves.  ``us`` are clobbered."""
        self.solve(fs, us, dts, [probe_steps] * self.ndom, [0.0] * self.ndom)
        t0, t1, _, team = self.domain_times()
        costs = [max(e - b, 1e-6) * max(s, 1) / probe_steps for b, e, s in zip(t0, t1, team)]
        self.set_costs(costs)
        return costs

    def tune(self, fs, us, dts, probe_steps=200, candidates=None, cache=None):
        """Autotune the launch shape: time a short solve per (minb, blocks/SM) candidate,
        then calibrate the per-domain costs at the chosen shape.  ``us`` are clobbered.
        ``cache`` (a JSON path) remembers the shape per device, domain count and size."""
        import json
        key = None
        known = {}
        if cache:
            dev = torch.cuda.get_device_properties(self.device)
            work = sum(p.NI * (12 * p.n + 24) for p in self.plans)
            key = f"{dev.name}|{dev.multi_processor_count}|{self.ndom}|{int(math.log2(work + 1))}"
            try:
                with open(cache) as fh:
                    known = json.load(fh)
            except (OSError, ValueError):
                known = {}
        if key and key in known:
            best = tuple(known[key])
            self.set_shape(*best)
        else:
            cands = candidates or (
                [(m, b, 256) for m in (1, 2, 3) for b in (1, 2, 3, 4) if b >= m - 1]
                + [(m, b, 512) for m in (1, 2) for b in (1, 2) if b >= m - 1]
                + [(1, 1, 768), (1, 1, 1024)])
            best, best_ms = None, float("inf")
            for (m, b, th) in cands:
                try:
                    self.set_shape(m, b, th)
                except RbffdError:
                    continue
                # costs measured at this shape, then a timed probe with them
                self.calibrate(fs, us, dts, probe_steps)
                self.solve(fs, us, dts, [probe_steps] * self.ndom, [0.0] * self.ndom)
                ms, _ = self.stats()
                if ms < best_ms:
                    best, best_ms = (m, b, th), ms
            if best is None:
                raise RbffdError(RBFFD_ERR_CAPACITY, "no launch shape fits")
            self.set_shape(*best)
            if cache and key:
                known[key] = list(best)
                with open(cache, "w") as fh:
                    json.dump(known, fh)
        self.calibrate(fs, us, dts, probe_steps)
        return best


class ExplicitSolver:
    """K explicit steps of Eq. 6 on a fixed node set, as a differentiable map.

    ``solver(f, g, w)`` returns u^K [N] from u^0 = 0 inside and g on the boundary
    (``g`` in the order of the boundary nodes, ascending).  Gradients flow to f, g
    and (if it requires grad) the weights w [NI, n].  The forward keeps every
    ``every``-th iterate (default ceil(sqrt(K))); the backward replays each
    segment from its checkpoint to get the iterates the weight gradient needs."""

    def __init__(self, xyz, is_bnd, interior, idx, K, dt, every=None, flags=0):
        self.xyz, self.is_bnd = xyz, is_bnd
        self.interior, self.idx = interior, idx
        self.K, self.dt = int(K), float(dt)
        self.every = int(every) if every else max(1, math.ceil(math.sqrt(max(self.K, 1))))
        self.flags = flags
        self.bnd = torch.nonzero(is_bnd).flatten()
        self.N = xyz.shape[1]
        self._plan, self._w_key = None, None

    def plan(self, w):
        key = (w.data_ptr(), w._version)
        if self._plan is None or self._w_key != key:
            if self._plan is not None:
                self._plan.destroy()
            self._plan = Plan(self.xyz, self.is_bnd, self.interior, self.idx, w.detach(),
                              self.flags)
            self._w_key = key
        return self._plan

    def __call__(self, f, g, w):
        return RBFFDExplicit.apply(f, g, w, self)


class RBFFDExplicit(torch.autograd.Function):
    """u^K of Eq. 6 with the adjoint (transposed stencil sweep) as its backward."""

    @staticmethod
    def forward(ctx, f, g, w, solver):
        plan = solver.plan(w)
        u = torch.zeros(solver.N, dtype=torch.float64, device=f.device)
        u[solver.bnd] = g
        ck = []
        done = 0
        while done < solver.K:
            ck.append(u.clone())
            steps = min(solver.every, solver.K - done)
            plan.solve_explicit(f.contiguous(), u, solver.dt, steps, 0.0)
            done += steps
        ckpt = torch.stack(ck) if ck else u.clone()[None]
        ctx.solver = solver
        ctx.save_for_backward(f, ckpt)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        solver = ctx.solver
        f, ckpt = ctx.saved_tensors
        plan = solver._plan
        grad_u = grad_u.contiguous()
        gw = None
        if ctx.needs_input_grad[2]:
            gw, gf, gg, _ = plan.adjoint_w(f.contiguous(), ckpt, solver.every, grad_u, solver.K,
                                           solver.dt)
        else:
            gf, gg, _ = plan.adjoint(grad_u, solver.K, solver.dt, want_lam0=False)
        # grad_g holds dL/dg at the boundary nodes (direct term included); g is
        # given in the order of the boundary nodes
        return gf, gg[solver.bnd], gw, None


def rbffd_plan_create(xyz, is_bnd, interior, idx, w, flags=0, seed=0) -> Plan:
    return Plan(xyz, is_bnd, interior, idx, w, flags, seed)


def rbffd_solve_explicit(plan: Plan, f, u, dt, max_steps, tol=0.0, precision=0):
    return plan.solve_explicit(f, u, dt, max_steps, tol, precision)


def rbffd_solve_dc(plan: Plan, f, u, dt, tol, max_outer, K_in, rho_in):
    return plan.solve_dc(f, u, dt, tol, max_outer, K_in, rho_in)


def rbffd_stable_dt(plan: Plan, v0, iters=200, safety=1.05):
    return plan.stable_dt(v0, iters, safety)


def rbffd_adjoint(plan: Plan, dLdu, K, dt):
    return plan.adjoint(dLdu, K, dt)


def rbffd_transpose(plan: Plan):
    return plan.transpose()


def monomial_count(d: int, m: int) -> int:
    """M = C(m + d, d) (Sec. II, text after Eq. 3)."""
    return math.comb(m + d, d)
