"""Thin ctypes binding of the C ABI in ``include/rcp.h`` (argument marshalling only).

Every function here forwards torch tensors' device pointers to the CUDA library
``_rcp_gb300.so``; no step of the method runs in Python.  Importing this module does not load
the library; the first call does, and raises ``RuntimeError`` if it is missing or if no CUDA
device is present (there is no CPU fallback).

Layout: the library is column-major.  A symmetric matrix needs no transpose (a contiguous
row-major ``n x n`` tensor is also its own column-major storage, ``lda = n``); after
:func:`rcp_factor` the multipliers sit in the library's strictly lower triangle, i.e. in the
tensor's strictly UPPER triangle (use :func:`unit_lower` to get L as a normal tensor).
Right-hand sides are ``(nrhs, n)`` tensors (column-major ``n x nrhs``, ``ldx = n``) or 1-D.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_rcp_gb300.so")
_lock = threading.Lock()
_lib = None

RCP_FP64, RCP_FP32, RCP_TF32, RCP_TF32X3, RCP_F16X3 = 0, 1, 2, 3, 4
PREC_NAMES = {"fp64": RCP_FP64, "fp32": RCP_FP32, "tf32": RCP_TF32, "tf32x3": RCP_TF32X3, "f16x3": RCP_F16X3}
STATUS = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT", -6: "ENOCONV",
          -7: "EUNSUPPORTED"}


class RcpError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")


class Opts(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("d", ctypes.c_int), ("q_mode", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("prec", ctypes.c_int), ("alpha", ctypes.c_double), ("omega", ctypes.c_void_p),
                ("grid", ctypes.c_int), ("guard_r", ctypes.c_int), ("guard_eps", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("growth_D", ctypes.c_double), ("max_abs_L", ctypes.c_double),
                ("min_sketch_ratio", ctypes.c_double), ("n_2x2", ctypes.c_int), ("info", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("device_flags", ctypes.c_int), ("berr", ctypes.c_double),
                ("anorm", ctypes.c_double), ("gmres_iters", ctypes.c_int), ("rank", ctypes.c_int),
                ("resketches", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    """Load the CUDA library (raises if it is not built or no GPU is visible)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"RCP CUDA library not built ({_LIB_PATH}); run paper_1710_00125_gb300.build.build()")
        if not torch.cuda.is_available():
            raise RuntimeError("RCP needs a CUDA device; there is no CPU fallback")
        torch.cuda.init()
        L = ctypes.CDLL(_LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.rcp_create.argtypes = [ctypes.POINTER(P)]
        L.rcp_destroy.argtypes = [P]
        L.rcp_destroy.restype = None
        L.rcp_status_string.argtypes = [I]
        L.rcp_status_string.restype = ctypes.c_char_p
        L.rcp_sync.argtypes = [P, P]
        L.rcp_reserve.argtypes = [P, I, I, ctypes.POINTER(Opts)]
        L.rcp_factor.argtypes = [P, I, P, I, P, P, P, ctypes.POINTER(Opts), P, ctypes.POINTER(Stats)]
        L.rcp_solve.argtypes = [P, I, I, P, I, P, P, P, I, P, I, P]
        L.rcp_refine.argtypes = [P, I, I, P, I, P, I, P, P, P, I, P, I, P, I, D, I, P, ctypes.POINTER(Stats)]
        L.rcp_exchange_latency.argtypes = [P, I, I, P, ctypes.POINTER(D)]
        L.rcp_wait_expiry.argtypes = [P, I, I, P, ctypes.POINTER(D)]
        L.rcp_wait_expiry.restype = ctypes.c_int
        L.rcp_l_norms.argtypes = [P, I, P, I, I, P, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.rcp_refine_gmres.argtypes = [P, I, I, P, I, P, I, P, P, P, I, P, I, P, I, D, I, I, I, P,
                                       ctypes.POINTER(Stats)]
        L.rcp_sysv.argtypes = [P, I, I, P, I, P, I, P, I, ctypes.POINTER(Opts), D, I, I, P, ctypes.POINTER(Stats)]
        L.rcp_omega.argtypes = [I, I, ctypes.c_uint64, P, P]
        L.rcp_sketch.argtypes = [I, I, P, I, I, ctypes.c_uint64, P, P, P]
        L.rcp_profile.argtypes = [P, I]
        L.rcp_set_speculation.argtypes = [P, I]
        L.rcp_profile_read.argtypes = [P, P, P, I]
        L.rcp_solve_noalloc.argtypes = [I, I, P, I, P, P, P, I, P, I, P]
        L.rcp_solve_noalloc.restype = ctypes.c_int
        L.rcp_panel_trace.argtypes = [P, P, I]
        L.rcp_panel_trace.restype = ctypes.c_int
        L.rcp_kernel_launches.argtypes = []
        L.rcp_kernel_launches.restype = ctypes.c_longlong
        L.rcp_factor_batched.argtypes = [P, I, I, P, P, P, P, P, P, P, P, ctypes.POINTER(Opts), P, P]
        L.rcp_refine_batched.argtypes = [P, I, I, I, P, P, P, P, P, P, P, P, I, P, P, P, P, D, I, P, P, P]
        L.rcp_factor_batched.restype = ctypes.c_int
        L.rcp_tune_batched.argtypes = [P, I, I, P, P, P, P, P, P, P, P, ctypes.POINTER(Opts), P, P,
                                       ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]
        L.rcp_tune_batched.restype = ctypes.c_int
        L.rcp_refine_batched.restype = ctypes.c_int
        L.rcp_set_batched_schedule.argtypes = [P, I, I]
        L.rcp_set_batched_schedule.restype = ctypes.c_int
        L.rcp_get_batched_schedule.argtypes = [P, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                               ctypes.POINTER(I)]
        L.rcp_get_batched_schedule.restype = ctypes.c_int
        for name in ("rcp_profile", "rcp_profile_read", "rcp_set_speculation", "rcp_create", "rcp_sync", "rcp_reserve", "rcp_factor", "rcp_solve", "rcp_refine", "rcp_sysv",
                     "rcp_omega", "rcp_sketch"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check(code, where, allow_info=False):
    if code < 0 or (code > 0 and not allow_info):
        raise RcpError(code, where)
    return code


def make_opts(b=64, d=None, seed=0, prec=RCP_FP64, alpha=None, omega=None, grid=0, q_mode=1, guard_r=0,
              guard_eps=0.0) -> Opts:
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    return Opts(b=b, d=(min(b + 16, 128) if d is None else d), q_mode=q_mode, seed=seed, prec=prec,
                alpha=(math.sqrt(2.0) / 2.0 if alpha is None else alpha),
                omega=(omega.data_ptr() if omega is not None else None), grid=grid, guard_r=guard_r,
                guard_eps=guard_eps)


class Handle:
    """Owns an ``rcp_handle`` (workspace); freed when garbage collected."""

    def __init__(self):
        self._lib = lib()
        h = ctypes.c_void_p()
        _check(self._lib.rcp_create(ctypes.byref(h)), "rcp_create")
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "h", None) and self.h.value:
                self._lib.rcp_destroy(self.h)
                self.h = ctypes.c_void_p()
        except Exception:
            pass


def rcp_create() -> Handle:
    return Handle()


def rcp_sync(h: Handle, stream=None) -> int:
    return _check(lib().rcp_sync(h.h, _stream(stream)), "rcp_sync")


def rcp_reserve(h: Handle, n: int, nrhs: int = 1, opts: Opts | None = None) -> None:
    _check(lib().rcp_reserve(h.h, n, nrhs, ctypes.byref(opts) if opts else None), "rcp_reserve")


def rcp_factor(h: Handle, A: torch.Tensor, Dd: torch.Tensor, Ds: torch.Tensor, perm: torch.Tensor,
               opts: Opts | None = None, stream=None, stats: bool = True):
    """Factor the symmetric ``A`` in place (n x n, contiguous, float64 for FP64 else float32).
    Returns (status, Stats) when ``stats``; status > 0 is LAPACK's info."""
    n = A.shape[0]
    assert A.is_cuda and A.is_contiguous() and A.shape == (n, n)
    st = Stats()
    code = lib().rcp_factor(h.h, n, _ptr(A), max(n, 1), _ptr(Dd), _ptr(Ds), _ptr(perm),
                            ctypes.byref(opts) if opts else None, _stream(stream),
                            ctypes.byref(st) if stats else None)
    _check(code, "rcp_factor", allow_info=True)
    return code, (st if stats else None)


def _rhs_view(X, n):
    if X.dim() == 1:
        return 1, n
    assert X.shape[1] == n and X.is_contiguous()
    return X.shape[0], n


def rcp_solve(h: Handle, LA: torch.Tensor, Dd, Ds, perm, prec, X: torch.Tensor, stream=None) -> None:
    """In place: X <- A^{-1} X using the factor (X float64, (nrhs, n) or (n,))."""
    n = LA.shape[0]
    nrhs, ldx = _rhs_view(X, n)
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    _check(lib().rcp_solve(h.h, n, nrhs, _ptr(LA), n, _ptr(Dd), _ptr(Ds), _ptr(perm), prec, _ptr(X), ldx,
                           _stream(stream)), "rcp_solve")


def rcp_solve_noalloc(LA: torch.Tensor, Dd, Ds, perm, prec, X: torch.Tensor, stream=None) -> None:
    """rcp_solve without any device allocation, for callers that cannot allocate when they
    solve (real-time loops, memory owned by another allocator): scratch comes from a fixed
    16 MiB device array shared by all calls."""
    n = LA.shape[0]
    nrhs, ldx = _rhs_view(X, n)
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    _check(lib().rcp_solve_noalloc(n, nrhs, _ptr(LA), n, _ptr(Dd), _ptr(Ds), _ptr(perm), prec, _ptr(X), ldx,
                                   _stream(stream)), "rcp_solve_noalloc")


def rcp_refine(h: Handle, A64, LA, Dd, Ds, perm, prec, Bv, X, tol=1e-12, max_iter=10, stream=None,
               stats: bool = True, raise_noconv: bool = False):
    n = A64.shape[0]
    nrhs, ldb = _rhs_view(Bv, n)
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    st = Stats()
    code = lib().rcp_refine(h.h, n, nrhs, _ptr(A64), n, _ptr(LA), n, _ptr(Dd), _ptr(Ds), _ptr(perm), prec,
                            _ptr(Bv), ldb, _ptr(X), ldb, float(tol), int(max_iter), _stream(stream),
                            ctypes.byref(st) if stats else None)
    if code == -6 and not raise_noconv:
        return code, st
    _check(code, "rcp_refine")
    return code, (st if stats else None)


def rcp_refine_gmres(h: Handle, A64, LA, Dd, Ds, perm, prec, Bv, X, tol=1e-12, max_outer=10, restart=0,
                     use_x=False, stream=None, raise_noconv: bool = False):
    """GMRES-based refinement (M^{-1} A preconditioned by the factor); returns (status, Stats)."""
    n = A64.shape[0]
    nrhs, ldb = _rhs_view(Bv, n)
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    st = Stats()
    code = lib().rcp_refine_gmres(h.h, n, nrhs, _ptr(A64), n, _ptr(LA), n, _ptr(Dd), _ptr(Ds), _ptr(perm), prec,
                                  _ptr(Bv), ldb, _ptr(X), ldb, float(tol), int(max_outer), int(restart),
                                  int(bool(use_x)), _stream(stream), ctypes.byref(st))
    if code == -6 and not raise_noconv:
        return code, st
    _check(code, "rcp_refine_gmres")
    return code, st


def rcp_sysv(h: Handle, A64, Bv, X, opts: Opts | None = None, tol=1e-12, max_iter=10, host_buffers=False,
             stream=None):
    """Solve A X = B end to end.  With host_buffers the tensors live in (pinned) host memory
    and the copies are part of the call."""
    n = A64.shape[0]
    nrhs, ldb = _rhs_view(Bv, n)
    st = Stats()
    code = lib().rcp_sysv(h.h, n, nrhs, _ptr(A64), n, _ptr(Bv), ldb, _ptr(X), ldb,
                          ctypes.byref(opts) if opts else None, float(tol), int(max_iter), int(bool(host_buffers)),
                          _stream(stream), ctypes.byref(st))
    if code != -6:
        _check(code, "rcp_sysv", allow_info=True)
    return code, st


PHASES = ("sketch", "panel", "interchange", "trailing", "solve", "residual", "h2d")


def rcp_profile(h: Handle, enable=True) -> None:
    """0/False: off; 1/True: per-phase events; 2: events plus per-step panel timestamps."""
    _check(lib().rcp_profile(h.h, int(enable)), "rcp_profile")


def rcp_set_speculation(h: Handle, mode: int) -> None:
    """FP32 panel speculation: -1 automatic, 0 off, 1 shadow sketch copy, 2 deferred update."""
    _check(lib().rcp_set_speculation(h.h, int(mode)), "rcp_set_speculation")


def rcp_l_norms(h: Handle, LA: torch.Tensor, prec, stream=None):
    """(||L||_1, estimate of ||L^{-1}||_1) of the factor ``LA`` from rcp_factor."""
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    nl, ni = ctypes.c_double(), ctypes.c_double()
    n = LA.shape[0]
    _check(lib().rcp_l_norms(h.h, n, _ptr(LA), n, prec, _stream(stream), ctypes.byref(nl), ctypes.byref(ni)),
           "rcp_l_norms")
    return nl.value, ni.value


def rcp_exchange_latency(h: Handle, grid: int = 0, rounds: int = 20000, stream=None) -> float:
    """Microseconds per round of the panel's grid-wide key exchange (latency floor of a pivot step)."""
    us = ctypes.c_double()
    _check(lib().rcp_exchange_latency(h.h, int(grid), int(rounds), _stream(stream), ctypes.byref(us)),
           "rcp_exchange_latency")
    return us.value


def rcp_wait_expiry(h: Handle, limit_us: int, grid: int = 0, stream=None):
    """Run a grid barrier that cannot complete, every wait bounded by limit_us: returns the
    status code (RCP_ETIMEOUT = -5 expected) and how long the first CTA waited (microseconds)."""
    us = ctypes.c_double()
    code = lib().rcp_wait_expiry(h.h, int(grid), int(limit_us), _stream(stream), ctypes.byref(us))
    return code, us.value


def rcp_panel_trace(h: Handle, n: int):
    """(n, 16) uint64 SM clock stamps of the panel steps of the last traced factorization."""
    import numpy as np
    out = np.zeros(n * 16, dtype=np.uint64)
    _check(lib().rcp_panel_trace(h.h, ctypes.c_void_p(out.ctypes.data), out.size), "rcp_panel_trace")
    return out.reshape(n, 16)


def rcp_profile_read(h: Handle) -> dict:
    """Per-phase milliseconds and bracketed-stretch counts since the last read."""
    k = len(PHASES)
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_int * k)()
    _check(lib().rcp_profile_read(h.h, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(cnt, ctypes.c_void_p), k),
           "rcp_profile_read")
    return {name: (ms[i], cnt[i]) for i, name in enumerate(PHASES)}


def rcp_omega(d: int, n: int, seed: int = 0, device="cuda", stream=None) -> torch.Tensor:
    """Omega as a (d, n) float64 tensor view of the column-major d x n array."""
    om = torch.empty((n, d), dtype=torch.float64, device=device)
    _check(lib().rcp_omega(d, n, seed, _ptr(om), _stream(stream)), "rcp_omega")
    return om.t()


def rcp_sketch(A: torch.Tensor, d: int, seed: int = 0, prec=RCP_FP64, omega: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """B = Omega A as a (d, n) tensor view (dtype follows ``prec``)."""
    n = A.shape[0]
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    dt = torch.float64 if prec == RCP_FP64 else torch.float32
    B = torch.empty((n, d), dtype=dt, device=A.device)
    om_ptr = None
    if omega is not None:
        om_cm = omega.t().contiguous()            # (n, d) row-major = d x n column-major
        om_ptr = _ptr(om_cm)
    _check(lib().rcp_sketch(n, d, _ptr(A), n, prec, seed, om_ptr, _ptr(B), _stream(stream)), "rcp_sketch")
    return B.t()


def unit_lower(LA: torch.Tensor) -> torch.Tensor:
    """L (unit lower triangular) from a factored tensor."""
    n = LA.shape[0]
    return torch.tril(LA.t(), -1) + torch.eye(n, dtype=LA.dtype, device=LA.device)


def block_d(Dd: torch.Tensor, Ds: torch.Tensor) -> torch.Tensor:
    D = torch.diag(Dd)
    off = Ds[:-1]
    D += torch.diag(off, -1) + torch.diag(off, 1)
    return D


def rcp_kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().rcp_kernel_launches())


# ---------------------------------------------------------------------------------------------
# batched ragged systems
# ---------------------------------------------------------------------------------------------
def rcp_factor_batched(h: Handle, batch: int, nmax: int, n, A64, lda64, A, lda, Dd, Ds, perm,
                       opts: Opts | None, info, stream=None) -> None:
    """One-to-one call of ``rcp_factor_batched``: every array argument is a device tensor
    (int32 per-system values, int64 pointer tables) or None for A64/lda64."""
    _check(lib().rcp_factor_batched(h.h, int(batch), int(nmax), _ptr(n), _ptr(A64), _ptr(lda64), _ptr(A),
                                    _ptr(lda), _ptr(Dd), _ptr(Ds), _ptr(perm),
                                    ctypes.byref(opts) if opts else None, _ptr(info), _stream(stream)),
           "rcp_factor_batched")


def rcp_refine_batched(h: Handle, batch: int, nmax: int, nrhs: int, n, A64, lda64, LA, ldla, Dd, Ds, perm,
                       prec, Bv, ldb, X, ldx, tol=1e-12, max_iter=10, berr=None, iters=None,
                       stream=None) -> None:
    """One-to-one call of ``rcp_refine_batched`` (A64/lda64 None: solve only)."""
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    _check(lib().rcp_refine_batched(h.h, int(batch), int(nmax), int(nrhs), _ptr(n), _ptr(A64), _ptr(lda64),
                                    _ptr(LA), _ptr(ldla), _ptr(Dd), _ptr(Ds), _ptr(perm), int(prec), _ptr(Bv),
                                    _ptr(ldb), _ptr(X), _ptr(ldx), float(tol), int(max_iter), _ptr(berr),
                                    _ptr(iters), _stream(stream)), "rcp_refine_batched")


def rcp_set_batched_schedule(h: Handle, threads: int = 0, split: int = 0) -> None:
    """One-to-one call of ``rcp_set_batched_schedule`` (0, 0: the tuned or default schedule)."""
    _check(lib().rcp_set_batched_schedule(h.h, int(threads), int(split)), "rcp_set_batched_schedule")


def rcp_get_batched_schedule(h: Handle, nmax: int, d: int = 0, prec="fp32") -> dict:
    """``rcp_get_batched_schedule``: the shape and CTA schedule rcp_factor_batched would use."""
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    b, dd, t, sp = (ctypes.c_int(0) for _ in range(4))
    _check(lib().rcp_get_batched_schedule(h.h, int(nmax), int(d), int(prec), ctypes.byref(b), ctypes.byref(dd),
                                          ctypes.byref(t), ctypes.byref(sp)), "rcp_get_batched_schedule")
    return {"b": b.value, "d": dd.value, "threads": t.value, "split": sp.value}


class Batch:
    """Pooled device storage and pointer tables for a ragged batch (argument marshalling only).

    System i owns an ``n_i x n_i`` FP64 original (``A64``), its factor (``F``: float64 for
    ``prec='fp64'``, else float32), ``Dd``/``Ds``/``perm`` of length n_i, right-hand sides
    ``B`` and solutions ``X`` (``nrhs x n_i`` row-major, i.e. column-major ``n_i x nrhs``).
    Each pool is one allocation; ``a64(i)``, ``b(i)``, ``x(i)`` ... return views."""

    def __init__(self, ns, nrhs: int, prec="fp32", device="cuda"):
        if isinstance(prec, str):
            prec = PREC_NAMES[prec]
        self.prec = prec
        self.ns = [int(v) for v in ns]
        self.batch = len(self.ns)
        self.nmax = max(self.ns) if self.ns else 0
        self.nrhs = int(nrhs)
        dev = torch.device(device)
        sq, ln, rh = [0], [0], [0]
        for v in self.ns:
            sq.append(sq[-1] + v * v)
            ln.append(ln[-1] + v)
            rh.append(rh[-1] + v * self.nrhs)
        self.off_sq, self.off_n, self.off_rhs = sq, ln, rh
        fdt = torch.float64 if prec == RCP_FP64 else torch.float32
        self.A64_pool = torch.zeros(max(sq[-1], 1), dtype=torch.float64, device=dev)
        self.F_pool = torch.zeros(max(sq[-1], 1), dtype=fdt, device=dev)
        self.Dd_pool = torch.zeros(max(ln[-1], 1), dtype=torch.float64, device=dev)
        self.Ds_pool = torch.zeros(max(ln[-1], 1), dtype=torch.float64, device=dev)
        self.perm_pool = torch.zeros(max(ln[-1], 1), dtype=torch.int32, device=dev)
        self.B_pool = torch.zeros(max(rh[-1], 1), dtype=torch.float64, device=dev)
        self.X_pool = torch.zeros(max(rh[-1], 1), dtype=torch.float64, device=dev)
        self.n = torch.tensor(self.ns, dtype=torch.int32, device=dev)
        self.ld = torch.tensor([max(v, 1) for v in self.ns], dtype=torch.int32, device=dev)
        self.info = torch.zeros(self.batch, dtype=torch.int32, device=dev)
        self.berr = torch.zeros(self.batch, dtype=torch.float64, device=dev)
        self.iters = torch.zeros(self.batch, dtype=torch.int32, device=dev)

        def table(pool, offs):
            base, es = pool.data_ptr(), pool.element_size()
            return torch.tensor([base + o * es for o in offs[:-1]], dtype=torch.int64, device=dev)

        self.p_A64 = table(self.A64_pool, sq)
        self.p_F = table(self.F_pool, sq)
        self.p_Dd = table(self.Dd_pool, ln)
        self.p_Ds = table(self.Ds_pool, ln)
        self.p_perm = table(self.perm_pool, ln)
        self.p_B = table(self.B_pool, rh)
        self.p_X = table(self.X_pool, rh)

    def _mat(self, pool, i):
        v = self.ns[i]
        return pool[self.off_sq[i]:self.off_sq[i] + v * v].view(v, v)

    def a64(self, i):
        return self._mat(self.A64_pool, i)

    def f(self, i):
        return self._mat(self.F_pool, i)

    def dd(self, i):
        return self.Dd_pool[self.off_n[i]:self.off_n[i + 1]]

    def ds(self, i):
        return self.Ds_pool[self.off_n[i]:self.off_n[i + 1]]

    def perm(self, i):
        return self.perm_pool[self.off_n[i]:self.off_n[i + 1]]

    def b(self, i):
        return self.B_pool[self.off_rhs[i]:self.off_rhs[i + 1]].view(self.nrhs, self.ns[i])

    def x(self, i):
        return self.X_pool[self.off_rhs[i]:self.off_rhs[i + 1]].view(self.nrhs, self.ns[i])

    def factor(self, h: Handle, opts: Opts | None = None, from_a64=True, stream=None) -> None:
        """rcp_factor_batched on every system (FP64 originals copied into the factors first)."""
        if opts is None:
            opts = Opts(b=32, d=40, q_mode=1, seed=0, prec=self.prec, alpha=math.sqrt(2.0) / 2.0, omega=None, grid=0)
        rcp_factor_batched(h, self.batch, self.nmax, self.n, self.p_A64 if from_a64 else None,
                           self.ld if from_a64 else None, self.p_F, self.ld, self.p_Dd, self.p_Ds, self.p_perm,
                           opts, self.info, stream)

    def tune(self, h: Handle, opts: Opts | None = None, stream=None):
        """rcp_tune_batched on this batch: returns (chosen b, its factor time in ms); later
        factor() calls with opts.b == 0 use the choice."""
        if opts is None:
            opts = Opts(b=0, d=40, q_mode=1, seed=0, prec=self.prec, alpha=math.sqrt(2.0) / 2.0, omega=None, grid=0)
        bb, ms = ctypes.c_int(0), ctypes.c_float(0.0)
        _check(lib().rcp_tune_batched(h.h, self.batch, self.nmax, _ptr(self.n), _ptr(self.p_A64), _ptr(self.ld),
                                      _ptr(self.p_F), _ptr(self.ld), _ptr(self.p_Dd), _ptr(self.p_Ds),
                                      _ptr(self.p_perm), ctypes.byref(opts), _ptr(self.info), _stream(stream),
                                      ctypes.byref(bb), ctypes.byref(ms)), "rcp_tune_batched")
        return bb.value, ms.value

    def refine(self, h: Handle, tol=1e-12, max_iter=10, refine=True, stream=None) -> None:
        """rcp_refine_batched: X = solve(B), then FP64 refinement when ``refine``."""
        rcp_refine_batched(h, self.batch, self.nmax, self.nrhs, self.n, self.p_A64 if refine else None,
                           self.ld if refine else None, self.p_F, self.ld, self.p_Dd, self.p_Ds, self.p_perm,
                           self.prec, self.p_B, self.ld, self.p_X, self.ld, tol, max_iter, self.berr, self.iters,
                           stream)

