"""Plain FP64 CPU oracle for randomized complete pivoting (RCP), Feng, Xiao and Gu.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` import this package.  The CUDA library never loads it, and this package
never loads the CUDA library.

The arithmetic lives in ``rcp_oracle.c`` (plain C, compiled with gcc by :func:`build`); this
module only marshals numpy arrays through ctypes and adds a few closed forms from the paper's
analysis section that the tests use as diagnostics.

Conventions: matrices are numpy float64 arrays; ``perm[i]`` is the original index that ends at
position ``i`` so that ``A[np.ix_(perm, perm)] == L @ D @ L.T``; ``Dd`` is the diagonal of D and
``Ds[i] = D[i+1, i]`` (zero for 1x1 blocks).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcp_oracle.c")
_SO = os.path.join(_HERE, "_rcp_oracle.so")
_lock = threading.Lock()
_lib = None

SQRT2_OVER_2 = math.sqrt(2.0) / 2.0           # alpha of the SBKP rule
BK_ALPHA = (1.0 + math.sqrt(17.0)) / 8.0      # alpha of Bunch-Kaufman / Bunch-Parlett


def build(force: bool = False) -> str:
    """Compile ``rcp_oracle.c`` into ``_rcp_oracle.so`` (plain gcc, portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Step(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("pi", ctypes.c_int), ("r", ctypes.c_int),
                ("kase", ctypes.c_int), ("s", ctypes.c_int),
                ("norm2", ctypes.c_double), ("lam", ctypes.c_double),
                ("norm2_next", ctypes.c_double), ("lam_next", ctypes.c_double),
                ("akk", ctypes.c_double), ("arr", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_philox4x64_10.argtypes = [P, P, P]
            lib.oracle_omega.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P]
            lib.oracle_sketch.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
            lib.oracle_rcp.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, P, P, P, P, P, P, P, P, P, P,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_uint64, P]
            lib.oracle_rcp.restype = ctypes.c_int
            for f in (lib.oracle_bk, lib.oracle_bp):
                f.argtypes = [ctypes.c_int, P, ctypes.c_double, P, P, P, P, P]
                f.restype = ctypes.c_int
            lib.oracle_ldlt_solve.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P]
            lib.oracle_berr.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
            lib.oracle_berr.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def philox4x64_10(counter, key):
    """One Philox4x64-10 block for a 4-word counter and a 2-word key."""
    lib = _load()
    c = np.asarray(counter, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib.oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def omega(seed: int, d: int, n: int, stream: int = 0) -> np.ndarray:
    """The d x n Gaussian sketch matrix drawn by Algorithm 1 (Philox + Box-Muller)."""
    lib = _load()
    om = np.zeros((d, n), dtype=np.float64, order="F")
    lib.oracle_omega(ctypes.c_uint64(seed), ctypes.c_uint64(stream), d, n, _ptr(om))
    return om


def sketch(om: np.ndarray, a: np.ndarray) -> np.ndarray:
    """B = Omega A by a plain triple loop."""
    lib = _load()
    om = _f64(om)
    a = _f64(a)
    d, n = om.shape
    b = np.zeros((d, n), dtype=np.float64, order="F")
    lib.oracle_sketch(n, d, _ptr(om), _ptr(a), _ptr(b))
    return b


def rcp(a, om, alpha: float = SQRT2_OVER_2, q_mode: int = 1, block: int = 64,
        record: bool = True, snapshots: bool = False, guard_r: int = 0, guard_eps: float = 0.0,
        seed: int = 0) -> dict:
    """RCP factorization (Algorithm 1, eager Schur complement).

    ``q_mode=1``: one sketch pivot per step; ``q_mode=2``: q = b (partial QRCP per block of
    ``block`` columns and one block sketch update per block).
    Returns L, Dd, Ds, perm, info, the per-step record and rho_elem, n_2x2, min sketch-norm
    ratio and max|L| (``stats``).  ``snapshots`` (tiny n only) adds the sketch B and the
    Schur-complement array after every step.  ``guard_r`` > 0 adds the safeguard of
    Algorithm 2 (q = 1; recomputed sketches drawn with ``seed``, Philox streams 1, 2, ...);
    ``rank`` and ``resketches`` report where it stopped and how often it recomputed.
    """
    lib = _load()
    a = _f64(a).copy(order="F")
    om = _f64(om)
    n = a.shape[0]
    d = om.shape[0]
    L = np.zeros((n, n), dtype=np.float64, order="F")
    Dd = np.zeros(n)
    Ds = np.zeros(n)
    perm = np.zeros(n, dtype=np.int32)
    steps = (_Step * max(n, 1))()
    nsteps = ctypes.c_int(0)
    stats = np.zeros(4)
    gout = np.zeros(2, dtype=np.int32)
    sb = np.zeros((max(n, 1), d, n), dtype=np.float64) if snapshots else None
    sa = np.zeros((max(n, 1), n, n), dtype=np.float64) if snapshots else None
    sp = np.zeros((max(n, 1), n), dtype=np.int32) if snapshots else None
    info = lib.oracle_rcp(n, _ptr(a), d, _ptr(om), float(alpha), int(q_mode), int(block),
                          _ptr(L), _ptr(Dd), _ptr(Ds), _ptr(perm),
                          ctypes.cast(steps, ctypes.c_void_p), ctypes.byref(nsteps),
                          _ptr(sb) if snapshots else None, _ptr(sa) if snapshots else None,
                          _ptr(sp) if snapshots else None, _ptr(stats),
                          int(guard_r), float(guard_eps), ctypes.c_uint64(seed), _ptr(gout))
    out = dict(L=L, Dd=Dd, Ds=Ds, perm=perm.astype(np.int64), info=int(info),
               rho_elem=float(stats[0]), n_2x2=int(stats[1]), min_sketch_ratio=float(stats[2]),
               max_abs_L=float(stats[3]), rank=int(gout[0]), resketches=int(gout[1]))
    if record:
        out["steps"] = [dict(k=s.k, pi=s.pi, r=s.r, kase=s.kase, s=s.s, norm2=s.norm2, lam=s.lam,
                             norm2_next=s.norm2_next, lam_next=s.lam_next, akk=s.akk, arr=s.arr)
                        for s in steps[: nsteps.value]]
    if snapshots:
        # snapshot arrays are C-ordered stacks of column-major d x n and n x n matrices
        ns = nsteps.value
        out["snap_B"] = [np.asarray(sb[t]).reshape(n, d).T.copy() for t in range(ns)]
        out["snap_A"] = [np.asarray(sa[t]).reshape(n, n).T.copy() for t in range(ns)]
        out["snap_perm"] = [sp[t].astype(np.int64).copy() for t in range(ns)]
    return out


def _pivoted(fn, a, alpha):
    lib = _load()
    a = _f64(a).copy(order="F")
    n = a.shape[0]
    L = np.zeros((n, n), dtype=np.float64, order="F")
    Dd = np.zeros(n)
    Ds = np.zeros(n)
    perm = np.zeros(n, dtype=np.int32)
    stats = np.zeros(2)
    info = fn(n, _ptr(a), float(alpha), _ptr(L), _ptr(Dd), _ptr(Ds), _ptr(perm), _ptr(stats))
    return dict(L=L, Dd=Dd, Ds=Ds, perm=perm.astype(np.int64), info=int(info),
                rho_elem=float(stats[0]), n_2x2=int(stats[1]))


def bk(a, alpha: float = BK_ALPHA) -> dict:
    """Bunch-Kaufman partial pivoting (comparison method of Section 2.3)."""
    return _pivoted(_load().oracle_bk, a, alpha)


def bp(a, alpha: float = BK_ALPHA) -> dict:
    """Bunch-Parlett complete pivoting (comparison method; textbook rule)."""
    return _pivoted(_load().oracle_bp, a, alpha)


def ldlt_solve(L, Dd, Ds, perm, rhs) -> np.ndarray:
    """x = Pi L^{-T} D^+ L^{-1} Pi^T b for one or several right-hand sides (D^+: a zero 1x1 block
    contributes 0)."""
    lib = _load()
    L = _f64(L)
    n = L.shape[0]
    rhs = np.asarray(rhs, dtype=np.float64)
    vec = rhs.ndim == 1
    x = _f64(rhs.reshape(n, -1)).copy(order="F")
    p32 = np.ascontiguousarray(perm, dtype=np.int32)
    lib.oracle_ldlt_solve(n, x.shape[1], _ptr(L), _ptr(np.ascontiguousarray(Dd, dtype=np.float64)),
                          _ptr(np.ascontiguousarray(Ds, dtype=np.float64)), _ptr(p32), _ptr(x))
    return x[:, 0].copy() if vec else x


def berr(a, x, rhs) -> float:
    """||A x - b||_inf / (||A||_inf ||x||_inf), the largest over right-hand sides."""
    lib = _load()
    a = _f64(a)
    n = a.shape[0]
    x = _f64(np.asarray(x, dtype=np.float64).reshape(n, -1))
    rhs = _f64(np.asarray(rhs, dtype=np.float64).reshape(n, -1))
    return float(lib.oracle_berr(n, x.shape[1], _ptr(a), _ptr(x), _ptr(rhs)))


def l_norms(L) -> tuple:
    """||L||_1 and ||L^{-1}||_1 of a unit lower triangular L (the stability diagnostics the
    paper's experiments report beside the growth factor), by their definitions: the largest
    column sum of |L| and of |L^{-1}|, L^{-1} from forward substitution against the identity."""
    L = np.asarray(L, dtype=np.float64)
    n = L.shape[0]
    Li = np.eye(n)
    for i in range(n):
        Li[i] -= L[i, :i] @ Li[:i]
    return float(np.abs(L).sum(axis=0).max()), float(np.abs(Li).sum(axis=0).max())


def decision_margins(steps, alpha: float = SQRT2_OVER_2) -> list:
    """(position, margin) of every step of an ``rcp`` record: the closest relative margin of the
    step's decisions -- the gap between the two largest sketch norms, between the two largest
    |a_ik| (lambda), and between |a_kk| (|a_rr| in cases 2/3) and alpha lambda.  A computation that
    rounds differently can decide a step the other way only where its margin is of the order of
    its rounding error."""
    out = []
    for st in steps:
        m = []
        if st["norm2"] > 0 and st["norm2_next"] >= 0:
            m.append((st["norm2"] - st["norm2_next"]) / st["norm2"])
        lam = st["lam"]
        if lam > 0:
            if st["lam_next"] >= 0:
                m.append((lam - st["lam_next"]) / lam)
            m.append(abs(st["akk"] - alpha * lam) / (alpha * lam))
            if st["kase"] >= 2 and st["arr"] >= 0:
                m.append(abs(st["arr"] - alpha * lam) / (alpha * lam))
        out.append((st["k"], min(m) if m else float("inf")))
    return out


def block_d(Dd, Ds) -> np.ndarray:
    """The block-diagonal D as a dense matrix."""
    n = len(Dd)
    D = np.diag(np.asarray(Dd, dtype=np.float64))
    for i in range(n - 1):
        if Ds[i] != 0.0:
            D[i + 1, i] = D[i, i + 1] = Ds[i]
    return D


def growth_d(Dd, Ds, a) -> float:
    """rho = ||D||_{1,inf} / ||A||_{1,inf} (largest |entry| of D over that of A)."""
    dm = max(np.max(np.abs(Dd)), np.max(np.abs(Ds)) if len(Ds) else 0.0)
    am = np.max(np.abs(a))
    return float(dm / am) if am > 0 else 0.0


def p_bound(n: int, eps: float, delta: float) -> int:
    """Smallest integer p with p >= 4/(eps^2 - eps^3) ln(n(n+1)/delta) (Lemma, norm preservation)."""
    return int(math.ceil(4.0 / (eps * eps - eps ** 3) * math.log(n * (n + 1) / delta)))


def l_entry_bound(n: int, k: int, eps: float, alpha: float = SQRT2_OVER_2) -> float:
    """Upper bound on |l_ik| from the theorem on the entries of L (holds with prob. 1 - delta)."""
    return (1.0 + math.sqrt((1 + eps) / (1 - eps)) * math.sqrt(n - k + 1)) / min(alpha, 1 - alpha * alpha)


def rho_col_bound(n: int, eps: float) -> float:
    """Column growth bound of the theorem with alpha = sqrt(2)/2 (holds with prob. 1 - delta)."""
    e = 3.0 + math.log(n - 1)
    return math.sqrt(2 * (1 + eps) / (1 - eps)) ** e * math.sqrt(n + 2) ** (2.0 + math.log(n - 1))
