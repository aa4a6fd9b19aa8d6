"""Seeded synthetic inputs for RCP: the matrix families of the paper's experiments section.

This module holds no step of the factorization, the sketch or the solve; it only draws
matrices and right-hand sides.  The CPU oracle (via the tests) and the CUDA path both take
their inputs from here, so that they always see identical inputs.

Random numbers come from numpy's Philox bit generator keyed by ``(seed, stream)``; every
family uses its own stream id.  Dense linear algebra used to *assemble* a family (a transpose,
a Householder product, a Gram matrix) runs in FP64 with numpy, or with torch on ``device``
when one is given (the values then differ from numpy's only by rounding).  Matrices are
returned symmetric, so row- and column-major layouts coincide; right-hand sides are returned
as ``(nrhs, n)`` arrays, i.e. column-major ``n x nrhs``.

Families (the paper's numbering):
  type 1  Bunch-Kaufman worst-case growth       type 6  Gaussian, symmetrized (G + G^T)/2
  type 3  Hankel                                 type 7  KKT [[H, W], [W^T, 0]]
  type 4  discrete sine transform                type 8  augmented [[I, W], [W^T, 0]]
  type 5  discrete cosine transform              type 10 rank deficient W diag(lam) W^T
  plus ``spectrum``: Q diag(lam) Q^T with Q a product of Householder reflectors and
  |lam| log-uniform over ``10^[0, kexp]`` (random signs), for conditioned indefinite tests.
"""
from __future__ import annotations

import math

import numpy as np

STREAM_A = 1        # matrix entries
STREAM_X = 2        # x_true
STREAM_V = 3        # Householder vectors
STREAM_LAM = 4      # eigenvalues
STREAM_SIZES = 5    # batched sizes
STREAM_W = 6        # off-diagonal blocks


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def _out(a: np.ndarray, device):
    if device is None:
        return a
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def _sym_from_gaussian(g: np.ndarray, device):
    if device is None:
        return 0.5 * (g + g.T)
    import torch
    t = torch.from_numpy(g).to(device)
    return (t + t.T) * 0.5


def gaussian_sym(n: int, seed: int = 0, device=None):
    """Type 6 as used here: A = (G + G^T)/2 with G i.i.d. N(0, 1)."""
    g = rng(seed, STREAM_A).standard_normal((n, n))
    return _sym_from_gaussian(g, device)


def spectrum(n: int, seed: int = 0, kexp: float = 4.0, nrefl: int = 64, device=None):
    """A = Q diag(lam) Q^T, Q = H_1 ... H_nrefl (Householder, v ~ N(0,1)),
    lam_i = s_i 10^{u_i}, u_i ~ U(0, kexp), s_i = +-1 with probability 1/2."""
    r = rng(seed, STREAM_LAM)
    u = r.uniform(0.0, kexp, n)
    s = np.where(r.random(n) < 0.5, -1.0, 1.0)
    lam = s * 10.0 ** u
    vs = rng(seed, STREAM_V).standard_normal((nrefl, n))
    if device is None:
        m = np.diag(lam)
        for v in vs[::-1]:
            beta = 2.0 / float(v @ v)
            w = m @ v
            m = m - beta * np.outer(v, w) - beta * np.outer(w, v) + beta * beta * float(v @ w) * np.outer(v, v)
        return 0.5 * (m + m.T)
    import torch
    m = torch.diag(torch.from_numpy(lam).to(device))
    for v in vs[::-1]:
        vt = torch.from_numpy(v.copy()).to(device)
        beta = 2.0 / float(v @ v)
        w = m @ vt
        vw = float(vt @ w)
        m.addr_(vt, w, alpha=-beta)
        m.addr_(w, vt, alpha=-beta)
        m.addr_(vt, vt, alpha=beta * beta * vw)
    return (m + m.T) * 0.5


def kkt(n1: int, n2: int, m: int | None = None, seed: int = 0, device=None):
    """Type 7 as used here: [[H, W^T], [W, 0]], H = M M^T / m + 1e-3 I (M n1 x m),
    W n2 x n1, all entries N(0, 1)."""
    m = n1 if m is None else m
    M = rng(seed, STREAM_A).standard_normal((n1, m))
    W = rng(seed, STREAM_W).standard_normal((n2, n1))
    n = n1 + n2
    if device is None:
        a = np.zeros((n, n))
        a[:n1, :n1] = M @ M.T / m + 1e-3 * np.eye(n1)
        a[n1:, :n1] = W
        a[:n1, n1:] = W.T
        return a
    import torch
    Mt = torch.from_numpy(M).to(device)
    Wt = torch.from_numpy(W).to(device)
    a = torch.zeros((n, n), dtype=torch.float64, device=device)
    h = Mt @ Mt.T / m
    h.diagonal().add_(1e-3)
    a[:n1, :n1] = (h + h.T) * 0.5
    a[n1:, :n1] = Wt
    a[:n1, n1:] = Wt.T
    return a


def bk_worst(n: int, eps: float = 1e-3, tilt: float = 1e-10, device=None):
    """Type 1: [[A1, (1-eps) I], [(1-eps) I, 0]] with A1 of order m = n/2 holding
    d_k = (1 + tilt) q^{1-k}/(1-q), q = 1 + 1/alpha, alpha = (1+sqrt 17)/8 on its first m-2
    diagonal entries and ones in its last two rows and columns (entries that underflow are 0).

    With tilt = 0 the construction sits exactly on the Bunch-Kaufman case-(1) boundary
    |a_kk| = alpha*lambda, and rounding in the Schur complements tips the comparison the
    other way after a few steps (LAPACK ?sytrf then shows bounded growth too); the small
    relative tilt keeps the intended 1x1 choice under rounding."""
    assert n % 2 == 0 and n >= 6
    m = n // 2
    alpha = (1.0 + math.sqrt(17.0)) / 8.0
    q = 1.0 + 1.0 / alpha
    a1 = np.zeros((m, m))
    for k in range(1, m - 1):
        a1[k - 1, k - 1] = (1.0 + tilt) * q ** (1 - k) / (1 - q)
    a1[m - 2:, :] = 1.0
    a1[:, m - 2:] = 1.0
    a = np.zeros((n, n))
    a[:m, :m] = a1
    a[:m, m:] = (1 - eps) * np.eye(m)
    a[m:, :m] = (1 - eps) * np.eye(m)
    return _out(a, device)


def hankel(n: int, seed: int = 0, device=None):
    """Type 3: a_ij = h_{i+j}, h i.i.d. N(0, 1) (2n-1 values)."""
    h = rng(seed, STREAM_A).standard_normal(2 * n - 1)
    idx = np.add.outer(np.arange(n), np.arange(n))
    return _out(h[idx], device)


def dst(n: int, device=None):
    """Type 4: a_ij = sqrt(2/(n+1)) sin(i j pi/(n+1)), i, j = 1..n."""
    i = np.arange(1, n + 1)
    return _out(math.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * math.pi / (n + 1)), device)


def dct(n: int, device=None):
    """Type 5: a_ij = cos((i-1)(j-1) pi/(n-1)), i, j = 1..n."""
    i = np.arange(n)
    return _out(np.cos(np.outer(i, i) * math.pi / (n - 1)), device)


def augmented(n1: int, n2: int, seed: int = 0, device=None):
    """Type 8: [[I, W], [W^T, 0]], W n1 x n2 i.i.d. N(0, 1)."""
    W = rng(seed, STREAM_W).standard_normal((n1, n2))
    n = n1 + n2
    a = np.zeros((n, n))
    a[:n1, :n1] = np.eye(n1)
    a[:n1, n1:] = W
    a[n1:, :n1] = W.T
    return _out(a, device)


def rank_deficient(n: int, seed: int = 0, device=None):
    """Type 10: W diag(lam) W^T with lam_i = q^{1-i}/(1-q), q = 1 + sqrt 2."""
    W = rng(seed, STREAM_W).standard_normal((n, n))
    q = 1.0 + math.sqrt(2.0)
    lam = np.array([q ** (1 - i) / (1 - q) for i in range(1, n + 1)])
    a = (W * lam) @ W.T
    return _out(0.5 * (a + a.T), device)


def x_true(n: int, nrhs: int = 1, seed: int = 0, device=None):
    """x_true ~ N(0, 1) as an (nrhs, n) array (column-major n x nrhs)."""
    return _out(rng(seed, STREAM_X).standard_normal((nrhs, n)), device)


def rhs_for(a, x):
    """b = A x_true in FP64; ``x`` and the result are (nrhs, n) arrays."""
    if isinstance(a, np.ndarray):
        return (a @ x.T).T.copy()
    return (a @ x.T).T.contiguous()


def batched_sizes(batch: int, lo: int = 32, hi: int = 512, seed: int = 0) -> np.ndarray:
    """Ragged orders n_i ~ U{lo..hi}."""
    return rng(seed, STREAM_SIZES).integers(lo, hi + 1, size=batch)


def batched_gaussian(sizes, seed: int = 0):
    """A_i = (G_i + G_i^T)/2 for every order in ``sizes`` (system i uses seed + i)."""
    return [gaussian_sym(int(n), seed=seed * 1000003 + i) for i, n in enumerate(sizes)]


def fill_batched_gaussian_device(sizes, offsets, pool, seed: int = 0) -> None:
    """Type 6 for a whole ragged batch, drawn on the device (for workloads too large to draw
    with numpy quickly): system i, of order sizes[i], gets A_i = (G_i + G_i^T)/2 written
    column-major at ``pool[offsets[i]:offsets[i] + n_i^2]`` (FP64).  G comes from torch's
    device generator seeded with ``seed``, drawn group by group of equal order (increasing
    order), so the values are reproducible on one device type but differ from
    ``batched_gaussian``'s numpy draws."""
    import torch
    g = torch.Generator(device=pool.device)
    g.manual_seed(int(seed))
    by_n = {}
    for i, n in enumerate(sizes):
        by_n.setdefault(int(n), []).append(i)
    for n in sorted(by_n):
        idx = by_n[n]
        if n == 0:
            continue
        G = torch.randn((len(idx), n, n), generator=g, device=pool.device, dtype=torch.float64)
        A = (G + G.transpose(1, 2)) * 0.5
        for j, i in enumerate(idx):
            pool[offsets[i]:offsets[i] + n * n].copy_(A[j].reshape(-1))


def fill_batched_rhs_device(sizes, offsets_sq, a_pool, offsets_rhs, b_pool, nrhs: int, seed: int = 0,
                            x_pool=None) -> None:
    """Right-hand sides b_i = A_i x_i with x_i i.i.d. N(0, 1) (nrhs columns, column-major
    ``n_i x nrhs`` at ``b_pool[offsets_rhs[i]:]``), drawn on the device; x_i is kept in
    ``x_pool`` when given."""
    import torch
    g = torch.Generator(device=a_pool.device)
    g.manual_seed(int(seed) + 1)
    for i, n in enumerate(sizes):
        n = int(n)
        if n == 0:
            continue
        A = a_pool[offsets_sq[i]:offsets_sq[i] + n * n].view(n, n)     # symmetric
        X = torch.randn((nrhs, n), generator=g, device=a_pool.device, dtype=torch.float64)
        b_pool[offsets_rhs[i]:offsets_rhs[i] + n * nrhs].view(nrhs, n).copy_(X @ A)
        if x_pool is not None:
            x_pool[offsets_rhs[i]:offsets_rhs[i] + n * nrhs].view(nrhs, n).copy_(X)
