"""GPU path vs the CPU oracle, through the C ABI.  Inputs come from the shared seeded
generators; expected values only from ``oracle``."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1710_00125_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def rcp():
    from paper_1710_00125_gb300 import rcp as r
    return r


@pytest.fixture(scope="module")
def handle(rcp):
    return rcp.rcp_create()


def _factor(rcp, handle, a, b, d, seed, prec="fp64", grid=0, q_mode=1):
    n = a.shape[0]
    dt = torch.float64 if prec == "fp64" else torch.float32
    A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dt)
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros(n, dtype=torch.float64, device=DEV)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=b, d=d, seed=seed, prec=prec, grid=grid,
                                                                      q_mode=q_mode))
    return code, st, A, Dd, Ds, perm


def _unit_lower(A):
    n = A.shape[0]
    return np.tril(A.cpu().double().numpy().T, -1) + np.eye(n)


# ------------------------------------------------------------------------------------------
# Omega and the sketch
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,seed", [(1, 5, 0), (7, 33, 1), (40, 256, 0), (80, 1000, 12345)])
def test_omega_matches_oracle(rcp, d, n, seed):
    got = rcp.rcp_omega(d, n, seed).cpu().numpy()
    ref = oracle.omega(seed, d, n)
    # same Philox words; Box-Muller through CUDA's and the C library's log/sin/cos
    assert np.allclose(got, ref, rtol=4e-15, atol=4e-15)


@pytest.mark.parametrize("n,d", [(1, 3), (63, 5), (130, 40), (257, 80),
                                 (2600, 80), (2048, 128)])   # the last two: the FP32 sketch in K slices
def test_sketch_matches_oracle(rcp, n, d):
    a = inputs.gaussian_sym(n, seed=n)
    A = torch.from_numpy(a).to(DEV)
    got = rcp.rcp_sketch(A, d, seed=9).cpu().numpy()
    om = oracle.omega(9, d, n)
    ref = oracle.sketch(om, a)
    scale = np.abs(om).max() * np.abs(a).max() * n
    assert np.max(np.abs(got - ref)) <= 1e-14 * scale
    got32 = rcp.rcp_sketch(A.float(), d, seed=9, prec="fp32").cpu().double().numpy()
    assert np.max(np.abs(got32 - ref)) <= 2e-6 * scale
    # tcgen05 with split TF32 operands (the sketch of the tensor-core precisions)
    for prec in ("tf32x3", "f16x3"):
        gtc = rcp.rcp_sketch(A.float(), d, seed=9, prec=prec).cpu().double().numpy()
        assert np.max(np.abs(gtc - ref)) <= 2e-6 * scale


@pytest.mark.parametrize("n,d", [(128, 16), (129, 1), (1000, 33), (4097, 80), (6144, 128)])
def test_tensor_core_sketch_entrywise(rcp, n, d):
    # every entry against the oracle's FP64 sketch of the FP32-rounded matrix, within a bound
    # of the split's rounding: |B_ij - B*_ij| <= 2^-20 sum_k |Omega_ik| |A_kj| + FP32 summation
    a = inputs.gaussian_sym(n, seed=n + 1)
    a32 = a.astype(np.float32).astype(np.float64)
    A = torch.from_numpy(a32).to(DEV).float()
    om = oracle.omega(5, d, n)
    om32 = om.astype(np.float32).astype(np.float64)
    ref = oracle.sketch(om32, a32)
    got = rcp.rcp_sketch(A, d, seed=5, prec="tf32x3").cpu().double().numpy()
    mag = np.abs(om32) @ np.abs(a32)
    bound = (2.0 ** -20 + 2.0 * n * 2.0 ** -24) * mag + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


# ------------------------------------------------------------------------------------------
# FP64 factorization: the same pivot sequence as the oracle
# ------------------------------------------------------------------------------------------

CASES = [
    (1, 8, 3, 0), (2, 8, 3, 1), (3, 8, 4, 2), (37, 8, 6, 3), (100, 8, 12, 4),     # many panels, ragged
    (256, 32, 40, 0),                                                               # the n = 256 workload
    (300, 32, 40, 5), (513, 64, 80, 6),                                             # ragged tails
]


@pytest.mark.parametrize("n,b,d,seed", CASES)
def test_fp64_factor_matches_oracle(rcp, handle, n, b, d, seed):
    a = inputs.gaussian_sym(n, seed=seed)
    ref = oracle.rcp(a, oracle.omega(seed, d, n), record=False)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, b, d, seed)
    assert code == 0
    assert np.array_equal(perm.cpu().numpy(), ref["perm"])
    ds = Ds.cpu().numpy()
    assert np.array_equal(ds != 0, ref["Ds"] != 0)
    scale = np.abs(a).max()
    assert np.allclose(Dd.cpu().numpy(), ref["Dd"], rtol=0, atol=1e-11 * scale * max(1, n / 64))
    assert np.allclose(ds, ref["Ds"], rtol=0, atol=1e-11 * scale * max(1, n / 64))
    L = _unit_lower(A)
    assert np.allclose(L, ref["L"], rtol=0, atol=1e-10 * max(1, n / 64))
    assert st.n_2x2 == ref["n_2x2"]
    assert st.growth_D == pytest.approx(oracle.growth_d(ref["Dd"], ref["Ds"], a), rel=1e-10)
    assert st.max_abs_L == pytest.approx(ref["max_abs_L"], rel=1e-9)


@pytest.mark.parametrize("grid", [1, 3, 16])
def test_fp64_factor_any_grid(rcp, handle, grid):
    # the result must not depend on how the indices are split over CTAs
    n, b, d, seed = 150, 16, 20, 8
    a = inputs.gaussian_sym(n, seed=seed)
    ref = oracle.rcp(a, oracle.omega(seed, d, n), record=False)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, b, d, seed, grid=grid)
    assert code == 0
    assert np.array_equal(perm.cpu().numpy(), ref["perm"])


@pytest.mark.parametrize("name", ["bk_worst", "kkt", "dst", "dct", "hankel", "augmented", "spectrum"])
def test_fp64_structured_families(rcp, handle, name):
    n = 64
    a = {"bk_worst": lambda: inputs.bk_worst(n), "kkt": lambda: inputs.kkt(40, 24, seed=1),
         "dst": lambda: inputs.dst(n), "dct": lambda: inputs.dct(n), "hankel": lambda: inputs.hankel(n, 2),
         "augmented": lambda: inputs.augmented(40, 24, 3), "spectrum": lambda: inputs.spectrum(n, 4, 4.0, 8)}[name]()
    d = 12
    ref = oracle.rcp(a, oracle.omega(2, d, n), record=False)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 16, d, 2)
    assert code == ref["info"]
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    L = _unit_lower(A)
    p = perm.cpu().numpy()
    recon = np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max()
    assert recon < 1e-12
    # growth within 1% of the oracle's (its pivot order may differ on exact ties)
    assert st.growth_D == pytest.approx(oracle.growth_d(ref["Dd"], ref["Ds"], a), rel=0.01)
    if name in ("bk_worst", "spectrum", "hankel"):
        assert np.array_equal(p, ref["perm"])


def test_empty_system(rcp, handle):
    # n = 0: nothing to factor, solve or refine; every call succeeds without launching work
    e = torch.empty((0, 0), dtype=torch.float64, device=DEV)
    v = torch.empty(0, dtype=torch.float64, device=DEV)
    p = torch.empty(0, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, e, v, v, p, rcp.make_opts(b=64, d=80, prec="fp64"))
    assert code == 0 and st.info == 0
    rcp.rcp_solve(handle, e, v, v, p, "fp64", torch.empty((1, 0), dtype=torch.float64, device=DEV))
    code, st = rcp.rcp_sysv(handle, e, torch.empty((1, 0), dtype=torch.float64, device=DEV),
                            torch.empty((1, 0), dtype=torch.float64, device=DEV), rcp.make_opts(prec="f16x3"))
    assert code == 0


def test_degenerate_inputs(rcp, handle):
    # zero matrix: every pivot is a zero 1x1 (SBKP case 0); info reports the first
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, np.zeros((5, 5)), 4, 3, 0)
    assert code == 1 and st.info == 1
    assert np.all(Dd.cpu().numpy() == 0)
    # [[0, 1], [1, 0]] needs a 2x2 pivot
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, np.array([[0.0, 1.0], [1.0, 0.0]]), 4, 3, 0)
    assert code == 0 and st.n_2x2 == 1 and Ds.cpu().numpy()[0] == 1.0
    # NaN input is reported, never trapped
    a = inputs.gaussian_sym(20, 1)
    a[3, 3] = np.nan
    code = None
    try:
        code, st, *_ = _factor(rcp, handle, a, 8, 4, 0)
    except rcp.RcpError as e:
        code = e.code
    assert code == -4
    # the handle stays usable afterwards
    a = inputs.gaussian_sym(20, 1)
    code, st, *_ = _factor(rcp, handle, a, 8, 4, 0)
    assert code == 0


def test_invalid_arguments(rcp, handle):
    lib = rcp.lib()
    assert lib.rcp_factor(handle.h, -1, None, 1, None, None, None, None, None, None) == -1
    assert lib.rcp_solve(handle.h, 4, 1, None, 4, None, None, None, 0, None, 4, None) == -1


# ------------------------------------------------------------------------------------------
# Solve and refinement
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,nrhs", [(1, 1), (65, 3), (256, 1), (300, 32)])
def test_solve_with_oracle_factor(rcp, handle, n, nrhs):
    # feed the oracle's factorization to the GPU solve and compare with the oracle's solve
    a = inputs.gaussian_sym(n, seed=n)
    ref = oracle.rcp(a, oracle.omega(1, 10, n), record=False)
    LA = torch.from_numpy(np.ascontiguousarray(ref["L"].T)).to(DEV)   # column-major L
    Dd = torch.from_numpy(ref["Dd"]).to(DEV)
    Ds = torch.from_numpy(ref["Ds"]).to(DEV)
    perm = torch.from_numpy(ref["perm"].astype(np.int32)).to(DEV)
    rhs = inputs.x_true(n, nrhs, seed=3)
    X = torch.from_numpy(rhs.copy()).to(DEV)
    rcp.rcp_solve(handle, LA, Dd, Ds, perm, "fp64", X)
    want = oracle.ldlt_solve(ref["L"], ref["Dd"], ref["Ds"], ref["perm"], rhs.T).T
    cond = np.linalg.cond(a)
    assert np.allclose(X.cpu().numpy(), want, rtol=0, atol=1e-13 * cond * np.abs(want).max())


def test_fp64_solve_backward_error(rcp, handle):
    n = 256
    a = inputs.gaussian_sym(n, seed=0)
    x = inputs.x_true(n, 1, seed=0)
    rhs = inputs.rhs_for(a, x)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 32, 40, 0)
    X = torch.from_numpy(rhs.copy()).to(DEV)
    rcp.rcp_solve(handle, A, Dd, Ds, perm, "fp64", X)
    be = oracle.berr(a, X.cpu().numpy().T, rhs.T)
    ref = oracle.rcp(a, oracle.omega(0, 40, n), record=False)
    be_ref = oracle.berr(a, oracle.ldlt_solve(ref["L"], ref["Dd"], ref["Ds"], ref["perm"], rhs.T), rhs.T)
    assert be <= max(1e-15, 10 * be_ref)


@pytest.mark.parametrize("prec", ["fp32"])
@pytest.mark.parametrize("kexp", [2.0, 4.0, 6.0])
def test_mixed_refine_reaches_fp64_backward_error(rcp, handle, prec, kexp):
    n = 384
    a = inputs.spectrum(n, seed=7, kexp=kexp, nrefl=16)
    x = inputs.x_true(n, 2, seed=7)
    rhs = inputs.rhs_for(a, x)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 32, 48, 1, prec=prec)
    assert code == 0
    A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Bv = torch.from_numpy(rhs.copy()).to(DEV)
    X = torch.zeros_like(Bv)
    code, rst = rcp.rcp_refine(handle, A64, A, Dd, Ds, perm, prec, Bv, X, tol=1e-12, max_iter=30)
    assert code == 0, rst.as_dict()
    xs = X.cpu().numpy()
    be = oracle.berr(a, xs.T, rhs.T)
    assert be <= 1e-12 and rst.berr <= 1e-12
    assert be == pytest.approx(rst.berr, rel=0.5, abs=1e-16)
    cond = np.linalg.cond(a)
    assert np.abs(xs - x).max() / np.abs(x).max() <= 50 * cond * 1e-12


@pytest.mark.parametrize("n,d,precs", [(200, 40, ("fp64", "fp32")),
                                        # several host copy blocks and K slices of the sketch: the
                                        # overlapped block-by-block path must give the same bits
                                        (700, 40, ("fp32", "f16x3")),
                                        # the tensor-core sketch in two K slices over 11 copy blocks
                                        (2600, 80, ("tf32x3", "f16x3"))])
def test_sysv_device_and_host_buffers(rcp, handle, n, d, precs):
    a = inputs.gaussian_sym(n, seed=11)
    x = inputs.x_true(n, 4, seed=11)
    rhs = inputs.rhs_for(a, x)
    for prec in precs:
        A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
        Bv = torch.from_numpy(rhs.copy()).to(DEV)
        X = torch.zeros_like(Bv)
        code, st = rcp.rcp_sysv(handle, A64, Bv, X, rcp.make_opts(b=32, d=d, prec=prec), tol=1e-12, max_iter=10)
        assert code == 0
        assert oracle.berr(a, X.cpu().numpy().T, rhs.T) <= 1e-12
        Ah = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        Bh = torch.from_numpy(rhs.copy()).pin_memory()
        Xh = torch.zeros_like(Bh).pin_memory()
        code, st2 = rcp.rcp_sysv(handle, Ah, Bh, Xh, rcp.make_opts(b=32, d=d, prec=prec), tol=1e-12, max_iter=10,
                                 host_buffers=True)
        assert code == 0
        assert np.array_equal(Xh.numpy(), X.cpu().numpy())


# ------------------------------------------------------------------------------------------
# FP32 factors: SIMT and tensor-core (tcgen05, split TF32 or scaled split FP16) trailing updates
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "f16x3"])
@pytest.mark.parametrize("n,b,d", [(300, 32, 40), (777, 64, 80), (1500, 128, 80)])
def test_fp32_factor_backward_error(rcp, handle, prec, n, b, d):
    # ||P A P^T - L D L^T||_max / ||A||_max computed in FP64 from the FP32 factor: a wrong
    # tile, swizzle or descriptor in the update makes this O(1)
    a = inputs.gaussian_sym(n, seed=n + b)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, b, d, 3, prec=prec)
    assert code == 0
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert sorted(p.tolist()) == list(range(n))
    err = np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max()
    assert err < 2e-5 * max(1.0, st.growth_D), err
    # the FP32 pivot sequence stays close to the oracle's FP64 one: same 2x2 count within 5%
    ref = oracle.rcp(a, oracle.omega(3, d, n), record=False)
    assert abs(st.n_2x2 - ref["n_2x2"]) <= max(3, 0.05 * ref["n_2x2"])


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
@pytest.mark.parametrize("n,grid", [(2000, 8), (1040, 4), (1200, 4)])
def test_fp32_panel_many_rows_per_cta(rcp, handle, prec, n, grid):
    # 250, 260 and 300 rows per CTA: the fused panel step makes 2, 3 and 3 passes of 128 rows (the
    # last with too little shared memory for the speculation's shadow sketch: the plain step)
    a = inputs.gaussian_sym(n, seed=n + grid)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 64, 40, 5, prec=prec, grid=grid)
    assert code == 0
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert sorted(p.tolist()) == list(range(n))
    err = np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max()
    assert err < 2e-5 * max(1.0, st.growth_D), err
    # the same factorization on the default grid: the pivot choices agree up to FP32 near-ties
    code2, st2, A2, _, _, perm2 = _factor(rcp, handle, a, 64, 40, 5, prec=prec)
    assert code2 == 0
    assert abs(st.n_2x2 - st2.n_2x2) <= max(3, 0.05 * st2.n_2x2)


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
@pytest.mark.parametrize("n,grid", [(1000, 0), (2000, 8), (1200, 4)])
def test_speculation_modes_give_identical_factors(rcp, prec, n, grid):
    # The FP32 panel's ways of preparing the next pivot step while it waits at a step's grid
    # barrier (a shadow copy of the sketch columns, the confirmed sketch update deferred to the next
    # step's pass, or no speculation) apply the same operations to every value: the pivot sequence,
    # D and L agree bit for bit.  300 rows per CTA (n = 1200 on 4 CTAs): the shadow copy does not
    # fit and is refused.
    a = inputs.gaussian_sym(n, seed=77 + n)
    h = rcp.rcp_create()
    got = {}
    for mode in (1, 2, 0, -1):
        rcp.rcp_set_speculation(h, mode)
        if mode == 1 and n == 1200:
            with pytest.raises(rcp.RcpError):
                _factor(rcp, h, a, 64, 40, 5, prec=prec, grid=grid)
            continue
        code, st, A, Dd, Ds, perm = _factor(rcp, h, a, 64, 40, 5, prec=prec, grid=grid)
        assert code == 0
        got[mode] = (perm.cpu().numpy(), Dd.cpu().numpy(), Ds.cpu().numpy(), A.cpu().numpy(), st.n_2x2)
    rcp.rcp_set_speculation(h, -1)
    ref = got[0]
    for mode, r in got.items():
        assert np.array_equal(r[0], ref[0]), mode
        for x, y in zip(r[1:4], ref[1:4]):
            assert np.array_equal(x, y), mode
        assert r[4] == ref[4]
    with pytest.raises(rcp.RcpError):
        rcp.rcp_set_speculation(h, 3)


@pytest.mark.parametrize("prec", ["tf32x3", "f16x3"])
@pytest.mark.parametrize("kexp", [2.0, 4.0, 6.0])
def test_tf32x3_refine_reaches_fp64_backward_error(rcp, handle, kexp, prec):
    n = 1024
    a = inputs.spectrum(n, seed=9, kexp=kexp, nrefl=16)
    x = inputs.x_true(n, 1, seed=9)
    rhs = inputs.rhs_for(a, x)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 128, 80, 2, prec=prec)
    assert code == 0
    A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Bv = torch.from_numpy(rhs.copy()).to(DEV)
    X = torch.zeros_like(Bv)
    code, rst = rcp.rcp_refine(handle, A64, A, Dd, Ds, perm, prec, Bv, X, tol=1e-12, max_iter=30)
    assert code == 0, rst.as_dict()
    assert oracle.berr(a, X.cpu().numpy().T, rhs.T) <= 1e-12
    assert rst.refine_iters <= 6


@pytest.mark.parametrize("scale", [1e-15, 1e15])
def test_f16x3_scaled_matrix(rcp, handle, scale):
    # the FP16 parts are formed after a power-of-two scaling by the panel maxima: matrices near
    # either end of the FP32 range (short of overflowing the FP32 sketch norms) factor to the same
    # relative accuracy as the TF32 split
    n, b, d = 777, 64, 80
    a = inputs.gaussian_sym(n, seed=11) * scale
    errs = {}
    for prec in ("tf32x3", "f16x3"):
        code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, b, d, 3, prec=prec)
        assert code == 0
        L = _unit_lower(A)
        D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
        p = perm.cpu().numpy()
        errs[prec] = np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max()
        assert errs[prec] < 2e-5 * max(1.0, st.growth_D), (prec, errs[prec])
    assert errs["f16x3"] < 8 * errs["tf32x3"] + 1e-7, errs


# ------------------------------------------------------------------------------------------
# q = b: block QRCP candidates, block sketch update (Section 3.1)
# ------------------------------------------------------------------------------------------

QB_CASES = [
    (37, 8, 12, 3), (100, 16, 20, 4),   # many blocks, ragged tails
    (256, 32, 40, 0),                  # the n = 256 workload with q = b
    (300, 32, 12, 5),                  # b > d: the QRCP ranks only d candidates per block
]


@pytest.mark.parametrize("n,b,d,seed", QB_CASES)
def test_fp64_qb_factor_matches_oracle(rcp, handle, n, b, d, seed):
    a = inputs.gaussian_sym(n, seed=seed)
    ref = oracle.rcp(a, oracle.omega(seed, d, n), q_mode=2, block=b, record=False)
    A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros(n, dtype=torch.float64, device=DEV)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=b, d=d, seed=seed, prec="fp64", q_mode=2))
    assert code == ref["info"]
    assert np.array_equal(perm.cpu().numpy(), ref["perm"])
    ds = Ds.cpu().numpy()
    assert np.array_equal(ds != 0, ref["Ds"] != 0)
    scale = np.abs(a).max()
    assert np.allclose(Dd.cpu().numpy(), ref["Dd"], rtol=0, atol=1e-11 * scale * max(1, n / 64))
    assert np.allclose(ds, ref["Ds"], rtol=0, atol=1e-11 * scale * max(1, n / 64))
    assert np.allclose(_unit_lower(A), ref["L"], rtol=0, atol=1e-10 * max(1, n / 64))
    assert st.n_2x2 == ref["n_2x2"]


def test_qb_differs_from_q1(rcp, handle):
    # the two modes pick different pivot sequences on the same input (the mode is really used)
    n, b, d, seed = 200, 16, 24, 7
    a = inputs.gaussian_sym(n, seed=seed)
    om = oracle.omega(seed, d, n)
    r1 = oracle.rcp(a, om, q_mode=1, record=False)
    r2 = oracle.rcp(a, om, q_mode=2, block=b, record=False)
    assert not np.array_equal(r1["perm"], r2["perm"])
    A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=b, d=d, seed=seed, prec="fp64", q_mode=2))
    assert np.array_equal(perm.cpu().numpy(), r2["perm"])


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "f16x3"])
def test_qb_mixed_refine_reaches_fp64_backward_error(rcp, handle, prec):
    n = 1000
    a = inputs.spectrum(n, seed=5, kexp=4.0, nrefl=16)
    x = inputs.x_true(n, 1, seed=5)
    rhs = inputs.rhs_for(a, x)
    A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV).float()
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=64, d=80, seed=1, prec=prec, q_mode=2))
    assert code == 0
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max() < 2e-5 * max(1.0, st.growth_D)
    A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Bv = torch.from_numpy(rhs.copy()).to(DEV)
    X = torch.zeros_like(Bv)
    code, rst = rcp.rcp_refine(handle, A64, A, Dd, Ds, perm, prec, Bv, X, tol=1e-12, max_iter=30)
    assert code == 0, rst.as_dict()
    assert oracle.berr(a, X.cpu().numpy().T, rhs.T) <= 1e-12


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "f16x3"])
@pytest.mark.parametrize("n", [300, 1000])
def test_qb_mixed_gaussian_ragged_blocks(rcp, handle, prec, n):
    # (G + G^T)/2: many 2x2 pivots, blocks of b and b + 1 columns and a ragged last block, with a
    # block QRCP (its own grid barriers) between consecutive panels
    a = inputs.gaussian_sym(n, seed=0)
    ref = oracle.rcp(a, oracle.omega(1, 80, n), q_mode=2, block=64, record=False)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 64, 80, 1, prec=prec, q_mode=2)
    assert code == 0
    assert torch.equal(torch.sort(perm.long())[0], torch.arange(n, device=DEV))
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max() < 2e-5 * max(1.0, st.growth_D)
    # FP32 decisions may part from the FP64 pivot sequence at near ties, not the growth's scale
    assert st.growth_D <= 3.0 * oracle.growth_d(ref["Dd"], ref["Ds"], a)
    assert abs(st.n_2x2 - ref["n_2x2"]) <= 0.1 * ref["n_2x2"] + 3


# ------------------------------------------------------------------------------------------
# Algorithm 2 (safeguard)
# ------------------------------------------------------------------------------------------

def _exact_rank_matrix(n, rho, seed):
    rng = np.random.default_rng(seed)
    V = rng.integers(-3, 4, size=(n, rho)).astype(np.float64)
    return V @ np.diag(rng.choice([-1.0, 1.0], size=rho)) @ V.T


def _guarded(rcp, handle, a, b, d, seed, prec, r, eps):
    n = a.shape[0]
    dt = torch.float64 if prec == "fp64" else torch.float32
    A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dt)
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, A, Dd, Ds, perm,
                              rcp.make_opts(b=b, d=d, seed=seed, prec=prec, guard_r=r, guard_eps=eps))
    return code, st, A, Dd, Ds, perm


@pytest.mark.parametrize("n,rho,b", [(300, 40, 64), (400, 150, 64)])
def test_guard_fp64_stops_at_the_rank_like_the_oracle(rcp, handle, n, rho, b):
    a = _exact_rank_matrix(n, rho, n + rho)
    ref = oracle.rcp(a, oracle.omega(7, 40, n), record=False, guard_r=1, guard_eps=1e-8, seed=7)
    assert ref["rank"] == rho
    code, st, A, Dd, Ds, perm = _guarded(rcp, handle, a, b, 40, 7, "fp64", 1, 1e-8)
    assert code == rho + 1 and st.info == rho + 1
    assert st.rank == rho and st.resketches == 0
    p = perm.cpu().numpy()
    assert np.array_equal(p[:rho], ref["perm"][:rho])
    assert sorted(p.tolist()) == list(range(n))
    L = _unit_lower(A)
    # the eliminated columns of L and D agree with the oracle's; rows are matched by original
    # index (the order of the tail, the zero Schur complement, may differ)
    rows = {int(v): i for i, v in enumerate(ref["perm"])}
    Lr = ref["L"][[rows[int(v)] for v in p], :rho]
    assert np.abs(L[:, :rho] - Lr).max() <= 1e-10
    assert np.allclose(Dd.cpu().numpy()[:rho], ref["Dd"][:rho], rtol=1e-11, atol=1e-11 * np.abs(a).max())
    assert np.all(Dd.cpu().numpy()[rho:] == 0.0) and np.all(Ds.cpu().numpy()[rho:] == 0.0)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() <= 1e-12 * np.abs(a).max()


def test_guard_fp64_recomputes_the_sketch_like_the_oracle(rcp, handle):
    # full rank, 80 of 200 eigenvalues near 1e-6: sqrt(eps) beta flags the small block, the
    # recomputed sketch passes eps beta (r = 2, eps = 1e-10)
    n, d = 200, 40
    rng = np.random.default_rng(8)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(1, 2, 120) * rng.choice([-1, 1], 120), 1e-6 * rng.uniform(1, 2, 80)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    ref = oracle.rcp(a, oracle.omega(5, d, n), record=False, guard_r=2, guard_eps=1e-10, seed=5)
    assert ref["resketches"] == 1 and ref["rank"] == n
    code, st, A, Dd, Ds, perm = _guarded(rcp, handle, a, 64, d, 5, "fp64", 2, 1e-10)
    assert code == 0 and st.resketches == 1 and st.rank == n
    p = perm.cpu().numpy()
    # the whole pivot sequence, including the steps that follow the recomputed sketch (Omega'
    # drawn from Philox stream 1 on both sides, then a fresh argmax)
    assert np.array_equal(p, ref["perm"])
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_guard_fp32_recomputes_the_sketch(rcp, handle, prec):
    # the FP32 re-sketch of the trailing submatrix (split-K sketch at an offset): 500 of 1200
    # eigenvalues near 1e-3, well above the FP32 rounding level of the Schur complement (~1e-5),
    # are flagged by sqrt(eps) beta = 1e-2 beta and accepted against eps beta after one recomputation
    n, d = 1200, 80
    rng = np.random.default_rng(9)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(1, 2, 700) * rng.choice([-1, 1], 700), 1e-3 * rng.uniform(1, 2, 500)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    code, st, A, Dd, Ds, perm = _guarded(rcp, handle, a, 64, d, 5, prec, 2, 1e-4)
    assert code == 0 and st.resketches == 1 and st.rank == n
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert sorted(p.tolist()) == list(range(n))
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() <= 2e-5 * max(1.0, st.growth_D) * np.abs(a).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_guard_that_never_fires_changes_nothing_on_the_gpu(rcp, handle, prec):
    a = inputs.gaussian_sym(300, seed=4)
    c0, s0, A0, Dd0, Ds0, p0 = _guarded(rcp, handle, a, 64, 40, 3, prec, 0, 0.0)
    c1, s1, A1, Dd1, Ds1, p1 = _guarded(rcp, handle, a, 64, 40, 3, prec, 3, 1e-300)
    assert c0 == c1 == 0 and s1.rank == 300 and s1.resketches == 0
    assert torch.equal(p0, p1) and torch.equal(A0, A1) and torch.equal(Dd0, Dd1)


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_guard_fp32_stops_at_the_rank(rcp, handle, prec):
    n, rho = 500, 40
    a = _exact_rank_matrix(n, rho, 11)
    code, st, A, Dd, Ds, perm = _guarded(rcp, handle, a, 64, 80, 2, prec, 1, 1e-4)
    assert st.rank == rho and code == rho + 1
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() <= 1e-5 * max(1.0, st.growth_D) * np.abs(a).max()


def test_guard_sysv_basic_solution_of_a_consistent_rank_deficient_system(rcp, handle):
    n, rho = 400, 60
    a = _exact_rank_matrix(n, rho, 12)
    x = inputs.x_true(n, 1, seed=12)
    rhs = inputs.rhs_for(a, x)
    A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Bv = torch.from_numpy(rhs.copy()).to(DEV)
    X = torch.zeros_like(Bv)
    code, st = rcp.rcp_sysv(handle, A64, Bv, X, rcp.make_opts(b=64, d=80, seed=3, prec="fp64", guard_r=1,
                                                              guard_eps=1e-8), tol=1e-12, max_iter=5)
    assert st.rank == rho and code == rho + 1   # info > 0: D is singular, x is the basic solution
    assert np.all(np.isfinite(X.cpu().numpy()))
    assert oracle.berr(a, X.cpu().numpy().T, rhs.T) <= 1e-12


def test_guard_option_checks(rcp, handle):
    a = inputs.gaussian_sym(100, seed=1)
    with pytest.raises(rcp.RcpError):
        A = torch.from_numpy(a).to(DEV)
        rcp.rcp_factor(handle, A, torch.zeros(100, dtype=torch.float64, device=DEV),
                       torch.zeros(100, dtype=torch.float64, device=DEV), torch.zeros(100, dtype=torch.int32, device=DEV),
                       rcp.make_opts(b=32, d=40, prec="fp64", q_mode=2, guard_r=1))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_l_norms_of_a_factor(rcp, handle, prec):
    n = 500
    a = inputs.gaussian_sym(n, seed=21)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 64, 40, 3, prec=prec)
    assert code == 0
    nl, ni = rcp.rcp_l_norms(handle, A, prec)
    L = _unit_lower(A)   # the factor's own values, in FP64
    el, ei = oracle.l_norms(L)
    assert nl == pytest.approx(el, rel=1e-12)
    # Higham's estimate: a lower bound (up to the solve's rounding), and close on random factors
    assert ei * 0.3 <= ni <= ei * (1 + (1e-10 if prec == "fp64" else 1e-4))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_l_norms_closed_form(rcp, handle, prec):
    # L = I - subdiagonal: ||L||_1 = 2 and ||L^{-1}||_1 = n (the lower triangle of ones)
    n = 777
    L = torch.zeros((n, n), dtype=torch.float64 if prec == "fp64" else torch.float32, device=DEV)
    idx = torch.arange(n - 1, device=DEV)
    L[idx, idx + 1] = -1.0    # column-major storage of the subdiagonal (the row-major transpose)
    nl, ni = rcp.rcp_l_norms(handle, L, prec)
    assert nl == 2.0 and ni == float(n)


def test_exchange_latency_probe(rcp, handle):
    # the panel's per-step grid exchange alone: a positive, finite time per round, and the
    # handle factors normally afterwards (barrier counter and key ring left zeroed)
    us = rcp.rcp_exchange_latency(handle, 0, 2000)
    assert 0.05 < us < 100.0
    us8 = rcp.rcp_exchange_latency(handle, 8, 2000)
    assert 0.0 < us8 < 100.0
    a = inputs.gaussian_sym(300, seed=1)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, 64, 40, 5, prec="fp32")
    assert code == 0
    L = _unit_lower(A)
    D = oracle.block_d(Dd.cpu().numpy(), Ds.cpu().numpy())
    p = perm.cpu().numpy()
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max() < 2e-5 * max(1.0, st.growth_D)


@pytest.mark.parametrize("grid,limit_us", [(0, 2000), (8, 20000)])
def test_bounded_wait_runs_out_and_the_handle_recovers(rcp, grid, limit_us):
    # a grid barrier that no launch can complete: every CTA gives up after the limit, records the
    # timeout and returns (no hang, no trap); the handle then reports RCP_ETIMEOUT until the next
    # factorization clears the status word, and that factorization matches the oracle exactly
    h = rcp.rcp_create()
    code, waited = rcp.rcp_wait_expiry(h, limit_us, grid=grid)
    assert code == -5, rcp.STATUS.get(code, code)
    assert limit_us <= waited < limit_us + 200000
    assert rcp.lib().rcp_sync(h.h, None) == -5
    n, b, d, seed = 200, 32, 40, 4
    a = inputs.gaussian_sym(n, seed=seed)
    code, st, A, Dd, Ds, perm = _factor(rcp, h, a, b, d, seed)
    assert code == 0 and st.device_flags == 0
    ref = oracle.rcp(a, oracle.omega(seed, d, n), record=False)
    assert np.array_equal(perm.cpu().numpy(), ref["perm"])
    assert rcp.lib().rcp_sync(h.h, None) == 0


def _mixed_system(rcp, handle, n, kexp, prec, seed=7, nrhs=1):
    a = inputs.spectrum(n, seed=seed, kexp=kexp, nrefl=16)
    x = inputs.x_true(n, nrhs, seed=seed)
    rhs = inputs.rhs_for(a, x)
    A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV).float()
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, _ = rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=64, d=80, seed=1, prec=prec))
    assert code == 0
    A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Bv = torch.from_numpy(rhs.copy()).to(DEV)
    return a, rhs, A64, A, Dd, Ds, perm, Bv


@pytest.mark.parametrize("n,prec", [(1000, "f16x3"), (4000, "f16x3"), (4000, "fp32")])
def test_gmres_refinement_where_classic_refinement_stalls(rcp, handle, n, prec):
    # condition number 1e10: the FP32 factor's error times kappa is far above one
    a, rhs, A64, A, Dd, Ds, perm, Bv = _mixed_system(rcp, handle, n, 10.0, prec)
    X = torch.zeros_like(Bv)
    code, st = rcp.rcp_refine(handle, A64, A, Dd, Ds, perm, prec, Bv, X, tol=1e-12, max_iter=10)
    assert code == -6 and st.berr > 1e-12   # stops early: a correction did not halve berr
    assert st.refine_iters <= 3
    X2 = torch.zeros_like(Bv)
    code, st = rcp.rcp_refine_gmres(handle, A64, A, Dd, Ds, perm, prec, Bv, X2, tol=1e-12, max_outer=10)
    assert code == 0 and st.berr <= 1e-12 and st.gmres_iters > 0
    assert oracle.berr(a, X2.cpu().numpy().T, rhs.T) <= 1e-12


def test_gmres_refinement_several_rhs_and_starting_iterate(rcp, handle):
    a, rhs, A64, A, Dd, Ds, perm, Bv = _mixed_system(rcp, handle, 700, 6.0, "f16x3", nrhs=3)
    X = torch.zeros_like(Bv)
    code, st = rcp.rcp_refine_gmres(handle, A64, A, Dd, Ds, perm, "f16x3", Bv, X, tol=1e-12, max_outer=10,
                                    restart=8)
    assert code == 0
    assert oracle.berr(a, X.cpu().numpy().T, rhs.T) <= 1e-12
    # from a converged iterate nothing is left to do
    code, st = rcp.rcp_refine_gmres(handle, A64, A, Dd, Ds, perm, "f16x3", Bv, X, tol=1e-12, use_x=True)
    assert code == 0 and st.refine_iters == 0 and st.gmres_iters == 0


@pytest.mark.parametrize("kexp,gmres", [(4.0, False), (10.0, True)])
def test_sysv_falls_back_to_gmres_refinement(rcp, handle, kexp, gmres):
    n = 2000
    a = inputs.spectrum(n, seed=3, kexp=kexp, nrefl=16)
    x = inputs.x_true(n, 1, seed=3)
    rhs = inputs.rhs_for(a, x)
    A64 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    Bv = torch.from_numpy(rhs.copy()).to(DEV)
    X = torch.zeros_like(Bv)
    code, st = rcp.rcp_sysv(handle, A64, Bv, X, rcp.make_opts(b=64, d=80, seed=1, prec="f16x3"), tol=1e-12,
                            max_iter=10)
    assert code == 0 and st.berr <= 1e-12
    assert (st.gmres_iters > 0) == gmres
    assert oracle.berr(a, X.cpu().numpy().T, rhs.T) <= 1e-12


# ------------------------------------------------------------------------------------------
# full sizes, in the bench's launch configuration: sampled entries of P^T A P - L D L^T (each
# computed in FP64 from one row of L), and the FP64 backward error of the refined solution
# ------------------------------------------------------------------------------------------

def _sampled_reconstruction(A64, LA, Dd, Ds, perm, samples=512, seed=0):
    """max over sampled (i, j), i >= j, of |A(perm[i], perm[j]) - (L D L^T)(i, j)| / max|A|."""
    n = A64.shape[0]
    g = np.random.default_rng(seed)
    ii = g.integers(0, n, samples)
    jj = g.integers(0, n, samples)
    i_t = torch.from_numpy(np.maximum(ii, jj)).to(DEV)
    j_t = torch.from_numpy(np.minimum(ii, jj)).to(DEV)
    # rows of L (unit lower, stored in the library's lower triangle = the tensor's upper one)
    Lr = lambda idx: torch.where(torch.arange(n, device=DEV)[None, :] < idx[:, None], LA.t()[idx].double(),
                                 (torch.arange(n, device=DEV)[None, :] == idx[:, None]).double())
    li, lj = Lr(i_t), Lr(j_t)
    # (L D)(i, :) with D block diagonal: D(k, k) = Dd[k], D(k+1, k) = D(k, k+1) = Ds[k]
    ds_up = torch.cat([torch.zeros(1, dtype=torch.float64, device=DEV), Ds[:-1]])
    ld = li * Dd[None, :] + torch.roll(li, -1, 1) * Ds[None, :] + torch.roll(li, 1, 1) * ds_up[None, :]
    rec = (ld * lj).sum(1)
    p = perm.long()
    a = A64[p[i_t], p[j_t]]
    return float((a - rec).abs().max() / A64.abs().max())


@pytest.mark.parametrize("prec", ["tf32x3", "f16x3"])
def test_full_size_mixed_n16384(rcp, handle, prec):
    n = 16384
    A64 = inputs.spectrum(n, seed=0, kexp=4.0, nrefl=64, device=DEV)
    xt = torch.from_numpy(inputs.x_true(n, 1, seed=0)).to(DEV)
    Bv = (A64 @ xt.T).T.contiguous()
    X = torch.zeros_like(Bv)
    opts = rcp.make_opts(b=256, d=80, seed=0, prec=prec)
    code, st = rcp.rcp_sysv(handle, A64, Bv, X, opts, tol=1e-12, max_iter=10)
    assert code == 0 and st.berr <= 1e-12
    r = Bv - (A64 @ X.T).T
    berr = float((r.abs().amax() / (A64.abs().sum(1).amax() * X.abs().amax())))
    assert berr <= 4e-12
    # the FP32 factor itself
    A = A64.float().contiguous()
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, fst = rcp.rcp_factor(handle, A, Dd, Ds, perm, opts)
    assert code == 0
    assert torch.equal(torch.sort(perm.long())[0], torch.arange(n, device=DEV))
    assert _sampled_reconstruction(A64, A, Dd, Ds, perm) < 1e-4 * max(1.0, fst.growth_D)


def test_full_size_mixed_n32768(rcp, handle):
    # 216 rows per panel CTA: two passes of the fused step per pivot; b = 128 (the panel block of W
    # rows for b = 256 does not fit in shared memory at this n)
    n = 32768
    A64 = inputs.spectrum(n, seed=1, kexp=4.0, nrefl=64, device=DEV)
    xt = torch.from_numpy(inputs.x_true(n, 1, seed=1)).to(DEV)
    Bv = (A64 @ xt.T).T.contiguous()
    X = torch.zeros_like(Bv)
    code, st = rcp.rcp_sysv(handle, A64, Bv, X, rcp.make_opts(b=128, d=80, seed=1, prec="f16x3"), tol=1e-12,
                            max_iter=10)
    assert code == 0 and st.berr <= 1e-12
    r = Bv - (A64 @ X.T).T
    berr = float((r.abs().amax() / (A64.abs().sum(1).amax() * X.abs().amax())))
    assert berr <= 4e-12
    del A64, Bv, X, r
    torch.cuda.empty_cache()


GOLDEN_C2 = os.path.join(os.path.dirname(__file__), "golden", "c2_n8192.json")


def test_full_size_fp64_n8192_matches_the_oracle(rcp, handle):
    # The plain FP64 path at order 8192 (Gaussian (G + G^T)/2, b = 64, d = 80, seed 0) against the
    # oracle's factorization of the same matrix with the same Omega (tests/golden/c2_n8192.json,
    # written by the oracle alone): the same pivot sequence and 2x2 pattern, growth and max|L|
    # within 1%, and the normwise backward error of the solve within 1e-12 of the oracle's
    # (Algorithm 1; experiments section, Eqs. "err" and "growth").  Where the oracle's decision
    # was a near tie, rounding may pick the other column; the sequence then must agree up to it.
    g = json.load(open(GOLDEN_C2))
    n = g["n"]
    a = inputs.gaussian_sym(n, seed=g["seed"])
    A64 = torch.from_numpy(a).to(DEV)
    A = A64.clone()
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=64, d=g["d"], seed=g["seed"], prec="fp64"))
    assert code == 0 and st.info == g["info"]
    p = perm.cpu().numpy()
    want = np.asarray(g["perm"])
    if np.array_equal(p, want):
        assert np.array_equal(np.flatnonzero(Ds.cpu().numpy() != 0.0), np.asarray(g["starts_2x2"]))
        assert st.n_2x2 == g["n_2x2"]
    else:
        first = int(np.flatnonzero(p != want)[0])
        ties = {k for k, _ in g["near_ties"]}
        assert first in ties or first - 1 in ties, f"pivot sequence leaves the oracle's at {first}, not a near tie"
    assert abs(st.growth_D - g["growth_D"]) <= 0.01 * g["growth_D"]
    assert abs(st.max_abs_L - g["max_abs_L"]) <= 0.01 * g["max_abs_L"]
    assert _sampled_reconstruction(A64, A, Dd, Ds, perm) < 1e-12 * max(1.0, st.growth_D) * n / 64
    for name, nrhs, seed in (("berr_1", 1, 0), ("berr_32", 32, 1)):
        rhs = inputs.rhs_for(a, inputs.x_true(n, nrhs, seed=seed))
        X = torch.from_numpy(rhs.copy()).to(DEV)
        rcp.rcp_solve(handle, A, Dd, Ds, perm, "fp64", X)
        torch.cuda.synchronize()
        be = oracle.berr(a, X.cpu().numpy().T, rhs.T)
        assert abs(be - g[name]) <= 1e-12 and be <= 1e-13, (name, be, g[name])


# ------------------------------------------------------------------------------------------
# Growth-stress and saddle-point systems (experiments section, Types 1 and 7)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("family", ["type1", "kkt"])
def test_growth_stress_rcp_against_bunch_kaufman_and_bunch_parlett(rcp, handle, family):
    # n = 2048 with the paper's sampling dimension p = 5: the GPU's growth equals the oracle's RCP
    # with the same Omega (within 1%); Bunch-Kaufman's growth explodes on Type 1 and is far larger
    # on the KKT system, while RCP stays within a small factor of Bunch-Parlett's complete pivoting
    n, b, d, seed = 2048, 64, 5, 1
    a = inputs.bk_worst(n) if family == "type1" else inputs.kkt(2 * n // 3, n - 2 * n // 3, seed=1)
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, b, d, seed)
    assert code == 0
    ref = oracle.rcp(a, oracle.omega(seed, d, n), record=False)
    rho = oracle.growth_d(ref["Dd"], ref["Ds"], a)
    assert abs(st.growth_D - rho) <= 0.01 * rho
    bk, bp = oracle.bk(a), oracle.bp(a)
    rho_bk = oracle.growth_d(bk["Dd"], bk["Ds"], a)
    rho_bp = oracle.growth_d(bp["Dd"], bp["Ds"], a)
    if family == "type1":
        assert st.growth_D < 1e-3 * rho_bk and st.growth_D < 10.0
    else:
        assert st.growth_D < 0.1 * rho_bk
    assert st.growth_D <= 10.0 * rho_bp


def test_kkt_n12288_fp64_and_mixed(rcp, handle):
    # the saddle-point system [[H, W^T], [W, 0]], H = M M^T / 8192 + 1e-3 I (M 8192 x 8192),
    # W 4096 x 8192, all N(0, 1): the FP64 factor solves it to FP64 backward error, and the
    # FP16-split factor with FP64 refinement reaches berr <= 1e-12
    n1, n2 = 8192, 4096
    n = n1 + n2
    A64 = inputs.kkt(n1, n2, m=8192, seed=4, device=DEV)
    xt = torch.from_numpy(inputs.x_true(n, 1, seed=4)).to(DEV)
    Bv = (A64 @ xt.T).T.contiguous()
    A = A64.clone()
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code, st = rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=64, d=80, seed=4, prec="fp64"))
    assert code == 0
    assert torch.equal(torch.sort(perm.long())[0], torch.arange(n, device=DEV))
    assert _sampled_reconstruction(A64, A, Dd, Ds, perm) < 1e-12 * max(1.0, st.growth_D) * n / 64
    assert st.growth_D < 1e3 and st.max_abs_L < 50.0
    X = Bv.clone()
    rcp.rcp_solve(handle, A, Dd, Ds, perm, "fp64", X)
    r = Bv - (A64 @ X.T).T
    berr = float((r.abs().amax() / (A64.abs().sum(1).amax() * X.abs().amax())))
    assert berr <= 1e-13
    del A
    X = torch.zeros_like(Bv)
    code, st2 = rcp.rcp_sysv(handle, A64, Bv, X, rcp.make_opts(b=256, d=80, seed=4, prec="f16x3"), tol=1e-12,
                             max_iter=10)
    assert code == 0 and st2.berr <= 1e-12
    r = Bv - (A64 @ X.T).T
    assert float((r.abs().amax() / (A64.abs().sum(1).amax() * X.abs().amax()))) <= 4e-12
    del A64, Bv, X, r
    torch.cuda.empty_cache()


# ------------------------------------------------------------------------------------------
# FP32 factors against the oracle, entry by entry, where every decision is well separated
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "f16x3"])
@pytest.mark.parametrize("n,b,d,seed", [(200, 32, 40, 2), (513, 64, 80, 7)])
def test_fp32_factor_matches_the_oracle_where_decisions_are_well_separated(rcp, handle, prec, n, b, d, seed):
    # The FP32 factors take their decisions on FP32 values (rounding ~1e-6 relative here); on inputs
    # whose every decision in the oracle clears its threshold by more than 2e-4 they must take the
    # oracle's decisions: the same pivot sequence and 2x2 pattern, and L and D equal to the oracle's
    # up to the FP32 arithmetic.
    a = inputs.gaussian_sym(n, seed=seed)
    ref = oracle.rcp(a, oracle.omega(seed, d, n), record=True)
    assert min(m for _, m in oracle.decision_margins(ref["steps"])) > 2e-4
    code, st, A, Dd, Ds, perm = _factor(rcp, handle, a, b, d, seed, prec=prec)
    assert code == 0
    assert np.array_equal(perm.cpu().numpy(), ref["perm"])
    ds = Ds.cpu().numpy()
    assert np.array_equal(ds != 0.0, ref["Ds"] != 0.0)
    scale = np.abs(a).max() * max(1.0, st.growth_D)
    assert np.abs(Dd.cpu().numpy() - ref["Dd"]).max() <= 1e-4 * scale
    assert np.abs(ds - ref["Ds"]).max() <= 1e-4 * scale
    assert np.abs(_unit_lower(A) - ref["L"]).max() <= 1e-4 * max(1.0, ref["max_abs_L"])
    rho = oracle.growth_d(ref["Dd"], ref["Ds"], a)
    assert abs(st.growth_D - rho) <= 0.01 * rho


# ------------------------------------------------------------------------------------------
# Graph capture: rcp_factor and rcp_solve (no host rcp_stats, workspace reserved first) replay
# from a CUDA graph with the results of the eager calls, replay after replay
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_factor_and_solve_replay_from_a_cuda_graph(rcp, prec):
    n, b, d, nrhs = 1500, 128, 80, 3
    a = inputs.gaussian_sym(n, seed=31)
    dt = torch.float64 if prec == "fp64" else torch.float32
    A0 = torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dt)
    rhs = torch.from_numpy(inputs.x_true(n, nrhs, seed=4)).to(DEV)
    h = rcp.rcp_create()
    opts = rcp.make_opts(b=b, d=d, seed=2, prec=prec)
    rcp.rcp_reserve(h, n, nrhs, opts)
    A = A0.clone()
    Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    X = rhs.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rcp.rcp_factor(h, A, Dd, Ds, perm, opts, stream=s, stats=False)
        rcp.rcp_solve(h, A, Dd, Ds, perm, prec, X, stream=s)
    s.synchronize()
    ref = [t.clone() for t in (A, Dd, Ds, perm, X)]
    assert torch.isfinite(X).all()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        A.copy_(A0)
        X.copy_(rhs)
        rcp.rcp_factor(h, A, Dd, Ds, perm, opts, stream=s, stats=False)
        rcp.rcp_solve(h, A, Dd, Ds, perm, prec, X, stream=s)
    for _ in range(3):
        A.fill_(float("nan"))      # the graph copies A and X in again
        X.fill_(float("nan"))
        for t in (Dd, Ds, perm):   # as before the eager call
            t.zero_()
        g.replay()
        torch.cuda.synchronize()
        for got, want in zip((A, Dd, Ds, perm, X), ref):
            assert torch.equal(got, want)
    assert rcp.rcp_sync(h) == 0
    be = oracle.berr(a, X.cpu().numpy().T, rhs.cpu().numpy().T)
    assert be < (1e-13 if prec == "fp64" else 1e-5), be
