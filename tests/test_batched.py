"""Batched ragged systems (rcp_factor_batched / rcp_refine_batched) against the CPU oracle,
system by system, through the C ABI.  Inputs come from the shared seeded generators; expected
values only from ``oracle``."""
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


def _opts(rcp, prec, b=32, d=40, seed=3):
    return rcp.make_opts(b=b, d=d, seed=seed, prec=prec)


def _load(bt, mats, nrhs=0, seed=0):
    rhs = []
    for i, a in enumerate(mats):
        if a.shape[0] == 0:
            rhs.append(None)
            continue
        bt.a64(i).copy_(torch.from_numpy(np.ascontiguousarray(a)))
        if nrhs:
            x = inputs.x_true(a.shape[0], nrhs, seed=seed + i)
            r = inputs.rhs_for(a, x)
            bt.b(i).copy_(torch.from_numpy(np.ascontiguousarray(r)))
            rhs.append(r)
    return rhs


def _unit_lower(F):
    n = F.shape[0]
    return np.tril(F.cpu().double().numpy().T, -1) + np.eye(n)


def _check_against_oracle(bt, i, a, seed, d, tol):
    n = a.shape[0]
    ref = oracle.rcp(a, oracle.omega(seed, d, n), record=False)
    assert int(bt.info[i]) == ref["info"], (i, n)
    assert np.array_equal(bt.perm(i).cpu().numpy(), ref["perm"]), (i, n)
    ds = bt.ds(i).cpu().numpy()
    assert np.array_equal(ds != 0, ref["Ds"] != 0)
    scale = max(np.abs(a).max(), 1e-300)
    assert np.allclose(bt.dd(i).cpu().numpy(), ref["Dd"], rtol=0, atol=tol * scale * max(1, n / 64))
    assert np.allclose(ds, ref["Ds"], rtol=0, atol=tol * scale * max(1, n / 64))
    assert np.allclose(_unit_lower(bt.f(i)), ref["L"], rtol=0, atol=10 * tol * max(1, n / 64))


# ------------------------------------------------------------------------------------------
# FP64 batched factor: every system gets the oracle's pivot sequence
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("b,d", [(32, 40), (8, 12), (5, 3)])
def test_batched_fp64_matches_oracle(rcp, handle, b, d):
    sizes = [129, 0, 1, 256, 2, 3, 31, 32, 33, 64, 100, 200, 17]
    mats = [inputs.gaussian_sym(n, seed=500 + i) for i, n in enumerate(sizes)]
    bt = rcp.Batch(sizes, 1, prec="fp64", device=DEV)
    _load(bt, mats)
    bt.factor(handle, _opts(rcp, "fp64", b, d, seed=11))
    torch.cuda.synchronize()
    for i, a in enumerate(mats):
        if a.shape[0]:
            _check_against_oracle(bt, i, a, 11, d, 1e-11)


def test_batched_fp64_structured(rcp, handle):
    # SBKP cases 2 and 3, 2x2 blocks at panel ends, zero pivots, an exactly singular system
    mats = [inputs.bk_worst(64), inputs.kkt(40, 24, seed=1), inputs.dst(50), inputs.dct(48),
            inputs.hankel(70, 2), inputs.augmented(40, 24, 3), inputs.spectrum(90, 4, 4.0, 8),
            np.zeros((9, 9)), np.array([[0.0, 1.0], [1.0, 0.0]]), inputs.rank_deficient(60, seed=2)]
    sizes = [m.shape[0] for m in mats]
    bt = rcp.Batch(sizes, 1, prec="fp64", device=DEV)
    _load(bt, mats)
    bt.factor(handle, _opts(rcp, "fp64", 8, 12, seed=2))
    torch.cuda.synchronize()
    for i, a in enumerate(mats):
        n = a.shape[0]
        ref = oracle.rcp(a, oracle.omega(2, 12, n), record=False)
        if i == len(mats) - 1:
            # numerical rank ~40: rounding-level pivots decide the tail, compare the leading ones
            assert np.array_equal(bt.perm(i).cpu().numpy()[:20], ref["perm"][:20])
            continue
        if i == 3:
            # the DCT-I matrix puts SBKP tests on a knife edge (a 1e-15 perturbation changes the
            # oracle's own pivots): check the factorization instead of the pivot sequence
            L = _unit_lower(bt.f(i))
            D = oracle.block_d(bt.dd(i).cpu().numpy(), bt.ds(i).cpu().numpy())
            p = bt.perm(i).cpu().numpy()
            assert sorted(p.tolist()) == list(range(n))
            assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() <= 1e-13 * n * np.abs(a).max()
            continue
        assert int(bt.info[i]) == ref["info"], i
        _check_against_oracle(bt, i, a, 2, 12, 1e-11)


def test_batched_equals_single_system_path(rcp, handle):
    # the batched kernel and rcp_factor take the same pivots (same Omega columns)
    sizes = [77, 256, 150]
    mats = [inputs.gaussian_sym(n, seed=40 + i) for i, n in enumerate(sizes)]
    bt = rcp.Batch(sizes, 1, prec="fp64", device=DEV)
    _load(bt, mats)
    bt.factor(handle, _opts(rcp, "fp64", 32, 40, seed=5))
    for i, a in enumerate(mats):
        n = a.shape[0]
        A = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
        Dd = torch.zeros(n, dtype=torch.float64, device=DEV)
        Ds = torch.zeros_like(Dd)
        perm = torch.zeros(n, dtype=torch.int32, device=DEV)
        rcp.rcp_factor(handle, A, Dd, Ds, perm, rcp.make_opts(b=32, d=40, seed=5, prec="fp64"))
        assert torch.equal(perm, bt.perm(i))
        assert torch.allclose(Dd, bt.dd(i), rtol=1e-12, atol=1e-12)


def test_batched_nonfinite_system_is_isolated(rcp, handle):
    mats = [inputs.gaussian_sym(50, seed=1), inputs.gaussian_sym(60, seed=2), inputs.gaussian_sym(40, seed=3)]
    mats[1] = mats[1].copy()
    mats[1][7, 3] = mats[1][3, 7] = np.nan
    bt = rcp.Batch([m.shape[0] for m in mats], 1, prec="fp32", device=DEV)
    _load(bt, mats)
    bt.factor(handle, _opts(rcp, "fp32", seed=4))
    torch.cuda.synchronize()
    assert int(bt.info[1]) == -4
    for i in (0, 2):
        assert int(bt.info[i]) == 0
        ref = oracle.rcp(mats[i], oracle.omega(4, 40, mats[i].shape[0]), record=False)
        assert np.array_equal(bt.perm(i).cpu().numpy(), ref["perm"])


# ------------------------------------------------------------------------------------------
# FP32 factor + FP64 refinement: the ragged workload of n ~ U{32..512}, 16 right-hand sides
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("threads", [512, 256, 128])
def test_batched_fp32_factor_backward_error(rcp, threads):
    # every CTA schedule: 512 threads keep the sketch in registers here, 256 and 128 in shared memory
    sizes = inputs.batched_sizes(24, 32, 512, seed=1).tolist() + [512, 32, 33]
    mats = inputs.batched_gaussian(sizes, seed=1)
    bt = rcp.Batch(sizes, 1, prec="fp32", device=DEV)
    _load(bt, mats)
    h = rcp.rcp_create()
    rcp.rcp_set_batched_schedule(h, threads, 0)
    bt.factor(h, _opts(rcp, "fp32", seed=6))
    torch.cuda.synchronize()
    assert (bt.info == 0).all()
    for i, a in enumerate(mats):
        n = a.shape[0]
        L = _unit_lower(bt.f(i))
        D = oracle.block_d(bt.dd(i).cpu().numpy(), bt.ds(i).cpu().numpy())
        p = bt.perm(i).cpu().numpy()
        assert sorted(p.tolist()) == list(range(n))
        growth = oracle.growth_d(bt.dd(i).cpu().numpy(), bt.ds(i).cpu().numpy(), a)
        err = np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max()
        assert err < 2e-5 * max(1.0, growth), (i, n, err)
        ref = oracle.rcp(a, oracle.omega(6, 40, n), record=False)
        n2 = int((bt.ds(i) != 0).sum())
        assert abs(n2 - ref["n_2x2"]) <= max(3, 0.05 * ref["n_2x2"])


def test_batched_refine_reaches_fp64_backward_error(rcp, handle):
    sizes = inputs.batched_sizes(40, 32, 512, seed=2).tolist() + [512, 32]
    mats = inputs.batched_gaussian(sizes, seed=2)
    nrhs = 16
    bt = rcp.Batch(sizes, nrhs, prec="fp32", device=DEV)
    rhs = _load(bt, mats, nrhs=nrhs, seed=100)
    bt.factor(handle, _opts(rcp, "fp32", seed=7))
    bt.refine(handle, tol=1e-12, max_iter=10)
    torch.cuda.synchronize()
    assert (bt.info == 0).all()
    berr = bt.berr.cpu().numpy()
    assert (berr <= 1e-12).all(), berr.max()
    assert int(bt.iters.max()) <= 6
    for i in range(0, len(mats), 5):
        x = bt.x(i).cpu().numpy()
        assert oracle.berr(mats[i], x.T, rhs[i].T) <= 1e-12
        # the device's berr is the same quantity, up to the rounding of its residual
        assert abs(oracle.berr(mats[i], x.T, rhs[i].T) - berr[i]) <= 1e-14


@pytest.mark.parametrize("nrhs", [1, 3, 16, 21])
def test_batched_fp64_solve_only(rcp, handle, nrhs):
    sizes = [1, 2, 45, 130, 256, 3]
    mats = [inputs.gaussian_sym(n, seed=70 + i) for i, n in enumerate(sizes)]
    bt = rcp.Batch(sizes, nrhs, prec="fp64", device=DEV)
    rhs = _load(bt, mats, nrhs=nrhs, seed=3)
    bt.factor(handle, _opts(rcp, "fp64", seed=8))
    bt.refine(handle, refine=False)
    torch.cuda.synchronize()
    for i, a in enumerate(mats):
        x = bt.x(i).cpu().numpy()
        assert oracle.berr(a, x.T, rhs[i].T) <= 1e-14, i
        ref = oracle.ldlt_solve(_unit_lower(bt.f(i)), bt.dd(i).cpu().numpy(), bt.ds(i).cpu().numpy(),
                                bt.perm(i).cpu().numpy(), rhs[i].T)
        # the same factor through two solve codes: they differ by rounding amplified by kappa(A)
        diff = np.abs(x.T - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert diff <= 1e-14 * max(1.0, np.linalg.cond(a)), (i, diff)


def test_batched_graph_capture_replays(rcp, handle):
    sizes = inputs.batched_sizes(30, 32, 300, seed=4).tolist()
    mats = inputs.batched_gaussian(sizes, seed=4)
    bt = rcp.Batch(sizes, 4, prec="fp32", device=DEV)
    _load(bt, mats, nrhs=4, seed=9)
    opts = _opts(rcp, "fp32", seed=1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bt.factor(handle, opts, stream=s)          # warm-up: grows the workspace, draws Omega
        bt.refine(handle, stream=s)
    s.synchronize()
    x_eager = bt.X_pool.clone()
    perm_eager = bt.perm_pool.clone()
    bt.X_pool.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bt.factor(handle, opts, stream=s)
        bt.refine(handle, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(bt.perm_pool, perm_eager)
    assert torch.equal(bt.X_pool, x_eager)
    assert (bt.berr <= 1e-12).all()


def test_batched_invalid_arguments(rcp, handle):
    bt = rcp.Batch([10, 20], 1, prec="fp64", device=DEV)
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_factor_batched(handle, -1, 20, bt.n, None, None, bt.p_F, bt.ld, bt.p_Dd, bt.p_Ds, bt.p_perm,
                               _opts(rcp, "fp64"), bt.info)
    assert e.value.code == -1
    with pytest.raises(rcp.RcpError) as e:
        # FP64 state of a 512-order system does not fit one CTA's shared memory
        rcp.rcp_factor_batched(handle, 2, 512, bt.n, None, None, bt.p_F, bt.ld, bt.p_Dd, bt.p_Ds, bt.p_perm,
                               _opts(rcp, "fp64"), bt.info)
    assert e.value.code == -7
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_factor_batched(handle, 2, 20, bt.n, None, None, bt.p_F, bt.ld, bt.p_Dd, bt.p_Ds, bt.p_perm,
                               _opts(rcp, "fp64", b=32, d=129), bt.info)
    assert e.value.code == -7
    with pytest.raises(rcp.RcpError) as e:
        # the Algorithm 2 safeguard is not offered on the batched path
        o = _opts(rcp, "fp64")
        o.guard_r = 1
        rcp.rcp_factor_batched(handle, 2, 20, bt.n, None, None, bt.p_F, bt.ld, bt.p_Dd, bt.p_Ds, bt.p_perm, o, bt.info)
    assert e.value.code == -7


@pytest.mark.parametrize("d", [40, 0])
def test_batched_autotuner(rcp, handle, d):
    # d = 40: the width alone is tuned; d = 0: the sketch follows the width (d = b + 8)
    sizes = inputs.batched_sizes(20, 32, 300, seed=5).tolist()
    mats = inputs.batched_gaussian(sizes, seed=5)
    bt = rcp.Batch(sizes, 1, prec="fp32", device=DEV)
    _load(bt, mats)
    h = rcp.rcp_create()
    b, ms = bt.tune(h, rcp.make_opts(b=0, d=d, seed=2, prec="fp32"))
    assert b in (8, 12, 16, 24, 32, 48, 64) and ms > 0
    sch = rcp.rcp_get_batched_schedule(h, bt.nmax, d, "fp32")
    assert sch["b"] == b and sch["d"] == (d if d else b + 8)
    assert (sch["threads"], sch["split"]) in ((512, 0), (256, 0), (128, 0), (512, min(256, bt.nmax // 2) & ~3))
    # the explicit shape and schedule the tuner chose give the same factorization as b = 0
    rcp.rcp_set_batched_schedule(h, sch["threads"], sch["split"])
    _load(bt, mats)
    bt.factor(h, rcp.make_opts(b=b, d=d if d else b + 8, seed=2, prec="fp32"))
    torch.cuda.synchronize()
    rcp.rcp_set_batched_schedule(h, 0, 0)
    perms = [bt.perm(i).cpu().numpy().copy() for i in range(len(sizes))]
    dds = [bt.dd(i).cpu().numpy().copy() for i in range(len(sizes))]
    _load(bt, mats)
    bt.factor(h, rcp.make_opts(b=0, d=d, seed=2, prec="fp32"))   # uses the tuned shape
    torch.cuda.synchronize()
    assert (bt.info == 0).all()
    for i in range(len(sizes)):
        assert np.array_equal(bt.perm(i).cpu().numpy(), perms[i]), i
        assert np.array_equal(bt.dd(i).cpu().numpy(), dds[i]), i
    for i, a in enumerate(mats):
        n = a.shape[0]
        L = _unit_lower(bt.f(i))
        D = oracle.block_d(bt.dd(i).cpu().numpy(), bt.ds(i).cpu().numpy())
        p = bt.perm(i).cpu().numpy()
        growth = oracle.growth_d(bt.dd(i).cpu().numpy(), bt.ds(i).cpu().numpy(), a)
        assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() / np.abs(a).max() < 2e-5 * max(1.0, growth)


# ------------------------------------------------------------------------------------------
# CTA schedules: 256-thread CTAs (two per SM) and the split by system order
# ------------------------------------------------------------------------------------------

def _factor_with(rcp, h, bt, mats, opts, threads, split):
    rcp.rcp_set_batched_schedule(h, threads, split)
    try:
        _load(bt, mats)
        bt.factor(h, opts)
        torch.cuda.synchronize()
    finally:
        rcp.rcp_set_batched_schedule(h, 0, 0)
    return ([bt.perm(i).cpu().numpy().copy() for i in range(bt.batch)],
            [bt.dd(i).cpu().numpy().copy() for i in range(bt.batch)],
            [bt.ds(i).cpu().numpy().copy() for i in range(bt.batch)],
            [bt.f(i).cpu().numpy().copy() for i in range(bt.batch)],
            bt.info.cpu().numpy().copy())


def _same(x, y):
    for u, v in zip(x[:4], y[:4]):
        for i, (p, q) in enumerate(zip(u, v)):
            assert np.array_equal(p, q), i
    assert np.array_equal(x[4], y[4])


@pytest.mark.parametrize("threads,split", [(256, 0), (128, 0), (512, 160), (0, 97)])
def test_batched_fp64_schedules_give_identical_factors(rcp, threads, split):
    # FP64 has one code path for every CTA size: the schedule moves work between threads only
    sizes = [300, 0, 1, 2, 97, 98, 160, 161, 33, 250, 5, 64]
    mats = [inputs.gaussian_sym(n, seed=700 + i) for i, n in enumerate(sizes)]
    bt = rcp.Batch(sizes, 1, prec="fp64", device=DEV)
    h = rcp.rcp_create()
    opts = _opts(rcp, "fp64", 16, 24, seed=4)
    ref = _factor_with(rcp, h, bt, mats, opts, 512, 0)
    got = _factor_with(rcp, h, bt, mats, opts, threads, split)
    _same(ref, got)
    for i, a in enumerate(mats):
        if a.shape[0]:
            _check_against_oracle(bt, i, a, 4, 24, 1e-11)


@pytest.mark.parametrize("threads", [128, 256])
def test_batched_fp32_small_ctas_with_register_sketch_give_identical_factors(rcp, threads):
    # orders <= the CTA size with d <= 48: every schedule keeps the sketch in registers
    sizes = inputs.batched_sizes(150, 1, threads, seed=threads).tolist() + [threads, 1, 0]
    mats = inputs.batched_gaussian(sizes, seed=threads)
    bt = rcp.Batch(sizes, 1, prec="fp32", device=DEV)
    h = rcp.rcp_create()
    opts = _opts(rcp, "fp32", 12, 20, seed=5)
    ref = _factor_with(rcp, h, bt, mats, opts, 512, 0)
    got = _factor_with(rcp, h, bt, mats, opts, threads, 0)
    _same(ref, got)


def test_batched_fp32_split_schedule_gives_identical_factors(rcp):
    # d <= 48: both launches keep the sketch in registers (the second one's order is 256), as the
    # single 512-thread launch does, so the factors are bit for bit the same
    sizes = inputs.batched_sizes(300, 32, 512, seed=9).tolist() + [256, 257, 1, 0]
    mats = inputs.batched_gaussian(sizes, seed=9)
    bt = rcp.Batch(sizes, 1, prec="fp32", device=DEV)
    h = rcp.rcp_create()
    opts = _opts(rcp, "fp32", 16, 24, seed=6)
    ref = _factor_with(rcp, h, bt, mats, opts, 512, 0)
    got = _factor_with(rcp, h, bt, mats, opts, 512, 256)
    _same(ref, got)
    assert (got[4] == 0).all()


@pytest.mark.parametrize("threads,b,d", [(256, 8, 16), (256, 16, 24), (256, 32, 40), (128, 8, 16), (128, 12, 20)])
def test_batched_fp32_small_ctas_refine_to_fp64_backward_error(rcp, threads, b, d):
    # 256- and 128-thread CTAs over systems up to order 512: the sketch stays in shared memory
    sizes = inputs.batched_sizes(200, 32, 512, seed=b).tolist()
    mats = inputs.batched_gaussian(sizes, seed=b)
    bt = rcp.Batch(sizes, 16, prec="fp32", device=DEV)
    h = rcp.rcp_create()
    rcp.rcp_set_batched_schedule(h, threads, 0)
    try:
        rhs = _load(bt, mats, nrhs=16, seed=b)
        bt.factor(h, _opts(rcp, "fp32", b, d, seed=1))
        bt.refine(h, tol=1e-12, max_iter=10)
        torch.cuda.synchronize()
    finally:
        rcp.rcp_set_batched_schedule(h, 0, 0)
    assert (bt.info.cpu().numpy() == 0).all()
    for i, a in enumerate(mats):
        be = oracle.berr(a, bt.x(i).cpu().numpy().T, rhs[i].T)
        assert be <= 1e-12, (i, a.shape[0], be)


def test_batched_schedule_graph_replay(rcp):
    # the split schedule's two launches replay from a CUDA graph with the same results
    sizes = inputs.batched_sizes(120, 32, 400, seed=12).tolist()
    mats = inputs.batched_gaussian(sizes, seed=12)
    bt = rcp.Batch(sizes, 1, prec="fp32", device=DEV)
    h = rcp.rcp_create()
    opts = _opts(rcp, "fp32", 16, 24, seed=8)
    ref = _factor_with(rcp, h, bt, mats, opts, 512, 200)
    rcp.rcp_set_batched_schedule(h, 512, 200)
    try:
        _load(bt, mats)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            bt.factor(h, opts, stream=s)   # warm-up: workspace and order array
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                bt.factor(h, opts, stream=s)
        for _ in range(2):
            _load(bt, mats)
            g.replay()
            torch.cuda.synchronize()
            got = ([bt.perm(i).cpu().numpy().copy() for i in range(bt.batch)],
                   [bt.dd(i).cpu().numpy().copy() for i in range(bt.batch)],
                   [bt.ds(i).cpu().numpy().copy() for i in range(bt.batch)],
                   [bt.f(i).cpu().numpy().copy() for i in range(bt.batch)],
                   bt.info.cpu().numpy().copy())
            _same(ref, got)
    finally:
        rcp.rcp_set_batched_schedule(h, 0, 0)


# every oracle decision of these systems (one Omega, seed 0, d = 40) clears its threshold by more
# than 2e-4 (checked below): the FP32 batched factor must take the oracle's decisions
WELL_SEPARATED = [(40, 1000), (97, 1000), (130, 1000), (200, 1001), (257, 1001), (300, 1000), (400, 1000),
                  (450, 1000), (512, 1002)]


@pytest.mark.parametrize("threads,split", [(512, 0), (256, 0), (128, 0), (512, 256)])
def test_batched_fp32_factor_matches_the_oracle_where_decisions_are_well_separated(rcp, threads, split):
    mats = [inputs.gaussian_sym(n, seed=s) for n, s in WELL_SEPARATED]
    refs = []
    for a in mats:
        ref = oracle.rcp(a, oracle.omega(0, 40, a.shape[0]), record=True)
        assert min(m for _, m in oracle.decision_margins(ref["steps"])) > 2e-4
        refs.append(ref)
    bt = rcp.Batch([a.shape[0] for a in mats], 1, prec="fp32", device=DEV)
    _load(bt, mats)
    h = rcp.rcp_create()
    rcp.rcp_set_batched_schedule(h, threads, split)
    bt.factor(h, _opts(rcp, "fp32", 16, 40, seed=0))
    torch.cuda.synchronize()
    assert (bt.info == 0).all()
    for i, (a, ref) in enumerate(zip(mats, refs)):
        assert np.array_equal(bt.perm(i).cpu().numpy(), ref["perm"]), i
        ds = bt.ds(i).cpu().numpy()
        assert np.array_equal(ds != 0.0, ref["Ds"] != 0.0), i
        rho = oracle.growth_d(ref["Dd"], ref["Ds"], a)
        scale = np.abs(a).max() * max(1.0, rho)
        assert np.abs(bt.dd(i).cpu().numpy() - ref["Dd"]).max() <= 1e-4 * scale, i
        assert np.abs(ds - ref["Ds"]).max() <= 1e-4 * scale, i
        assert np.abs(_unit_lower(bt.f(i)) - ref["L"]).max() <= 1e-4 * max(1.0, ref["max_abs_L"]), i
