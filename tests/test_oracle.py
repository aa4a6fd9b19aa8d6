"""Pins for the CPU oracle: checks against facts the paper and mathematics fix, not against the
oracle's own formulas.  Runs without a GPU."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from paper_1710_00125_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")
ALPHA = math.sqrt(2.0) / 2.0


def _recon_err(a, r):
    D = oracle.block_d(r["Dd"], r["Ds"])
    p = r["perm"]
    return np.max(np.abs(a[np.ix_(p, p)] - r["L"] @ D @ r["L"].T)) / np.max(np.abs(a))


# ---------------------------------------------------------------------------------------------
# Philox and the Gaussian sketch matrix
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ctr,key", [([0, 0, 0, 0], [0, 0]), ([3, 0, 0, 0], [7, 0]),
                                     ([12345, 6, 7, 0], [2**63 + 5, 99]),
                                     ([2**64 - 2, 2**64 - 1, 5, 1], [1, 2**64 - 1])])
def test_philox_matches_numpy_bit_generator(ctr, key):
    # numpy's Philox (4x64, 10 rounds) bumps the 256-bit counter before each block
    bg = np.random.Philox(key=key[0] + (key[1] << 64), counter=np.array(ctr, dtype=np.uint64))
    ref = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    if c[0] == 0:
        c[1] = (c[1] + 1) % 2**64
    got = oracle.philox4x64_10(c, key)
    assert np.array_equal(got, np.asarray(ref, dtype=np.uint64))


def test_omega_uses_philox_words_as_documented():
    # entries (2t, 2t+1) of column j come from the block with counter (j, t, stream, 0)
    seed, d, n = 11, 7, 5
    om = oracle.omega(seed, d, n, stream=0)
    j, t = 3, 2
    bg = np.random.Philox(key=seed, counter=[j - 1, t, 0, 0])
    w = bg.random_raw(4)
    u1 = ((int(w[0]) >> 11) + 1) * 2.0 ** -53
    u2 = (int(w[1]) >> 11) * 2.0 ** -53
    rho = math.sqrt(-2.0 * math.log(u1))
    assert om[2 * t, j] == pytest.approx(rho * math.cos(2 * math.pi * u2), rel=1e-14, abs=1e-15)
    assert om[2 * t + 1, j] == pytest.approx(rho * math.sin(2 * math.pi * u2), rel=1e-14, abs=1e-15)


def test_omega_is_standard_normal():
    om = oracle.omega(3, 40, 5000)
    x = om.ravel()
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1.0) < 0.02
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-3
    # the cosine and sine halves are uncorrelated, and columns are not repeated
    assert abs(np.corrcoef(om[0], om[1])[0, 1]) < 0.05
    assert abs(np.corrcoef(om[0, :-1], om[0, 1:])[0, 1]) < 0.05
    assert not np.allclose(oracle.omega(3, 4, 8), oracle.omega(4, 4, 8))


def test_omega_columns_and_rows_do_not_depend_on_the_draw_size():
    # column j and row pair (2t, 2t+1) come from counter (j, t): a d x n draw is the leading
    # block of any larger draw with the same seed (a ragged batch shares one d x nmax draw)
    big = oracle.omega(7, 21, 300)
    for d, n in ((21, 97), (20, 300), (5, 1), (1, 33)):
        assert np.array_equal(oracle.omega(7, d, n), big[:d, :n]), (d, n)


def test_sketch_is_the_matrix_product():
    a = inputs.gaussian_sym(37, seed=2)
    om = oracle.omega(5, 9, 37)
    assert np.allclose(oracle.sketch(om, a), om @ a, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------------------------
# The factorization
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,d", [(1, 3), (2, 3), (3, 4), (8, 5), (33, 8), (96, 12)])
def test_rcp_reconstructs_and_has_ldlt_structure(n, d):
    a = inputs.gaussian_sym(n, seed=n)
    r = oracle.rcp(a, oracle.omega(1, d, n))
    assert _recon_err(a, r) < 1e-13
    L = r["L"]
    assert np.allclose(np.diag(L), 1.0) and np.allclose(np.triu(L, 1), 0.0)
    assert sorted(r["perm"].tolist()) == list(range(n))
    # multipliers inside a 2x2 block are zero: L(k+1, k) = 0
    for i in range(n - 1):
        if r["Ds"][i] != 0.0:
            assert L[i + 1, i] == 0.0


def test_sbkp_block_properties():
    # 2x2 blocks: |a_kk|, |a_rr| < alpha*lambda and |a_rk| = lambda give det < 0 and
    # |det| > (1 - alpha^2) lambda^2 = lambda^2/2 (Section 4.3, case pivot[k] = 2);
    # case (1) columns have |l| <= 1/alpha (Section 4.2, case (1)).
    n = 160
    a = inputs.gaussian_sym(n, seed=4)
    r = oracle.rcp(a, oracle.omega(2, 10, n))
    seen = {0: 0, 1: 0, 2: 0, 3: 0}
    for st in r["steps"]:
        k = st["k"]
        seen[st["kase"]] += 1
        if st["s"] == 2:
            a11, a21, a22 = r["Dd"][k], r["Ds"][k], r["Dd"][k + 1]
            det = a11 * a22 - a21 * a21
            assert abs(a21) == pytest.approx(st["lam"], rel=0, abs=0)
            assert det < 0 and abs(det) >= 0.5 * st["lam"] ** 2 * (1 - 1e-12)
        if st["kase"] == 1:
            assert np.max(np.abs(r["L"][k + 1:, k]), initial=0.0) <= 1.0 / ALPHA * (1 + 1e-14)
        if st["kase"] == 2:
            assert abs(r["Dd"][k]) >= ALPHA * st["lam"] * (1 - 1e-14)
    assert seen[1] > 0 and seen[2] > 0 and seen[3] > 0


def test_sketch_identity_holds_at_every_step():
    # B^{(k)} = Omega~_2 A^{(k)} (Eq. "Update matrix B"): the updated sketch equals a fresh
    # projection of the current Schur complement with the permuted Omega.
    n, d = 30, 6
    a = inputs.gaussian_sym(n, seed=9)
    om = oracle.omega(8, d, n)
    r = oracle.rcp(a, om, snapshots=True)
    scale = np.linalg.norm(om, 2) * np.linalg.norm(a, 2)
    for st, B, S, p in zip(r["steps"], r["snap_B"], r["snap_A"], r["snap_perm"]):
        k1 = st["k"] + st["s"]
        if k1 >= n:
            continue
        direct = om[:, p[k1:]] @ S[k1:, k1:]
        assert np.max(np.abs(B[:, k1:] - direct)) <= 1e-12 * scale


def test_identity_sketch_picks_largest_schur_column():
    # Omega = I_n (d = n): the sketch columns are the Schur-complement columns, so the
    # pivot is the deterministic largest-column-norm rule; checked by brute force.
    n = 24
    a = inputs.gaussian_sym(n, seed=5)
    r = oracle.rcp(a, np.eye(n), snapshots=True)
    prev = a.copy()
    for st, S in zip(r["steps"], r["snap_A"]):
        k = st["k"]
        norms = np.sum(prev[k:, k:] ** 2, axis=0)
        # the step's interchange k <-> pi happens before SBKP; compare norms, which are
        # permutation invariant, and the chosen value
        assert st["norm2"] == pytest.approx(norms.max(), rel=1e-12)
        prev = S


def test_inertia_and_determinant():
    # Sylvester's law of inertia: D and A have the same numbers of positive and negative
    # eigenvalues; |det A| = |det D| since det L = 1.
    for n, seed in ((10, 1), (12, 2), (40, 3)):
        a = inputs.gaussian_sym(n, seed=seed)
        r = oracle.rcp(a, oracle.omega(seed, 5, n))
        ea = np.linalg.eigvalsh(a)
        ed = np.linalg.eigvalsh(oracle.block_d(r["Dd"], r["Ds"]))
        assert (ea > 0).sum() == (ed > 0).sum() and (ea < 0).sum() == (ed < 0).sum()
        if n <= 12:
            assert abs(np.linalg.det(a)) == pytest.approx(abs(np.linalg.det(oracle.block_d(r["Dd"], r["Ds"]))),
                                                          rel=1e-10)


def test_zero_and_degenerate_inputs():
    # case (0) of SBKP: lambda = 0 takes a_kk as a 1x1 pivot with zero multipliers; a zero
    # pivot is reported LAPACK style in info.
    n = 6
    r = oracle.rcp(np.zeros((n, n)), oracle.omega(1, 3, n))
    assert r["info"] == 1 and np.all(r["Dd"] == 0.0)
    diag = np.diag([3.0, -2.0, 5.0, 1.0])
    r = oracle.rcp(diag, oracle.omega(1, 3, 4))
    assert r["info"] == 0 and r["n_2x2"] == 0
    assert sorted(np.abs(r["Dd"]).tolist()) == [1.0, 2.0, 3.0, 5.0]
    # a pure 2x2 indefinite block [[0, 1], [1, 0]] forces a 2x2 pivot
    r = oracle.rcp(np.array([[0.0, 1.0], [1.0, 0.0]]), oracle.omega(1, 3, 2))
    assert r["n_2x2"] == 1 and r["info"] == 0


def test_bunch_kaufman_matches_lapack_sytrf():
    # scipy.linalg.ldl runs LAPACK ?sytrf (Bunch-Kaufman, alpha = (1+sqrt 17)/8): same
    # block pattern and same D for the unblocked sizes.
    for n, seed in ((9, 1), (31, 2), (60, 3)):
        a = inputs.gaussian_sym(n, seed=seed)
        r = oracle.bk(a)
        _, dref, _ = scipy.linalg.ldl(a, lower=True)
        D = oracle.block_d(r["Dd"], r["Ds"])
        assert np.allclose(D, dref, rtol=1e-10, atol=1e-12)
        assert _recon_err(a, r) < 1e-13


def test_bunch_kaufman_sigma_excludes_the_diagonal():
    # lambda = |a_10| = 1 (r = 1), sigma = the largest off-diagonal |a_i1| = 1: case (3) takes a_11
    # = 1000 as the first pivot (an interchange); counting a_11 in sigma would accept a_00 = 1e-3
    a = np.array([[1e-3, 1.0, 0.0], [1.0, 1000.0, 0.1], [0.0, 0.1, 1.0]])
    r = oracle.bk(a)
    assert r["perm"][0] == 1 and r["Dd"][0] == 1000.0
    sl = pytest.importorskip("scipy.linalg")
    _, d_lapack, _ = sl.ldl(a, lower=True)
    assert np.isclose(np.abs(np.diag(d_lapack)).max(), 1000.0)


def test_bunch_parlett_first_pivot_is_global():
    # complete pivoting: the first pivot is the largest diagonal (1x1) or the largest
    # off-diagonal pair (2x2), found by brute force
    for seed in range(5):
        n = 9
        a = inputs.gaussian_sym(n, seed=seed)
        r = oracle.bp(a)
        off = np.abs(np.tril(a, -1))
        mu0 = off.max()
        mu1 = np.abs(np.diag(a)).max()
        if mu1 >= oracle.BK_ALPHA * mu0:
            assert abs(r["Dd"][0]) == pytest.approx(mu1)
            assert r["Ds"][0] == 0.0
        else:
            assert abs(r["Ds"][0]) == pytest.approx(mu0)
        assert _recon_err(a, r) < 1e-13


def test_type1_growth_bk_exponential_rcp_bounded():
    # Type 1 is the Bunch-Kaufman worst case: BK's growth explodes, RCP and BP stay small
    n = 40
    a = inputs.bk_worst(n)
    g_bk = oracle.bk(a)["rho_elem"]
    g_rcp = oracle.rcp(a, oracle.omega(0, 8, n))["rho_elem"]
    g_bp = oracle.bp(a)["rho_elem"]
    assert g_bk > 1e6
    assert g_rcp < 10 and g_bp < 10
    g_bk_small = oracle.bk(inputs.bk_worst(20))["rho_elem"]
    assert g_bk > 1e3 * g_bk_small
    # LAPACK's Bunch-Kaufman (scipy.linalg.ldl) shows the same growth on this matrix
    _, dref, _ = scipy.linalg.ldl(a, lower=True)
    assert np.abs(dref).max() / np.abs(a).max() == pytest.approx(g_bk, rel=1e-6)


def test_solve_and_backward_error():
    n = 256
    a = inputs.gaussian_sym(n, seed=0)
    r = oracle.rcp(a, oracle.omega(0, 40, n), record=False)
    x = inputs.x_true(n, 3, seed=0)
    b = inputs.rhs_for(a, x)
    xs = oracle.ldlt_solve(r["L"], r["Dd"], r["Ds"], r["perm"], b.T)
    u = 2.0 ** -53
    be = oracle.berr(a, xs, b.T)
    assert be <= 10 * n * u
    # backward error measured independently with numpy (the residual itself is at rounding
    # level, so the two evaluations agree only to within a small factor)
    worst = max(np.abs(a @ xs[:, c] - b[c]).max() / (np.abs(a).sum(1).max() * np.abs(xs[:, c]).max())
                for c in range(3))
    assert worst <= 10 * n * u and be <= 10 * worst + 4 * u and worst <= 10 * be + 4 * u
    # a wrong solve is caught by the same measure
    bad = xs.copy()
    bad[0, 0] += 1e-6
    assert oracle.berr(a, bad, b.T) > 1e-9
    cond = np.linalg.cond(a)
    assert np.abs(xs.T - x).max() / np.abs(x).max() <= cond * 50 * n * u


def test_berr_definition_on_known_values():
    a = np.array([[2.0, 1.0], [1.0, -3.0]])
    x = np.array([1.0, 2.0])
    b = np.array([4.5, -5.0])          # A x = [4, -5]; residual 0.5
    # ||A||_inf = 4, ||x||_inf = 2
    assert oracle.berr(a, x, b) == pytest.approx(0.5 / 8.0)


def test_q_equals_b_mode():
    n, d, blk = 70, 20, 8
    a = inputs.gaussian_sym(n, seed=6)
    om = oracle.omega(3, d, n)
    r = oracle.rcp(a, om, q_mode=2, block=blk, snapshots=True)
    assert _recon_err(a, r) < 1e-13
    # after every completed block the block-updated sketch equals a fresh projection of the
    # Schur complement (the L11^{-T} reading of the block update)
    scale = np.linalg.norm(om, 2) * np.linalg.norm(a, 2)
    done, checked = 0, 0
    for st, B, S, p in zip(r["steps"], r["snap_B"], r["snap_A"], r["snap_perm"]):
        done += st["s"]
        k1 = st["k"] + st["s"]
        if done >= blk and k1 < n:
            assert np.max(np.abs(B[:, k1:] - om[:, p[k1:]] @ S[k1:, k1:])) <= 1e-11 * scale
            done = 0
            checked += 1
    assert checked >= 3


def test_argmax_ties_go_to_the_smallest_position():
    # Omega = I (d = n): B = A, and columns 0 and 1 have equal norms; the pivot is column 0
    a = np.array([[2.0, 0.0, 0.5], [0.0, 2.0, 0.5], [0.5, 0.5, 1.0]])
    r = oracle.rcp(a, np.eye(3))
    assert r["steps"][0]["pi"] == 0 and r["perm"][0] == 0


def test_sbkp_lambda_is_the_off_diagonal_maximum_of_the_pivot_column():
    # step 0 (nothing eliminated yet): lambda = max_{i != pi} |A(i, pi)| of the input itself
    for seed in range(5):
        a = inputs.gaussian_sym(12, seed=20 + seed)
        a[np.diag_indices(12)] *= 8.0   # diagonals larger than the column's other entries
        st0 = oracle.rcp(a, oracle.omega(seed, 6, 12))["steps"][0]
        col = np.delete(a[:, st0["pi"]], st0["pi"])
        assert st0["lam"] == np.abs(col).max()


def test_qb_block_candidates_match_lapack_qrcp():
    # the partial QRCP of the sketch picks the same columns as LAPACK's ?geqp3 (Businger-Golub
    # pivoting); on a strongly diagonal SPD matrix SBKP keeps case (1), so positions 0..b-1 after
    # the first step hold the candidates in QRCP order
    sl = pytest.importorskip("scipy.linalg")
    n, d, blk = 60, 16, 8
    rng = np.random.default_rng(11)
    g = rng.standard_normal((n, n))
    a = g @ g.T / n + 4.0 * np.eye(n)
    om = oracle.omega(4, d, n)
    r = oracle.rcp(a, om, q_mode=2, block=blk, snapshots=True)
    assert all(st["kase"] == 1 for st in r["steps"][:blk])
    _, _, piv = sl.qr(om @ a, pivoting=True, mode="economic")
    assert np.array_equal(r["snap_perm"][0][:blk], piv[:blk])


def test_paper_p_bound_example():
    g = json.load(open(GOLDEN))["p_bound_example"]
    assert oracle.p_bound(g["n"], g["eps"], g["delta"]) == g["p"]


def test_random_inputs_respect_the_probabilistic_bounds():
    # the L-entry and column-growth bounds hold with high probability; on these inputs they
    # hold with a wide margin (a violation would be logged, not failed, in larger sweeps)
    n = 128
    a = inputs.gaussian_sym(n, seed=7)
    r = oracle.rcp(a, oracle.omega(7, 12, n))
    assert r["max_abs_L"] <= oracle.l_entry_bound(n, 1, 0.5)
    assert r["rho_elem"] <= math.sqrt(n) * oracle.rho_col_bound(n, 0.5)


def test_generators_are_symmetric_and_seeded():
    for a in (inputs.gaussian_sym(20, 1), inputs.spectrum(20, 1, 3.0, 8), inputs.kkt(12, 8, seed=1),
              inputs.bk_worst(20), inputs.hankel(20, 1), inputs.dst(20), inputs.dct(20),
              inputs.augmented(12, 8, 1), inputs.rank_deficient(20, 1)):
        assert np.array_equal(a, a.T)
    assert np.array_equal(inputs.gaussian_sym(10, 3), inputs.gaussian_sym(10, 3))
    ev = np.abs(np.linalg.eigvalsh(inputs.spectrum(64, 2, 4.0, 16)))
    assert 1e3 < ev.max() / ev.min() <= 1e4 * 1.0001


# ------------------------------------------------------------------------------------------
# Algorithm 2 (safeguard): threshold eps^delta * beta on the pivot's sketch column norm
# ------------------------------------------------------------------------------------------

def _exact_rank_matrix(n, rho, seed):
    # integer V (n x rho) and D = diag(+-1): A = V D V^T has exact rank rho
    rng = np.random.default_rng(seed)
    V = rng.integers(-3, 4, size=(n, rho)).astype(np.float64)
    D = np.diag(rng.choice([-1.0, 1.0], size=rho))
    return V @ D @ V.T


def test_guard_stops_at_the_exact_rank():
    n, rho, d = 24, 7, 12
    a = _exact_rank_matrix(n, rho, 5)
    assert np.linalg.matrix_rank(a) == rho
    r = oracle.rcp(a, oracle.omega(3, d, n), guard_r=1, guard_eps=1e-8, seed=3)
    assert r["rank"] == rho and r["resketches"] == 0
    assert r["info"] == rho + 1
    assert np.all(r["Dd"][rho:] == 0.0) and np.all(r["Ds"][rho - 1:] == 0.0)
    L, p = r["L"], r["perm"]
    assert np.array_equal(L[rho:, rho:], np.eye(n - rho))
    D = oracle.block_d(r["Dd"], r["Ds"])
    assert np.abs(a[np.ix_(p, p)] - L @ D @ L.T).max() <= 1e-12 * np.abs(a).max()


def test_guard_recomputes_once_then_stops():
    n, rho, d = 24, 7, 12
    a = _exact_rank_matrix(n, rho, 6)
    # delta = 1/2 then 1: both thresholds sit far above the rounding-level Schur complement
    r = oracle.rcp(a, oracle.omega(3, d, n), guard_r=2, guard_eps=1e-8, seed=3)
    assert r["rank"] == rho and r["resketches"] == 1


def test_guard_recomputation_can_accept_a_small_but_real_schur_complement():
    # full rank with a block 1e-6 times smaller: sqrt(eps) * beta (eps = 1e-10) flags it, the
    # recomputed sketch is checked against eps * beta and accepted
    n, d = 20, 10
    rng = np.random.default_rng(8)
    g = rng.standard_normal((n, n))
    q, _ = np.linalg.qr(g)
    lam = np.concatenate([rng.uniform(1, 2, 12) * rng.choice([-1, 1], 12), 1e-6 * rng.uniform(1, 2, 8)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    r = oracle.rcp(a, oracle.omega(2, d, n), guard_r=2, guard_eps=1e-10, seed=2)
    assert r["rank"] == n and r["resketches"] == 1 and r["info"] == 0
    D = oracle.block_d(r["Dd"], r["Ds"])
    p = r["perm"]
    assert np.abs(a[np.ix_(p, p)] - r["L"] @ D @ r["L"].T).max() <= 1e-13 * np.abs(a).max()


def test_guard_that_never_fires_changes_nothing():
    a = inputs.gaussian_sym(40, seed=4)
    om = oracle.omega(1, 12, 40)
    r0 = oracle.rcp(a, om)
    r1 = oracle.rcp(a, om, guard_r=3, guard_eps=1e-300, seed=1)
    assert np.array_equal(r0["perm"], r1["perm"]) and np.array_equal(r0["L"], r1["L"])
    assert r1["rank"] == 40 and r1["resketches"] == 0


def test_pseudo_inverse_solve_and_basic_solution():
    # D = diag(2, 0, 4), L = I, perm = id: x = (b0 / 2, 0, b2 / 4)
    L = np.eye(3)
    x = oracle.ldlt_solve(L, np.array([2.0, 0.0, 4.0]), np.zeros(3), np.arange(3), np.array([[6.0, 5.0, 8.0]]).T)
    assert np.array_equal(x.ravel(), [3.0, 0.0, 2.0])
    # a consistent rank-deficient system: the basic solution has a small backward error
    n, rho = 24, 7
    a = _exact_rank_matrix(n, rho, 9)
    r = oracle.rcp(a, oracle.omega(3, 12, n), guard_r=1, guard_eps=1e-8, seed=3)
    xt = np.random.default_rng(1).standard_normal((n, 1))
    b = a @ xt
    x = oracle.ldlt_solve(r["L"], r["Dd"], r["Ds"], r["perm"], b.copy())
    assert oracle.berr(a, x, b) <= 1e-13


def test_l_norms_closed_forms():
    # L = I - (subdiagonal of ones): L^{-1} is the lower triangle of ones, ||L^{-1}||_1 = n
    n = 9
    L = np.eye(n) - np.eye(n, k=-1)
    assert oracle.l_norms(L) == (2.0, float(n))
    # [[1, 0], [e, 1]]: both norms 1 + |e|
    e = -0.375
    assert oracle.l_norms(np.array([[1.0, 0.0], [e, 1.0]])) == (1.0 + abs(e), 1.0 + abs(e))
    # against numpy's inverse on a random unit lower triangle
    rng = np.random.default_rng(2)
    L = np.tril(rng.uniform(-1, 1, (30, 30)), -1) + np.eye(30)
    nl, ni = oracle.l_norms(L)
    assert nl == pytest.approx(np.abs(L).sum(0).max())
    assert ni == pytest.approx(np.abs(np.linalg.inv(L)).sum(0).max(), rel=1e-8)


# ---------------------------------------------------------------------------------------------
# The growth factor rho = max|D_ij| / max|A_ij| (experiments section, Eq. "growth")
# ---------------------------------------------------------------------------------------------

def test_growth_closed_form_one_by_one_pivots():
    # A = [[1, t], [t, 1]], t = 1.2: lambda = t and |a_kk| = 1 >= alpha t, so a 1x1 pivot,
    # D = diag(1, 1 - t^2) whichever column the sketch picks; max|A| = t sits off the diagonal
    t = 1.2
    a = np.array([[1.0, t], [t, 1.0]])
    r = oracle.rcp(a, oracle.omega(0, 2, 2), record=False)
    assert r["n_2x2"] == 0
    assert oracle.growth_d(r["Dd"], r["Ds"], a) == pytest.approx(1.0 / t, rel=1e-15)


def test_growth_closed_form_largest_entry_in_a_2x2_block():
    # the 5 couples two small diagonal entries: SBKP case (3) takes the whole 2x2 block, so the
    # largest entry of D is its off-diagonal 5 = max|A| and rho = 1 (without D's sub-diagonal the
    # ratio would be 0.2 / 5)
    a = np.array([[0.1, 5.0, 0.0], [5.0, 0.2, 0.0], [0.0, 0.0, 1.0]])
    for seed in range(4):
        r = oracle.rcp(a, oracle.omega(seed, 3, 3), record=False)
        assert r["n_2x2"] == 1
        assert oracle.growth_d(r["Dd"], r["Ds"], a) == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("n,seed", [(60, 0), (61, 3), (90, 7)])
def test_growth_equals_the_largest_entry_of_the_reconstructed_d(n, seed):
    # D rebuilt without Dd/Ds: L^{-1} (P A P^T) L^{-T} from the factor's L and the input alone
    a = inputs.gaussian_sym(n, seed=seed)
    r = oracle.rcp(a, oracle.omega(seed, 12, n), record=False)
    assert r["n_2x2"] > 0
    p = r["perm"]
    Li = scipy.linalg.solve_triangular(r["L"], np.eye(n), lower=True, unit_diagonal=True)
    d_full = Li @ a[np.ix_(p, p)] @ Li.T
    rho = np.max(np.abs(d_full)) / np.max(np.abs(a))
    assert oracle.growth_d(r["Dd"], r["Ds"], a) == pytest.approx(rho, rel=1e-10)


def test_decision_margins_closed_forms():
    # Omega = I: the sketch is A itself.  diag(2, 1): squared column norms 4 and 1, lambda = 0 at the
    # first step, so the only decision is the argmax with relative gap (4 - 1) / 4
    om = np.eye(2)
    r = oracle.rcp(np.diag([2.0, 1.0]), om)
    assert oracle.decision_margins(r["steps"])[0] == (0, pytest.approx(0.75, rel=1e-15))
    # [[1, t], [t, 1]]: equal column norms (a tie, margin 0)
    r = oracle.rcp(np.array([[1.0, 0.5], [0.5, 1.0]]), om)
    assert oracle.decision_margins(r["steps"])[0][1] == 0.0
    # [[3, 1], [1, 0.5]], Omega = I: norms^2 10 and 1.25; lambda = 1, |a_kk| = 3 against alpha
    r = oracle.rcp(np.array([[3.0, 1.0], [1.0, 0.5]]), om)
    want = min((10.0 - 1.25) / 10.0, abs(3.0 - oracle.SQRT2_OVER_2) / oracle.SQRT2_OVER_2)
    assert oracle.decision_margins(r["steps"])[0][1] == pytest.approx(want, rel=1e-14)
