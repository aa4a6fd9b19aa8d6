"""rcp_solve_noalloc, the solve for callers that cannot allocate device memory when they solve
(real-time loops that must not block in the allocator, programs whose device memory belongs to
another allocator).  It must give the same solutions as rcp_solve, call after call, with its
scratch taken from one fixed device array that every call reuses.  Collected last so that a
failure here cannot hide the other tests."""
import numpy as np
import pytest
import torch

from paper_1710_00125_gb300 import inputs

pytestmark = pytest.mark.gpu


def _factor(rcp, h, n, prec, seed):
    a = inputs.gaussian_sym(n, seed=seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    A = torch.from_numpy(a).cuda().to(dt).contiguous()
    Dd = torch.zeros(n, dtype=torch.float64, device="cuda")
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    code, _ = rcp.rcp_factor(h, A, Dd, Ds, perm, rcp.make_opts(b=32, d=40, seed=seed, prec=prec))
    assert code == 0
    return A, Dd, Ds, perm


def _identity_factor(n, prec):
    """L = I (zero strict lower triangle), D = I, perm = identity: the solve returns X = B."""
    dt = torch.float64 if prec == "fp64" else torch.float32
    L = torch.zeros((n, n), dtype=dt, device="cuda")
    Dd = torch.ones(n, dtype=torch.float64, device="cuda")
    Ds = torch.zeros_like(Dd)
    perm = torch.arange(n, dtype=torch.int32, device="cuda")
    return L, Dd, Ds, perm


# precision and size change from one call to the next: every call must clear what an earlier
# call of another shape or precision left in the shared scratch
SEQUENCE = [("fp64", 1000, 3), ("fp32", 300, 1), ("fp64", 300, 2), ("f16x3", 700, 4), ("fp32", 1000, 1),
            ("fp64", 1, 1)]


def test_noalloc_solve_matches_rcp_solve_over_a_sequence_of_shapes():
    from paper_1710_00125_gb300 import rcp
    h = rcp.rcp_create()
    for prec, n, nrhs in SEQUENCE:
        A, Dd, Ds, perm = _factor(rcp, h, n, prec, seed=n)
        rhs = torch.from_numpy(inputs.x_true(n, nrhs, seed=5)).cuda()
        want = rhs.clone()
        rcp.rcp_solve(h, A, Dd, Ds, perm, prec, want)
        for _ in range(2):                    # two calls in a row share the same scratch
            got = rhs.clone()
            rcp.rcp_solve_noalloc(A, Dd, Ds, perm, prec, got)
            torch.cuda.synchronize()
            assert torch.isfinite(got).all()
            assert torch.equal(got, want), (prec, n, nrhs)


def test_noalloc_fp32_after_fp64_doubles_that_look_like_published_words():
    # An FP64 call through the identity factor leaves the right-hand side's doubles in the
    # scratch.  Their high 32 bits are 1, 2, 3, ...: the FP32 solves take a 64-bit word as
    # published when its high half equals the call's epoch (a small counter), so without the
    # clearing some of these leftovers would pass for results of the next FP32 call.
    from paper_1710_00125_gb300 import rcp
    h = rcp.rcp_create()
    n64, nrhs64 = 4096, 16
    L, Dd1, Ds1, p1 = _identity_factor(n64, "fp64")
    hi = np.arange(1, n64 * nrhs64 + 1, dtype=np.uint64)
    bits = (hi << np.uint64(32)) | np.uint64(12345)
    rhs64 = torch.from_numpy(bits.view(np.float64).reshape(nrhs64, n64).copy()).cuda()
    n32, nrhs32 = 4096, 8                     # its two word arrays cover the same 65536 words
    A, Dd, Ds, perm = _factor(rcp, h, n32, "fp32", seed=7)
    rhs = torch.from_numpy(inputs.x_true(n32, nrhs32, seed=9)).cuda()
    want = rhs.clone()
    rcp.rcp_solve(h, A, Dd, Ds, perm, "fp32", want)
    for _ in range(3):
        x64 = rhs64.clone()
        rcp.rcp_solve_noalloc(L, Dd1, Ds1, p1, "fp64", x64)
        got = rhs.clone()
        rcp.rcp_solve_noalloc(A, Dd, Ds, perm, "fp32", got)
        torch.cuda.synchronize()
        assert torch.equal(x64, rhs64)        # the identity factor returns the right-hand sides
        assert torch.equal(got, want)


@pytest.mark.parametrize("prec,nrhs_max", [("fp64", 63), ("fp32", 12)])
def test_noalloc_size_limit_at_order_16384(prec, nrhs_max):
    # the largest right-hand-side count the 16 MiB scratch holds at n = 16384 runs; one more is
    # refused before anything is launched
    from paper_1710_00125_gb300 import rcp
    n = 16384
    L, Dd, Ds, perm = _identity_factor(n, prec)
    rhs = torch.from_numpy(inputs.x_true(n, nrhs_max, seed=3)).cuda()
    if prec != "fp64":
        rhs = rhs.float().double()            # exact through the FP32 solve
    x = rhs.clone()
    rcp.rcp_solve_noalloc(L, Dd, Ds, perm, prec, x)
    torch.cuda.synchronize()
    assert torch.equal(x, rhs)
    lib = rcp.lib()
    code = rcp.PREC_NAMES[prec]
    fake = 1 << 20
    assert lib.rcp_solve_noalloc(n, nrhs_max + 1, fake, n, fake, fake, fake, code, fake, n, None) == -7
    del L, x, rhs
    torch.cuda.empty_cache()


def test_noalloc_solve_rejects_sizes_beyond_its_scratch():
    from paper_1710_00125_gb300 import rcp
    lib = rcp.lib()
    # n * nrhs * 8 bytes beyond 16 MiB: refused before touching any pointer
    fake = 1 << 20
    assert lib.rcp_solve_noalloc(4096, 600, fake, 4096, fake, fake, fake, 0, fake, 4096, None) == -7
