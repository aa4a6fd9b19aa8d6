"""rcp_solve_noalloc, the solve for callers that cannot allocate device memory (for example
while a stream is being captured into a CUDA graph): it must give the same solutions as
rcp_solve, call after call, with its scratch taken from a fixed device array.  Collected last so
that a failure here cannot hide the other tests."""
import numpy as np
import pytest
import torch

from paper_1710_00125_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,n,nrhs", [("fp64", 300, 3), ("fp32", 1000, 1), ("fp64", 1, 1)])
def test_noalloc_solve_matches_rcp_solve(prec, n, nrhs):
    from paper_1710_00125_gb300 import rcp
    h = rcp.rcp_create()
    a = inputs.gaussian_sym(n, seed=n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    A = torch.from_numpy(a).cuda().to(dt).contiguous()
    Dd = torch.zeros(n, dtype=torch.float64, device="cuda")
    Ds = torch.zeros_like(Dd)
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    code, _ = rcp.rcp_factor(h, A, Dd, Ds, perm, rcp.make_opts(b=32, d=40, seed=1, prec=prec))
    assert code == 0
    rhs = torch.from_numpy(inputs.x_true(n, nrhs, seed=5)).cuda()
    want = rhs.clone()
    rcp.rcp_solve(h, A, Dd, Ds, perm, prec, want)
    for _ in range(2):                        # two calls in a row share the same scratch
        got = rhs.clone()
        rcp.rcp_solve_noalloc(A, Dd, Ds, perm, prec, got)
        torch.cuda.synchronize()
        assert torch.allclose(got, want, rtol=1e-12, atol=1e-12 * float(want.abs().max()))


def test_noalloc_solve_rejects_sizes_beyond_its_scratch():
    from paper_1710_00125_gb300 import rcp
    lib = rcp.lib()
    # n * nrhs * 8 bytes beyond 16 MiB: refused before touching any pointer
    fake = 1 << 20
    assert lib.rcp_solve_noalloc(4096, 600, fake, 4096, fake, fake, fake, 0, fake, 4096, None) == -7
