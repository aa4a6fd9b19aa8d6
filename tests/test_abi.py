"""The C ABI without a GPU: the library loads, exports every function ``include/rcp.h``
declares, and its host-only helpers compute what they document (no device work)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rcp.h")


@pytest.fixture(scope="module")
def clib():
    from paper_1710_00125_gb300 import build
    return ctypes.CDLL(build.build())   # compiles only when a source is newer than the library


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(rcp_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rcp_create", "rcp_destroy", "rcp_factor", "rcp_solve", "rcp_refine", "rcp_refine_gmres",
                 "rcp_sysv", "rcp_factor_batched", "rcp_refine_batched", "rcp_omega", "rcp_sketch"):
        assert must in names


def test_library_exports_every_declared_function(clib):
    missing = [nm for nm in _declared() if not hasattr(clib, nm)]
    assert missing == []


def test_status_strings(clib):
    clib.rcp_status_string.restype = ctypes.c_char_p
    clib.rcp_status_string.argtypes = [ctypes.c_int]
    assert clib.rcp_status_string(0) == b"ok"
    assert clib.rcp_status_string(-6) == b"refinement did not reach the tolerance"
    assert clib.rcp_status_string(-7) == b"unsupported size or option"


def _lsq(clib, H, beta):
    k = H.shape[1]
    Hf = np.asfortranarray(H, dtype=np.float64)
    y = np.zeros(max(k, 1))
    res = ctypes.c_double(-1.0)
    clib.rcp_gmres_lsq.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double)]
    code = clib.rcp_gmres_lsq(k, Hf.ctypes.data, H.shape[0], beta, y.ctypes.data, ctypes.byref(res))
    return code, y[:k], res.value


@pytest.mark.parametrize("k", [1, 2, 5, 17, 30, 64])
def test_gmres_lsq_matches_numpy_lstsq(clib, k):
    rng = np.random.default_rng(k)
    H = np.triu(rng.standard_normal((k + 1, k)), -1)
    beta = 2.5
    code, y, res = _lsq(clib, H, beta)
    assert code == 0
    rhs = np.zeros(k + 1)
    rhs[0] = beta
    yref = np.linalg.lstsq(H, rhs, rcond=None)[0]
    # forward error bounded by the conditioning of H; the residual is optimal and reported
    assert np.abs(y - yref).max() <= 1e-14 * np.linalg.cond(H) * np.abs(yref).max()
    assert np.linalg.norm(rhs - H @ y) == pytest.approx(np.linalg.norm(rhs - H @ yref), rel=1e-9, abs=1e-13)
    assert res == pytest.approx(np.linalg.norm(rhs - H @ yref), rel=1e-9, abs=1e-13)


def test_gmres_lsq_ignores_entries_below_the_subdiagonal(clib):
    rng = np.random.default_rng(3)
    H = np.triu(rng.standard_normal((7, 6)), -1)
    noisy = H + np.tril(rng.standard_normal((7, 6)), -2)
    assert np.array_equal(_lsq(clib, H, 1.0)[1], _lsq(clib, noisy, 1.0)[1])


def test_gmres_lsq_exact_breakdown(clib):
    # H(k, k-1) = 0 (an invariant Krylov space): the square part is solved exactly
    rng = np.random.default_rng(4)
    k = 6
    H = np.triu(rng.standard_normal((k + 1, k)), -1)
    H[k, k - 1] = 0.0
    code, y, res = _lsq(clib, H, 1.0)
    assert code == 0 and res < 1e-14
    e1 = np.zeros(k)
    e1[0] = 1.0
    assert np.allclose(H[:k] @ y, e1, atol=1e-12)


def test_gmres_lsq_rejects_bad_arguments(clib):
    res = ctypes.c_double()
    clib.rcp_gmres_lsq.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double)]
    H = np.zeros((3, 2), order="F")
    y = np.zeros(2)
    assert clib.rcp_gmres_lsq(2, H.ctypes.data, 2, 1.0, y.ctypes.data, ctypes.byref(res)) == -1   # ldh < k + 1
    assert clib.rcp_gmres_lsq(-1, H.ctypes.data, 3, 1.0, y.ctypes.data, ctypes.byref(res)) == -1
    # k = 0: the residual is beta
    assert clib.rcp_gmres_lsq(0, None, 1, 3.0, None, ctypes.byref(res)) == 0 and res.value == 3.0


def test_product_path_fails_loudly_without_a_gpu_or_library(monkeypatch, tmp_path):
    # no CPU fallback: the binding raises instead of computing anything on the host
    import torch

    from paper_1710_00125_gb300 import rcp
    monkeypatch.setattr(rcp, "_lib", None)
    monkeypatch.setattr(rcp, "_LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        rcp.lib()
    if not torch.cuda.is_available():
        from paper_1710_00125_gb300 import build
        monkeypatch.setattr(rcp, "_LIB_PATH", build.build())
        with pytest.raises(RuntimeError, match="CUDA device"):
            rcp.lib()


def test_package_never_imports_the_oracle():
    # the oracle is test infrastructure: no module of the package names it in an import
    pkg = os.path.join(ROOT, "paper_1710_00125_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), name
            assert "import oracle" not in src and "from oracle" not in src, name


def test_plain_c_program_compiles_links_and_calls_the_abi(clib, tmp_path):
    # a C (not C++) consumer of include/rcp.h: the header is valid C, the library links, and the
    # host-only entry points answer (no device work)
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1710_00125_gb300 import build
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include "rcp.h"
int main(void) {
    double H[6] = {2.0, 1.0, 0.0, 1.0, 3.0, 1.0};   /* 3 x 2 Hessenberg, column-major */
    double y[2], res = -1.0;
    rcp_opts o = {0};
    rcp_stats st = {0};
    (void)o; (void)st;
    if (rcp_gmres_lsq(2, H, 3, 1.0, y, &res) != RCP_OK) return 2;
    if (rcp_factor(NULL, 4, NULL, 4, NULL, NULL, NULL, NULL, NULL, NULL) != RCP_EINVAL) return 3;
    printf("%s|%.17g\n", rcp_status_string(RCP_EUNSUPPORTED), res);
    return 0;
}
""")
    exe = tmp_path / "abi"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", inc, str(src), lib, "-o", str(exe),
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    msg, res = out.stdout.strip().split("|")
    assert msg == "unsupported size or option"
    # the least-squares residual of the 3 x 2 Hessenberg problem, by numpy
    Hm = np.array([[2.0, 1.0], [1.0, 3.0], [0.0, 1.0]])
    e1 = np.array([1.0, 0.0, 0.0])
    yref = np.linalg.lstsq(Hm, e1, rcond=None)[0]
    assert float(res) == pytest.approx(np.linalg.norm(e1 - Hm @ yref), rel=1e-12)


def test_batched_schedule_setter_and_getter_on_the_host(clib):
    # the schedule lives in the handle: no device work, so this runs without a GPU
    P, I = ctypes.c_void_p, ctypes.c_int
    clib.rcp_create.argtypes = [ctypes.POINTER(P)]
    clib.rcp_destroy.argtypes = [P]
    clib.rcp_set_batched_schedule.argtypes = [P, I, I]
    clib.rcp_get_batched_schedule.argtypes = [P, I, I, I] + [ctypes.POINTER(I)] * 4
    h = P()
    assert clib.rcp_create(ctypes.byref(h)) == 0

    def get(nmax, d=0, prec=1):
        out = [I(-1) for _ in range(4)]
        assert clib.rcp_get_batched_schedule(h, nmax, d, prec, *[ctypes.byref(o) for o in out]) == 0
        return tuple(o.value for o in out)

    try:
        assert get(512) == (32, 40, 512, 0)              # default shape and schedule
        assert get(512, 24) == (32, 24, 512, 0)
        for bad in ((64, 0), (-1, 0), (512, -1), (256, 100), (128, 100), (1024, 0)):
            assert clib.rcp_set_batched_schedule(h, *bad) == -1, bad
        assert clib.rcp_set_batched_schedule(h, 256, 0) == 0
        assert get(512)[2:] == (256, 0)
        assert clib.rcp_set_batched_schedule(h, 0, 200) == 0
        assert get(512)[2:] == (512, 200)
        assert get(200)[2:] == (512, 0)                  # a split at or above nmax is no split
        assert clib.rcp_set_batched_schedule(h, 0, 0) == 0
        assert get(512)[2:] == (512, 0)
        assert clib.rcp_set_batched_schedule(None, 0, 0) == -1
    finally:
        clib.rcp_destroy(h)
