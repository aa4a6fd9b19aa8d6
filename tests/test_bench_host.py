"""Host-side arithmetic of the bench on CPU: the flop count, the bytes the host-buffer path
copies, and the roofline records (no GPU)."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_flop_count_is_the_operation_count_table():
    # factorization n^3/3, solve 2 n^2 per right-hand side
    assert bench.flops(16384, 1) == 16384 ** 3 / 3 + 2 * 16384 ** 2
    assert bench.flops(3, 4) == 9 + 72


@pytest.mark.parametrize("n,cols", [(1, 256), (255, 256), (256, 256), (700, 256), (1000, 96)])
def test_host_copy_bytes_counts_the_copied_rectangles(n, cols):
    # brute force: mark every element the rectangles (from each block's diagonal down) cover
    copied = np.zeros((n, n), dtype=bool)
    for j0 in range(0, n, cols):
        copied[j0:, j0:j0 + cols] = True
    assert bench.host_copy_bytes(n, cols) == int(copied.sum()) * 8
    # the rectangles hold the whole lower triangle and less than one block more per block
    assert copied[np.tril_indices(n)].all()


def _args(**kw):
    a = dict(n=16384, b=256, d=80, prec="f16x3")
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_panel_roofline_record():
    r = bench.roofline_for("panel", 76.0, 64, _args(), 6685.5, {"hbm_gbs": 6685.5}, "of measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(r["achieved"] / 6685.5)
    # algorithmic bytes of the average launch over its time
    m = 16384 / 2.0
    byts = (2 * 80 * m + 256 * m * 1.5 + 2 * 256 * m) * 4
    assert r["achieved"] == pytest.approx(byts / (76.0 / 64 * 1e-3) / 1e9)
    # DRAM traffic needs a profiler capture; the timed run reports none
    assert r["traffic"] is None


def test_trailing_roofline_record():
    peaks = {"bf16_tflops": 1944.0, "sm_max_mhz": 2070.0}
    r = bench.roofline_for("trailing", 10.0, 64, _args(), 6685.5, peaks, "")
    assert r["bound"] == "tensor" and r["peak"] == 1944.0
    assert r["achieved"] == pytest.approx(16384 ** 3 / 3 / 64 / (10.0 / 64 * 1e-3) / 1e12)
    assert bench.roofline_for("trailing", 10.0, 64, _args(prec="tf32x3"), 6685.5, peaks, "")["peak"] == 972.0
    assert bench.roofline_for("trailing", 10.0, 64, _args(prec="fp32"), 6685.5, peaks, "")["bound"] == "alu"


@pytest.mark.parametrize("n,b", [(1, 64), (7, 3), (64, 64), (300, 64), (513, 32)])
def test_trailing_flops_count_the_lower_triangle_updates(n, b):
    # brute force: for every panel, every lower entry (i >= j) of the trailing block gets one
    # multiply and one add per panel column
    fl = 0
    for k0 in range(0, n, b):
        kend = min(n, k0 + b)
        for j in range(kend, n):
            fl += 2 * (n - j) * (kend - k0)
    assert bench.trailing_flops(n, b) == fl


def test_trailing_flops_approach_n_cubed_over_three():
    n = 16384
    assert bench.trailing_flops(n, 64) == pytest.approx(n ** 3 / 3, rel=0.01)
