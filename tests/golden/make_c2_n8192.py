"""Writes ``c2_n8192.json``: the CPU oracle's RCP factorization of the plain FP64 Gaussian
system of order 8192 (A = (G + G^T)/2, G i.i.d. N(0, 1) from the seeded generator, seed 0;
Omega 80 x 8192 from Philox with seed 0), the reference the GPU's FP64 path is compared with
at that size (Algorithm 1 with b = q = 1; the GPU's panel width only changes when the deferred
update is applied, not the pivots).

It calls only ``oracle`` and the seeded input generators, never the CUDA library:

    python tests/golden/make_c2_n8192.py        (about 15 minutes on one core)

Stored values:
  perm            the pivot sequence (perm[i] = original index at position i)
  starts_2x2      positions k where a 2x2 block D(k:k+2, k:k+2) starts
  growth_D        rho = max|D_ij| / max|A_ij| (experiments section, Eq. "growth")
  max_abs_L       max |L_ij|, i > j
  berr_1, berr_32 normwise backward error (Eq. "err") of the oracle's solve of A x = b with
                  b = A x_true, x_true = x_true(n, 1, seed=0), resp. x_true(n, 32, seed=1)
                  (max over the right-hand sides)
  near_ties       [position, margin] for every step whose closest decision margin is below 1e-6:
                  the relative gap between the two largest sketch norms, between the two
                  largest |a_ik| (lambda), or between |a_kk| (|a_rr|) and alpha lambda.  A
                  computation that rounds differently may decide such a step the other way
                  (several results are then correct); every other step must match exactly.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1710_00125_gb300 import inputs  # noqa: E402

N, D, SEED = 8192, 80, 0
OUT = os.path.join(HERE, "c2_n8192.json")


def main(n=N, path=OUT):
    t0 = time.time()
    a = inputs.gaussian_sym(n, seed=SEED)
    om = oracle.omega(SEED, D, n)
    r = oracle.rcp(a, om, record=True)
    t1 = time.time()
    rhs1 = inputs.rhs_for(a, inputs.x_true(n, 1, seed=0))
    rhs32 = inputs.rhs_for(a, inputs.x_true(n, 32, seed=1))
    be = {}
    for name, rhs in (("berr_1", rhs1), ("berr_32", rhs32)):
        x = oracle.ldlt_solve(r["L"], r["Dd"], r["Ds"], r["perm"], rhs.T)
        be[name] = oracle.berr(a, x, rhs.T)
    ties = [[k, m] for k, m in oracle.decision_margins(r["steps"]) if m < 1e-6]
    rec = {
        "_comment": "Written by tests/golden/make_c2_n8192.py from the CPU oracle only "
                    "(Algorithm 1, b = q = 1, eager Schur complement).",
        "n": n, "d": D, "seed": SEED, "family": "gaussian_sym(n, seed=0)",
        "omega": "oracle.omega(0, 80, n)",
        "perm": [int(p) for p in r["perm"]],
        "starts_2x2": [int(i) for i in np.flatnonzero(r["Ds"] != 0.0)],
        "n_2x2": r["n_2x2"], "info": r["info"],
        "growth_D": oracle.growth_d(r["Dd"], r["Ds"], a),
        "max_abs_L": r["max_abs_L"],
        "berr_1": be["berr_1"], "berr_32": be["berr_32"],
        "rhs": {"berr_1": "x_true(n, 1, seed=0)", "berr_32": "x_true(n, 32, seed=1)"},
        "near_ties": ties,
        "oracle_seconds": round(t1 - t0, 1),
    }
    with open(path, "w") as f:
        json.dump(rec, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {path}: {len(ties)} near ties, growth {rec['growth_D']:.4f}, "
          f"berr {be['berr_1']:.2e}/{be['berr_32']:.2e}, {t1 - t0:.0f} s")


if __name__ == "__main__":
    main()
