"""Randomized complete pivoting (RCP) for dense symmetric indefinite systems on GB300 (sm_103a).

Feng, Xiao and Gu, "Randomized complete pivoting for solving symmetric indefinite linear
systems": the block factorization Pi^T A Pi = L D L^T whose pivots come from a Gaussian sketch
B = Omega A, with SBKP 1x1 / 2x2 pivots (Algorithm 1; q = 1 or q = b), the Algorithm 2
safeguard, the solves, and FP64 iterative refinement of FP32 factors (classic, or GMRES-based
when the factor is too inaccurate for it).

Modules:
  rcp     ctypes binding of the C ABI in include/rcp.h (argument marshalling only; it raises
          when the CUDA library or a GPU is missing: there is no CPU path)
  build   in-tree nvcc build of csrc/*.cu into _rcp_gb300.so
  inputs  seeded synthetic matrices and right-hand sides (the paper's matrix families)

Typical use:
    from paper_1710_00125_gb300 import rcp
    h = rcp.rcp_create()
    code, stats = rcp.rcp_sysv(h, A64, B, X, rcp.make_opts(b=256, d=80, prec="f16x3"))
"""
