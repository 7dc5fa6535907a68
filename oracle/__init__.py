"""Plain, slow FP64 CPU oracle of the HDCR hot path (arXiv:1611.06944).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA path (``paper_1611_06944_gb300``); the only
common module is ``synth`` (seeded input generators, no method arithmetic).

Everything is numpy complex128.  Each function cites the passage of the paper
it follows; where the paper is silent the reading used is stated in the
function's docstring.

Modules
-------
``dwf``        the fine operator H = Gamma5 D_dwf (Section 3) and its hop pieces
``krylov``     conjugate residual (Section 3) and flexible GCR (Section 4)
``multigrid``  subspace, block projection, little Dirac operator, coarse solve,
               the two-level preconditioner and the HDCR solve (Section 4)
``force``      gauge-link gradient of Re(eta^dag H^-1 b) (not in the paper)
``redblack``   red-black (even-odd) preconditioned CGNE, the comparison solver of
               Section 5 (Table 1)

Layouts follow ``synth``: gauge ``(4, Lt, Lz, Ly, Lx, 3, 3)``; fermion
``(..., Lt, Lz, Ly, Lx, Ls, 4, 3)`` with optional leading batch axes.
"""
