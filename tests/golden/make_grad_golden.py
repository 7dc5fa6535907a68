"""Writes grad_8x8x8x16_ls8.json: the oracle's gradient of the differentiation
workload (8^3 x 16, Ls = 8), the expected values of the GPU gradient tests.

Only ``oracle/`` (and the seeded input generators of ``synth/``) are called:
x and y come from the oracle's conjugate residual (Section 3) converged to a
relative residual of 1e-13, the gradient from ``oracle.force.solve_gradient``.
The loss is L = Re(eta^dag x) with H x = b; stored are L, the full norms of
dL/dU and dL/db, and their values on a seeded sample of links and components.

    python tests/golden/make_grad_golden.py      (several minutes of CPU time)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import dwf, force  # noqa: E402
from oracle.krylov import cr  # noqa: E402

L, LS, EPS, M5, MF, BC = (8, 8, 8, 16), 8, 0.5, 1.8, 0.05, 1
SEED_U, SEED_B, SEED_ETA, SEED_SAMPLE = 6000, 6001, 6002, 6005
N_LINKS, N_COMP = 64, 32
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grad_8x8x8x16_ls8.json")


def main() -> None:
    U = synth.gauge_field(L, EPS, SEED_U)
    b = synth.gaussian_fermion(L, LS, SEED_B)
    eta = synth.gaussian_fermion(L, LS, SEED_ETA)
    H = lambda v: dwf.apply_H(U, v, M5, MF, BC)
    x, ix = cr(H, b, tol=1e-13, maxiter=100000)
    y, iy = cr(H, eta, tol=1e-13, maxiter=100000)
    gU, gb = force.solve_gradient(U, x, y, BC)
    gU = gU.reshape(4, -1, 3, 3)                       # (mu, x4, a, b)
    gbl = np.swapaxes(gb.reshape(-1, LS, 12), -1, -2)  # library layout (x4, c, s)
    rng = synth.rng(SEED_SAMPLE)
    links = [(int(rng.integers(4)), int(rng.integers(gU.shape[1]))) for _ in range(N_LINKS)]
    comps = [(int(rng.integers(gbl.shape[0])), int(rng.integers(12)), int(rng.integers(LS))) for _ in range(N_COMP)]
    d = {
        "what": "oracle gradient of L = Re(eta^dag x), H x = b, for the differentiation workload",
        "lattice": list(L), "Ls": LS, "eps": EPS, "M5": M5, "mf": MF, "bc_t": BC,
        "seeds": {"U": SEED_U, "b": SEED_B, "eta": SEED_ETA, "sample": SEED_SAMPLE},
        "cr_iters": [ix.iters, iy.iters], "cr_true_resid": [ix.true_resid, iy.true_resid],
        "loss": float(np.vdot(eta, x).real),
        "grad_U_norm": float(np.linalg.norm(gU)), "grad_b_norm": float(np.linalg.norm(gb)),
        "links": [[mu, x4, [[gU[mu, x4, a, c].real, gU[mu, x4, a, c].imag] for a in range(3) for c in range(3)]]
                  for mu, x4 in links],
        "grad_b": [[x4, c, s, gbl[x4, c, s].real, gbl[x4, c, s].imag] for x4, c, s in comps],
    }
    with open(OUT, "w") as f:
        json.dump(d, f, indent=1)
    print(f"wrote {OUT}: loss {d['loss']:.12e}, CR iterations {d['cr_iters']}")


if __name__ == "__main__":
    main()
