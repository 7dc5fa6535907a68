"""Profiling driver: repeated applications of one kernel on random device data.

    python -m paper_1611_06944_gb300.probe stencil L dtype [reps]

applies H = Gamma5 D_dwf ``reps`` times (default 4) on an L^4 x 16 lattice with
random links and field (dtype f32 or f64), for ncu captures of a single kernel.
"""
from __future__ import annotations

import sys

import torch

import paper_1611_06944_gb300 as hd


def stencil(n: int, dtype: str, reps: int = 4) -> None:
    dt = torch.complex64 if dtype == "f32" else torch.complex128
    lat = hd.Lattice((n, n, n, n), 16)
    g = torch.Generator(device="cuda").manual_seed(0)
    U = torch.randn(4, lat.V4, 3, 3, dtype=dt, device="cuda", generator=g)
    x = torch.randn(lat.V4, 12, 16, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(reps):
        hd.apply_g5dwf(lat, U, x, 1.8, 0.01, out=y)
    torch.cuda.synchronize()
    # event-timed launches (the inputs exceed L2 at n = 16, so every launch reads from HBM)
    hd.stencil_timer(True)
    for _ in range(reps):
        hd.apply_g5dwf(lat, U, x, 1.8, 0.01, out=y)
    torch.cuda.synchronize()
    t = hd.stencil_timer_read(dt)
    hd.stencil_timer(False)
    us = t["ms"] / max(t["launches"], 1) * 1e3
    real = 4 if dtype == "f32" else 8
    per_site = 2 * 24 * real + 4 * 18 * real / 16   # psi in + out, links shared by the 16 s-sites
    print(f"ok {dtype} L={n} Ls=16: {us:.2f} us per launch, {lat.V4 * 16 * per_site / (us * 1e-6) / 1e9:.1f} GB/s")


def main(argv=None) -> int:
    a = sys.argv[1:] if argv is None else argv
    if len(a) >= 3 and a[0] == "stencil":
        stencil(int(a[1]), a[2], int(a[3]) if len(a) > 3 else 4)
        return 0
    print(__doc__)
    return 2


if __name__ == "__main__":
    sys.exit(main())
