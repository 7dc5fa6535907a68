"""Profiling driver: repeated applications of one kernel on random device data.

    python -m paper_1611_06944_gb300.probe stencil L dtype [reps]
    python -m paper_1611_06944_gb300.probe coarse L nvec dtype [reps]

``L`` is one extent (an L^4 lattice) or four comma-separated extents
(e.g. 24,24,24,48); Ls = 16.  ``stencil`` applies H = Gamma5 D_dwf ``reps``
times (default 4) with random links and field (dtype f32, f64, or h16 for
FP16-stored fields); ``coarse``
builds the little Dirac operator ``reps`` times (default 3; dtype f64, f32, or
f32fast for single-pass TF32 projections) from nvec random basis vectors on 4^4
blocks of that lattice and reports its time in units of
one fine application of H of the same precision.  For ncu captures of single
kernels.
"""
from __future__ import annotations

import sys

import torch

import paper_1611_06944_gb300 as hd


def _extents(spec: str) -> tuple:
    parts = [int(v) for v in spec.split(",")]
    return tuple(parts) if len(parts) == 4 else (parts[0],) * 4


def stencil(L: tuple, dtype: str, reps: int = 4) -> None:
    h16 = dtype == "h16"  # FP16 storage, FP32 arithmetic and links
    dt = torch.complex64 if dtype in ("f32", "h16") else torch.complex128
    lat = hd.Lattice(L, 16)
    g = torch.Generator(device="cuda").manual_seed(0)
    U = torch.randn(4, lat.V4, 3, 3, dtype=dt, device="cuda", generator=g)
    x = torch.randn(lat.V4, 12, 16, dtype=dt, device="cuda", generator=g)
    if h16:
        x = hd.encode_h16(lat, x)
    y = torch.empty_like(x)
    apply = (lambda: hd.apply_g5dwf_h16(lat, U, x, 1.8, 0.01, out=y)) if h16 else \
        (lambda: hd.apply_g5dwf(lat, U, x, 1.8, 0.01, out=y))
    for _ in range(reps):
        apply()
    torch.cuda.synchronize()
    # event-timed launches (the inputs exceed L2 at n = 16, so every launch reads from HBM)
    hd.stencil_timer(True)
    for _ in range(reps):
        apply()
    torch.cuda.synchronize()
    t = hd.stencil_timer_read("h16" if h16 else dt)
    hd.stencil_timer(False)
    us = t["ms"] / max(t["launches"], 1) * 1e3
    real = 4 if dtype == "f32" else 8
    per_site = 2 * 24 * real + 4 * 18 * real / 16   # psi in + out, links shared by the 16 s-sites
    if h16:
        per_site = 2 * 52 + 4 * 18 * 4 / 16         # half2 spinor + FP32 scale, in and out; FP32 links
    print(f"ok {dtype} L={L} Ls=16: {us:.2f} us per launch, {lat.V4 * 16 * per_site / (us * 1e-6) / 1e9:.1f} GB/s")


def coarse(L: tuple, nvec: int, dtype: str, reps: int = 3) -> None:
    fast = dtype == "f32fast"  # single-pass TF32 projections
    dt = torch.complex64 if dtype in ("f32", "f32fast") else torch.complex128
    lat = hd.Lattice(L, 16)
    g = torch.Generator(device="cuda").manual_seed(0)
    U = torch.randn(4, lat.V4, 3, 3, dtype=torch.complex128, device="cuda", generator=g)
    v = torch.randn(nvec, lat.V4, 12, 16, dtype=torch.complex128, device="cuda", generator=g)
    sub = hd.subspace_from_vectors(lat, (4, 4, 4, 4), v, store_dtype=dt)
    del v
    torch.cuda.empty_cache()
    hd.build_coarse_op(sub, U, 1.8, 0.01, op_dtype=dt, fast=fast).close()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        hd.build_coarse_op(sub, U, 1.8, 0.01, op_dtype=dt, fast=fast).close()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    Ud = U.to(dt)
    x = torch.randn(lat.V4, 12, 16, dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(3):
        hd.apply_g5dwf(lat, Ud, x, 1.8, 0.01, out=y)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        hd.apply_g5dwf(lat, Ud, x, 1.8, 0.01, out=y)
    e1.record()
    torch.cuda.synchronize()
    mv = e0.elapsed_time(e1) / 10
    sub.close()
    print(f"ok coarse {dtype} L={L} Ls=16 nvec={nvec}: build {ms:.2f} ms = {ms / mv:.1f} fine matvecs ({mv:.3f} ms)")


def main(argv=None) -> int:
    a = sys.argv[1:] if argv is None else argv
    if len(a) >= 3 and a[0] == "stencil":
        stencil(_extents(a[1]), a[2], int(a[3]) if len(a) > 3 else 4)
        return 0
    if len(a) >= 4 and a[0] == "coarse":
        coarse(_extents(a[1]), int(a[2]), a[3], int(a[4]) if len(a) > 4 else 3)
        return 0
    print(__doc__)
    return 2


if __name__ == "__main__":
    sys.exit(main())
