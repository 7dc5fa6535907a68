"""The FP32 little Dirac operator (Eq. 4.5), whose projections run on the
tensor cores, against the FP64 build from the same basis (itself checked
against the oracle in test_gpu_multigrid).  The cases cover the operand
shapes the kernel pads differently (2 nvec = 16, 48, 64, 128 rows), chunks of
the contraction dimension that end ragged, and coarse extents of 2 (legs that
reach the same coarse site)."""
import numpy as np
import pytest

import synth
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


# (L, Ls, block, nvec, bc)
CASES = [
    ((4, 4, 4, 4), 8, (2, 2, 2, 2), 8, 1),
    ((6, 4, 4, 6), 5, (3, 2, 2, 3), 24, -1),
    ((8, 8, 4, 4), 6, (4, 4, 2, 2), 32, 1),
    ((4, 4, 4, 8), 4, (2, 2, 2, 4), 64, 1),
]


@pytest.mark.parametrize("L,Ls,block,nvec,bc", CASES)
def test_fp32_coarse_op_matches_fp64_build(hd, L, Ls, block, nvec, bc):
    U = synth.gauge_field(L, 0.5, 5100)
    rng = synth.rng(5101)
    lat = hd.Lattice(L, Ls, bc)
    shape = (nvec, lat.V4, 12, Ls)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    sub64 = hd.subspace_from_vectors(lat, block, dev(v), store_dtype=torch.complex128)
    sub32 = hd.subspace_from_vectors(lat, block, dev(v), store_dtype=torch.complex64)
    Ud = dev(links(U))
    A64 = host(hd.build_coarse_op(sub64, Ud, 1.8, 0.01).op())
    A32 = host(hd.build_coarse_op(sub32, Ud, 1.8, 0.01, op_dtype=torch.complex64).op())
    # Bound: the FP32 basis differs from the FP64 one by ~1e-7 relative.  Each
    # product of the projection (three TF32 passes: hi*hi + hi*lo + lo*hi) is good
    # to ~2^-20 relative and the tensor-core accumulator (not rounded to nearest)
    # drifts by about as much over a 512-term segment, so an entry is good to
    # ~1e-6 of sum |phi_j| |Y_k|.  For random bases the entries are smaller than
    # that sum by the cancellation of ~sqrt(K) random-sign terms (K = 12 Ls |block|
    # up to 1536 here), i.e. up to ~40x: 1e-5 relative overall, 1e-4 per leg.
    assert relerr(A32, A64) < 1e-5
    # leg by leg, so that a wrong leg cannot hide behind the large diagonal one
    for leg in range(9):
        assert relerr(A32[:, leg], A64[:, leg]) < 1e-4


@pytest.mark.parametrize("L,Ls,block,nvec,bc", [CASES[0], CASES[2], CASES[3]])
def test_single_pass_tf32_coarse_op(hd, L, Ls, block, nvec, bc):
    """fast=True: one pass of TF32 products.  Each operand is rounded to TF32
    (11 significant bits, relative error <= 2^-11), so a product is good to about
    2^-10 ~ 1e-3 and, the rounding errors being as random in sign as the terms
    themselves, an entry to about 1e-3 of its size: 4e-3 overall, 1e-2 per leg.
    It must also differ from the three-pass build (the mode took effect)."""
    U = synth.gauge_field(L, 0.5, 5300)
    rng = synth.rng(5301)
    lat = hd.Lattice(L, Ls, bc)
    shape = (nvec, lat.V4, 12, Ls)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Ud = dev(links(U))
    sub64 = hd.subspace_from_vectors(lat, block, dev(v), store_dtype=torch.complex128)
    sub32 = hd.subspace_from_vectors(lat, block, dev(v), store_dtype=torch.complex64)
    A64 = host(hd.build_coarse_op(sub64, Ud, 1.8, 0.01).op())
    A3 = host(hd.build_coarse_op(sub32, Ud, 1.8, 0.01, op_dtype=torch.complex64).op())
    A1 = host(hd.build_coarse_op(sub32, Ud, 1.8, 0.01, op_dtype=torch.complex64, fast=True).op())
    e1 = relerr(A1, A64)
    assert e1 < 4e-3
    assert e1 > 10 * relerr(A3, A64)
    for leg in range(9):
        assert relerr(A1[:, leg], A64[:, leg]) < 1e-2


def test_hdcr_solve_with_single_pass_coarse_op(hd):
    """The mixed-precision solve recovers full accuracy with the single-pass build:
    true residual <= 1e-10, recomputed by the oracle."""
    from oracle import dwf
    from gpu_util import natural, planes
    L, Ls, block, nvec, mf = (4, 4, 4, 4), 8, (2, 2, 2, 2), 8, 0.01
    lat = hd.Lattice(L, Ls)
    Uh = synth.gauge_field(L, 0.3, 1000)
    U = dev(links(Uh))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 3001, count=nvec // 2)))
    sub = hd.build_subspace(lat, U, noise, 1.8, mf, block, kind="chebyshev", order=100, lam_cut=0.3,
                            store_dtype=torch.complex64)
    co = hd.build_coarse_op(sub, U, 1.8, mf, op_dtype=torch.complex64, fast=True)
    b = synth.gaussian_fermion(L, Ls, 2000)
    x, st = hd.hdcr_solve(co, U, dev(planes(b)), tol=1e-10, inner_dtype=torch.complex64, max_outer=2000,
                          restart=16)
    xg = natural(host(x), L, Ls)
    res = np.sqrt(dwf.norm2(b - dwf.apply_H(Uh, xg, 1.8, mf)) / dwf.norm2(b))
    assert st["status"] == 0 and res <= 1.01e-10


# 8^4 x 4 with 4^4 blocks: K = 256 x 4 x 12 = 12288 per block (384 chunks of 32),
# so every leg-0 projection is split over 24 CTAs and summed by the reduction
# kernel; nvec 24 and 32 run the M = 64 variant, 48 and 64 the M = 128 one with
# two tasks per thread.
@pytest.mark.parametrize("nvec", [24, 32, 48, 64])
def test_tensor_core_coarse_op_matches_oracle(hd, nvec):
    """The FP32 tensor-core builds (three-pass and single-pass TF32) against
    oracle.multigrid.coarse_op evaluated in FP64 on the same FP32-rounded basis,
    leg by leg.  Bounds as derived in the tests above: three passes 1e-5 overall
    and 1e-4 per leg; one pass 4e-3 overall and 1e-2 per leg."""
    from oracle import multigrid as mg
    L, Ls, block, bc, mf = (8, 8, 8, 8), 4, (4, 4, 4, 4), -1, 0.01
    U = synth.gauge_field(L, 0.5, 5400 + nvec)
    rng = synth.rng(5500 + nvec)
    lat = hd.Lattice(L, Ls, bc)
    shape = (nvec, lat.V4, 12, Ls)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    sub32 = hd.subspace_from_vectors(lat, block, dev(v), store_dtype=torch.complex64)
    Ud = dev(links(U))
    A3 = host(hd.build_coarse_op(sub32, Ud, 1.8, mf, op_dtype=torch.complex64).op())
    A1 = host(hd.build_coarse_op(sub32, Ud, 1.8, mf, op_dtype=torch.complex64, fast=True).op())
    # the oracle on the basis the GPU stored (FP32 values, evaluated in FP64)
    g = mg.Geometry(L, Ls, block)
    phi = natural(host(sub32.vectors()), L, Ls)
    osub = mg.Subspace(g, mg.to_blocks(g, phi))
    A = mg.coarse_op(U, osub, 1.8, mf, bc)
    assert relerr(A3, A) < 1e-5
    assert relerr(A1, A) < 4e-3
    for leg in range(9):
        assert relerr(A3[:, leg], A[:, leg]) < 1e-4
        assert relerr(A1[:, leg], A[:, leg]) < 1e-2


def test_fp32_build_of_a_complex128_operator_matches_oracle(hd):
    """fp32_build=True: a complex128 basis, the FP32-exact tensor-core build on its
    FP32 rounding, stored as complex128.  Against the oracle on the complex128 basis
    the basis rounding (~1e-7 relative) adds to the three-pass bounds above, which
    still hold; the operator keeps the solve's complex128 interface (a solve with the
    dense coarse inverse reaches 1e-10)."""
    from oracle import dwf, multigrid as mg
    L, Ls, block, bc, mf, nvec = (8, 8, 8, 8), 4, (4, 4, 4, 4), 1, 0.05, 24
    U = synth.gauge_field(L, 0.5, 5600)
    rng = synth.rng(5601)
    lat = hd.Lattice(L, Ls, bc)
    shape = (nvec, lat.V4, 12, Ls)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    sub64 = hd.subspace_from_vectors(lat, block, dev(v), store_dtype=torch.complex128)
    Ud = dev(links(U))
    co = hd.build_coarse_op(sub64, Ud, 1.8, mf, fp32_build=True)
    At = co.op()
    assert At.dtype == torch.complex128
    At = host(At)
    g = mg.Geometry(L, Ls, block)
    phi = natural(host(sub64.vectors()), L, Ls)
    A = mg.coarse_op(U, mg.Subspace(g, mg.to_blocks(g, phi)), 1.8, mf, bc)
    assert relerr(At, A) < 1e-5
    for leg in range(9):
        assert relerr(At[:, leg], A[:, leg]) < 1e-4
    # the FP64 build of the same basis agrees to the same bound
    A64 = host(hd.build_coarse_op(sub64, Ud, 1.8, mf).op())
    assert relerr(At, A64) < 1e-5
    b = synth.gaussian_fermion(L, Ls, 5602)
    x, st = hd.hdcr_solve(co, Ud, dev(planes(b)), tol=1e-10, max_outer=500, restart=16)
    res = np.sqrt(dwf.norm2(b - dwf.apply_H(U, natural(host(x), L, Ls), 1.8, mf, bc)) / dwf.norm2(b))
    assert st["status"] == 0 and res <= 1.01e-10
