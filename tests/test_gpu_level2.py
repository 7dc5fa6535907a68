"""The third level (recursion of Section 5 on the coarse operator) on the GPU against
the oracle (oracle/level2.py): the level-2 basis from the same coarse noise, A2 on the
basis the GPU built, the recursive coarse solve against LU, and an HDCR solve that
uses it to a true residual of 1e-10 recomputed by the oracle."""
import numpy as np
import pytest

import synth
from oracle import dwf, level2 as l2, multigrid as mg
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M5 = 1.8


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


def _setup(hd, dtype, L=(8, 8, 8, 8), Ls=4, block=(2, 2, 2, 2), nvec=8, mf=0.05, seed=1500):
    g = mg.Geometry(L, Ls, block)
    U = synth.gauge_field(L, 0.5, seed)
    sub = mg.build_subspace(U, synth.gaussian_fermion(L, Ls, seed + 1, count=nvec // 2), g, M5, mf,
                            smooth_iters=10)
    lat = hd.Lattice(L, Ls)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    gsub = hd.subspace_from_vectors(lat, block, dev(planes(mg.from_blocks(g, sub.Phi))), store_dtype=tdt)
    co = hd.build_coarse_op(gsub, dev(links(U)), M5, mf, op_dtype=tdt)
    return g, U, lat, gsub, co


@pytest.mark.parametrize("dtype,tol_basis,tol_op", [("c128", 1e-10, 1e-12), ("c64", 1e-3, 1e-5)])
def test_level2_basis_and_operator_match_oracle(hd, dtype, tol_basis, tol_op):
    """The basis: FP64 agrees to rounding; in FP32 the six CR smoothing steps amplify the
    FP32 rounding (as for the fine subspace's FP32 filter), so 1e-3.  A2 is compared on
    the basis the GPU stored."""
    g, U, lat, gsub, co = _setup(hd, dtype)
    A = host(co.op())                                  # the GPU's level-1 operator (checked elsewhere)
    gc = l2.CoarseGeometry(g.Lc, 8, (2, 2, 2, 2))
    rng = synth.rng(1600)
    noise = rng.standard_normal((4, gc.Vc, 8)) + 1j * rng.standard_normal((4, gc.Vc, 8))
    hd.build_level2(co, dev(noise), (2, 2, 2, 2), smooth_iters=6, cycle_smooth=4)
    vec, op = hd.level2_get(co)
    vec, op = host(vec), host(op)
    want_phi = l2.from_blocks(gc, l2.build_level2(A, gc, noise, smooth_iters=6))
    for k in range(8):
        assert relerr(vec[k], want_phi[k]) < tol_basis, k
    # A2 from the basis the GPU stored, leg by leg
    A2 = l2.level2_op(A, gc, l2.to_blocks(gc, vec))
    assert relerr(op, A2) < tol_op
    for leg in range(9):
        assert relerr(op[:, leg], A2[:, leg]) < 10 * tol_op


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-10), ("c64", 1e-5)])
def test_recursive_coarse_solve_matches_lu(hd, dtype, tol):
    g, U, lat, gsub, co = _setup(hd, dtype)
    gc = l2.CoarseGeometry(g.Lc, 8, (2, 2, 2, 2))
    rng = synth.rng(1700)
    noise = rng.standard_normal((4, gc.Vc, 8)) + 1j * rng.standard_normal((4, gc.Vc, 8))
    hd.build_level2(co, dev(noise), (2, 2, 2, 2), smooth_iters=6, cycle_smooth=4)
    A = host(co.op())
    D = mg.coarse_dense(A, mg.Geometry(g.L, g.Ls, g.block))
    b = rng.standard_normal((gc.Vc, 8)) + 1j * rng.standard_normal((gc.Vc, 8))
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    x, it = hd.coarse_solve_level2(co, dev(b, tdt), tol=tol, max_iter=200)
    want = np.linalg.solve(D, b.ravel()).reshape(b.shape)
    xg = host(x).astype(np.complex128)
    cond = np.linalg.cond(D)
    assert relerr(xg, want) < 10 * cond * tol
    assert np.linalg.norm(D @ xg.ravel() - b.ravel()) <= 2 * tol * np.linalg.norm(b) + 1e-6 * (dtype == "c64")
    print(f"{dtype}: recursive coarse solve {it} iterations, condition number {cond:.1f}")


@pytest.mark.parametrize("inner", ["c128", "c64"])
def test_hdcr_solve_with_recursive_coarse_solve(hd, inner):
    """8^4 x 8 with 2^4 blocks (4^4 coarse lattice, 2048 coarse unknowns) and a 2^4
    level-2 lattice: the FP64 flexible GCR with the V-cycle whose coarse solve is the
    recursive one reaches a true residual of 1e-10, recomputed by the oracle."""
    L, Ls, mf = (8, 8, 8, 8), 8, 0.01
    lat = hd.Lattice(L, Ls)
    Uh = synth.gauge_field(L, 0.5, 1800)
    U = dev(links(Uh))
    tdt = torch.complex128 if inner == "c128" else torch.complex64
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 1801, count=12)))
    sub = hd.build_subspace(lat, U, noise, M5, mf, (2, 2, 2, 2), kind="chebyshev", order=100, lam_cut=0.5,
                            store_dtype=tdt)
    co = hd.build_coarse_op(sub, U, M5, mf, op_dtype=tdt)
    rng = synth.rng(1802)
    n2 = rng.standard_normal((24, sub.Vc, 24)) + 1j * rng.standard_normal((24, sub.Vc, 24))
    hd.build_level2(co, dev(n2), (2, 2, 2, 2), smooth_iters=50, cycle_smooth=8)
    b = synth.gaussian_fermion(L, Ls, 1803)
    x, st = hd.hdcr_solve(co, U, dev(planes(b)), tol=1e-10, max_outer=100, restart=16, coarse_solver="recursive",
                          coarse_tol=1e-6, coarse_max=100, inner_dtype=tdt)
    xg = natural(host(x), L, Ls)
    res = np.sqrt(dwf.norm2(b - dwf.apply_H(Uh, xg, M5, mf)) / dwf.norm2(b))
    print(f"{inner}: HDCR with the recursive coarse solve: {st['iters']} outer iterations, "
          f"{st['coarse_matvecs']} coarse GCR iterations, true residual {res:.2e}")
    assert st["status"] == 0 and res <= 1.01e-10
    # the recursive coarse solve reaches its tolerance instead of running to its cap
    assert st["coarse_matvecs"] < 50 * st["iters"]
