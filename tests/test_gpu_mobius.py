"""The Moebius domain-wall operator with c5 = 0 (b5 D_W + D_5; Section 3's Shamir
operator is b5 = 1) through the library, against the oracle's own definition of
it: the operator in FP64 and FP32, and the CR and red-black CGNE solves of its
system, each certified by the oracle."""
import numpy as np
import pytest

import synth
from oracle import dwf
from oracle.krylov import cr
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M5 = 1.8


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


@pytest.mark.parametrize("b5", [0.7, 1.5])
def test_mobius_operator_matches_oracle(hd, b5):
    L, Ls, mf, bc = (4, 4, 2, 6), 8, 0.02, -1
    U = synth.gauge_field(L, 0.5, 9300)
    psi = synth.gaussian_fermion(L, Ls, 9301)
    lat = hd.Lattice(L, Ls, bc)
    want = dwf.apply_H_mobius(U, psi, M5, mf, b5, bc)
    Ub, M5s, mfs = hd.mobius_to_shamir(dev(links(U)), M5, mf, b5)
    assert abs(M5s - (4 - b5 * (4 - M5))) < 1e-15 and mfs == mf
    out = hd.apply_g5dwf(lat, Ub, dev(planes(psi)), M5s, mfs)
    assert relerr(natural(host(out), L, Ls), want) <= 1e-13
    # FP32: the oracle sees the FP32-rounded links and field
    U32 = links(U).astype(np.complex64)
    p32 = planes(psi).astype(np.complex64)
    Ub32, M5s, mfs = hd.mobius_to_shamir(dev(U32), M5, mf, b5)
    out32 = hd.apply_g5dwf(lat, Ub32, dev(p32), M5s, mfs)
    want32 = dwf.apply_H_mobius(U32.astype(np.complex128).reshape(U.shape),
                                natural(p32.astype(np.complex128), L, Ls), M5, mf, b5, bc)
    assert relerr(natural(host(out32).astype(np.complex128), L, Ls), want32) <= 1e-6


def test_mobius_solves_match_oracle(hd):
    L, Ls, mf, b5 = (4, 4, 4, 4), 8, 0.05, 1.5
    lat = hd.Lattice(L, Ls)
    Uh = synth.gauge_field(L, 0.3, 9400)
    b = synth.gaussian_fermion(L, Ls, 9401)
    Ub, M5s, mfs = hd.mobius_to_shamir(dev(links(Uh)), M5, mf, b5)
    bd = dev(planes(b))
    H = lambda v: dwf.apply_H_mobius(Uh, v, M5, mf, b5)
    xo, info = cr(H, b, tol=1e-12, maxiter=50000)
    assert info.converged

    def check(x, name):
        xg = natural(host(x), L, Ls)
        res = np.sqrt(dwf.norm2(b - H(xg)) / dwf.norm2(b))
        assert res <= 1.01e-10, (name, res)
        assert relerr(xg, xo) < 1e-6, name

    x, st = hd.cr_solve(lat, Ub, bd, M5s, mfs, tol=1e-10)
    check(x, "cr")
    x, st = hd.cgne_rb_solve(lat, Ub, bd, M5s, mfs, tol=1e-10)
    check(x, "cgne_rb")


def test_mobius_hdcr_solve_with_scaled_windows(hd):
    """HDCR on the Moebius operator (b5 = 2 through the Shamir form): b5 stretches the
    spectrum of H, so the filter's upper edge (8 b5) and the smoother's window
    ([b5^2, 64 b5^2] on H^2) are scaled with it; the solve then reaches a true
    residual of 1e-10 of the oracle's Moebius operator (8^4 x 8, 4^4 blocks, nvec 24,
    about 27 outer iterations)."""
    L, Ls, mf, b5 = (8, 8, 8, 8), 8, 0.01, 2.0
    lat = hd.Lattice(L, Ls)
    Uh = synth.gauge_field(L, 0.5, 1900)
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 1901, count=12)))
    b = synth.gaussian_fermion(L, Ls, 1903)
    Ub, M5s, mfs = hd.mobius_to_shamir(dev(links(Uh)), M5, mf, b5)
    sub = hd.build_subspace(lat, Ub, noise, M5s, mfs, (4, 4, 4, 4), kind="chebyshev", order=200,
                            lam_cut=0.5 * b5, lam_max=8.0 * b5)
    co = hd.build_coarse_op(sub, Ub, M5s, mfs)
    x, st = hd.hdcr_solve(co, Ub, dev(planes(b)), tol=1e-10, max_outer=100, restart=8,
                          cheb_lo=b5 * b5, cheb_hi=64.0 * b5 * b5)
    xg = natural(host(x), L, Ls)
    res = np.sqrt(dwf.norm2(b - dwf.apply_H_mobius(Uh, xg, M5, mf, b5)) / dwf.norm2(b))
    assert st["status"] == 0 and res <= 1.01e-10
    assert st["iters"] < 60


def test_mobius_rejects_bad_scale(hd):
    U = dev(links(synth.gauge_field((2, 2, 2, 2), 0.5, 9500)))
    with pytest.raises(hd.HDCRError) as e:
        hd.mobius_to_shamir(U, M5, 0.01, 0.0)
    assert e.value.status == -1
