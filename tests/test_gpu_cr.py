"""GPU conjugate residual (Section 3) against the oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import dwf
from oracle.krylov import cr
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


def test_cr_fp64_tiny_workload_matches_oracle(hd):
    """4^4 x 8, eps = 0.3, M5 = 1.8, mf = 0.01: unpreconditioned CR to 1e-10."""
    L, Ls = (4, 4, 4, 4), 8
    U = synth.gauge_field(L, 0.3, 1000)
    b = synth.gaussian_fermion(L, Ls, 2000)
    lat = hd.Lattice(L, Ls)
    x, st = hd.cr_solve(lat, dev(links(U)), dev(planes(b)), 1.8, 0.01, tol=1e-10, max_iter=20000)
    assert st["status"] == 0 and st["true_resid"] <= 1e-10
    xg = natural(host(x), L, Ls)
    # the true residual recomputed by the oracle agrees
    r = b - dwf.apply_H(U, xg, 1.8, 0.01)
    assert np.sqrt(dwf.norm2(r) / dwf.norm2(b)) <= 1.01e-10
    xo, io = cr(lambda v: dwf.apply_H(U, v, 1.8, 0.01), b, tol=1e-10, maxiter=40000)
    # both solve the same system: differences are bounded by cond * tol
    assert relerr(xg, xo) < 1e-6



def test_cr_iterates_match_oracle_step_by_step(hd):
    """The same recursion: after k iterations the GPU iterate equals the oracle's
    k-th iterate up to rounding (checked before rounding drift accumulates; over
    ~1000 iterations the counts to reach 1e-10 differ by a few percent)."""
    L, Ls = (4, 4, 4, 4), 8
    U = synth.gauge_field(L, 0.3, 1000)
    b = synth.gaussian_fermion(L, Ls, 2000)
    H = lambda v: dwf.apply_H(U, v, 1.8, 0.01)
    # For an indefinite H with a nearly symmetric spectrum gamma = <r, H r> is a sum
    # with heavy cancellation, so alpha (and the iterate) carry a relative rounding
    # error far above machine epsilon; a wrong sign or term gives O(1) differences.
    for k, tol in ((1, 1e-9), (2, 1e-9), (7, 1e-9), (30, 1e-9)):
        # the not-converged call leaves its k-th iterate in x
        xd = dev(np.zeros_like(planes(b)))
        with pytest.raises(hd.HDCRError) as e:
            hd.cr_solve_into(hd.Lattice(L, Ls), dev(links(U)), dev(planes(b)), xd, 1.8, 0.01,
                             tol=1e-14, max_iter=k)
        assert e.value.status == -3
        xo, _ = cr(H, b, fixed_iters=k)
        assert relerr(natural(host(xd), L, Ls), xo) < tol


def test_cr_fp32_true_residual_is_reported_honestly(hd):
    """FP32 CR: the recursive residual reaches the tolerance while the true residual
    stalls higher (the FP32 residual gap); the reported true residual must be the
    one the oracle measures for the returned x."""
    L, Ls = (4, 4, 4, 4), 8
    U = synth.gauge_field(L, 0.3, 1000)
    b = synth.gaussian_fermion(L, Ls, 2001)
    lat = hd.Lattice(L, Ls)
    U32 = links(U).astype(np.complex64)
    b32 = planes(b).astype(np.complex64)
    x, st = hd.cr_solve(lat, dev(U32), dev(b32), 1.8, 0.01, tol=1e-4, max_iter=20000)
    assert st["status"] == 0
    xg = natural(host(x).astype(np.complex128), L, Ls)
    Ur = U32.astype(np.complex128).reshape(U.shape)
    br = natural(b32.astype(np.complex128), L, Ls)
    true = np.sqrt(dwf.norm2(br - dwf.apply_H(Ur, xg, 1.8, 0.01)) / dwf.norm2(br))
    assert true < 1e-2
    assert abs(st["true_resid"] - true) <= 0.05 * true


def test_cr_reports_non_convergence(hd):
    L, Ls = (4, 4, 4, 4), 4
    U = synth.gauge_field(L, 0.3, 1000)
    b = synth.gaussian_fermion(L, Ls, 2002)
    with pytest.raises(hd.HDCRError) as e:
        hd.cr_solve(hd.Lattice(L, Ls), dev(links(U)), dev(planes(b)), 1.8, 0.01, tol=1e-10, max_iter=3)
    assert e.value.status == -3


def test_cr_reports_nonfinite_source(hd):
    L, Ls = (4, 4, 4, 4), 4
    U = synth.gauge_field(L, 0.3, 1000)
    b = planes(synth.gaussian_fermion(L, Ls, 2003))
    b.reshape(-1)[17] = np.nan
    with pytest.raises(hd.HDCRError) as e:
        hd.cr_solve(hd.Lattice(L, Ls), dev(links(U)), dev(b), 1.8, 0.01, tol=1e-10, max_iter=100)
    assert e.value.status == -4


def test_cr_fp32_on_many_site_groups(hd):
    """FP32 CR (the fused stencil + <r, H r> kernel, which loops over 4d-site groups
    when they outnumber its reduction grid) on a 16^3 x 12 lattice (1536 groups of
    32 sites).  The first iterate x1 = alpha b with alpha = <b, Hb> / |Hb|^2 is
    checked against the FP64 oracle within FP32 rounding amplified by the
    cancellation in <b, Hb> (H is indefinite), and a converged FP32 solve must
    report the true residual the oracle measures (which stalls above the
    recursive residual, the FP32 residual gap)."""
    L, Ls = (16, 16, 16, 12), 4
    U = synth.gauge_field(L, 0.5, 1001)
    b = synth.gaussian_fermion(L, Ls, 2004)
    U32 = links(U).astype(np.complex64)
    b32 = planes(b).astype(np.complex64)
    Ur = U32.astype(np.complex128).reshape(U.shape)
    br = natural(b32.astype(np.complex128), L, Ls)
    lat = hd.Lattice(L, Ls)
    Hb = dwf.apply_H(Ur, br, 1.8, 0.01)
    amp = np.sqrt(dwf.norm2(br) * dwf.norm2(Hb)) / abs(np.vdot(br, Hb).real)
    xd = torch.zeros_like(dev(b32))
    with pytest.raises(hd.HDCRError) as e:
        hd.cr_solve_into(lat, dev(U32), dev(b32), xd, 1.8, 0.01, tol=1e-14, max_iter=1)
    assert e.value.status == -3
    x1 = natural(host(xd).astype(np.complex128), L, Ls)
    alpha = np.vdot(br, Hb).real / dwf.norm2(Hb)
    assert relerr(x1, alpha * br) < 20 * 6e-8 * amp
    x, st = hd.cr_solve(lat, dev(U32), dev(b32), 1.8, 0.01, tol=1e-5, max_iter=20000)
    assert st["status"] == 0
    xg = natural(host(x).astype(np.complex128), L, Ls)
    true = np.sqrt(dwf.norm2(br - dwf.apply_H(Ur, xg, 1.8, 0.01)) / dwf.norm2(br))
    assert true < 1e-2          # FP32 recursion: the true residual stalls above the recursive one
    assert abs(st["true_resid"] - true) <= 0.05 * true
