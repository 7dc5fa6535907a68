"""GPU parity of red-black CGNE (the comparison solver of Section 5, Table 1)
against the oracle's own red-black CGNE and the oracle's H, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import dwf
from oracle import redblack as rb
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


@pytest.mark.parametrize("L,Ls,bc,mf", [((4, 2, 2, 4), 8, -1, 0.05), ((4, 4, 4, 4), 16, 1, 0.01)])
def test_cgne_rb_matches_oracle(hd, L, Ls, bc, mf):
    U = synth.gauge_field(L, 0.5, 8400)
    b = synth.gaussian_fermion(L, Ls, 8401)
    lat = hd.Lattice(L, Ls, bc)
    x, st = hd.cgne_rb_solve(lat, dev(links(U)), dev(planes(b)), 1.8, mf, tol=1e-12)
    xg = natural(host(x), L, Ls)
    res = np.sqrt(dwf.norm2(b - dwf.apply_H(U, xg, 1.8, mf, bc)) / dwf.norm2(b))
    assert st["status"] == 0 and res <= 2e-12 and abs(st["true_resid"] - res) <= 1e-3 * res + 1e-15
    xo, it, res_o = rb.cgne_rb_solve(U, b, 1.8, mf, bc, tol=1e-12)
    assert res_o <= 2e-12
    assert relerr(xg, xo) <= 1e-9
    # the same Krylov method: iteration counts within a few (checked every 4 on the GPU)
    assert abs(st["iters"] - it) <= 6


def test_cgne_rb_solution_equals_cr_solution(hd):
    """The two comparison solvers (red-black CGNE and plain CR on H) reach the same
    solution (8^4 x 8), each certified by the oracle's H."""
    L, Ls, mf = (8, 8, 8, 8), 8, 0.05
    U = synth.gauge_field(L, 0.3, 8500)
    b = synth.gaussian_fermion(L, Ls, 8501)
    lat = hd.Lattice(L, Ls, 1)
    Ud, bd = dev(links(U)), dev(planes(b))
    x1, st1 = hd.cgne_rb_solve(lat, Ud, bd, 1.8, mf, tol=1e-11)
    x2, st2 = hd.cr_solve(lat, Ud, bd, 1.8, mf, tol=1e-11, max_iter=100000)
    for x in (x1, x2):
        res = np.sqrt(dwf.norm2(b - dwf.apply_H(U, natural(host(x), L, Ls), 1.8, mf)) / dwf.norm2(b))
        assert res <= 1.01e-11
    assert float(torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x2)) < 1e-8


def test_cgne_rb_rejects_odd_extent(hd):
    L, Ls = (3, 4, 4, 4), 4
    U = dev(links(synth.gauge_field(L, 0.5, 8600)))
    b = dev(planes(synth.gaussian_fermion(L, Ls, 8601)))
    with pytest.raises(hd.HDCRError) as e:
        hd.cgne_rb_solve(hd.Lattice(L, Ls), U, b, 1.8, 0.05)
    assert e.value.status == -2
