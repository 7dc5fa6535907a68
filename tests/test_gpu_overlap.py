"""The continued-fraction overlap operator of Section 3 on the GPU against the oracle
(oracle/overlap.py): the application in FP64 and FP32 for the printed five-component
form and for three and seven components, and CR on it to a true residual of 1e-10
recomputed by the oracle."""
import numpy as np
import pytest

import synth
from oracle import overlap as ov
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M5 = 1.8


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


@pytest.mark.parametrize("beta,R,L,bc", [((1.3, 0.9, 1.7, 0.6), 0.35, (4, 4, 4, 4), 1),
                                         ((0.8, 1.2), -0.2, (6, 4, 2, 4), -1),
                                         ((1.1, 0.7, 1.9, 0.5, 1.4, 0.8), 0.5, (4, 2, 4, 6), 1)])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-13), ("c64", 1e-6)])
def test_cf_overlap_matches_oracle(hd, beta, R, L, bc, dtype, tol):
    n = len(beta) + 1
    U = synth.gauge_field(L, 0.5, 9000)
    psi = synth.gaussian_fermion(L, n, 9001, count=2)
    lat = hd.Lattice(L, n, bc)
    npdt = np.complex128 if dtype == "c128" else np.complex64
    Ud = links(U).astype(npdt)
    pd = planes(psi).astype(npdt)
    got = natural(host(hd.apply_cf_overlap(lat, dev(Ud), dev(pd), M5, beta, R)).astype(np.complex128), L, n)
    Ur = Ud.astype(np.complex128).reshape(U.shape)
    pr = natural(pd.astype(np.complex128), L, n)
    for r in range(2):
        assert relerr(got[r], ov.apply_cf(Ur, pr[r], M5, beta, R, bc)) < tol


def test_cf_overlap_cr_solve(hd):
    L, beta, R = (4, 4, 4, 8), (1.3, 0.9, 1.7, 0.6), 0.35
    n = len(beta) + 1
    U = synth.gauge_field(L, 0.3, 9100)
    b = synth.gaussian_fermion(L, n, 9101)
    lat = hd.Lattice(L, n)
    x, st = hd.cf_cr_solve(lat, dev(links(U)), dev(planes(b)), M5, beta, R, tol=1e-10)
    xg = natural(host(x), L, n)
    res = np.sqrt(np.vdot(b - ov.apply_cf(U, xg, M5, beta, R), b - ov.apply_cf(U, xg, M5, beta, R)).real /
                  np.vdot(b, b).real)
    assert st["status"] == 0 and res <= 1.01e-10 and abs(res - st["true_resid"]) < 1e-11
