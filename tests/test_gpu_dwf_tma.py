"""The shared-memory (TMA-staged) FP32 operator, tuner variant 6 (columns of
16 x 4 x 2 sites times one quad of s, marching in t):
bit for bit the same as the L1 kernel (variant 0) for every epilogue -- the plain
application, the fused Re <in, H in> of CR and the fused Chebyshev step of the
filter -- and within the FP32 bound of the oracle.  The lattices cover several
columns and t-chunks per CTA, both walls of the fifth dimension inside and across
quads (Ls = 8 and 16), the antiperiodic time boundary and several right-hand sides."""
import numpy as np
import pytest

import synth
from oracle import dwf
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (L, Ls, bc, variant, nrhs)
CASES = [
    ((16, 8, 4, 6), 16, -1, 6, 2),
    ((16, 4, 2, 4), 8, 1, 6, 1),
    ((16, 4, 4, 8), 8, -1, 6, 3),
    ((16, 16, 16, 16), 16, 1, 6, 1),
]


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


def _forced(hd, v, fn):
    try:
        hd.stencil_tune(1, v)
        return fn()
    finally:
        hd.stencil_tune(1, -1)


@pytest.mark.parametrize("L,Ls,bc,variant,nrhs", CASES)
def test_tma_stencil_matches_l1_kernel_and_oracle(hd, L, Ls, bc, variant, nrhs):
    U = synth.gauge_field(L, 0.5, 8100)
    psi = synth.gaussian_fermion(L, Ls, 8101, count=nrhs)
    lat = hd.Lattice(L, Ls, bc)
    U32 = dev(links(U).astype(np.complex64))
    p32 = dev(planes(psi).astype(np.complex64))
    a = _forced(hd, 0, lambda: host(hd.apply_g5dwf(lat, U32, p32, 1.8, 0.01)))
    b = _forced(hd, variant, lambda: host(hd.apply_g5dwf(lat, U32, p32, 1.8, 0.01)))
    assert np.array_equal(a, b)
    # against the oracle on sampled fields (all of them on the small lattices)
    Ur = links(U).astype(np.complex64).astype(np.complex128).reshape(U.shape)
    pin = natural(host(p32).astype(np.complex128), L, Ls)
    if nrhs == 1:
        pin = pin[None]
    got = natural(b.astype(np.complex128), L, Ls)
    if nrhs == 1:
        got = got[None]
    for r in range(min(nrhs, 2) if lat.V4 > 8192 else nrhs):
        want = dwf.apply_H(Ur, pin[r], 1.8, 0.01, bc)
        assert relerr(got[r], want) <= 1e-6


@pytest.mark.parametrize("L,Ls,bc,variant,nrhs", CASES[:3])
def test_tma_stencil_cr_and_filter_match_l1_kernel(hd, L, Ls, bc, variant, nrhs):
    """FP32 CR (the fused Re <r, H r> epilogue) and the FP32 Chebyshev filter (the fused
    recurrence epilogue) give the same bits with the shared-memory kernel."""
    U = synth.gauge_field(L, 0.5, 8200)
    lat = hd.Lattice(L, Ls, bc)
    Ud = dev(links(U))
    U32 = dev(links(U).astype(np.complex64))
    b = dev(planes(synth.gaussian_fermion(L, Ls, 8201)).astype(np.complex64))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 8202, count=2)))
    block = tuple(2 if L[i] >= 4 else 1 for i in range(4))

    def run():
        x = torch.zeros_like(b)
        try:
            hd.cr_solve_into(lat, U32, b, x, 1.8, 0.05, tol=1e-9, max_iter=40)
        except hd.HDCRError:
            pass  # 40 iterations of FP32 CR: x holds the last iterate
        sub = hd.build_subspace(lat, Ud, noise, 1.8, 0.05, block, kind="chebyshev", order=12,
                                filter_dtype=torch.complex64, store_dtype=torch.complex64)
        v = host(sub.vectors())
        sub.close()
        return host(x), v

    x0, v0 = _forced(hd, 0, run)
    x1, v1 = _forced(hd, variant, run)
    assert np.abs(x0).max() > 0 and np.array_equal(x0, x1)
    assert np.array_equal(v0, v1)
