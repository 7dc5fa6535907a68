"""FP16 storage of the fermion fields (half2 per complex number, one FP32 scale per
5d site) and the FP32 operator H = Gamma5 D_dwf (Section 3) on it, against the FP64
oracle through the C ABI.  Bounds: a stored half is rounded to 2^-11 of its site's
largest |re|, |im| (the scale), so a decoded component is good to that much; the
operator's output is re-encoded the same way, after FP32 arithmetic (~1e-6)."""
import numpy as np
import pytest

import synth
from oracle import dwf
from gpu_util import dev, host, links, natural, planes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HALF_ULP = 2.0 ** -11


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


CASES = [((4, 4, 4, 4), 8, 1), ((6, 4, 4, 10), 16, -1), ((3, 5, 2, 6), 6, -1)]


def _site_max(a, L, Ls):
    """largest |re|, |im| of every 5d site of natural-layout fields (..., Lt,Lz,Ly,Lx,Ls,4,3)."""
    r = np.maximum(np.abs(a.real), np.abs(a.imag))
    return r.max(axis=(-1, -2))


@pytest.mark.parametrize("L,Ls,bc", CASES)
def test_h16_roundtrip(hd, L, Ls, bc):
    lat = hd.Lattice(L, Ls, bc)
    psi = synth.gaussian_fermion(L, Ls, 6100, count=2)
    psi[1] *= 1e-12  # the scale carries the magnitude: tiny fields keep their relative accuracy
    for dt in (torch.complex128, torch.complex64):
        buf = hd.encode_h16(lat, dev(planes(psi)).to(dt))
        assert buf.shape == (2, 52 * lat.V5)
        back = natural(host(hd.decode_h16(lat, buf, torch.complex128)), L, Ls)
        err = np.maximum(np.abs((back - psi).real), np.abs((back - psi).imag)).max(axis=(-1, -2))
        assert np.all(err <= HALF_ULP * _site_max(psi, L, Ls) * 1.001 + 1e-30)


@pytest.mark.parametrize("L,Ls,bc", CASES)
def test_h16_apply_matches_oracle(hd, L, Ls, bc):
    lat = hd.Lattice(L, Ls, bc)
    U = synth.gauge_field(L, 0.5, 6200)
    U32 = links(U).astype(np.complex64)
    psi = synth.gaussian_fermion(L, Ls, 6201, count=3)
    buf = hd.encode_h16(lat, dev(planes(psi)))
    out = hd.apply_g5dwf_h16(lat, dev(U32), buf, 1.8, 0.01)
    # the oracle on exactly what the kernel read: the decoded input and the FP32 links
    xin = natural(host(hd.decode_h16(lat, buf, torch.complex128)), L, Ls)
    want = dwf.apply_H(U32.astype(np.complex128).reshape(U.shape), xin, 1.8, 0.01, bc)
    got = natural(host(hd.decode_h16(lat, out, torch.complex128)), L, Ls)
    m = _site_max(want, L, Ls)
    err = np.maximum(np.abs((got - want).real), np.abs((got - want).imag)).max(axis=(-1, -2))
    assert np.all(err <= (HALF_ULP * 1.001 + 2e-6) * m + 1e-6 * m.max())
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-3
    # the same fields one at a time give the same bits
    per = 52 * lat.V5
    for r in range(3):
        one = hd.apply_g5dwf_h16(lat, dev(U32), buf.reshape(-1)[r * per:(r + 1) * per].contiguous(), 1.8, 0.01)
        assert torch.equal(one.reshape(-1), out.reshape(-1)[r * per:(r + 1) * per])


def test_h16_agrees_with_fp32_kernel(hd):
    """FP16 storage and the FP32 kernel on the same (decoded) input: the difference is the
    output's FP16 rounding."""
    L, Ls = (8, 6, 4, 8), 16
    lat = hd.Lattice(L, Ls, 1)
    U32 = dev(links(synth.gauge_field(L, 0.5, 6300)).astype(np.complex64))
    buf = hd.encode_h16(lat, dev(planes(synth.gaussian_fermion(L, Ls, 6301))))
    x32 = hd.decode_h16(lat, buf, torch.complex64)
    y32 = natural(host(hd.apply_g5dwf(lat, U32, x32, 1.8, 0.01)).astype(np.complex128), L, Ls)
    y16 = natural(host(hd.decode_h16(lat, hd.apply_g5dwf_h16(lat, U32, buf, 1.8, 0.01), torch.complex128)), L, Ls)
    m = _site_max(y32, L, Ls)
    err = np.maximum(np.abs((y16 - y32).real), np.abs((y16 - y32).imag)).max(axis=(-1, -2))
    assert np.all(err <= (HALF_ULP * 1.001 + 1e-6) * m)


def test_h16_rejects_odd_ls(hd):
    L, Ls = (4, 4, 4, 4), 5
    lat = hd.Lattice(L, Ls, 1)
    U32 = dev(links(synth.gauge_field(L, 0.5, 6400)).astype(np.complex64))
    buf = hd.encode_h16(lat, dev(planes(synth.gaussian_fermion(L, Ls, 6401))))
    with pytest.raises(hd.HDCRError) as e:
        hd.apply_g5dwf_h16(lat, U32, buf, 1.8, 0.01)
    assert e.value.status == -1
