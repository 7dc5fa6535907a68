"""GPU parity of the fine operator H = Gamma5 D_dwf (Section 3) and its field
utilities against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import dwf
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (L, Ls, bc_t, eps): the tiny 4^4 x 8 workload, a ragged odd lattice spanning several
# thread blocks with a partial last block, and two multi-block cases
CASES = [
    ((4, 4, 4, 4), 8, 1, 0.3),
    ((3, 5, 2, 6), 5, -1, 0.5),
    ((8, 6, 4, 8), 8, -1, 0.5),
    ((6, 4, 4, 10), 16, 1, 0.5),
    ((3, 5, 2, 6), 6, -1, 0.5),   # even Ls on a volume that leaves the last 32-site group ragged
    ((4, 2, 2, 4), 2, 1, 0.5),    # Ls = 2: both domain walls inside one fifth-dimension pair
]


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


def _inputs(L, Ls, eps, seed, count=None):
    U = synth.gauge_field(L, eps, seed)
    psi = synth.gaussian_fermion(L, Ls, seed + 1, count=count)
    return U, psi


@pytest.mark.parametrize("L,Ls,bc,eps", CASES)
def test_apply_fp64_matches_oracle(hd, L, Ls, bc, eps):
    U, psi = _inputs(L, Ls, eps, 1000)
    lat = hd.Lattice(L, Ls, bc)
    out = hd.apply_g5dwf(lat, dev(links(U)), dev(planes(psi)), 1.8, 0.01)
    want = dwf.apply_H(U, psi, 1.8, 0.01, bc)
    assert relerr(natural(host(out), L, Ls), want) <= 1e-13


@pytest.mark.parametrize("L,Ls,bc,eps", CASES)
def test_apply_fp32_matches_oracle(hd, L, Ls, bc, eps):
    U, psi = _inputs(L, Ls, eps, 1100)
    U32 = links(U).astype(np.complex64)
    p32 = planes(psi).astype(np.complex64)
    out = hd.apply_g5dwf(hd.Lattice(L, Ls, bc), dev(U32), dev(p32), 1.8, 0.01)
    # the oracle sees the same FP32-rounded inputs, in FP64
    Ur = U32.astype(np.complex128).reshape(U.shape)
    pr = natural(p32.astype(np.complex128), L, Ls)
    want = dwf.apply_H(Ur, pr, 1.8, 0.01, bc)
    assert relerr(natural(host(out).astype(np.complex128), L, Ls), want) <= 1e-6


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_multi_rhs(hd, dtype):
    L, Ls = (4, 2, 6, 4), 6
    U, psi = _inputs(L, Ls, 0.5, 1200, count=3)
    npdt = np.complex128 if dtype == "c128" else np.complex64
    Ud, pd = links(U).astype(npdt), planes(psi).astype(npdt)
    out = hd.apply_g5dwf(hd.Lattice(L, Ls, -1), dev(Ud), dev(pd), 1.8, 0.05)
    got = natural(host(out).astype(np.complex128), L, Ls)
    Ur = Ud.astype(np.complex128).reshape(U.shape)
    pr = natural(pd.astype(np.complex128), L, Ls)
    for r in range(3):
        want = dwf.apply_H(Ur, pr[r], 1.8, 0.05, -1)
        assert relerr(got[r], want) <= (1e-13 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_full_size_sampled(hd, dtype):
    """16^4 x 16 (the two-level FP64 workload): the whole field on the GPU, checked
    at sampled sites (including every boundary corner class) by the site-wise oracle."""
    L, Ls = (16, 16, 16, 16), 16
    U = synth.gauge_field(L, 0.5, 1300)
    psi = synth.gaussian_fermion(L, Ls, 1301)
    npdt = np.complex128 if dtype == "c128" else np.complex64
    Ud, pd = links(U).astype(npdt), planes(psi).astype(npdt)
    out = host(hd.apply_g5dwf(hd.Lattice(L, Ls, 1), dev(Ud), dev(pd), 1.8, 0.01))
    got = natural(out.astype(np.complex128), L, Ls)
    rng = synth.rng(1302)
    sites = [tuple(int(rng.integers(0, e)) for e in L + (Ls,)) for _ in range(48)]
    sites += [(0, 0, 0, 0, 0), (15, 15, 15, 15, 15), (0, 15, 0, 15, 7), (15, 0, 15, 0, 8)]
    Ur = Ud.astype(np.complex128).reshape(U.shape)
    pr = natural(pd.astype(np.complex128), L, Ls)
    want = dwf.apply_H_at(Ur, pr, sites, 1.8, 0.01, 1)
    g = np.array([got[t, z, y, x, s] for (x, y, z, t, s) in sites])
    assert relerr(g, want) <= (1e-13 if dtype == "c128" else 1e-6)


def test_hermiticity_on_gpu(hd):
    L, Ls = (4, 4, 4, 6), 8
    U = synth.gauge_field(L, 0.5, 1400)
    x = dev(planes(synth.gaussian_fermion(L, Ls, 1401)))
    y = dev(planes(synth.gaussian_fermion(L, Ls, 1402)))
    lat = hd.Lattice(L, Ls, -1)
    Ud = dev(links(U))
    a = hd.cdot(x, hd.apply_g5dwf(lat, Ud, y, 1.8, 0.01))
    b = hd.cdot(hd.apply_g5dwf(lat, Ud, x, 1.8, 0.01), y)
    assert abs(a - b) / abs(a) < 1e-13


def test_gamma5_r5_and_layouts(hd):
    L, Ls = (3, 2, 4, 2), 5
    psi = synth.gaussian_fermion(L, Ls, 1500, count=2)
    lat = hd.Lattice(L, Ls)
    pd = dev(planes(psi))
    g = natural(host(hd.apply_gamma5_r5(lat, pd)), L, Ls)
    for r in range(2):
        assert relerr(g[r], dwf.gamma5_r5(psi[r])) == 0.0
    nat = dev(psi)
    assert np.array_equal(host(hd.pack(lat, nat)), planes(psi))
    assert np.array_equal(host(hd.unpack(lat, pd)), psi)
    c = hd.convert(pd, torch.complex64)
    assert np.array_equal(host(c), planes(psi).astype(np.complex64))


def test_reductions_fp64_deterministic(hd):
    rng = synth.rng(1600)
    n = 1_000_003
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ud, vd = dev(u), dev(v)
    d1 = hd.cdot(ud, vd)
    d2 = hd.cdot(ud, vd)
    assert d1 == d2                                   # bitwise reproducible
    want = np.vdot(u, v)
    assert abs(d1 - want) / abs(want) < 1e-13
    assert abs(hd.norm2(ud) - np.vdot(u, u).real) / np.vdot(u, u).real < 1e-14
    u32 = dev(u.astype(np.complex64))
    assert abs(hd.norm2(u32) - np.vdot(u.astype(np.complex64), u.astype(np.complex64)).real) < 1e-6 * n


def test_apply_fp32_unaligned_fields_take_the_scalar_kernel(hd):
    """The packed two-site FP32 kernel needs 16-byte aligned fields; fields that are
    only 8-byte aligned go to the one-site kernel, and both agree with the oracle."""
    L, Ls, bc = (4, 4, 2, 6), 8, -1
    U, psi = _inputs(L, Ls, 0.5, 1700)
    lat = hd.Lattice(L, Ls, bc)
    U32 = dev(links(U).astype(np.complex64))
    p32 = planes(psi).astype(np.complex64)
    n = p32.size
    buf_in = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
    buf_out = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
    x_off = buf_in[1:]                       # 8 bytes past a 256-byte boundary
    x_off.copy_(dev(p32).reshape(-1))
    y_off = buf_out[1:]
    hd.apply_g5dwf(lat, U32, x_off, 1.8, 0.01, out=y_off)
    y_al = hd.apply_g5dwf(lat, U32, dev(p32), 1.8, 0.01)
    assert x_off.data_ptr() % 16 == 8 and y_al.data_ptr() % 16 == 0
    pr = natural(p32.astype(np.complex128), L, Ls)
    want = dwf.apply_H(links(U).astype(np.complex64).astype(np.complex128).reshape(U.shape), pr, 1.8, 0.01,
                       bc_t=bc)
    got_off = natural(host(y_off).astype(np.complex128).reshape(p32.shape), L, Ls)
    got_al = natural(host(y_al).astype(np.complex128), L, Ls)
    assert relerr(got_off, want) <= 1e-6
    assert relerr(got_al, want) <= 1e-6
    assert relerr(got_al, got_off) <= 1e-6


@pytest.mark.parametrize("Ls", [8, 16])
def test_fp32_tile_variants_identical(hd, Ls):
    """Every tile shape of the FP32 kernel gives the same bits (the tile only changes
    which CTA computes a site), matches the oracle, and the autotuner picks one of them."""
    L = (16, 4, 4, 6)
    U, psi = _inputs(L, Ls, 0.5, 1300)
    U32 = dev(links(U).astype(np.complex64))
    p32 = dev(planes(psi).astype(np.complex64))
    lat = hd.Lattice(L, Ls, -1)
    Ur = links(U).astype(np.complex64).astype(np.complex128).reshape(U.shape)
    want = dwf.apply_H(Ur, natural(host(p32).astype(np.complex128), L, Ls), 1.8, 0.01, -1)
    outs = []
    try:
        for v in range(7):
            hd.stencil_tune(1, v)
            outs.append(host(hd.apply_g5dwf(lat, U32, p32, 1.8, 0.01)))
        hd.stencil_tune(2, -1)
        tuned = host(hd.apply_g5dwf(lat, U32, p32, 1.8, 0.01))
        info = hd.stencil_tune_info(lat)
    finally:
        hd.stencil_tune(1, -1)
    assert relerr(natural(outs[0].astype(np.complex128), L, Ls), want) <= 1e-6
    for v, o in enumerate(outs):
        assert np.array_equal(o, outs[0]), f"tile variant {v} differs"
    assert np.array_equal(tuned, outs[0])
    assert 0 <= info["variant"] < 7 and info["us"][info["variant"]] > 0
    assert all(u > 0 for u in info["us"][:6])  # every tile divides this lattice
    assert info["us"][6] > 0                   # the shared-memory column 16 x 4 x 2 fits too
    assert all(u == -1 for u in info["us"][7:])
