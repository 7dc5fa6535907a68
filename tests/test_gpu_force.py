"""GPU gauge force and the differentiable HDCR solve against the FP64 oracle and
against central finite differences."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import dwf, force
from oracle.krylov import cr
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M5 = 1.8


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-13), ("c64", 1e-5)])
@pytest.mark.parametrize("L,Ls,bc", [((4, 4, 2, 6), 4, -1), ((3, 2, 4, 4), 5, 1)])
def test_force_kernel_matches_oracle(hd, dtype, tol, L, Ls, bc):
    x = synth.gaussian_fermion(L, Ls, 4000)
    w = synth.gaussian_fermion(L, Ls, 4001)
    npdt = np.complex128 if dtype == "c128" else np.complex64
    xd, wd = planes(x).astype(npdt), planes(w).astype(npdt)
    F = host(hd.gauge_force(hd.Lattice(L, Ls, bc), dev(xd), dev(wd))).astype(np.complex128)
    want = force.gauge_force(np.zeros((4,) + synth.lattice_shape(L) + (3, 3), complex),
                             natural(xd.astype(np.complex128), L, Ls), natural(wd.astype(np.complex128), L, Ls), bc)
    assert relerr(F, want.reshape(F.shape)) < tol
    # the gradient layout: G[mu, x4, a, b] = conj(F_ba)
    G = host(hd.gauge_grad(hd.Lattice(L, Ls, bc), dev(xd), dev(wd))).astype(np.complex128)
    assert relerr(G, np.conj(np.swapaxes(want, -1, -2)).reshape(G.shape)) < tol


def _loss_and_grad(hd, lat, U, b, eta, noise, block, nvec_kw):
    Ut = dev(links(U)).requires_grad_(True)
    bt = dev(planes(b)).requires_grad_(True)
    x = hd.solve_autograd(lat, Ut, bt, dev(planes(noise)), M5, 0.05, block,
                          filter_kw=nvec_kw, solve_kw=dict(tol=1e-12, max_outer=500))
    loss = torch.vdot(dev(planes(eta)).reshape(-1), x.reshape(-1)).real
    loss.backward()
    return float(loss.detach()), host(Ut.grad), host(bt.grad)


def test_autograd_matches_oracle_gradient(hd):
    """4^4 x 8: d Re(eta^dag x) / dU and / db from the GPU backward (adjoint HDCR solve +
    force kernel) against the oracle's gradient from tightly converged CR solves."""
    L, Ls, block = (4, 4, 4, 4), 8, (2, 2, 2, 2)
    U = synth.gauge_field(L, 0.3, 5000)
    b = synth.gaussian_fermion(L, Ls, 5001)
    eta = synth.gaussian_fermion(L, Ls, 5002)
    noise = synth.gaussian_fermion(L, Ls, 5003, count=4)
    lat = hd.Lattice(L, Ls)
    loss, gU, gb = _loss_and_grad(hd, lat, U, b, eta, noise, block, dict(kind="chebyshev", order=60))
    H = lambda v: dwf.apply_H(U, v, M5, 0.05)
    x, _ = cr(H, b, tol=1e-13, maxiter=100000)
    y, _ = cr(H, eta, tol=1e-13, maxiter=100000)
    gU_o, gb_o = force.solve_gradient(U, x, y)
    assert abs(loss - np.vdot(eta, x).real) < 1e-9 * abs(loss)
    assert relerr(gU, gU_o.reshape(gU.shape)) < 1e-6
    assert relerr(natural(gb, L, Ls), gb_o) < 1e-6


def test_autograd_vs_finite_differences(hd):
    """8^3 x 16, Ls = 8 (the differentiation workload), complex128: central
    differences with h = 1e-6 along U -> exp(i h T) U on 20 random links agree with
    the backward's gradient to 1e-6 relative.

    The loss Re(eta^dag x) is O(1e3) while its derivative is O(1), so the
    difference is taken of the corrections: with x0 the solution at U,
    x(U') = x0 + d with H(U') d = b - H(U') x0, and
    L(U+) - L(U-) = Re eta^dag (d+ - d-); the large common part cancels exactly and
    the corrections need only a moderate relative tolerance."""
    L, Ls, block, mf = (8, 8, 8, 16), 8, (4, 4, 4, 4), 0.05
    U = synth.gauge_field(L, 0.5, 6000)
    b = synth.gaussian_fermion(L, Ls, 6001)
    eta = synth.gaussian_fermion(L, Ls, 6002)
    noise = synth.gaussian_fermion(L, Ls, 6003, count=8)
    lat = hd.Lattice(L, Ls)
    Ut = dev(links(U)).requires_grad_(True)
    x = hd.solve_autograd(lat, Ut, dev(planes(b)), dev(planes(noise)), M5, mf, block,
                          filter_kw=dict(kind="chebyshev", order=100),
                          solve_kw=dict(tol=1e-12, max_outer=500))
    etad = dev(planes(eta)).reshape(-1)
    torch.vdot(etad, x.reshape(-1)).real.backward()
    F = np.conj(np.swapaxes(host(Ut.grad), -1, -2))          # grad_U = F^dag
    bd = dev(planes(b))
    x0, _ = hd.cr_solve(lat, dev(links(U)), bd, M5, mf, tol=1e-12, max_iter=200000)

    def dloss(Ua):
        Ud = dev(Ua)
        r = bd - hd.apply_g5dwf(lat, Ud, x0, M5, mf)
        d, _ = hd.cr_solve(lat, Ud, r.contiguous(), M5, mf, tol=1e-9, max_iter=200000)
        return float(torch.vdot(etad, d.reshape(-1)).real)

    rng = synth.rng(6004)
    Ul = links(U)
    h = 1e-6
    for _ in range(20):
        mu = int(rng.integers(4))
        x4 = int(rng.integers(Ul.shape[1]))
        G = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        T = 0.5 * (G + G.conj().T)
        T -= np.trace(T) / 3 * np.eye(3)
        w_, V = np.linalg.eigh(T)
        E = lambda s: (V * np.exp(1j * s * h * w_)) @ V.conj().T
        Up, Um = Ul.copy(), Ul.copy()
        Up[mu, x4] = E(1) @ Ul[mu, x4]
        Um[mu, x4] = E(-1) @ Ul[mu, x4]
        fd = (dloss(Up) - dloss(Um)) / (2 * h)
        an = np.trace(1j * T @ Ul[mu, x4] @ F[mu, x4]).real
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(F).max()), (mu, x4, fd, an)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grad_8x8x8x16_ls8.json")


@pytest.mark.parametrize("dtype,tol,bound", [("c128", 1e-12, 1e-6), ("c64", 1e-7, 1e-4)])
def test_autograd_differentiation_workload_matches_oracle(hd, dtype, tol, bound):
    """The differentiation workload (8^3 x 16, Ls = 8) in complex128 and complex64:
    the backward's dL/dU and dL/db on a seeded sample of links and components against
    the oracle's gradient from CR converged to 1e-13 (tests/golden, written by
    make_grad_golden.py from the oracle alone).  complex64: inputs, outputs and the
    force kernel in FP32, V-cycle in FP32, outer iteration in FP64 to 1e-7; the error
    against the FP64 oracle is printed and must stay below 1e-4 (about 1700 FP32 roundings
    of 2^-24; 6e-6 is measured); complex128 must agree to 1e-6."""
    with open(GOLDEN) as f:
        gd = json.load(f)
    L, Ls, mf = tuple(gd["lattice"]), gd["Ls"], gd["mf"]
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    U = synth.gauge_field(L, gd["eps"], gd["seeds"]["U"])
    b = synth.gaussian_fermion(L, Ls, gd["seeds"]["b"])
    eta = synth.gaussian_fermion(L, Ls, gd["seeds"]["eta"])
    noise = synth.gaussian_fermion(L, Ls, 6003, count=8)
    lat = hd.Lattice(L, Ls, gd["bc_t"])
    Ut = dev(links(U), tdt).requires_grad_(True)
    bt = dev(planes(b), tdt).requires_grad_(True)
    x = hd.solve_autograd(lat, Ut, bt, dev(planes(noise)), gd["M5"], mf, (4, 4, 4, 4),
                          filter_kw=dict(kind="chebyshev", order=100),
                          solve_kw=dict(tol=tol, max_outer=500))
    assert x.dtype == tdt
    loss = torch.vdot(dev(planes(eta), tdt).reshape(-1), x.reshape(-1)).real
    loss.backward()
    assert Ut.grad.dtype == tdt and bt.grad.dtype == tdt
    gU = host(Ut.grad).astype(np.complex128)
    gb = host(bt.grad).astype(np.complex128)
    got = np.array([gU[mu, x4].reshape(-1) for mu, x4, _ in gd["links"]])
    want = np.array([[complex(r, i) for r, i in v] for _, _, v in gd["links"]])
    gotb = np.array([gb[x4, c, s] for x4, c, s, _, _ in gd["grad_b"]])
    wantb = np.array([complex(r, i) for _, _, _, r, i in gd["grad_b"]])
    eU, eb = relerr(got, want), relerr(gotb, wantb)
    el = abs(float(loss.detach()) - gd["loss"]) / abs(gd["loss"])
    print(f"{dtype}: gradient error vs FP64 oracle: dL/dU {eU:.2e}, dL/db {eb:.2e}, loss {el:.2e}")
    assert eU < bound and eb < bound and el < bound
