"""Pins for the oracle gauge force: central finite differences of
L(U) = Re(eta^dag H(U)^{-1} b) along U_mu(x) -> exp(i h T) U_mu(x)."""
import numpy as np
import pytest

import synth
from oracle import dwf, force
from oracle.krylov import cr
from pins import dense_H_from_stencil, relerr

M5, MF = 1.8, 0.05


def gell_mann():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l / 2


def _loss(U, b, eta, Ls, bc_t):
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF, bc_t)
    x = np.linalg.solve(Hd, b.ravel())
    return float(np.vdot(eta.ravel(), x).real)


def _expiT(T, h):
    w, V = np.linalg.eigh(T)
    return (V * np.exp(1j * h * w)) @ V.conj().T


@pytest.mark.parametrize("bc_t", [1, -1])
def test_force_matches_central_differences(bc_t):
    L, Ls = (2, 2, 2, 2), 4
    U = synth.gauge_field(L, 0.5, 500)
    b = synth.gaussian_fermion(L, Ls, 501)
    eta = synth.gaussian_fermion(L, Ls, 502)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF, bc_t)
    x = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    y = np.linalg.solve(Hd, eta.ravel()).reshape(b.shape)
    F = force.gauge_force(U, x, dwf.gamma5_r5(y), bc_t)
    rng = synth.rng(503)
    links = [(int(rng.integers(4)), tuple(int(v) for v in rng.integers(0, 2, 4))) for _ in range(3)]
    links.append((3, (1, 0, 1, 1)))                 # a t-link across the boundary (t = Lt-1)
    T8 = gell_mann()
    h = 1e-5
    for mu, (t, z, yy, xx) in links:
        for T in T8[[1, 7]]:
            Up, Um = U.copy(), U.copy()
            Up[mu, t, z, yy, xx] = _expiT(T, h) @ U[mu, t, z, yy, xx]
            Um[mu, t, z, yy, xx] = _expiT(T, -h) @ U[mu, t, z, yy, xx]
            fd = (_loss(Up, b, eta, Ls, bc_t) - _loss(Um, b, eta, Ls, bc_t)) / (2 * h)
            an = np.trace(1j * T @ U[mu, t, z, yy, xx] @ F[mu, t, z, yy, xx]).real
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(F).max())


def test_force_random_direction_all_links():
    """One directional derivative moving every link at once."""
    L, Ls = (2, 2, 2, 2), 4
    U = synth.gauge_field(L, 0.5, 510)
    b = synth.gaussian_fermion(L, Ls, 511)
    eta = synth.gaussian_fermion(L, Ls, 512)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF)
    x = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    y = np.linalg.solve(Hd, eta.ravel()).reshape(b.shape)
    F = force.gauge_force(U, x, dwf.gamma5_r5(y))
    rng = synth.rng(513)
    G = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    T = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    h = 1e-5
    E = lambda s: np.stack([[_expiT(Tm, s * h) for Tm in Tmu.reshape(-1, 3, 3)] for Tmu in T]).reshape(U.shape)
    Up, Um = E(1) @ U, E(-1) @ U
    fd = (_loss(Up, b, eta, Ls, 1) - _loss(Um, b, eta, Ls, 1)) / (2 * h)
    an = np.einsum("...ab,...bc,...ca->...", 1j * T, U, F).sum().real
    assert abs(fd - an) <= 1e-6 * abs(fd)


def test_solve_gradient_torch_convention_and_cr_solves():
    """grad_U = F^dag satisfies dL = Re sum conj(grad_U) dU, and the gradient from
    tightly converged CR solves equals the one from dense solves."""
    L, Ls = (2, 2, 2, 2), 4
    U = synth.gauge_field(L, 0.5, 520)
    b = synth.gaussian_fermion(L, Ls, 521)
    eta = synth.gaussian_fermion(L, Ls, 522)
    H = lambda v: dwf.apply_H(U, v, M5, MF)
    x, _ = cr(H, b, tol=1e-14, maxiter=20000)
    y, _ = cr(H, eta, tol=1e-14, maxiter=20000)
    gU, gb = force.solve_gradient(U, x, y)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF)
    xd = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    yd = np.linalg.solve(Hd, eta.ravel()).reshape(b.shape)
    gUd, _ = force.solve_gradient(U, xd, yd)
    assert relerr(gU, gUd) < 1e-9
    assert relerr(gb, yd) < 1e-9
    rng = synth.rng(523)
    dU = 1e-6 * (rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    fd = _loss(U + dU, b, eta, Ls, 1) - _loss(U - dU, b, eta, Ls, 1)
    lin = 2 * np.vdot(gU, dU).real
    assert abs(fd - lin) <= 1e-6 * abs(lin)
