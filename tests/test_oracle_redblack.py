"""Pins of the red-black CGNE oracle (the paper's comparison solver, Section 5 and
Table 1): the even-odd split is exact, M5^{-1} inverts M5 and has the closed form
of a bidiagonal matrix, the Schur complement is Gamma5-hermitian, and the solve
reproduces a dense LU solution of H x = b."""
import numpy as np

import synth
from oracle import dwf
from oracle import redblack as rb
from pins import dense_H_assembled


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def test_split_is_exact_and_hops_change_parity():
    L, Ls = (4, 2, 4, 2), 4
    U = synth.gauge_field(L, 0.5, 8000)
    psi = synth.gaussian_fermion(L, Ls, 8001)
    full = dwf.ddwf(U, psi, 1.8, 0.05, -1)
    assert _rel(rb.m5_apply(psi, 1.8, 0.05) + rb.dhop_apply(U, psi, 1.8, -1), full) < 1e-14
    odd = rb.parity_mask(L)
    for p in (0, 1):
        h = rb.dhop_apply(U, rb.on_parity(psi, odd, p), 1.8, -1)
        assert np.abs(rb.on_parity(h, odd, p)).max() == 0.0   # D_hop joins opposite parities only
        assert np.abs(rb.on_parity(h, odd, 1 - p)).max() > 0.1


def test_m5_inverse_inverts_and_matches_closed_form():
    L, Ls, M5, mf = (2, 2, 2, 2), 8, 1.8, 0.03
    psi = synth.gaussian_fermion(L, Ls, 8100)
    assert _rel(rb.m5_apply(rb.m5_inverse(psi, M5, mf), M5, mf), psi) < 1e-14
    # closed form at mf = 0: for the upper spins M5 = a - (shift s -> s+1), lower-bidiagonal,
    # so (M5^{-1})[s, s'] = a^{-(s - s' + 1)} for s >= s', 0 above; the lower spins transposed
    a = 5.0 - M5
    Minv = np.linalg.inv(rb.m5_matrix(Ls, M5, 0.0))
    s, sp = np.meshgrid(np.arange(Ls), np.arange(Ls), indexing="ij")
    want_up = np.where(s >= sp, a ** (-(s - sp + 1.0)), 0.0)
    assert np.allclose(Minv[0], want_up, rtol=1e-14, atol=1e-16)
    assert np.allclose(Minv[2], want_up.T, rtol=1e-14, atol=1e-16)
    # the walls: with mf != 0 the corner couples s = 0 and Ls - 1 (the last column of the
    # upper-spin inverse is no longer zero above the diagonal)
    Minv_mf = np.linalg.inv(rb.m5_matrix(Ls, M5, mf))
    assert abs(Minv_mf[0][0, Ls - 1]) > 0


def test_schur_complement_is_gamma5_hermitian():
    L, Ls, M5, mf = (4, 2, 2, 4), 4, 1.8, 0.02
    U = synth.gauge_field(L, 0.5, 8200)
    odd = rb.parity_mask(L)
    x = rb.on_parity(synth.gaussian_fermion(L, Ls, 8201), odd, 1)
    y = rb.on_parity(synth.gaussian_fermion(L, Ls, 8202), odd, 1)
    lhs = dwf.inner(x, rb.schur_apply(U, y, odd, M5, mf))
    rhs = dwf.inner(rb.schur_dag_apply(U, x, odd, M5, mf), y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_cgne_rb_matches_dense_lu():
    L, Ls, M5, mf = (4, 2, 2, 2), 4, 1.8, 0.05
    U = synth.gauge_field(L, 0.5, 8300)
    b = synth.gaussian_fermion(L, Ls, 8301)
    x, it, res = rb.cgne_rb_solve(U, b, M5, mf, -1, tol=1e-12)
    assert res <= 1e-11
    H = dense_H_assembled(dwf, U, Ls, M5, mf, -1)
    xo = np.linalg.solve(H, b.ravel()).reshape(b.shape)
    assert _rel(x, xo) < 1e-9
    # CGNE on the Schur complement needs at most its dimension (N / 2) steps in exact
    # arithmetic; far fewer here
    assert 0 < it < b.size // 2
