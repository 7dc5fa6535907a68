"""Pins for the oracle's fine operator H = Gamma5 D_dwf (Section 3)."""
import numpy as np
import pytest

import synth
from oracle import dwf
from pins import (covariance_error, dense_H_assembled, dense_H_from_stencil,
                  gamma_algebra_error, hermiticity_error, p0_det_error,
                  plane_wave_error, relerr)


def test_gamma_algebra_chiral_basis():
    assert gamma_algebra_error(dwf) < 1e-15
    np.testing.assert_allclose(np.diag(dwf.GAMMA5).real, [1, 1, -1, -1])
    # P_pm are complementary projectors
    assert np.abs(dwf.P_PLUS @ dwf.P_PLUS - dwf.P_PLUS).max() < 1e-15
    assert np.abs(dwf.P_PLUS + dwf.P_MINUS - np.eye(4)).max() < 1e-15


@pytest.mark.parametrize("bc_t", [1, -1])
@pytest.mark.parametrize("L,Ls", [((4, 4, 4, 4), 8), ((3, 2, 4, 5), 3)])
def test_hermiticity(L, Ls, bc_t):
    U = synth.gauge_field(L, 0.5, 11)
    x = synth.gaussian_fermion(L, Ls, 12)
    y = synth.gaussian_fermion(L, Ls, 13)
    assert hermiticity_error(dwf, U, x, y, 1.8, 0.01, bc_t) < 1e-13


def test_gamma5_squares_to_one():
    L, Ls = (2, 3, 2, 2), 5
    x = synth.gaussian_fermion(L, Ls, 3)
    assert relerr(dwf.gamma5_r5(dwf.gamma5_r5(x)), x) == 0.0


@pytest.mark.parametrize("bc_t", [1, -1])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 3), (3, 1, 1, 0)])
def test_free_field_plane_wave(n, bc_t):
    L, Ls = (4, 6, 4, 8), 6
    chi = synth.gaussian_fermion((1, 1, 1, 1), Ls, 21)[0, 0, 0, 0]
    assert plane_wave_error(dwf, L, Ls, 1.8, 0.03, n, chi, bc_t) < 1e-14


@pytest.mark.parametrize("Ls", [4, 8, 12])
def test_zero_momentum_wall_mass(Ls):
    assert p0_det_error(dwf, Ls, 1.8, 0.01) < 1e-10
    assert p0_det_error(dwf, Ls, 1.3, 0.2) < 1e-10


@pytest.mark.parametrize("bc_t", [1, -1])
def test_gauge_covariance(bc_t):
    L, Ls = (4, 4, 2, 6), 4
    U = synth.gauge_field(L, 0.5, 31)
    Om = synth.random_su3_field(L, 32)
    psi = synth.gaussian_fermion(L, Ls, 33)
    assert covariance_error(dwf, U, Om, psi, 1.8, 0.01, bc_t) < 1e-14


@pytest.mark.parametrize("bc_t", [1, -1])
def test_dense_stencil_equals_assembled_matrix(bc_t):
    L, Ls = (3, 2, 2, 2), 3
    U = synth.gauge_field(L, 0.7, 41)
    Hs = dense_H_from_stencil(dwf, U, Ls, 1.8, 0.05, bc_t)
    Ha = dense_H_assembled(dwf, U, Ls, 1.8, 0.05, bc_t)
    assert relerr(Hs, Ha) < 1e-15
    assert relerr(Hs, Hs.conj().T) < 1e-15          # Hermitian
    ev = np.linalg.eigvalsh(Hs)
    assert ev.min() < 0 < ev.max()                  # indefinite (Section 3)


def test_hop_pieces_sum_to_operator():
    """H = Gamma5 [(4 - M5 + D5) - 1/2 sum hops]: the hop pieces used by the coarse
    operator add up with the local part to H."""
    L, Ls = (4, 2, 4, 4), 4
    U = synth.gauge_field(L, 0.5, 51)
    psi = synth.gaussian_fermion(L, Ls, 52)
    local = dwf.gamma5_r5((4 - 1.8) * psi + dwf.d5(psi, 0.01))
    tot = local + sum(dwf.apply_H_hop(U, psi, mu, s, -1) for mu in range(4) for s in (1, -1))
    assert relerr(tot, dwf.apply_H(U, psi, 1.8, 0.01, -1)) < 1e-15


def test_synthetic_links_are_su3():
    U = synth.gauge_field((2, 2, 2, 2), 0.5, 7)
    M = U.reshape(-1, 3, 3)
    err_u = np.abs(M @ np.conj(np.swapaxes(M, -1, -2)) - np.eye(3)).max()
    err_d = np.abs(np.linalg.det(M) - 1).max()
    assert err_u < 1e-14 and err_d < 1e-14


def test_device_gaussian_is_seeded_and_standard():
    """The device-side noise of the large workloads: the same seed gives the same
    numbers, and Re, Im are independent N(0, 1) (here drawn on the CPU device)."""
    torch = pytest.importorskip("torch")
    a = synth.device_gaussian(2, 4096, 11, device="cpu")
    b = synth.device_gaussian(2, 4096, 11, device="cpu")
    c = synth.device_gaussian(2, 4096, 12, device="cpu")
    assert a.shape == (2, 4096 * 12) and a.dtype == torch.complex128
    assert torch.equal(a, b) and not torch.equal(a, c)
    re, im = a.real.numpy().ravel(), a.imag.numpy().ravel()
    n = re.size
    for x in (re, im):  # mean 0, variance 1 within a few standard errors
        assert abs(x.mean()) < 5 / np.sqrt(n)
        assert abs(x.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.corrcoef(re, im)[0, 1]) < 5 / np.sqrt(n)
    assert synth.device_gaussian(1, 8, 3, device="cpu", dtype=torch.complex64).dtype == torch.complex64


def test_sitewise_evaluation_matches_field_apply():
    L, Ls = (3, 4, 2, 5), 4
    U = synth.gauge_field(L, 0.5, 61)
    psi = synth.gaussian_fermion(L, Ls, 62)
    full = dwf.apply_H(U, psi, 1.8, 0.02, -1)
    rng = synth.rng(63)
    sites = [tuple(int(rng.integers(0, e)) for e in L + (Ls,)) for _ in range(40)]
    sites += [(0, 0, 0, 0, 0), (2, 3, 1, 4, Ls - 1)]
    got = dwf.apply_H_at(U, psi, sites, 1.8, 0.02, -1)
    want = np.array([full[t, z, y, x, s] for (x, y, z, t, s) in sites])
    assert relerr(got, want) < 1e-15


# ------------------------------------------------------------ Moebius, c5 = 0
def test_mobius_b5_one_is_shamir():
    L, Ls = (2, 3, 2, 4), 5
    U = synth.gauge_field(L, 0.5, 9000)
    psi = synth.gaussian_fermion(L, Ls, 9001)
    assert relerr(dwf.ddwf_mobius(U, psi, 1.8, 0.03, 1.0, -1), dwf.ddwf(U, psi, 1.8, 0.03, -1)) == 0.0


@pytest.mark.parametrize("b5", [0.6, 1.7])
def test_mobius_hermiticity(b5):
    L, Ls = (2, 2, 4, 2), 6
    U = synth.gauge_field(L, 0.5, 9100)
    x = synth.gaussian_fermion(L, Ls, 9101)
    y = synth.gaussian_fermion(L, Ls, 9102)
    lhs = dwf.inner(x, dwf.apply_H_mobius(U, y, 1.8, 0.02, b5, -1))
    rhs = dwf.inner(dwf.apply_H_mobius(U, x, 1.8, 0.02, b5, -1), y)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 3)])
def test_mobius_free_field_plane_wave(n):
    L, Ls = (4, 6, 4, 8), 6
    chi = synth.gaussian_fermion((1, 1, 1, 1), Ls, 9200)[0, 0, 0, 0]
    assert plane_wave_error(dwf, L, Ls, 1.8, 0.03, n, chi, 1, b5=1.5) < 1e-14
