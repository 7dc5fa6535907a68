"""Pins for the oracle's Krylov solvers: CR (Section 3) and flexible GCR (Section 4)."""
import numpy as np
import pytest

import synth
from oracle import dwf
from oracle.krylov import cr, fgcr
from pins import dense_H_from_stencil, relerr


def _system(L, Ls, mf, seed):
    U = synth.gauge_field(L, 0.5, seed)
    Hd = dense_H_from_stencil(dwf, U, Ls, 1.8, mf)
    b = synth.gaussian_fermion(L, Ls, seed + 1)
    return U, Hd, b


@pytest.mark.parametrize("L,Ls", [((2, 2, 2, 2), 4), ((2, 2, 2, 4), 4)])
def test_cr_matches_dense_lu(L, Ls):
    U, Hd, b = _system(L, Ls, 0.05, 100)
    H = lambda v: dwf.apply_H(U, v, 1.8, 0.05)
    x, info = cr(H, b, tol=1e-12, maxiter=5000)
    x_lu = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    cond = np.linalg.cond(Hd)
    assert info.converged
    assert info.true_resid < 1e-11
    assert relerr(x, x_lu) < cond * 1e-11
    # minimal residual: |r_k| never increases
    h = np.array(info.resid_history)
    assert np.all(np.diff(h) <= 1e-12 * h[:-1])


def test_cr_terminates_after_distinct_eigenvalue_count():
    """The Krylov space of a Hermitian A with d distinct eigenvalues has dimension d,
    so CR reaches the exact solution in d steps (up to rounding)."""
    rng = synth.rng(5)
    n = 60
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Qm, _ = np.linalg.qr(G)
    lam = np.array([-3.0, -1.0, 0.5, 2.0, 4.0])[np.arange(n) % 5]   # indefinite, 5 distinct
    A = (Qm * lam) @ Qm.conj().T
    b = rng.standard_normal(n) + 0j
    x, info = cr(lambda v: A @ v, b, tol=1e-11, maxiter=50)
    assert info.converged and info.iters == 5
    assert relerr(x, np.linalg.solve(A, b)) < 1e-11


def test_gcr_with_identity_preconditioner_is_cr():
    """Unpreconditioned GCR on a Hermitian operator reproduces CR's residual norms."""
    L, Ls = (2, 2, 2, 2), 4
    U, _, b = _system(L, Ls, 0.1, 200)
    H = lambda v: dwf.apply_H(U, v, 1.8, 0.1)
    _, icr = cr(H, b, tol=1e-8, maxiter=30)
    _, igcr = fgcr(H, lambda r: r, b, tol=1e-8, restart=60, maxiter=30)
    k = min(len(icr.resid_history) - 1, len(igcr.resid_history), 25)
    np.testing.assert_allclose(igcr.resid_history[:k], icr.resid_history[1:k + 1], rtol=1e-7)


def test_fgcr_with_nonlinear_preconditioner_matches_lu():
    L, Ls = (2, 2, 2, 2), 4
    U, Hd, b = _system(L, Ls, 0.05, 300)
    H = lambda v: dwf.apply_H(U, v, 1.8, 0.05)
    prec = lambda r: cr(H, r, fixed_iters=8)[0]            # nonlinear in r
    x, info = fgcr(H, prec, b, tol=1e-10, restart=16, maxiter=400)
    assert info.converged and info.true_resid <= 1e-10
    x_lu = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    assert relerr(x, x_lu) < np.linalg.cond(Hd) * 1e-10


def test_fixed_iteration_cr_counts_matvecs():
    L, Ls = (2, 2, 2, 2), 4
    U, _, b = _system(L, Ls, 0.05, 400)
    calls = []
    H = lambda v: (calls.append(1), dwf.apply_H(U, v, 1.8, 0.05))[1]
    cr(H, b, fixed_iters=8)
    assert len(calls) == 8          # zero guess: one apply per step, none after the last


def test_cr_needs_no_more_matvecs_than_cgne():
    """Section 3: CGNE's N-th iterate lies in the Krylov space that 2N steps of CR on
    H minimise over (D^dag D = H^2 and D^dag b = H Gamma5 b), so CR reaches at least as
    small a residual with the same number of operator applications.  CGNE here is
    plain CG on H^2 x = H b' (b' = Gamma5 b, the normal equations of D x = b), two
    applications of H per step; both start from zero."""
    L, Ls, mf = (2, 2, 2, 4), 4, 0.05
    U = synth.gauge_field(L, 0.5, 8700)
    b = synth.gaussian_fermion(L, Ls, 8701)
    H = lambda v: dwf.apply_H(U, v, 1.8, mf)
    nb = np.sqrt(dwf.norm2(b))
    # CG on H^2 x = H b, recording |b - H x| after each step (2 applications of H)
    x = np.zeros_like(b)
    r = H(b)  # normal-equation residual H b - H^2 x at x = 0
    p = r.copy()
    rr = dwf.norm2(r)
    cgne = []
    for _ in range(30):
        q = H(H(p))
        a = rr / np.real(dwf.inner(p, q))
        x = x + a * p
        r = r - a * q
        rn = dwf.norm2(r)
        p = r + (rn / rr) * p
        rr = rn
        cgne.append(np.sqrt(dwf.norm2(b - H(x))) / nb)
    for n_steps in (1, 2, 5, 10, 20, 30):
        _, info = cr(H, b, fixed_iters=2 * n_steps)
        r_cr = info.resid_history[-1]
        assert r_cr <= cgne[n_steps - 1] * (1 + 1e-8), (n_steps, r_cr, cgne[n_steps - 1])
        # CR needs roughly as many matvecs as CGNE: here it is better by under 1%
        assert r_cr >= 0.95 * cgne[n_steps - 1], (n_steps, r_cr, cgne[n_steps - 1])
