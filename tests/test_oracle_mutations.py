"""Planted mistakes in the oracle (on the CPU) must be caught by a pin.

Each test swaps one piece of the oracle for a plausible wrong version (a
dropped term, a wrong sign, a wrong index, a transposed operand) and checks
that the corresponding pin reports a large error, so the pins are shown to
constrain the oracle rather than just agree with it.
"""
import numpy as np
import pytest

import synth
from oracle import dwf, force, krylov, multigrid as mg
from pins import (covariance_error, hermiticity_error, p0_det_error,
                  plane_wave_error, relerr, dense_H_from_stencil)

L4, LS = (4, 4, 2, 6), 4


def _cov():
    U = synth.gauge_field(L4, 0.5, 31)
    Om = synth.random_su3_field(L4, 32)
    psi = synth.gaussian_fermion(L4, LS, 33)
    return covariance_error(dwf, U, Om, psi, 1.8, 0.01, -1)


def _herm():
    U = synth.gauge_field(L4, 0.5, 11)
    x = synth.gaussian_fermion(L4, LS, 12)
    y = synth.gaussian_fermion(L4, LS, 13)
    return hermiticity_error(dwf, U, x, y, 1.8, 0.01, -1)


def _pw(bc_t=1):
    chi = synth.gaussian_fermion((1, 1, 1, 1), LS, 21)[0, 0, 0, 0]
    return plane_wave_error(dwf, (4, 6, 4, 8), LS, 1.8, 0.03, (1, 0, 2, 3), chi, bc_t)


def test_unmutated_oracle_passes_all():
    assert _cov() < 1e-14 and _herm() < 1e-13 and _pw(1) < 1e-14 and _pw(-1) < 1e-14
    assert p0_det_error(dwf, 8, 1.8, 0.01) < 1e-10


def test_backward_hop_with_wrong_link_is_caught(monkeypatch):
    orig = dwf.hop

    def bad(U, psi, mu, sign, bc_t):
        if sign > 0:
            return orig(U, psi, mu, sign, bc_t)
        t = dwf.color_mul_dag(U[mu], dwf.shift_fermion(psi, mu, -1, bc_t))   # U(x) not U(x-mu)
        return dwf.spin_mul(dwf.IDENT4 + dwf.GAMMA[mu], t)

    monkeypatch.setattr(dwf, "hop", bad)
    assert _cov() > 1e-3


def test_missing_dagger_on_backward_link_is_caught(monkeypatch):
    def bad(U, psi, mu, sign, bc_t):
        if sign > 0:
            t = dwf.color_mul(U[mu], dwf.shift_fermion(psi, mu, +1, bc_t))
            return dwf.spin_mul(dwf.IDENT4 - dwf.GAMMA[mu], t)
        t = dwf.color_mul(dwf.shift_links(U[mu], mu, -1), dwf.shift_fermion(psi, mu, -1, bc_t))
        return dwf.spin_mul(dwf.IDENT4 + dwf.GAMMA[mu], t)

    monkeypatch.setattr(dwf, "hop", bad)
    assert _herm() > 1e-3 or _cov() > 1e-3


def test_dropped_half_is_caught(monkeypatch):
    orig = dwf.hop
    monkeypatch.setattr(dwf, "hop", lambda U, psi, mu, s, bc: 2.0 * orig(U, psi, mu, s, bc))
    assert _pw() > 1e-3


def test_swapped_wilson_projectors_are_caught(monkeypatch):
    def bad(U, psi, mu, sign, bc_t):                     # (1 + g) forward, (1 - g) backward
        if sign > 0:
            t = dwf.color_mul(U[mu], dwf.shift_fermion(psi, mu, +1, bc_t))
            return dwf.spin_mul(dwf.IDENT4 + dwf.GAMMA[mu], t)
        t = dwf.color_mul_dag(dwf.shift_links(U[mu], mu, -1), dwf.shift_fermion(psi, mu, -1, bc_t))
        return dwf.spin_mul(dwf.IDENT4 - dwf.GAMMA[mu], t)

    monkeypatch.setattr(dwf, "hop", bad)
    assert _pw() > 1e-3


def test_missing_R5_is_caught(monkeypatch):
    monkeypatch.setattr(dwf, "gamma5_r5", lambda psi: dwf.spin_mul(dwf.GAMMA5, psi))
    assert _herm() > 1e-3


def test_wrong_mf_sign_is_caught(monkeypatch):
    orig = dwf.d5
    monkeypatch.setattr(dwf, "d5", lambda psi, mf: orig(psi, -mf))
    assert p0_det_error(dwf, 8, 1.8, 0.01) > 1e-3


def test_missing_antiperiodic_phase_is_caught(monkeypatch):
    orig = dwf.shift_fermion
    monkeypatch.setattr(dwf, "shift_fermion", lambda psi, mu, s, bc: orig(psi, mu, s, 1))
    assert _pw(-1) > 1e-3


def test_swapped_coarse_legs_are_caught(monkeypatch):
    g = mg.Geometry((4, 6, 4, 4), 2, (2, 2, 2, 2))           # coarse extent 3 in y
    U = synth.gauge_field(g.L, 0.5, 90)
    noise = synth.gaussian_fermion(g.L, g.Ls, 91, count=2)
    sub = mg.build_subspace(U, noise, g, 1.8, 0.05, smooth_iters=2)
    orig = mg.leg_index
    monkeypatch.setattr(mg, "leg_index", lambda mu, s: orig(mu, -s) if mu == 1 else orig(mu, s))
    A = mg.coarse_op(U, sub, 1.8, 0.05)
    monkeypatch.setattr(mg, "leg_index", orig)
    c = synth.gaussian_fermion((1, 1, 1, 1), 1, 92)[0, 0, 0, 0, 0].ravel()
    c = np.resize(c, (g.Vc, sub.nvec))
    lhs = mg.coarse_apply(A, g, c)
    rhs = mg.restrict(sub, dwf.apply_H(U, mg.prolong(sub, c), 1.8, 0.05))
    assert relerr(lhs, rhs) > 1e-3


def test_single_pass_unnormalised_gram_schmidt_is_caught(monkeypatch):
    def bad(Phi, rank_tol=1e-12):
        Phi = Phi.copy()
        for a in range(Phi.shape[1]):
            for k in range(Phi.shape[0]):
                for j in range(k):
                    Phi[k, a] -= np.vdot(Phi[j, a], Phi[k, a]) * Phi[j, a]
        return Phi

    monkeypatch.setattr(mg, "block_orthonormalise", bad)
    g = mg.Geometry((4, 4, 4, 4), 2, (2, 2, 2, 2))
    vs = mg.chiral_split(synth.gaussian_fermion(g.L, g.Ls, 3, count=2))
    Phi = mg.basis_from_vectors(g, vs).Phi
    gram = np.einsum("jak,iak->aji", np.conj(Phi), Phi)
    assert np.abs(gram - np.eye(4)[None]).max() > 1e-3


def test_force_without_dagger_on_second_term_is_caught(monkeypatch):
    def bad(U, x, w, bc_t=1):
        F = np.zeros_like(U)
        for mu in range(4):
            xf = dwf.shift_fermion(x, mu, +1, bc_t)
            wf = dwf.shift_fermion(w, mu, +1, bc_t)
            h = dwf.spin_mul(dwf.IDENT4 - dwf.GAMMA[mu], xf)
            gq = dwf.spin_mul(dwf.IDENT4 + dwf.GAMMA[mu], x)
            B = np.einsum("...sib,...sia->...ba", h, np.conj(w))
            C = np.einsum("...sib,...sia->...ba", gq, np.conj(wf))
            F[mu] = 0.5 * (B + C)
        return F

    L, Ls = (2, 2, 2, 2), 4
    U = synth.gauge_field(L, 0.5, 510)
    b = synth.gaussian_fermion(L, Ls, 511)
    eta = synth.gaussian_fermion(L, Ls, 512)
    Hd = dense_H_from_stencil(dwf, U, Ls, 1.8, 0.05)
    x = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    y = np.linalg.solve(Hd, eta.ravel()).reshape(b.shape)
    good = force.gauge_force(U, x, dwf.gamma5_r5(y))
    monkeypatch.setattr(force, "gauge_force", bad)
    wrong = force.gauge_force(U, x, dwf.gamma5_r5(y))
    # the directional derivative along a random Lie-algebra direction differs
    rng = synth.rng(513)
    G = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    T = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    d_good = np.einsum("...ab,...bc,...ca->...", 1j * T, U, good).sum().real
    d_bad = np.einsum("...ab,...bc,...ca->...", 1j * T, U, wrong).sum().real
    assert abs(d_good - d_bad) > 1e-3 * abs(d_good)


def test_inverted_cr_beta_is_caught(monkeypatch):
    """A CR with beta = gamma / gamma' no longer reaches the dense solution."""
    rng = synth.rng(5)
    n = 40
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Qm, _ = np.linalg.qr(G)
    A = (Qm * np.linspace(-3, 4, n)) @ Qm.conj().T
    b = rng.standard_normal(n) + 0j

    def bad_cr(apply, b, tol=1e-10, maxiter=200):
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        Ar = apply(r)
        Ap = Ar.copy()
        gam = np.vdot(r, Ar).real
        for _ in range(maxiter):
            al = gam / np.vdot(Ap, Ap).real
            x = x + al * p
            r = r - al * Ap
            Ar = apply(r)
            gn = np.vdot(r, Ar).real
            beta = gam / gn
            gam = gn
            p = r + beta * p
            Ap = Ar + beta * Ap
        return x

    x = bad_cr(lambda v: A @ v, b, maxiter=60)
    assert relerr(x, np.linalg.solve(A, b)) > 1e-3
    x_ok, _ = krylov.cr(lambda v: A @ v, b, tol=1e-12, maxiter=400)
    assert relerr(x_ok, np.linalg.solve(A, b)) < 1e-9


# ------------------------------------------------------------ red-black CGNE and Moebius
from oracle import redblack as rb  # noqa: E402
from pins import dense_H_assembled  # noqa: E402


def _rb_lu_error():
    """Red-black CGNE against the independently assembled dense H (the pin of
    test_oracle_redblack): relative error of the solution."""
    L, Ls, M5, mf = (4, 2, 2, 2), 4, 1.8, 0.05
    U = synth.gauge_field(L, 0.5, 8300)
    b = synth.gaussian_fermion(L, Ls, 8301)
    x, _, _ = rb.cgne_rb_solve(U, b, M5, mf, -1, tol=1e-12, maxiter=3000)
    H = dense_H_assembled(dwf, U, Ls, M5, mf, -1)
    xo = np.linalg.solve(H, b.ravel()).reshape(b.shape)
    return relerr(x, xo)


def _m5inv_error():
    psi = synth.gaussian_fermion((2, 2, 2, 2), 8, 8100)
    return relerr(rb.m5_apply(rb.m5_inverse(psi, 1.8, 0.03), 1.8, 0.03), psi)


def _schur_herm_error():
    L, Ls, M5, mf = (4, 2, 2, 4), 4, 1.8, 0.02
    U = synth.gauge_field(L, 0.5, 8200)
    odd = rb.parity_mask(L)
    x = rb.on_parity(synth.gaussian_fermion(L, Ls, 8201), odd, 1)
    y = rb.on_parity(synth.gaussian_fermion(L, Ls, 8202), odd, 1)
    lhs = dwf.inner(x, rb.schur_apply(U, y, odd, M5, mf))
    rhs = dwf.inner(rb.schur_dag_apply(U, x, odd, M5, mf), y)
    return abs(lhs - rhs) / abs(lhs)


def test_unmutated_redblack_and_mobius_pass():
    assert _rb_lu_error() < 1e-9 and _m5inv_error() < 1e-14 and _schur_herm_error() < 1e-13
    chi = synth.gaussian_fermion((1, 1, 1, 1), LS, 21)[0, 0, 0, 0]
    assert plane_wave_error(dwf, (4, 6, 4, 8), LS, 1.8, 0.03, (1, 0, 2, 3), chi, 1, b5=1.5) < 1e-14


def test_schur_without_m5_inverse_is_caught(monkeypatch):
    def bad(U, v, odd, M5, mf, bc_t=1):  # D_oe D_eo in place of D_oe M5^{-1} D_eo
        a = rb.on_parity(rb.dhop_apply(U, v, M5, bc_t), odd, 0)
        c = rb.on_parity(rb.dhop_apply(U, a, M5, bc_t), odd, 1)
        return rb.on_parity(rb.m5_apply(v, M5, mf), odd, 1) - c

    monkeypatch.setattr(rb, "schur_apply", bad)
    assert _rb_lu_error() > 1e-3


def test_transposed_m5_inverse_is_caught(monkeypatch):
    def bad(psi, M5, mf):
        Ls = psi.shape[-3]
        Minv = np.linalg.inv(rb.m5_matrix(Ls, M5, mf))
        return np.einsum("pts,...tpc->...spc", Minv, psi)  # Minv^T

    monkeypatch.setattr(rb, "m5_inverse", bad)
    assert _m5inv_error() > 1e-3


def test_schur_adjoint_without_gamma5_is_caught(monkeypatch):
    monkeypatch.setattr(rb, "schur_dag_apply", lambda U, v, odd, M5, mf, bc_t=1: rb.schur_apply(U, v, odd, M5, mf, bc_t))
    assert _schur_herm_error() > 1e-3


def test_mobius_with_unscaled_mass_term_is_caught(monkeypatch):
    def bad(U, psi, M5, mf, b5, bc_t=1):  # b5 on the hops only, not on (4 - M5)
        hops = dwf.wilson(U, psi, M5, bc_t) - (4.0 - M5) * psi
        return b5 * hops + (4.0 - M5) * psi + dwf.d5(psi, mf)

    monkeypatch.setattr(dwf, "ddwf_mobius", bad)
    chi = synth.gaussian_fermion((1, 1, 1, 1), LS, 21)[0, 0, 0, 0]
    assert plane_wave_error(dwf, (4, 6, 4, 8), LS, 1.8, 0.03, (1, 0, 2, 3), chi, 1, b5=1.5) > 1e-3


# ------------------------------------------------------------- third level (oracle/level2.py)
def _l2_galerkin_error():
    """|A2 (densified) - P2^dag A P2| / |P2^dag A P2| with dense matrices built independently."""
    from oracle import level2 as l2
    from test_oracle_level2 import _dense_A, _dense_P2
    g = l2.CoarseGeometry((6, 4, 4, 6), 4, (3, 2, 2, 3))
    A = l2.random_coarse_op(g, 61)
    rng = np.random.default_rng(62)
    v = rng.standard_normal((4, g.Vc, 4)) + 1j * rng.standard_normal((4, g.Vc, 4))
    Phi2 = l2.basis_from_vectors(g, v)
    P = _dense_P2(g, Phi2)
    brute = np.conj(P.T) @ _dense_A(A, g) @ P
    return np.abs(l2.level2_dense(l2.level2_op(A, g, Phi2), g) - brute).max() / np.abs(brute).max()


def test_unmutated_level2_oracle_passes():
    assert _l2_galerkin_error() < 1e-12


def test_level2_leg_without_block_mask_is_caught(monkeypatch):
    from oracle import level2 as l2
    monkeypatch.setattr(l2, "crossing_mask", lambda g, mu, sign: np.ones((g.Vc, 1)))
    assert _l2_galerkin_error() > 1e-3


def test_level2_leg_in_the_wrong_direction_is_caught(monkeypatch):
    from oracle import level2 as l2
    orig = l2.apply_leg
    monkeypatch.setattr(l2, "apply_leg", lambda A, g, c, mu, sign: orig(A, g, c, mu, -sign))
    assert _l2_galerkin_error() > 1e-3


def test_level2_projection_without_conjugate_is_caught(monkeypatch):
    from oracle import level2 as l2
    orig_conj = l2.np.conj

    class NoConjNp:
        def __getattr__(self, name):
            return getattr(np, name)

        @staticmethod
        def conj(x):
            return x

    monkeypatch.setattr(l2, "np", NoConjNp())
    try:
        err = _l2_galerkin_error()
    finally:
        monkeypatch.setattr(l2, "np", np)
    assert orig_conj is np.conj and err > 1e-3


def test_coarse_gamma5_with_wrong_ordering_is_caught(monkeypatch):
    """The split must follow the level-1 basis's chirality ordering (the P_+ half first);
    alternating signs would mix chiralities, which the definite-chirality pin sees."""
    from oracle import level2 as l2
    monkeypatch.setattr(l2, "gamma5_coarse", lambda nvec: np.array([(-1.0) ** i for i in range(nvec)]))
    g5_true = np.concatenate([np.ones(3), -np.ones(3)])
    rng = np.random.default_rng(63)
    v = rng.standard_normal((2, 16, 6)) + 1j * rng.standard_normal((2, 16, 6))
    s = l2.chiral_split(v, 6)
    assert not np.allclose(s[:2] * g5_true, s[:2])


# ------------------------------------------------------------- continued fraction (oracle/overlap.py)
def _cf_printed_error():
    from oracle import overlap as ov
    from test_oracle_overlap import BETA, R, _dense_cf, _printed_matrix
    U = synth.gauge_field((2, 2, 2, 2), 0.5, 81)
    P = _printed_matrix(U, BETA, R)
    return np.abs(_dense_cf(U, BETA, R) - P).max() / np.abs(P).max()


def test_unmutated_cf_oracle_passes():
    assert _cf_printed_error() < 1e-13


def test_cf_without_alternating_signs_is_caught(monkeypatch):
    from oracle import overlap as ov
    orig = ov.diag_scales
    monkeypatch.setattr(ov, "diag_scales", lambda beta: np.abs(orig(beta)))
    assert _cf_printed_error() > 1e-3


def test_cf_last_coupling_with_both_betas_is_caught(monkeypatch):
    """The last coupling is 1/sqrt(beta_{N-2}), not 1/sqrt(beta_{N-2} beta_0)."""
    from oracle import overlap as ov
    orig = ov.couplings

    def bad(beta):
        c = orig(beta).copy()
        c[-1] = 1.0 / np.sqrt(beta[-1] * beta[0])
        return c

    monkeypatch.setattr(ov, "couplings", bad)
    assert _cf_printed_error() > 1e-3


def test_cf_without_gamma5_on_the_kernel_is_caught(monkeypatch):
    from oracle import overlap as ov
    monkeypatch.setattr(ov, "apply_HW", lambda U, psi, M5, bc_t=1: dwf.wilson(U, psi, M5, bc_t))
    assert _cf_printed_error() > 1e-3


# ------------------------------------- two-level pieces on the continued fraction, cycle shapes
def _cf_galerkin_error():
    """max over two random coarse vectors of |A c - P^dag H_cf P c| / |P^dag H_cf P c| on a
    3^4 coarse lattice (the pin of test_oracle_overlap_coarse)."""
    from oracle import overlap as ov
    L, N, block, nvec, beta, R = (6, 6, 6, 6), 3, (2, 2, 2, 2), 4, [1.2, 0.7], 0.3
    g = mg.Geometry(L, N, block)
    U = synth.gauge_field(L, 0.5, 710)
    sub = mg.basis_from_vectors(g, synth.gaussian_fermion(L, N, 711, count=nvec))
    A = ov.cf_coarse_op(U, sub, 1.8, beta, R)
    rng = synth.rng(712)
    err = 0.0
    for _ in range(2):
        c = rng.standard_normal((g.Vc, nvec)) + 1j * rng.standard_normal((g.Vc, nvec))
        want = mg.restrict(sub, ov.apply_cf(U, mg.prolong(sub, c), 1.8, beta, R))
        err = max(err, relerr(mg.coarse_apply(A, g, c), want))
    return err


def test_unmutated_cf_coarse_oracle_passes():
    assert _cf_galerkin_error() < 1e-13


def test_cf_hop_without_component_factor_is_caught(monkeypatch):
    """The hop part of H_cf without the component's factor (-1)^i / beta_0 puts the wrong
    hops into the legs and leaves their difference in the self leg."""
    from oracle import overlap as ov

    def bad(U, psi, mu, sign, beta, bc_t=1):
        return dwf.spin_mul(dwf.GAMMA5, -0.5 * dwf.hop(U, psi, mu, sign, bc_t))

    monkeypatch.setattr(ov, "apply_cf_hop", bad)
    assert _cf_galerkin_error() > 1e-3


def test_cf_leg_with_the_wrong_crossing_mask_is_caught(monkeypatch):
    """The face of the opposite side taken as the block crossing of a hop."""
    orig = mg.crossing_mask
    monkeypatch.setattr(mg, "crossing_mask", lambda g, mu, sign: orig(g, mu, -sign))
    assert _cf_galerkin_error() > 1e-3


def _post_cycle_error(cycle="post"):
    """|v - B H v - (1 - S H)(1 - Q H) v| / |.| for one random v with a linear S and exact Q."""
    from test_oracle_multigrid import _tiny_two_level, M5 as M5m, MF as MFm
    g, U, sub, A, Hd, P, Q, _ = _tiny_two_level()
    N = Hd.shape[0]
    Sm = 0.05 * Hd + 0.01 * np.eye(N)
    S = lambda v: (Sm @ v.ravel()).reshape(v.shape)
    Ad = mg.coarse_dense(A, g)
    Qc = lambda c: np.linalg.solve(Ad, c.ravel()).reshape(c.shape)
    p = mg.HDCRParams(M5=M5m, mf=MFm)
    v = synth.rng(131).standard_normal(N) + 1j * synth.rng(132).standard_normal(N)
    got = v - mg.vcycle(U, sub, A, (Hd @ v).reshape(g.fine_shape()), p, S=S, Qc=Qc, cycle=cycle).ravel()
    want = (np.eye(N) - Sm @ Hd) @ ((np.eye(N) - Q @ Hd) @ v)
    return relerr(got, want)


def test_unmutated_post_cycle_passes():
    assert _post_cycle_error() < 1e-11


def test_post_cycle_smoothing_r_instead_of_the_residual_is_caught(monkeypatch):
    """Smoothing the input r instead of r - H z1 (the residual after the coarse step)."""
    orig = mg.vcycle

    def bad(U, sub, A, r, p, S=None, Qc=None, cycle="symmetric"):
        if cycle != "post":
            return orig(U, sub, A, r, p, S=S, Qc=Qc, cycle=cycle)
        z1 = mg.prolong(sub, Qc(mg.restrict(sub, r)))
        return z1 + S(r)

    monkeypatch.setattr(mg, "vcycle", bad)
    assert _post_cycle_error() > 1e-3
