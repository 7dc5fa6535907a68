"""Pins for the oracle's two-level construction (Section 4, Eqs. 4.1-4.6)."""
import numpy as np
import pytest

import synth
from oracle import dwf, multigrid as mg
from pins import dense_H_from_stencil, relerr

M5, MF = 1.8, 0.05


def _subspace(L, Ls, block, nvec, seed, eps=0.5, bc_t=1, iters=4):
    g = mg.Geometry(L, Ls, block)
    U = synth.gauge_field(L, eps, seed)
    noise = synth.gaussian_fermion(L, Ls, seed + 1, count=nvec // 2)
    sub = mg.build_subspace(U, noise, g, M5, MF, bc_t, smooth_iters=iters)
    return g, U, sub


def test_block_layout_matches_coordinates():
    g = mg.Geometry((4, 6, 2, 4), 2, (2, 3, 1, 2))
    Lx, Ly, Lz, Lt = g.L
    t, z, y, x = np.indices((Lt, Lz, Ly, Lx))
    field = np.zeros(g.fine_shape(), dtype=np.complex128)
    field[...] = (x + 100 * y + 10000 * z + 1000000 * t)[..., None, None, None]
    blk = mg.to_blocks(g, field)
    Xc, Yc, Zc, Tc = g.Lc
    for a in range(g.Vc):
        xc = a % Xc
        yc = (a // Xc) % Yc
        zc = (a // (Xc * Yc)) % Zc
        tc = a // (Xc * Yc * Zc)
        v = blk[a].real.astype(int)
        assert np.all(v % 100 // 2 == xc)
        assert np.all(v // 100 % 100 // 3 == yc)
        assert np.all(v // 10000 % 100 // 1 == zc)
        assert np.all(v // 1000000 // 2 == tc)
    assert relerr(mg.from_blocks(g, blk), field) == 0.0


def test_subspace_orthonormal_chiral_and_spanning():
    L, Ls = (4, 4, 4, 4), 4
    g = mg.Geometry(L, Ls, (2, 2, 2, 2))
    U = synth.gauge_field(L, 0.5, 10)
    noise = synth.gaussian_fermion(L, Ls, 11, count=3)
    sm = np.stack([mg.smooth_noise(U, x0, M5, MF, 1, 4) for x0 in noise])
    vs = mg.chiral_split(sm)
    sub = mg.basis_from_vectors(g, vs)
    Phi = sub.Phi
    # P^dag P = 1 in every block (Eq. 4.3 is a projector)
    gram = np.einsum("jak,iak->aji", np.conj(Phi), Phi)
    assert np.abs(gram - np.eye(6)[None]).max() < 1e-13
    # chirality: first half Gamma5-even, second half Gamma5-odd (orthonormalising
    # inside a block keeps this, since Gamma5 acts inside a block)
    full = mg.from_blocks(g, Phi)
    assert relerr(dwf.gamma5_r5(full[:3]), full[:3]) < 1e-14
    assert relerr(dwf.gamma5_r5(full[3:]), -full[3:]) < 1e-14
    # span{phi_k} in span{phi_k^b} (Eq. 4.2): P P^dag reproduces each vector
    for v in vs:
        assert relerr(mg.prolong(sub, mg.restrict(sub, v)), v) < 1e-13
    # the smoothed vectors are normalised
    np.testing.assert_allclose([dwf.norm2(v) for v in sm], 1.0, rtol=1e-14)


def test_smoothing_lowers_rayleigh_quotient():
    """Ten CR steps on H x = 0 shrink |H x| / |x| relative to the noise (near-null space)."""
    L, Ls = (4, 4, 4, 4), 8
    U = synth.gauge_field(L, 0.3, 12)
    x0 = synth.gaussian_fermion(L, Ls, 13)
    x = mg.smooth_noise(U, x0, 1.8, 0.01, 1, 10)
    r0 = np.sqrt(dwf.norm2(dwf.apply_H(U, x0, 1.8, 0.01)) / dwf.norm2(x0))
    r1 = np.sqrt(dwf.norm2(dwf.apply_H(U, x, 1.8, 0.01)))
    assert r1 < 0.5 * r0


def test_rank_deficiency_detected():
    L, Ls = (4, 4, 4, 4), 2
    g = mg.Geometry(L, Ls, (2, 2, 2, 2))
    v = synth.gaussian_fermion(L, Ls, 3, count=1)
    vs = mg.chiral_split(np.concatenate([v, v]))      # duplicates
    with pytest.raises(mg.RankDeficient):
        mg.basis_from_vectors(g, vs)


def _dense_coarse_by_definition(U, sub, bc_t=1):
    """<phi_j^a | H | phi_k^b> for all a, b by applying H to each block-restricted vector."""
    g = sub.geom
    nvec, Vc, _ = sub.Phi.shape
    D = np.zeros((Vc * nvec, Vc * nvec), dtype=np.complex128)
    for b in range(Vc):
        blk = np.zeros((nvec, Vc, g.K), dtype=np.complex128)
        blk[:, b] = sub.Phi[:, b]
        vk = mg.from_blocks(g, blk)
        Hv = dwf.apply_H(U, vk, M5, MF, bc_t)
        c = mg.restrict(sub, Hv)                       # (nvec_k, Vc, nvec_j)
        for k in range(nvec):
            D[:, b * nvec + k] = c[k].reshape(-1)
    return D


@pytest.mark.parametrize("bc_t", [1, -1])
def test_coarse_op_equals_brute_force_projection_extent2(bc_t):
    """Densified 9-point stencil == P^dag H P on a 2^4 coarse lattice (legs alias)."""
    g, U, sub = _subspace((4, 4, 4, 4), 4, (2, 2, 2, 2), 4, 60, bc_t=bc_t)
    A = mg.coarse_op(U, sub, M5, MF, bc_t)
    D = _dense_coarse_by_definition(U, sub, bc_t)
    assert relerr(mg.coarse_dense(A, g), D) < 1e-14
    assert relerr(D, D.conj().T) < 1e-14


@pytest.mark.slow
def test_coarse_op_nine_point_sparsity_extent3():
    """On a 3^4 coarse lattice every leg is a distinct block and exactly 9 block columns
    of each block row of P^dag H P are nonzero (the sparsity after Eq. 4.6)."""
    g, U, sub = _subspace((6, 6, 6, 6), 2, (2, 2, 2, 2), 4, 70, iters=2)
    A = mg.coarse_op(U, sub, M5, MF)
    D = _dense_coarse_by_definition(U, sub)
    nvec, Vc = sub.nvec, g.Vc
    idx = np.arange(Vc)
    for a in range(Vc):
        nz = [b for b in range(Vc)
              if np.abs(D[a * nvec:(a + 1) * nvec, b * nvec:(b + 1) * nvec]).max() > 0]
        assert len(nz) == 9
        blk = D[a * nvec:(a + 1) * nvec, a * nvec:(a + 1) * nvec]
        assert relerr(A[a, 0], blk) < 1e-14
        for mu in range(4):
            for s in (1, -1):
                b = mg.coarse_neighbour(idx[:, None], g, mu, s)[a, 0]
                blk = D[a * nvec:(a + 1) * nvec, b * nvec:(b + 1) * nvec]
                assert relerr(A[a, mg.leg_index(mu, s)], blk) < 1e-14


def test_coarse_op_hermitian_legs():
    """A^{a,a+mu} = (A^{a+mu,a}_{-mu})^dag and A^{aa} Hermitian."""
    g, U, sub = _subspace((4, 6, 4, 6), 2, (2, 2, 2, 2), 4, 80, bc_t=-1)
    A = mg.coarse_op(U, sub, M5, MF, -1)
    idx = np.arange(g.Vc)
    assert np.abs(A[:, 0] - np.conj(np.swapaxes(A[:, 0], -1, -2))).max() < 1e-14
    for mu in range(4):
        nb = mg.coarse_neighbour(idx[:, None], g, mu, +1)[:, 0]
        fwd = A[:, mg.leg_index(mu, +1)]
        bwd = A[nb, mg.leg_index(mu, -1)]
        assert np.abs(fwd - np.conj(np.swapaxes(bwd, -1, -2))).max() < 1e-14


def test_galerkin_identity():
    """apply_coarse(c) = P^dag H P c (Eq. 4.5: A represents M exactly on the subspace)."""
    g, U, sub = _subspace((4, 6, 6, 4), 4, (2, 2, 3, 2), 6, 90)
    A = mg.coarse_op(U, sub, M5, MF)
    rng = synth.rng(91)
    c = rng.standard_normal((g.Vc, sub.nvec)) + 1j * rng.standard_normal((g.Vc, sub.nvec))
    lhs = mg.coarse_apply(A, g, c)
    rhs = mg.restrict(sub, dwf.apply_H(U, mg.prolong(sub, c), M5, MF))
    assert relerr(lhs, rhs) < 1e-14


def _tiny_two_level():
    L, Ls = (4, 2, 2, 2), 4
    g, U, sub = _subspace(L, Ls, (2, 1, 1, 1), 4, 120)
    A = mg.coarse_op(U, sub, M5, MF)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF)
    N = Hd.shape[0]
    E = np.eye(N, dtype=np.complex128).reshape((N,) + g.fine_shape())
    P = mg.prolong(sub, np.eye(g.Vc * sub.nvec).reshape(-1, g.Vc, sub.nvec)).reshape(-1, N).T
    Ad = mg.coarse_dense(A, g)
    Q = P @ np.linalg.solve(Ad, P.conj().T)
    return g, U, sub, A, Hd, P, Q, E


def test_projector_identities():
    """P_L = 1 - M Q and P_R = 1 - Q M: P_L M Q = 0, Q M Q = Q, P_L M = M P_R (Section 4)."""
    g, U, sub, A, Hd, P, Q, _ = _tiny_two_level()
    N = Hd.shape[0]
    assert relerr(P.conj().T @ Hd @ P, mg.coarse_dense(A, g)) < 1e-14
    PL = np.eye(N) - Hd @ Q
    PR = np.eye(N) - Q @ Hd
    scale = np.linalg.norm(Hd, 2) * np.linalg.norm(Q, 2)
    assert np.linalg.norm(PL @ Hd @ Q, 2) / scale < 1e-13
    assert relerr(Q @ Hd @ Q, Q) < 1e-11
    assert relerr(PL @ Hd, Hd @ PR) < 1e-11
    assert relerr(PL @ PL, PL) < 1e-11


def test_vcycle_equals_composite_M_outer():
    """With a fixed linear smoother S and exact Q, the V-cycle equals
    M_outer = S P_L + P_R S + Q - S P_L H S (Section 4)."""
    g, U, sub, A, Hd, P, Q, _ = _tiny_two_level()
    N = Hd.shape[0]
    rng = synth.rng(130)
    Sm = 0.05 * Hd + 0.01 * np.eye(N)                    # a fixed linear smoother
    S = lambda v: (Sm @ v.ravel()).reshape(v.shape)
    Ad = mg.coarse_dense(A, g)
    Qc = lambda c: np.linalg.solve(Ad, c.ravel()).reshape(c.shape)
    p = mg.HDCRParams(M5=M5, mf=MF)
    r = rng.standard_normal(g.fine_shape()) + 1j * rng.standard_normal(g.fine_shape())
    z = mg.vcycle(U, sub, A, r, p, S=S, Qc=Qc)
    PL = np.eye(N) - Hd @ Q
    PR = np.eye(N) - Q @ Hd
    Mo = Sm @ PL + PR @ Sm + Q - Sm @ PL @ Hd @ Sm
    assert relerr(z.ravel(), Mo @ r.ravel()) < 1e-12


def test_post_only_cycle_error_propagator():
    """The post-smoothing cycle (coarse correction, then the smoother) has the error
    propagator (1 - B H) = (1 - S H)(1 - Q H), the product of the two corrections in
    that order; the symmetric cycle's is (1 - S H)(1 - Q H)(1 - S H).  Checked on
    random errors v: v - B H v against the products applied to v."""
    g, U, sub, A, Hd, P, Q, _ = _tiny_two_level()
    N = Hd.shape[0]
    Sm = 0.05 * Hd + 0.01 * np.eye(N)
    S = lambda v: (Sm @ v.ravel()).reshape(v.shape)
    Ad = mg.coarse_dense(A, g)
    Qc = lambda c: np.linalg.solve(Ad, c.ravel()).reshape(c.shape)
    p = mg.HDCRParams(M5=M5, mf=MF)
    E_s, E_q = np.eye(N) - Sm @ Hd, np.eye(N) - Q @ Hd
    rng = synth.rng(131)
    for _ in range(3):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        Hv = (Hd @ v).reshape(g.fine_shape())
        post = v - mg.vcycle(U, sub, A, Hv, p, S=S, Qc=Qc, cycle="post").ravel()
        sym = v - mg.vcycle(U, sub, A, Hv, p, S=S, Qc=Qc, cycle="symmetric").ravel()
        assert relerr(post, E_s @ (E_q @ v)) < 1e-11
        assert relerr(sym, E_s @ (E_q @ (E_s @ v))) < 1e-11
    with pytest.raises(ValueError):
        mg.vcycle(U, sub, A, Hv, p, S=S, Qc=Qc, cycle="pre")


def test_chiral_split_keeps_low_spectrum():
    """Section 4: the gamma5-compatible split eliminates near-zero coarse eigenvalues.
    Built from exact low eigenvectors of H, the coarse operator's smallest |eigenvalue|
    equals H's when the split uses Gamma5 = gamma5 R5, but falls far below it when
    the split uses the 4d gamma5 alone (the reading's evidence)."""
    L, Ls = (4, 2, 2, 2), 4
    g = mg.Geometry(L, Ls, (2, 1, 1, 1))
    U = synth.gauge_field(L, 0.5, 120)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF)
    ev, V = np.linalg.eigh(Hd)
    order = np.argsort(np.abs(ev))
    low = np.stack([V[:, order[i]].reshape(g.fine_shape()) for i in range(4)])
    sub = mg.basis_from_vectors(g, mg.chiral_split(low))
    ea = np.linalg.eigvalsh(mg.coarse_dense(mg.coarse_op(U, sub, M5, MF), g))
    assert abs(np.abs(ea).min() - np.abs(ev).min()) < 1e-10
    g5 = np.concatenate([dwf.spin_mul(dwf.P_PLUS, low), dwf.spin_mul(dwf.P_MINUS, low)])
    sub4 = mg.basis_from_vectors(g, g5)
    ea4 = np.linalg.eigvalsh(mg.coarse_dense(mg.coarse_op(U, sub4, M5, MF), g))
    assert np.abs(ea4).min() < 0.2 * np.abs(ev).min()


def test_hdcr_solve_matches_lu():
    g, U, sub, A, Hd, P, Q, _ = _tiny_two_level()
    b = synth.gaussian_fermion(g.L, g.Ls, 140)
    p = mg.HDCRParams(M5=M5, mf=MF, tol=1e-10, restart=16, max_outer=400)
    x, info = mg.hdcr_solve(U, sub, A, b, p)
    assert info.converged and info.true_resid <= 1e-10
    x_lu = np.linalg.solve(Hd, b.ravel()).reshape(b.shape)
    assert relerr(x, x_lu) < np.linalg.cond(Hd) * 1e-10


def test_coarse_solve_reaches_tolerance():
    g, U, sub, A, *_ = _tiny_two_level()
    rng = synth.rng(150)
    rhs = rng.standard_normal((g.Vc, sub.nvec)) + 0j
    c, info = mg.coarse_solve(A, g, rhs, tol=1e-4)
    assert info.converged
    assert relerr(mg.coarse_apply(A, g, c), rhs) <= 1e-4 * 1.0001


# ------------------------------------------------------------------ Chebyshev
def test_chebyshev_coefficients_closed_form():
    """1/(a + b cos th) = (1/sqrt(a^2 - b^2)) [1 + 2 sum_k (-q)^k cos k th],
    q = (a - sqrt(a^2 - b^2))/b: the series coefficients of 1/y on [lo, hi]."""
    for lo, hi, n in [(1.0, 64.0, 10), (0.25, 9.0, 30), (2.0, 3.0, 5)]:
        a, b = 0.5 * (hi + lo), 0.5 * (hi - lo)
        s = np.sqrt(a * a - b * b)
        q = (a - s) / b
        want = 2.0 / s * (-q) ** np.arange(n + 1)
        got = mg.chebyshev_inverse_coeffs(lo, hi, n)
        # quadrature on 4(n+1) nodes aliases the far tail of the series: ~q^(8n) relative
        assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()


def _cheb_eval(c, t):
    """c_0/2 + sum c_k T_k(t) at a scalar t, T_k(t) = cos(k arccos t) on [-1, 1]."""
    k = np.arange(len(c))
    return float(np.sum(c * np.cos(k * np.arccos(np.clip(t, -1, 1)))) - 0.5 * c[0])


def test_chebyshev_smoother_on_eigenvectors():
    """S v = lambda p(lambda^2) v for an eigenvector (H v = lambda v): the smoother is
    the polynomial H p(H^2) of Section 4, and y p(y) ~ 1 on [1, 64]."""
    L, Ls = (2, 2, 2, 2), 4
    U = synth.gauge_field(L, 0.5, 400)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF)
    ev, V = np.linalg.eigh(Hd)
    p = mg.HDCRParams(M5=M5, mf=MF)
    c = mg.chebyshev_inverse_coeffs(1.0, 64.0, 10)
    shape = (2, 2, 2, 2, Ls, 4, 3)
    for i in [0, len(ev) // 3, np.argmin(np.abs(ev)), len(ev) - 1]:
        lam = ev[i]
        v = V[:, i].reshape(shape)
        Sv = mg.chebyshev_smoother(U, v, p)
        pl = _cheb_eval(c, (2 * lam * lam - 65.0) / 63.0) if 1.0 <= lam * lam <= 64.0 else None
        ratio = np.vdot(v, Sv) / np.vdot(v, v)
        assert relerr(Sv, ratio * v) < 1e-12                 # eigenvector is kept
        if pl is not None:
            assert abs(ratio - lam * pl) < 1e-10 * abs(lam * pl)


def test_chebyshev_filter_on_eigenvectors():
    """The filter maps an eigenvector combination v1 + v2 to T_n(t(l1^2)) v1 + T_n(t(l2^2)) v2
    (up to normalisation): low modes (|l| < lam_cut) are enhanced."""
    L, Ls = (2, 2, 2, 2), 4
    U = synth.gauge_field(L, 0.5, 410)
    Hd = dense_H_from_stencil(dwf, U, Ls, M5, MF)
    ev, V = np.linalg.eigh(Hd)
    i1 = int(np.argmin(np.abs(ev)))
    i2 = int(np.argmax(np.abs(ev) > 2.0))
    shape = (2, 2, 2, 2, Ls, 4, 3)
    x0 = (V[:, i1] + V[:, i2]).reshape(shape)
    lc, lm, n = 1.0, 8.0, 12
    out = mg.chebyshev_filter(U, x0, M5, MF, 1, lc, lm, n)
    tf = lambda lam: (2 * lam * lam - (lm * lm + lc * lc)) / (lm * lm - lc * lc)
    T = lambda t: np.cosh(n * np.arccosh(abs(t))) * (np.sign(t) ** n) if abs(t) > 1 else np.cos(n * np.arccos(t))
    a1, a2 = T(tf(ev[i1])), T(tf(ev[i2]))
    want = (a1 * V[:, i1] + a2 * V[:, i2]).reshape(shape)
    want = want / np.sqrt(dwf.norm2(want))
    assert relerr(out, want) < 1e-10 or relerr(out, -want) < 1e-10
    assert abs(a1) > 10 * abs(a2)
