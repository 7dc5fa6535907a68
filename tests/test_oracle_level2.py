"""Pins of the third-level oracle (oracle/level2.py), independent of the oracle's own
formulas: the level-2 operator against the brute-force Galerkin product P2^dag A P2
of dense matrices, its sparsity (9 nonzero block columns), Hermitian legs, the chiral
split, and the three-level solve against a dense LU solve."""
import numpy as np
import pytest

from oracle import level2 as l2
from oracle import multigrid as mg


def _dense_A(A, g):
    """The 9-point coarse operator as a dense matrix, built by applying it to unit vectors."""
    n = g.Vc * g.nvec
    D = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        D[:, i] = l2.apply_A(A, g, e.reshape(g.Vc, g.nvec)).ravel()
    return D


def _dense_P2(g, Phi2):
    """P2 as a dense (Vc*nvec) x (Vc2*n2) matrix, column (B, j) = phi2_j^B placed in its block."""
    n2 = Phi2.shape[0]
    P = np.zeros((g.Vc * g.nvec, g.Vc2 * n2), dtype=np.complex128)
    for B in range(g.Vc2):
        for j in range(n2):
            blk = np.zeros((g.Vc2, g.K2), dtype=np.complex128)
            blk[B] = Phi2[j, B]
            P[:, B * n2 + j] = l2.from_blocks(g, blk).ravel()
    return P


@pytest.mark.parametrize("Lc,block,nvec,n2", [((4, 4, 4, 4), (2, 2, 2, 2), 4, 4),
                                              ((6, 4, 4, 6), (3, 2, 2, 3), 4, 6)])
def test_level2_op_is_the_galerkin_product(Lc, block, nvec, n2):
    """A2 = P2^dag A P2 with dense matrices (the densified 9-point A2), on a level-2
    lattice of extent 2 (legs alias) and a mixed 3/2 one."""
    g = l2.CoarseGeometry(Lc, nvec, block)
    A = l2.random_coarse_op(g, 11)
    rng = np.random.default_rng(12)
    v = rng.standard_normal((n2, g.Vc, nvec)) + 1j * rng.standard_normal((n2, g.Vc, nvec))
    Phi2 = l2.basis_from_vectors(g, v)
    A2 = l2.level2_op(A, g, Phi2)
    P = _dense_P2(g, Phi2)
    brute = np.conj(P.T) @ _dense_A(A, g) @ P
    assert np.abs(l2.level2_dense(A2, g) - brute).max() < 1e-12 * np.abs(brute).max()
    # P2 has orthonormal columns (block Gram-Schmidt)
    assert np.abs(np.conj(P.T) @ P - np.eye(P.shape[1])).max() < 1e-12


def test_level2_op_has_nine_points_and_hermitian_legs():
    """On a 3^4 level-2 lattice every block row of A2 has exactly 9 nonzero block
    columns, the self leg is Hermitian and A2^{B,B+mu} = (A2^{B+mu,B}_{(-mu)})^dag."""
    g = l2.CoarseGeometry((6, 6, 6, 6), 2, (2, 2, 2, 2))
    A = l2.random_coarse_op(g, 21)
    rng = np.random.default_rng(22)
    v = rng.standard_normal((2, g.Vc, 2)) + 1j * rng.standard_normal((2, g.Vc, 2))
    Phi2 = l2.basis_from_vectors(g, v)
    A2 = l2.level2_op(A, g, Phi2)
    D = l2.level2_dense(A2, g)
    n2 = 2
    for B in range(g.Vc2):
        nz = sum(np.abs(D[B * n2:(B + 1) * n2, C * n2:(C + 1) * n2]).max() > 1e-12 for C in range(g.Vc2))
        assert nz == 9
    assert np.abs(D - np.conj(D.T)).max() < 1e-12 * np.abs(D).max()
    idx = np.arange(g.Vc2)
    for mu in range(4):
        nb = l2.level2_neighbour(idx, g, mu, +1)
        d = A2[:, mg.leg_index(mu, 1)] - np.conj(np.swapaxes(A2[nb, mg.leg_index(mu, -1)], -1, -2))
        assert np.abs(d).max() < 1e-12 * np.abs(A2).max()


def test_chiral_split_has_definite_coarse_chirality():
    g = l2.CoarseGeometry((4, 4, 4, 4), 6, (2, 2, 2, 2))
    rng = np.random.default_rng(31)
    v = rng.standard_normal((3, g.Vc, 6)) + 1j * rng.standard_normal((3, g.Vc, 6))
    s = l2.chiral_split(v, 6)
    g5 = l2.gamma5_coarse(6)
    assert np.allclose(s[:3] * g5, s[:3]) and np.allclose(s[3:] * g5, -s[3:])
    assert np.allclose(s[:3] + s[3:], v)


def test_three_level_solve_matches_lu():
    """FGCR on the little Dirac operator of the fine oracle (8^4 x 4, 2^4 blocks, nvec 8)
    preconditioned by the level-2 V-cycle (2^4 level-2 blocks, 8 level-2 vectors)
    reaches the LU solution, in fewer outer iterations than plain CR needs."""
    import synth
    from oracle.krylov import cr
    L, Ls, M5, mf = (8, 8, 8, 8), 4, 1.8, 0.05
    U = synth.gauge_field(L, 0.5, 1500)
    g1 = mg.Geometry(L, Ls, (2, 2, 2, 2))
    sub = mg.build_subspace(U, synth.gaussian_fermion(L, Ls, 1501, count=4), g1, M5, mf, smooth_iters=10)
    A = mg.coarse_op(U, sub, M5, mf)
    g = l2.CoarseGeometry(g1.Lc, 8, (2, 2, 2, 2))
    rng = np.random.default_rng(42)
    noise2 = rng.standard_normal((4, g.Vc, 8)) + 1j * rng.standard_normal((4, g.Vc, 8))
    Phi2 = l2.build_level2(A, g, noise2, smooth_iters=10)
    A2 = l2.level2_op(A, g, Phi2)
    b = rng.standard_normal((g.Vc, 8)) + 1j * rng.standard_normal((g.Vc, 8))
    x, info = l2.solve_A(A, g, Phi2, A2, b, tol=1e-11, smooth_iters=4)
    want = np.linalg.solve(_dense_A(A, g), b.ravel()).reshape(b.shape)
    assert info.true_resid <= 1e-11
    assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
    _, icr = cr(lambda c: l2.apply_A(A, g, c), b, tol=1e-11, maxiter=20000)
    assert info.iters < icr.iters
