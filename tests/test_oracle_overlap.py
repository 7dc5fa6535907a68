"""Pins of the continued-fraction overlap oracle (oracle/overlap.py): the stencil
form against the block matrix printed in Section 3 assembled from an independently
assembled dense Wilson kernel, Hermiticity, and the Schur complement on the last
component against the continued fraction in H evaluated on H's eigenvalues."""
import numpy as np
import pytest

import synth
from oracle import dwf, overlap as ov
from pins import dense_H_assembled

L = (2, 2, 2, 2)
M5 = 1.8
BETA = (1.3, 0.9, 1.7, 0.6)   # four coefficients: the printed five-component form
R = 0.35


def _dense_cf(U, beta, R):
    """The oracle's operator as a dense matrix from its action on unit vectors."""
    n = len(beta) + 1
    shp = U.shape[1:5] + (n, 4, 3)
    N = int(np.prod(shp))
    E = np.eye(N, dtype=np.complex128).reshape((N,) + shp)
    return ov.apply_cf(U, E, M5, beta, R).reshape(N, N).T


def _printed_matrix(U, beta, R):
    """The block matrix of Section 3 written out, in the field index
    ((x4*N + i)*4 + spin)*3 + colour, with H = gamma5 D_W assembled site by site
    (pins.dense_H_assembled with Ls = 1 and mf = -1, where the wall term vanishes)."""
    n = len(beta) + 1
    H = dense_H_assembled(dwf, U, 1, M5, -1.0)          # (V4*12)^2
    V4 = H.shape[0] // 12
    c = [1.0 / np.sqrt(beta[i] * beta[i + 1]) for i in range(n - 2)] + [1.0 / np.sqrt(beta[n - 2])]
    blocks = [[np.zeros((12 * V4, 12 * V4), dtype=np.complex128) for _ in range(n)] for _ in range(n)]
    for i in range(n - 1):
        blocks[i][i] = (-1.0) ** i * H
        blocks[i][i + 1] = c[i] * np.eye(12 * V4)
        blocks[i + 1][i] = c[i] * np.eye(12 * V4)
    g5 = np.kron(np.eye(V4), np.kron(dwf.GAMMA5, np.eye(3)))
    blocks[n - 1][n - 1] = R * g5 + beta[0] * H
    # component-major block matrix -> the field's site-major index
    B = np.block(blocks)                                 # index (i, x4, spin, colour)
    perm = np.arange(n * 12 * V4).reshape(n, V4, 12).transpose(1, 0, 2).ravel()
    return B[np.ix_(perm, perm)]


def test_stencil_is_the_printed_matrix():
    U = synth.gauge_field(L, 0.5, 71)
    D = _dense_cf(U, BETA, R)
    P = _printed_matrix(U, BETA, R)
    assert np.abs(D - P).max() < 1e-13 * np.abs(P).max()


def test_hermitian():
    U = synth.gauge_field((4, 4, 2, 4), 0.5, 72)
    rng = synth.rng(73)
    shp = (4, 2, 4, 4, 5, 4, 3)
    x = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    y = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    lhs = np.vdot(x, ov.apply_cf(U, y, M5, BETA, R))
    rhs = np.vdot(ov.apply_cf(U, x, M5, BETA, R), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("beta", [(0.8,), (1.3, 0.9, 1.7, 0.6), (1.1, 0.7, 1.9, 0.5, 1.4, 0.8)])
def test_schur_complement_is_the_continued_fraction(beta):
    """Eliminating the first N - 1 components leaves R gamma5 + f(H) on the last, with f
    the continued fraction of the eigenvalues of H (N = 2, 5, 7)."""
    U = synth.gauge_field(L, 0.5, 74)
    n = len(beta) + 1
    D = _dense_cf(U, beta, R)
    V4 = D.shape[0] // (12 * n)
    idx = np.arange(D.shape[0]).reshape(V4, n, 12)
    last = idx[:, n - 1, :].ravel()
    rest = idx[:, :n - 1, :].ravel()
    S = D[np.ix_(last, last)] - D[np.ix_(last, rest)] @ np.linalg.solve(D[np.ix_(rest, rest)], D[np.ix_(rest, last)])
    H = dense_H_assembled(dwf, U, 1, M5, -1.0)
    lam, V = np.linalg.eigh(H)
    g5 = np.kron(np.eye(V4), np.kron(dwf.GAMMA5, np.eye(3)))
    want = ov.schur_last(lam, beta, R, g5, V)
    assert np.abs(S - want).max() < 1e-10 * np.abs(want).max()
