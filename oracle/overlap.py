"""Oracle: the continued-fraction overlap operator of Section 3.  Test
infrastructure only (the tests and the CPU baseline use it; the CUDA library
never does).

Section 3 notes that the continued-fraction form of the overlap operator with
the Hermitian Wilson kernel H = H_W is already Hermitian indefinite and prints
it for five components: a block-tridiagonal matrix whose diagonal blocks are
H, -H, H, -H and R gamma5 + beta_0 H, and whose off-diagonal blocks are the
scalars 1/sqrt(beta_0 beta_1), 1/sqrt(beta_1 beta_2), 1/sqrt(beta_2 beta_3) and
1/sqrt(beta_3) (symmetric).

Readings:
* H = gamma5 D_W, D_W the Wilson operator of ``oracle.dwf`` with mass -M5 (the
  kernel of the domain-wall operator of the same section).
* Other sizes: N components (N >= 2) with N - 1 coefficients beta_0..beta_{N-2};
  diagonal (-1)^i H for i < N - 1 and R gamma5 + beta_0 H for the last; coupling
  1/sqrt(beta_i beta_{i+1}) between components i and i + 1 for i < N - 2 and
  1/sqrt(beta_{N-2}) between N - 2 and N - 1.  N = 5 is the printed matrix.
* A field stores its N components where a domain-wall field stores s: shape
  (..., Lt, Lz, Ly, Lx, N, 4, 3).

Eliminating the first N - 1 components leaves, on the last one, the Schur
complement R gamma5 + beta_0 H - c_{N-2}^2 K_{N-2}(H)^{-1} with the continued
fraction K_0 = H, K_i = (-1)^i H - c_{i-1}^2 K_{i-1}^{-1} (c_i the couplings): a
rational function of H, which is how the overlap's sign function enters.
"""
from __future__ import annotations

import numpy as np

from . import dwf


def couplings(beta) -> np.ndarray:
    """The N - 1 off-diagonal scalars of the Section 3 continued-fraction matrix for
    N = len(beta) + 1 components."""
    b = np.asarray(beta, dtype=float)
    n = len(b)
    c = np.empty(n)
    for i in range(n - 1):
        c[i] = 1.0 / np.sqrt(b[i] * b[i + 1])
    c[n - 1] = 1.0 / np.sqrt(b[n - 1])
    return c


def diag_scales(beta) -> np.ndarray:
    """The factor of H on each diagonal block of the Section 3 continued-fraction matrix:
    (-1)^i, and beta_0 on the last."""
    n = len(beta) + 1
    s = np.array([(-1.0) ** i for i in range(n)])
    s[-1] = beta[0]
    return s


def apply_HW(U, psi, M5: float, bc_t: int = 1) -> np.ndarray:
    """H_W = gamma5 D_W on every component (the Hermitian Wilson kernel of Section 3)."""
    return dwf.spin_mul(dwf.GAMMA5, dwf.wilson(U, psi, M5, bc_t))


def apply_cf(U, psi, M5: float, beta, R: float, bc_t: int = 1) -> np.ndarray:
    """The continued-fraction operator of Section 3 on an N-component field (N = len(beta) + 1)."""
    n = psi.shape[-3]
    if n != len(beta) + 1:
        raise ValueError("the field must have len(beta) + 1 components")
    hw = apply_HW(U, psi, M5, bc_t)
    s = diag_scales(beta)
    c = couplings(beta)
    out = hw * s[:, None, None]
    out[..., n - 1, :, :] += R * dwf.spin_mul(dwf.GAMMA5, psi[..., n - 1, :, :])
    for i in range(n - 1):
        out[..., i, :, :] += c[i] * psi[..., i + 1, :, :]
        out[..., i + 1, :, :] += c[i] * psi[..., i, :, :]
    return out


def schur_last(hw_eigvals, beta, R, g5, V):
    """The Schur complement of the Section 3 matrix on the last component from the continued fraction of
    the eigenvalues of H (V its eigenvectors as columns, g5 gamma5 as a matrix in
    the same basis as V's rows): R g5 + V diag(f(lambda)) V^dag."""
    c = couplings(beta)
    n = len(beta) + 1
    lam = np.asarray(hw_eigvals, dtype=float)
    K = lam.copy()                       # K_0 = lambda
    for i in range(1, n - 1):
        K = (-1.0) ** i * lam - c[i - 1] ** 2 / K
    f = beta[0] * lam - c[n - 2] ** 2 / K if n > 1 else beta[0] * lam
    return R * g5 + (V * f) @ np.conj(V.T)


# ------------------------------------------------ the two-level method on it
def apply_cf_hop(U, psi, mu: int, sign: int, beta, bc_t: int = 1) -> np.ndarray:
    """The part of the Section 3 continued-fraction operator made of the single 4d hop reading
    psi(x + sign*mu): component i gets (-1)^i (beta_0 on the last) times
    gamma5 (-1/2) hop(mu, sign) of its own component (the couplings and R gamma5 are
    site-local and belong to no hop)."""
    s = diag_scales(beta)
    h = dwf.spin_mul(dwf.GAMMA5, -0.5 * dwf.hop(U, psi, mu, sign, bc_t))
    return h * s[:, None, None]


def cf_coarse_op(U, sub, M5: float, beta, R: float, bc_t: int = 1) -> np.ndarray:
    """Little operator of the continued-fraction operator on the block basis ``sub``
    (an ``oracle.multigrid.Subspace`` whose fifth coordinate holds the N components):
    A[a, d, j, k] = <phi_j^a | H_cf | phi_k^{a+d}>, the construction of Section 4
    applied to H_cf.  As for the domain-wall operator, leg d = (mu, sign) keeps the
    hops reading x + sign*mu that leave the block and the self leg keeps the rest
    (the components' couplings and R gamma5 are site-local, so they stay in it)."""
    from . import multigrid as mg
    g = sub.geom
    nvec = sub.nvec
    A = np.zeros((g.Vc, mg.NLEGS, nvec, nvec), dtype=np.complex128)
    phit = np.conj(np.transpose(sub.Phi, (1, 0, 2)))             # (Vc, j, K)
    phis = [mg.from_blocks(g, sub.Phi[k]) for k in range(nvec)]

    def project(Y):                                             # Y: (k, Vc, K)
        return np.matmul(phit, np.transpose(Y, (1, 2, 0)))

    Yself = np.stack([mg.to_blocks(g, apply_cf(U, p, M5, beta, R, bc_t)) for p in phis])
    for mu in range(4):
        for s in (+1, -1):
            m = mg.crossing_mask(g, mu, s)[..., None, None, None]
            Yd = np.stack([mg.to_blocks(g, m * apply_cf_hop(U, p, mu, s, beta, bc_t)) for p in phis])
            Yself -= Yd
            A[:, mg.leg_index(mu, s)] = project(Yd)
    A[:, 0] = project(Yself)
    return A
