"""Oracle: red-black (even-odd) preconditioned CGNE, the paper's comparison solver.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 5 compares HDCR with red-black preconditioned CGNE on the same operator (Table 1).
The paper does not write the red-black decomposition out; the standard one for
the Shamir domain-wall operator of ``dwf`` is taken:

* Colour the 4d sites by parity p(x) = (x + y + z + t) mod 2 (all extents even),
  even = 0, odd = 1.  The fifth dimension is site-local, so a 5d site has the
  parity of its 4d site.
* D_dwf = M5 + D_hop with
      M5 psi    = (4 - M5) psi + D_5 psi      (the site-local part: the Wilson mass
                                               term and the fifth-dimension hop),
      D_hop psi = D_W psi - (4 - M5) psi      (the 4d hops; they join opposite
                                               parities only).
* In even-odd blocks D = [[M5, D_eo], [D_oe, M5]]; the Schur complement on the odd
  sites is S = M5 - D_oe M5^{-1} D_eo, and D psi = eta becomes
      eta~_o = eta_o - D_oe M5^{-1} eta_e,   S psi_o = eta~_o,
      psi_e  = M5^{-1} (eta_e - D_eo psi_o).
* CGNE: conjugate gradient on the normal equations S^dag S psi_o = S^dag eta~_o,
  S^dag = Gamma5 S Gamma5 (Gamma5 = gamma5 R5 is site-local, so S inherits the
  Gamma5-hermiticity of D).  The iteration tracks the Schur residual
  t = eta~_o - S psi_o as well; its norm is the norm of the full residual.
* The HDCR solve is posed as H x = b (H = Gamma5 D_dwf), i.e. D x = Gamma5 b.

M5^{-1} is applied here as the inverse of the explicit Ls x Ls matrix of M5 (per
spin, the same for every 4d site and colour), built by applying M5 to the unit
vectors of the fifth dimension.
"""
from __future__ import annotations

import numpy as np

from . import dwf


def parity_mask(L) -> np.ndarray:
    """Boolean (Lt, Lz, Ly, Lx) array: True on odd 4d sites (x + y + z + t odd): the site
    colouring of the red-black CGNE of Section 5, as the header reads it."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2) == 1


def on_parity(psi: np.ndarray, odd: np.ndarray, parity: int) -> np.ndarray:
    """psi with the sites of the other parity set to zero (the red-black split of the header)."""
    keep = odd if parity == 1 else ~odd
    return psi * keep[..., None, None, None]


def m5_apply(psi: np.ndarray, M5: float, mf: float) -> np.ndarray:
    """M5 psi = (4 - M5) psi + D_5 psi (site-local; the diagonal block of the red-black
    decomposition in the header)."""
    return (4.0 - M5) * psi + dwf.d5(psi, mf)


def dhop_apply(U, psi: np.ndarray, M5: float, bc_t: int = 1) -> np.ndarray:
    """The 4d hopping part of D_dwf: D_W psi - (4 - M5) psi (the off-diagonal blocks D_eo,
    D_oe of the red-black decomposition in the header)."""
    return dwf.wilson(U, psi, M5, bc_t) - (4.0 - M5) * psi


def m5_matrix(Ls: int, M5: float, mf: float) -> np.ndarray:
    """(4, Ls, Ls): per spin, the matrix of M5 over the fifth coordinate (for M5^{-1}, see the header)."""
    out = np.zeros((4, Ls, Ls), dtype=np.complex128)
    for s in range(Ls):
        e = np.zeros((1, 1, 1, 1, Ls, 4, 3), dtype=np.complex128)
        e[..., s, :, 0] = 1.0  # unit vector in s, every spin, colour 0
        col = m5_apply(e, M5, mf)[0, 0, 0, 0, :, :, 0]  # (Ls, 4)
        out[:, :, s] = col.T
    return out


def m5_inverse(psi: np.ndarray, M5: float, mf: float) -> np.ndarray:
    """M5^{-1} psi with the inverted Ls x Ls matrices (per spin), as the header reads it."""
    Ls = psi.shape[-3]
    Minv = np.linalg.inv(m5_matrix(Ls, M5, mf))  # (4, Ls, Ls)
    # out[..., s, sp, c] = sum_s' Minv[sp, s, s'] psi[..., s', sp, c]
    return np.einsum("pst,...tpc->...spc", Minv, psi)


def schur_apply(U, v: np.ndarray, odd: np.ndarray, M5: float, mf: float, bc_t: int = 1) -> np.ndarray:
    """Schur complement of the red-black reading in the header: S v = M5 v - D_oe M5^{-1} D_eo v
    on the odd sites (v supported on odd sites)."""
    a = on_parity(dhop_apply(U, v, M5, bc_t), odd, 0)
    b = m5_inverse(a, M5, mf)
    c = on_parity(dhop_apply(U, b, M5, bc_t), odd, 1)
    return on_parity(m5_apply(v, M5, mf), odd, 1) - c


def schur_dag_apply(U, v, odd, M5, mf, bc_t=1):
    """S^dag v = Gamma5 S Gamma5 v (the Gamma5-hermiticity of the Section 3 operator, which S inherits)."""
    return dwf.gamma5_r5(schur_apply(U, dwf.gamma5_r5(v), odd, M5, mf, bc_t))


def cgne_rb_solve(U, b: np.ndarray, M5: float, mf: float, bc_t: int = 1, tol: float = 1e-10,
                  maxiter: int = 100000):
    """H x = b by red-black CGNE, the comparison solver of Section 5 (Table 1), in the
    reading of the header.  Returns (x, iterations, |b - H x| / |b|)."""
    L = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    odd = parity_mask(L)
    eta = dwf.gamma5_r5(b)  # D x = Gamma5 b
    eta_e, eta_o = on_parity(eta, odd, 0), on_parity(eta, odd, 1)
    eta_t = eta_o - on_parity(dhop_apply(U, m5_inverse(eta_e, M5, mf), M5, bc_t), odd, 1)
    x = np.zeros_like(b)
    t = eta_t.copy()
    r = schur_dag_apply(U, t, odd, M5, mf, bc_t)
    p = r.copy()
    rr = dwf.norm2(r)
    stop2 = (tol ** 2) * dwf.norm2(eta)
    it = 0
    while dwf.norm2(t) > stop2 and it < maxiter:
        q = schur_apply(U, p, odd, M5, mf, bc_t)
        alpha = rr / dwf.norm2(q)
        x = x + alpha * p
        t = t - alpha * q
        r = r - alpha * schur_dag_apply(U, q, odd, M5, mf, bc_t)
        rr_new = dwf.norm2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    # psi_e = M5^{-1} (eta_e - D_eo psi_o)
    x_e = m5_inverse(eta_e - on_parity(dhop_apply(U, x, M5, bc_t), odd, 0), M5, mf)
    x = x + on_parity(x_e, odd, 0)
    res = np.sqrt(dwf.norm2(b - dwf.apply_H(U, x, M5, mf, bc_t)) / dwf.norm2(b))
    return x, it, res
