"""Oracle: gauge-link gradient of a solve through H = Gamma5 D_dwf.

Not in the paper (which has no gradient); derived from the operator of
``oracle.dwf``.  For the loss L = Re(eta^dag x) with H x = b:

    dL = -Re(y^dag dH x),  H y = eta  (H is Hermitian),
       = -Re(w^dag dD x),  w = Gamma5 y,

and only the Wilson hops of D depend on U.  Collecting the terms of one link
U_mu(x) gives dL = Re sum_{x,mu} tr(dU_mu(x) F_mu(x)) with

    F_mu(x) = 1/2 sum_s [ B + C^dag ],
    B_{ba} = sum_alpha [(1 - gamma_mu) x(x+mu, s)]_{alpha b} conj(w(x, s)_{alpha a})
    C_{ba} = sum_alpha [(1 + gamma_mu) x(x, s)]_{alpha b}    conj(w(x+mu, s)_{alpha a})

(the t-boundary phase bc_t enters through x(x+mu), w(x+mu)).  Hence
dL/dRe U_{ab} = Re F_{ba}, dL/dIm U_{ab} = -Im F_{ba}, and the derivative along
U -> exp(i h T) U is Re tr(i T U F).  The torch convention for a real loss of a
complex tensor (dL/dRe + i dL/dIm) is therefore F^dag per link.
"""
from __future__ import annotations

import numpy as np

from . import dwf


def gauge_force(U, x, w, bc_t: int = 1) -> np.ndarray:
    """F with dL = Re sum tr(dU F), derived in the header from the Section 3 operator (the paper
    has no gradient); shape (4, Lt, Lz, Ly, Lx, 3, 3), F[mu, ..., p, q] = F_pq."""
    F = np.zeros_like(U)
    for mu in range(4):
        xf = dwf.shift_fermion(x, mu, +1, bc_t)
        wf = dwf.shift_fermion(w, mu, +1, bc_t)
        h = dwf.spin_mul(dwf.IDENT4 - dwf.GAMMA[mu], xf)
        gq = dwf.spin_mul(dwf.IDENT4 + dwf.GAMMA[mu], x)
        B = np.einsum("...sib,...sia->...ba", h, np.conj(w))
        C = np.einsum("...sib,...sia->...ba", gq, np.conj(wf))
        F[mu] = 0.5 * (B + np.conj(np.swapaxes(C, -1, -2)))
    return F


def solve_gradient(U, x, y, bc_t: int = 1):
    """Gradients of L = Re(eta^dag x), H x = b, given x and the adjoint solution y (H y = eta),
    as derived in the header (the paper has no gradient).

    Returns (grad_U, grad_b) in the torch convention: grad_U = F^dag per link,
    grad_b = y.
    """
    w = dwf.gamma5_r5(y)
    F = gauge_force(U, x, w, bc_t)
    return np.conj(np.swapaxes(F, -1, -2)), y
