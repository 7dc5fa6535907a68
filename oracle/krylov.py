"""Oracle: Krylov solvers for a Hermitian (indefinite) operator.

* ``cr`` -- conjugate residual, the solver Section 3 of the paper builds on:
  unlike conjugate gradients it needs the operator to be Hermitian only, not
  positive definite.  The paper does not print the
  recursion; the textbook form used here is:

      r = b - A x,  p = r,  Ar = A r,  Ap = Ar,  gamma = <r, Ar>
      repeat:  alpha = gamma / |Ap|^2
               x += alpha p;   r -= alpha Ap
               Ar = A r;  gamma' = <r, Ar>;  beta = gamma' / gamma
               p = r + beta p;  Ap = Ar + beta Ap

  <r, Ar> is real for Hermitian A; its real part is used.  The stopping test
  is on the recursively updated residual, |r| <= tol |b|.

* ``fgcr`` -- flexible (variable-preconditioned) GCR(m), the outer iteration
  of Section 4, which the paper calls standard and does not document.  The
  reading: z_i = B(r); w_i = A z_i; modified Gram-Schmidt of w_i against the
  earlier w_j of the cycle with the same coefficients applied to z_i;
  normalise; a = <w_i, r>; x += a z_i; r -= a w_i.  After m steps (restart)
  or on convergence of the recursive residual the true residual b - A x is
  recomputed; the solve ends when the TRUE relative residual is <= tol.

Vectors are numpy arrays of any shape; inner products run over all entries.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _dot(u, v) -> complex:
    return complex(np.vdot(u, v))


def _nrm(u) -> float:
    return float(np.sqrt(np.vdot(u, u).real))


@dataclass
class SolveInfo:
    iters: int = 0
    matvecs: int = 0
    converged: bool = False
    resid_history: list = field(default_factory=list)   # |r_k| / |b| (recursive)
    true_resid: float = float("nan")                    # |b - A x| / |b|


def cr(apply, b, x0=None, tol: float = 1e-10, maxiter: int = 10000,
       fixed_iters: int | None = None):
    """Conjugate residual on A x = b (Section 3).

    ``fixed_iters`` runs exactly that many iterations with no convergence test
    (used for the subspace smoothing and the smoother).  Returns (x, SolveInfo).
    """
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if x0 is None or not np.any(x0):
        r = b.copy()
    else:
        r = b - apply(x)
        info.matvecs += 1
    bnorm = _nrm(b)
    scale = bnorm if bnorm > 0 else _nrm(r)
    if scale == 0.0:
        info.converged = True
        info.true_resid = 0.0
        return x, info
    info.resid_history.append(_nrm(r) / scale)
    niter = fixed_iters if fixed_iters is not None else maxiter
    if fixed_iters is None and info.resid_history[-1] <= tol:
        info.converged = True
        info.true_resid = info.resid_history[-1]
        return x, info
    p = r.copy()
    Ar = apply(r)
    info.matvecs += 1
    Ap = Ar.copy()
    gamma = _dot(r, Ar).real
    for k in range(niter):
        alpha = gamma / _dot(Ap, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        info.iters = k + 1
        rn = _nrm(r) / scale
        info.resid_history.append(rn)
        if fixed_iters is None and rn <= tol:
            info.converged = True
            break
        if k == niter - 1:
            break
        Ar = apply(r)
        info.matvecs += 1
        gamma_new = _dot(r, Ar).real
        beta = gamma_new / gamma
        gamma = gamma_new
        p = r + beta * p
        Ap = Ar + beta * Ap
    if fixed_iters is None:
        info.true_resid = _nrm(b - apply(x)) / scale
    return x, info


def fgcr(apply, precond, b, x0=None, tol: float = 1e-10, restart: int = 8,
         maxiter: int = 500):
    """Flexible GCR(m) with a (possibly nonlinear) preconditioner (Section 4).

    Returns (x, SolveInfo) with ``iters`` = outer iterations and ``matvecs``
    = applications of ``apply`` made by the outer loop itself.
    """
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = _nrm(b)
    if bnorm == 0.0:
        info.converged = True
        info.true_resid = 0.0
        return x, info
    r = b - apply(x)
    info.matvecs += 1
    it = 0
    while it < maxiter:
        Z, W = [], []
        for _ in range(restart):
            z = precond(r)
            w = apply(z)
            info.matvecs += 1
            for zj, wj in zip(Z, W):
                beta = _dot(wj, w)
                w = w - beta * wj
                z = z - beta * zj
            nw = _nrm(w)
            w = w / nw
            z = z / nw
            a = _dot(w, r)
            x = x + a * z
            r = r - a * w
            Z.append(z)
            W.append(w)
            it += 1
            rn = _nrm(r) / bnorm
            info.resid_history.append(rn)
            if rn <= tol or it >= maxiter:
                break
        # restart: true residual
        r = b - apply(x)
        info.matvecs += 1
        true = _nrm(r) / bnorm
        if true <= tol:
            info.converged = True
            break
    info.iters = it
    info.true_resid = _nrm(b - apply(x)) / bnorm
    return x, info
