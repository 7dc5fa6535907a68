"""Oracle: the two-level HDCR preconditioner of Section 4.

Steps, in the paper's order and notation:

1. Subspace vectors phi_k: inverse iteration on Gaussian noise vectors
   (Section 4, option i).  Reading: each noise vector x0 gets a fixed number
   of conjugate-residual iterations on H x = 0 starting from x0 (10 by
   default), then is normalised.
2. Chiral split (Section 4: each vector is split into its left- and
   right-handed parts, which keeps the coarse operator compatible with
   gamma5 and removes near-zero
   eigenvalues of the coarse operator).  Reading: the chirality is that of
   Gamma5 = gamma5 R5, the involution with D_dwf^dag = Gamma5 D_dwf Gamma5
   (the 5d counterpart of gamma5 for Wilson fermions), so each vector v
   becomes P_+ v and P_- v with P_pm = (1 pm Gamma5)/2.  With this split the
   coarse operator built from exact low eigenvectors keeps the smallest
   |eigenvalue| of H, whereas a split by the 4d gamma5 alone creates spurious
   near-zero coarse eigenvalues (both shown in the tests).  Ordering read
   here: the nvec/2 P_+ vectors first, then the nvec/2 P_- vectors
   (chirality-major); the coarse dimension is nvec.
3. Block restriction phi_k^b (Eq. 4.1), blocks of ``block`` = (bx, by, bz, bt)
   sites times the full fifth dimension.
4. Block orthonormalisation so that P_S = sum |phi_k^b><phi_k^b| (Eq. 4.3) is
   a projector.  The paper leaves it implicit; reading: modified
   Gram-Schmidt per block in the fixed order k = 0..nvec-1, applied twice,
   rank deficiency when the remaining norm is < 1e-12 of the original.
5. Little Dirac operator A^{ab}_{jk} = <phi_j^a | H | phi_k^b> (Eq. 4.5).
   Nonzero only for b = a and the 8 nearest coarse neighbours (the sparsity
   noted after Eq. 4.6).  It is stored as 9 legs per coarse site, leg 0 the
   self block and leg 1 + 2 mu + (0 for +mu, 1 for -mu) the hop to a + mu /
   a - mu.  A leg collects only the fine hops in its own direction, so on a
   coarse extent of 2 the +mu and -mu legs reach the same site and are summed.
6. Coarse inverse Q = P A^{-1} P^dag (Eq. 4.6) by conjugate residual on A
   from a zero guess (relative residual 1e-4 by default).
7. Preconditioner, applied as the V-cycle  z1 = S r;  z2 = z1 + Q (r - H z1);
   z = z2 + S (r - H z2),  which for a fixed linear S and exact Q equals the
   composite M_outer = S P_L + P_R S + Q - S P_L H S of Section 4 (the
   calligraphic H there is read as the fine operator).  The smoother S read
   here is a fixed number (8) of CR steps from zero; the order-10 Chebyshev
   smoother of the paper is a variant.
8. Outer flexible GCR on H (``oracle.krylov.fgcr``).

Block-form arrays: a basis is ``Phi`` of shape (nvec, Vc, K), coarse site
a = ((tc*Zc + zc)*Yc + yc)*Xc + xc, K = bt*bz*by*bx*Ls*4*3 in the order
(t, z, y, x inside the block, s, spin, colour).  Coarse vectors are (Vc, nvec).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dwf
from .krylov import cr, fgcr

NLEGS = 9


class RankDeficient(RuntimeError):
    pass


def leg_index(mu: int, sign: int) -> int:
    return 1 + 2 * mu + (0 if sign > 0 else 1)


@dataclass
class Geometry:
    L: tuple          # (Lx, Ly, Lz, Lt)
    Ls: int
    block: tuple      # (bx, by, bz, bt)

    def __post_init__(self):
        self.L = tuple(int(v) for v in self.L)
        self.block = tuple(int(v) for v in self.block)
        for mu in range(4):
            if self.L[mu] % self.block[mu] != 0:
                raise ValueError("block does not divide the lattice")
            if self.L[mu] // self.block[mu] < 2:
                raise ValueError("coarse extent must be at least 2")

    @property
    def Lc(self):
        return tuple(self.L[mu] // self.block[mu] for mu in range(4))

    @property
    def Vc(self):
        return int(np.prod(self.Lc))

    @property
    def K(self):
        return int(np.prod(self.block)) * self.Ls * 12

    def fine_shape(self):
        Lx, Ly, Lz, Lt = self.L
        return (Lt, Lz, Ly, Lx, self.Ls, 4, 3)

    def coarse_shape(self):
        Xc, Yc, Zc, Tc = self.Lc
        return (Tc, Zc, Yc, Xc)


# ----------------------------------------------------------- block reshapes
def to_blocks(g: Geometry, psi: np.ndarray) -> np.ndarray:
    """Fine field(s) (..., Lt,Lz,Ly,Lx,Ls,4,3) -> (..., Vc, K): the block restriction of Eq. 4.1
    laid out per block (step 3 of the header)."""
    lead = psi.shape[:-7]
    bx, by, bz, bt = g.block
    Xc, Yc, Zc, Tc = g.Lc
    n = len(lead)
    a = psi.reshape(lead + (Tc, bt, Zc, bz, Yc, by, Xc, bx, g.Ls, 4, 3))
    perm = list(range(n)) + [n + i for i in (0, 2, 4, 6, 1, 3, 5, 7, 8, 9, 10)]
    a = a.transpose(perm)
    return a.reshape(lead + (g.Vc, g.K))


def from_blocks(g: Geometry, blk: np.ndarray) -> np.ndarray:
    """Inverse of ``to_blocks``."""
    lead = blk.shape[:-2]
    bx, by, bz, bt = g.block
    Xc, Yc, Zc, Tc = g.Lc
    n = len(lead)
    a = blk.reshape(lead + (Tc, Zc, Yc, Xc, bt, bz, by, bx, g.Ls, 4, 3))
    perm = list(range(n)) + [n + i for i in (0, 4, 1, 5, 2, 6, 3, 7, 8, 9, 10)]
    a = a.transpose(perm)
    return np.ascontiguousarray(a.reshape(lead + g.fine_shape()))


def crossing_mask(g: Geometry, mu: int, sign: int) -> np.ndarray:
    """Sites x (4d, shape (Lt,Lz,Ly,Lx)) whose neighbour x + sign*mu lies in another block
    (the hops that connect neighbouring blocks, the sparsity noted after Eq. 4.6)."""
    Lx, Ly, Lz, Lt = g.L
    coords = np.indices((Lt, Lz, Ly, Lx))        # t, z, y, x
    c = coords[3 - mu]
    b = g.block[mu]
    return (c % b) == (b - 1 if sign > 0 else 0)


# ------------------------------------------------------------------ subspace
def smooth_noise(U, x0, M5, mf, bc_t=1, iters: int = 10):
    """Inverse-iteration-like smoothing (Section 4, option i; step 1 of the header):
    ``iters`` CR steps on H x = 0 from x0, normalised."""
    H = lambda v: dwf.apply_H(U, v, M5, mf, bc_t)
    x, _ = cr(H, np.zeros_like(x0), x0=x0, fixed_iters=iters)
    return x / np.sqrt(dwf.norm2(x))


def chiral_split(vs: np.ndarray) -> np.ndarray:
    """Chiral split of Section 4 (step 2 of the header).
    (h, fine...) -> (2h, fine...): [P_+ v_0..P_+ v_{h-1}, P_- v_0..P_- v_{h-1}],
    P_pm = (1 pm Gamma5)/2 with Gamma5 = gamma5 R5."""
    g = dwf.gamma5_r5(vs)
    plus = 0.5 * (vs + g)
    minus = 0.5 * (vs - g)
    return np.concatenate([plus, minus], axis=0)


def block_orthonormalise(Phi: np.ndarray, rank_tol: float = 1e-12) -> np.ndarray:
    """Block orthonormalisation so that P_S of Eq. 4.3 is a projector (step 4 of the header,
    a reading): modified Gram-Schmidt (twice) inside every block, order k = 0..nvec-1.

    Phi: (nvec, Vc, K).  Returns a new array whose vectors are orthonormal in
    each block.  Raises RankDeficient when a vector has nothing left.
    """
    Phi = Phi.copy()
    nvec, Vc, _ = Phi.shape
    for a in range(Vc):
        for k in range(nvec):
            v = Phi[k, a].copy()
            n0 = np.sqrt(np.vdot(v, v).real)
            for _ in range(2):
                for j in range(k):
                    v = v - np.vdot(Phi[j, a], v) * Phi[j, a]
            n = np.sqrt(np.vdot(v, v).real)
            if not (n > rank_tol * n0):
                raise RankDeficient(f"block {a}: vector {k} is linearly dependent")
            Phi[k, a] = v / n
    return Phi


@dataclass
class Subspace:
    geom: Geometry
    Phi: np.ndarray        # (nvec, Vc, K), block-orthonormal

    @property
    def nvec(self):
        return self.Phi.shape[0]


def build_subspace(U, noise, geom: Geometry, M5, mf, bc_t=1, smooth_iters: int = 10) -> Subspace:
    """Section 4: noise -> smoothing -> chiral split -> block restriction -> orthonormalise.

    ``noise``: (nvec/2, Lt,Lz,Ly,Lx,Ls,4,3) Gaussian fields (drawn by the caller).
    """
    sm = np.stack([smooth_noise(U, x0, M5, mf, bc_t, smooth_iters) for x0 in noise])
    vs = chiral_split(sm)
    return Subspace(geom, block_orthonormalise(to_blocks(geom, vs)))


def basis_from_vectors(geom: Geometry, vectors: np.ndarray) -> Subspace:
    """Subspace from given full fine vectors (already split), block-orthonormalised
    (steps 3-4 of the header: Eq. 4.1, Eq. 4.3)."""
    return Subspace(geom, block_orthonormalise(to_blocks(geom, vectors)))


# --------------------------------------------------------- restrict/prolong
def restrict(sub: Subspace, v: np.ndarray) -> np.ndarray:
    """P^dag v: c[a, j] = <phi_j^a, v> (Eq. 4.3 as a map to coarse coordinates)."""
    vb = to_blocks(sub.geom, v)
    return np.einsum("jak,...ak->...aj", np.conj(sub.Phi), vb)


def prolong(sub: Subspace, c: np.ndarray) -> np.ndarray:
    """P c: v = sum_{a,j} c[a, j] phi_j^a (Eq. 4.3: the basis of P_S, from coarse coordinates
    back to the fine field)."""
    vb = np.einsum("jak,...aj->...ak", sub.Phi, c)
    return from_blocks(sub.geom, vb)


# ------------------------------------------------------------ coarse operator
def coarse_op(U, sub: Subspace, M5, mf, bc_t=1) -> np.ndarray:
    """Little Dirac operator A (Vc, 9, nvec, nvec), A[a, d, j, k] = <phi_j^a|H|phi_k^{a+d}>.

    Leg d = (mu, sign) keeps only the fine hops reading x + sign*mu that leave
    the block; the self leg keeps H minus every block-crossing hop.  For each
    leg the images Y_k of all nvec basis vectors are formed first; the block
    inner products <phi_j^a | Y_k^a> of every (j, k) are then one batched matrix
    product per leg (the same sums as Eq. 4.5 term by term).
    """
    g = sub.geom
    nvec = sub.nvec
    A = np.zeros((g.Vc, NLEGS, nvec, nvec), dtype=np.complex128)
    masks = {(mu, s): crossing_mask(g, mu, s)[..., None, None, None]
             for mu in range(4) for s in (+1, -1)}
    phit = np.conj(np.transpose(sub.Phi, (1, 0, 2)))             # (Vc, nvec j, K)
    phis = [from_blocks(g, sub.Phi[k]) for k in range(nvec)]

    def project(Y):                                             # Y: (nvec k, Vc, K)
        return np.matmul(phit, np.transpose(Y, (1, 2, 0)))      # (Vc, j, k)

    Yself = np.stack([to_blocks(g, dwf.apply_H(U, phik, M5, mf, bc_t)) for phik in phis])
    for mu in range(4):
        for s in (+1, -1):
            Yd = np.stack([to_blocks(g, masks[(mu, s)] * dwf.apply_H_hop(U, phik, mu, s, bc_t))
                           for phik in phis])
            Yself -= Yd
            A[:, leg_index(mu, s)] = project(Yd)
    A[:, 0] = project(Yself)
    return A


def coarse_neighbour(c: np.ndarray, g: Geometry, mu: int, sign: int) -> np.ndarray:
    """c(a + sign*mu) on the periodic coarse lattice; c is (Vc, nvec) (the coarse neighbour
    a leg of Eq. 4.5 reaches)."""
    cs = c.reshape(g.coarse_shape() + c.shape[1:])
    ax = 3 - mu
    return np.roll(cs, -sign, axis=ax).reshape(c.shape)


def coarse_apply(A: np.ndarray, g: Geometry, c: np.ndarray) -> np.ndarray:
    """9-point coarse stencil: y[a] = sum_d A[a, d] c[a + d] (A of Eq. 4.5 with the sparsity
    noted after Eq. 4.6)."""
    y = np.einsum("ajk,ak->aj", A[:, 0], c)
    for mu in range(4):
        for s in (+1, -1):
            y = y + np.einsum("ajk,ak->aj", A[:, leg_index(mu, s)], coarse_neighbour(c, g, mu, s))
    return y


def coarse_dense(A: np.ndarray, g: Geometry) -> np.ndarray:
    """The coarse operator of Eq. 4.5 as a dense (Vc*nvec)^2 matrix (legs that alias are summed)."""
    Vc, _, nvec, _ = A.shape
    D = np.zeros((Vc * nvec, Vc * nvec), dtype=np.complex128)
    idx = np.arange(Vc)
    for mu in range(4):
        for s in (+1, -1):
            nb = coarse_neighbour(idx[:, None], g, mu, s)[:, 0]
            for a in range(Vc):
                D[a * nvec:(a + 1) * nvec, nb[a] * nvec:(nb[a] + 1) * nvec] += A[a, leg_index(mu, s)]
    for a in range(Vc):
        D[a * nvec:(a + 1) * nvec, a * nvec:(a + 1) * nvec] += A[a, 0]
    return D


# ------------------------------------------------------------------- solves
def coarse_solve(A, g: Geometry, rhs, tol: float = 1e-4, maxiter: int = 1000):
    """A^{-1} rhs by conjugate residual from zero (Eq. 4.6)."""
    return cr(lambda c: coarse_apply(A, g, c), rhs, tol=tol, maxiter=maxiter)


@dataclass
class HDCRParams:
    M5: float = 1.8
    mf: float = 0.01
    bc_t: int = 1
    tol: float = 1e-10
    restart: int = 8
    max_outer: int = 500
    smoother_steps: int = 8
    coarse_tol: float = 1e-4
    coarse_max: int = 1000


def smoother(U, r, p: HDCRParams):
    """S r: a fixed number of CR steps on H z = r from z = 0 (the CR smoother read in step 7
    of the header; Section 4 uses the Chebyshev one below)."""
    H = lambda v: dwf.apply_H(U, v, p.M5, p.mf, p.bc_t)
    z, _ = cr(H, r, fixed_iters=p.smoother_steps)
    return z


def vcycle(U, sub: Subspace, A, r, p: HDCRParams, S=None, Qc=None, cycle: str = "symmetric"):
    """B r = z2 + S (r - H z2),  z2 = z1 + Q (r - H z1),  z1 = S r  (Section 4).

    ``S`` (fine smoother) and ``Qc`` (coarse inverse on coarse vectors) may be
    replaced by callables, e.g. a linear smoother and an exact coarse solve.
    cycle="post" (a reading, not the paper's composite): the first smoothing is
    dropped, B r = z1 + S (r - H z1) with z1 = Q r.
    """
    H = lambda v: dwf.apply_H(U, v, p.M5, p.mf, p.bc_t)
    if S is None:
        S = lambda v: smoother(U, v, p)
    if Qc is None:
        Qc = lambda c: coarse_solve(A, sub.geom, c, p.coarse_tol, p.coarse_max)[0]
    if cycle == "post":
        z1 = prolong(sub, Qc(restrict(sub, r)))
        return z1 + S(r - H(z1))
    if cycle != "symmetric":
        raise ValueError("cycle must be 'symmetric' or 'post'")
    z1 = S(r)
    r1 = r - H(z1)
    z2 = z1 + prolong(sub, Qc(restrict(sub, r1)))
    r2 = r - H(z2)
    return z2 + S(r2)


def hdcr_solve(U, sub: Subspace, A, b, p: HDCRParams, x0=None):
    """Outer flexible GCR on H preconditioned by the V-cycle (Section 4)."""
    H = lambda v: dwf.apply_H(U, v, p.M5, p.mf, p.bc_t)
    B = lambda r: vcycle(U, sub, A, r, p)
    return fgcr(H, B, b, x0=x0, tol=p.tol, restart=p.restart, maxiter=p.max_outer)


# ------------------------------------------------- Chebyshev variants (Section 4, Fig. 1)
def chebyshev_inverse_coeffs(lo: float, hi: float, order: int) -> np.ndarray:
    """Coefficients c_0..c_order of the truncated Chebyshev series of f(y) = 1/y on
    [lo, hi] (Section 4's smoother: order 10 on [1, 64]), from Chebyshev-Gauss quadrature with 4*(order+1) nodes:
    p(y) = c_0/2 + sum_{k>=1} c_k T_k(t), t = (2y - hi - lo)/(hi - lo)."""
    m = 4 * (order + 1)
    theta = np.pi * (np.arange(m) + 0.5) / m
    y = 0.5 * (hi + lo) + 0.5 * (hi - lo) * np.cos(theta)
    f = 1.0 / y
    return np.array([2.0 / m * np.sum(f * np.cos(k * theta)) for k in range(order + 1)])


def chebyshev_smoother(U, r, p: HDCRParams, lo: float = 1.0, hi: float = 64.0, order: int = 10):
    """S r = H p(H^2) r with p the Chebyshev approximation of 1/y on [lo, hi] (Section 4).

    Reading: the interval of the paper's smoother refers to y = H^2 (the
    spectrum of H reaches |lambda| ~ 8, so [1, 64] covers 1 <= |lambda| <= 8), and
    S = H p(H^2) approximates H^{-1} there.  Linear in r.  The three-term
    recurrence T_{k+1} = 2 t T_k - T_{k-1} runs on vectors with t = (2 H^2 - hi - lo)/(hi - lo)."""
    H = lambda v: dwf.apply_H(U, v, p.M5, p.mf, p.bc_t)
    c = chebyshev_inverse_coeffs(lo, hi, order)
    a, b = 2.0 / (hi - lo), -(hi + lo) / (hi - lo)
    tmap = lambda v: a * H(H(v)) + b * v
    v = H(r)
    t_prev = v
    acc = 0.5 * c[0] * t_prev
    if order >= 1:
        t_cur = tmap(v)
        acc = acc + c[1] * t_cur
        for k in range(2, order + 1):
            t_next = 2.0 * tmap(t_cur) - t_prev
            acc = acc + c[k] * t_next
            t_prev, t_cur = t_cur, t_next
    return acc


def chebyshev_filter(U, x0, M5, mf, bc_t=1, lam_cut: float = 0.5, lam_max: float = 8.0,
                     order: int = 500):
    """T_order(t(H^2)) x0, normalised: the Chebyshev low-pass filter of Fig. 1 (right)
    applied to Gaussian noise (Section 4, option iii).  t maps [lam_cut^2, lam_max^2] onto
    [-1, 1], where |T| <= 1, while modes with |lambda| < lam_cut are enhanced.  The
    recurrence is rescaled every 8 steps (a common factor keeps it exact)."""
    H = lambda v: dwf.apply_H(U, v, M5, mf, bc_t)
    lo, hi = lam_cut * lam_cut, lam_max * lam_max
    a, b = 2.0 / (hi - lo), -(hi + lo) / (hi - lo)
    tmap = lambda v: a * H(H(v)) + b * v
    t_prev = x0
    t_cur = tmap(x0)
    for k in range(2, order + 1):
        t_prev, t_cur = t_cur, 2.0 * tmap(t_cur) - t_prev
        if k % 8 == 0:
            s = 1.0 / np.sqrt(dwf.norm2(t_cur))
            t_prev, t_cur = t_prev * s, t_cur * s
    return t_cur / np.sqrt(dwf.norm2(t_cur))
