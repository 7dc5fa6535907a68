"""Oracle: a third level -- the two-level construction of Section 4 applied to the
little Dirac operator itself (Section 5 names recursion as the way to solve the
coarse system more exactly).  Test infrastructure only: the tests and the CPU
baseline use it; the CUDA library never does.

Reading of the recursion (the paper gives none of the details): every step of
Section 4 is repeated with the coarse operator A (Eq. 4.5) in place of H and the
coarse lattice in place of the fine one.

1. Level-2 vectors: Gaussian noise on the coarse lattice, each smoothed by a
   fixed number of conjugate-residual steps on A x = 0 (Section 4's inverse
   iteration on Gaussian noise, with A in place of H), then normalised.
2. Chiral split with the coarse Gamma5.  Every level-1 basis vector has definite
   Gamma5 chirality (the nvec/2 P_+ vectors first, then the P_- ones), so
   P^dag Gamma5 P = Gamma5c = diag(+1 x nvec/2, -1 x nvec/2) on every coarse site;
   a level-2 vector v becomes (1 + Gamma5c) v / 2 and (1 - Gamma5c) v / 2.
3. Blocks of b2 coarse sites times all nvec components (Eq. 4.1 on the coarse
   lattice); modified Gram-Schmidt, twice, in each block, order k = 0..n2-1.
4. A2^{BC}_{jk} = <phi_j^B | A | phi_k^C> (Eq. 4.5 with A for H), nonzero for
   C = B and the 8 nearest level-2 neighbours; a leg collects the coarse hops of
   A from block B into block B +- mu, the self leg everything else.
5. The coarse solve of the two-level V-cycle becomes a solve of A by flexible GCR
   preconditioned with the same V-cycle one level down: smoother S_A (CR steps on
   A from zero), the level-2 correction P2 A2^{-1} P2^dag (exact), smoother again.

Array conventions: coarse vectors (Vc, nvec) with a = ((tc*Zc + zc)*Yc + yc)*Xc + xc;
a level-2 basis Phi2 (n2, Vc2, K2), K2 = bt*bz*by*bx*nvec in the order (t, z, y, x
inside the block, component); A2 (Vc2, 9, n2, n2) with the leg numbering of
``oracle.multigrid``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .krylov import cr, fgcr
from .multigrid import NLEGS, RankDeficient, leg_index


@dataclass
class CoarseGeometry:
    Lc: tuple        # coarse extents (Xc, Yc, Zc, Tc)
    nvec: int        # components per coarse site (level-1 basis size)
    block: tuple     # level-2 block (bx, by, bz, bt) in coarse sites

    def __post_init__(self):
        self.Lc = tuple(int(v) for v in self.Lc)
        self.block = tuple(int(v) for v in self.block)
        for mu in range(4):
            if self.Lc[mu] % self.block[mu] != 0:
                raise ValueError("level-2 block does not divide the coarse lattice")
            if self.Lc[mu] // self.block[mu] < 2:
                raise ValueError("level-2 extent must be at least 2")

    @property
    def Vc(self):
        return int(np.prod(self.Lc))

    @property
    def L2(self):
        return tuple(self.Lc[mu] // self.block[mu] for mu in range(4))

    @property
    def Vc2(self):
        return int(np.prod(self.L2))

    @property
    def K2(self):
        return int(np.prod(self.block)) * self.nvec

    def shape(self):
        Xc, Yc, Zc, Tc = self.Lc
        return (Tc, Zc, Yc, Xc)


def gamma5_coarse(nvec: int) -> np.ndarray:
    """Gamma5c on one coarse site (step 2 of the header): +1 for the nvec/2 P_+ basis vectors,
    -1 for the rest."""
    return np.concatenate([np.ones(nvec // 2), -np.ones(nvec // 2)])


def neighbour(c: np.ndarray, g: CoarseGeometry, mu: int, sign: int) -> np.ndarray:
    """c(a + sign*mu) on the periodic coarse lattice (the neighbour a leg of Eq. 4.5 reaches);
    c is (..., Vc, nvec)."""
    lead = c.shape[:-2]
    cs = c.reshape(lead + g.shape() + (g.nvec,))
    ax = len(lead) + 3 - mu
    return np.roll(cs, -sign, axis=ax).reshape(c.shape)


def apply_leg(A: np.ndarray, g: CoarseGeometry, c: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """The one leg (mu, sign) of the 9-point coarse stencil of Eq. 4.5: y[a] = A[a, leg] c[a + sign mu]."""
    return np.einsum("ajk,ak->aj", A[:, leg_index(mu, sign)], neighbour(c, g, mu, sign))


def apply_A(A: np.ndarray, g: CoarseGeometry, c: np.ndarray) -> np.ndarray:
    """The 9-point coarse stencil y[a] = sum_d A[a, d] c[a + d] (the operator of Eq. 4.5)."""
    y = np.einsum("ajk,ak->aj", A[:, 0], c)
    for mu in range(4):
        for s in (+1, -1):
            y = y + apply_leg(A, g, c, mu, s)
    return y


# ----------------------------------------------------------- level-2 blocks
def to_blocks(g: CoarseGeometry, c: np.ndarray) -> np.ndarray:
    """Coarse vector(s) (..., Vc, nvec) -> (..., Vc2, K2): the block restriction of Eq. 4.1
    on the coarse lattice (step 3 of the header)."""
    lead = c.shape[:-2]
    bx, by, bz, bt = g.block
    X2, Y2, Z2, T2 = g.L2
    n = len(lead)
    a = c.reshape(lead + (T2, bt, Z2, bz, Y2, by, X2, bx, g.nvec))
    perm = list(range(n)) + [n + i for i in (0, 2, 4, 6, 1, 3, 5, 7, 8)]
    return a.transpose(perm).reshape(lead + (g.Vc2, g.K2))


def from_blocks(g: CoarseGeometry, b: np.ndarray) -> np.ndarray:
    """Inverse of ``to_blocks``."""
    lead = b.shape[:-2]
    bx, by, bz, bt = g.block
    X2, Y2, Z2, T2 = g.L2
    n = len(lead)
    a = b.reshape(lead + (T2, Z2, Y2, X2, bt, bz, by, bx, g.nvec))
    perm = list(range(n)) + [n + i for i in (0, 4, 1, 5, 2, 6, 3, 7, 8)]
    return np.ascontiguousarray(a.transpose(perm).reshape(lead + (g.Vc, g.nvec)))


def crossing_mask(g: CoarseGeometry, mu: int, sign: int) -> np.ndarray:
    """(Vc, 1): coarse sites whose neighbour a + sign*mu lies in another level-2 block (the
    hops that make the legs of step 4)."""
    Xc, Yc, Zc, Tc = g.Lc
    coords = np.indices((Tc, Zc, Yc, Xc))
    c = coords[3 - mu]
    b = g.block[mu]
    return ((c % b) == (b - 1 if sign > 0 else 0)).reshape(-1, 1)


def block_orthonormalise(Phi: np.ndarray, rank_tol: float = 1e-12) -> np.ndarray:
    """Step 3 (the projector of Eq. 4.3 on the coarse lattice, a reading): modified Gram-Schmidt
    (twice) inside every level-2 block, order k = 0..n2-1."""
    Phi = Phi.copy()
    n2, Vc2, _ = Phi.shape
    for a in range(Vc2):
        for k in range(n2):
            v = Phi[k, a].copy()
            n0 = np.sqrt(np.vdot(v, v).real)
            for _ in range(2):
                for j in range(k):
                    v = v - np.vdot(Phi[j, a], v) * Phi[j, a]
            n = np.sqrt(np.vdot(v, v).real)
            if not (n > rank_tol * n0):
                raise RankDeficient(f"level-2 block {a}: vector {k} is linearly dependent")
            Phi[k, a] = v / n
    return Phi


def chiral_split(vs: np.ndarray, nvec: int) -> np.ndarray:
    """Step 2 (the chiral split of Section 4 with the coarse Gamma5):
    (h, Vc, nvec) -> (2h, Vc, nvec): [P+ v_0..P+ v_{h-1}, P- v_0..P- v_{h-1}] with
    P+- = (1 +- Gamma5c)/2."""
    g5 = gamma5_coarse(nvec)
    plus = 0.5 * (vs + vs * g5)
    minus = 0.5 * (vs - vs * g5)
    return np.concatenate([plus, minus], axis=0)


def build_level2(A: np.ndarray, g: CoarseGeometry, noise: np.ndarray, smooth_iters: int = 10) -> np.ndarray:
    """Steps 1-3: level-2 basis Phi2 (n2, Vc2, K2) from noise (n2/2, Vc, nvec)."""
    op = lambda c: apply_A(A, g, c)
    sm = []
    for x0 in noise:
        x, _ = cr(op, np.zeros_like(x0), x0=x0, fixed_iters=smooth_iters)
        sm.append(x / np.sqrt(np.vdot(x, x).real))
    vs = chiral_split(np.stack(sm), g.nvec)
    return block_orthonormalise(to_blocks(g, vs))


def basis_from_vectors(g: CoarseGeometry, vectors: np.ndarray) -> np.ndarray:
    """Level-2 basis from given coarse vectors (n2, Vc, nvec), block-orthonormalised (step 3)."""
    return block_orthonormalise(to_blocks(g, vectors))


def restrict(g: CoarseGeometry, Phi2: np.ndarray, c: np.ndarray) -> np.ndarray:
    """P2^dag c: c2[B, j] = <phi2_j^B, c> (Eq. 4.3 on the coarse lattice, to level-2 coordinates)."""
    return np.einsum("jbk,...bk->...bj", np.conj(Phi2), to_blocks(g, c))


def prolong(g: CoarseGeometry, Phi2: np.ndarray, c2: np.ndarray) -> np.ndarray:
    """P2 c2 = sum_{B, j} c2[B, j] phi2_j^B (Eq. 4.3 on the coarse lattice, back to coarse vectors)."""
    return from_blocks(g, np.einsum("jbk,...bj->...bk", Phi2, c2))


def level2_op(A: np.ndarray, g: CoarseGeometry, Phi2: np.ndarray) -> np.ndarray:
    """Step 4: A2 (Vc2, 9, n2, n2), A2[B, d, j, k] = <phi2_j^B | A | phi2_k^{B+d}>.  Leg d
    keeps the coarse hops of A leaving block B in its direction; the self leg keeps A
    minus every block-crossing hop."""
    n2 = Phi2.shape[0]
    A2 = np.zeros((g.Vc2, NLEGS, n2, n2), dtype=np.complex128)
    for k in range(n2):
        phik = from_blocks(g, Phi2[k])
        Yself = apply_A(A, g, phik)
        for mu in range(4):
            for s in (+1, -1):
                Yd = crossing_mask(g, mu, s) * apply_leg(A, g, phik, mu, s)
                Yself = Yself - Yd
                A2[:, leg_index(mu, s), :, k] = np.einsum("jbk,bk->bj", np.conj(Phi2), to_blocks(g, Yd))
        A2[:, 0, :, k] = np.einsum("jbk,bk->bj", np.conj(Phi2), to_blocks(g, Yself))
    return A2


def level2_neighbour(idx: np.ndarray, g: CoarseGeometry, mu: int, sign: int) -> np.ndarray:
    """Level-2 block index B + sign*mu (periodic) for an array of block indices (the block a
    leg of step 4 reaches)."""
    X2, Y2, Z2, T2 = g.L2
    c = [idx % X2, (idx // X2) % Y2, (idx // (X2 * Y2)) % Z2, idx // (X2 * Y2 * Z2)]
    c[mu] = (c[mu] + sign) % g.L2[mu]
    return ((c[3] * Z2 + c[2]) * Y2 + c[1]) * X2 + c[0]


def level2_dense(A2: np.ndarray, g: CoarseGeometry) -> np.ndarray:
    """A2 of step 4 as a dense (Vc2*n2)^2 matrix (legs reaching the same block add up)."""
    Vc2, _, n2, _ = A2.shape
    D = np.zeros((Vc2 * n2, Vc2 * n2), dtype=np.complex128)
    for B in range(Vc2):
        D[B * n2:(B + 1) * n2, B * n2:(B + 1) * n2] += A2[B, 0]
        for mu in range(4):
            for s in (+1, -1):
                C = int(level2_neighbour(np.array(B), g, mu, s))
                D[B * n2:(B + 1) * n2, C * n2:(C + 1) * n2] += A2[B, leg_index(mu, s)]
    return D


def apply_A2(A2: np.ndarray, g: CoarseGeometry, c2: np.ndarray) -> np.ndarray:
    """The 9-point level-2 stencil (A2 of step 4) on (Vc2, n2) vectors."""
    idx = np.arange(g.Vc2)
    y = np.einsum("bjk,bk->bj", A2[:, 0], c2)
    for mu in range(4):
        for s in (+1, -1):
            y = y + np.einsum("bjk,bk->bj", A2[:, leg_index(mu, s)], c2[level2_neighbour(idx, g, mu, s)])
    return y


# ------------------------------------------------------------------- solve
def vcycle2(A: np.ndarray, g: CoarseGeometry, Phi2: np.ndarray, A2inv: np.ndarray, r: np.ndarray,
            smooth_iters: int = 4) -> np.ndarray:
    """Step 5's preconditioner on a coarse residual r:  z1 = S_A r;
    z2 = z1 + P2 A2^{-1} P2^dag (r - A z1);  z = z2 + S_A (r - A z2),  S_A a fixed number of
    CR steps on A from zero, A2^{-1} exact (a dense inverse)."""
    op = lambda c: apply_A(A, g, c)
    S = lambda v: cr(op, v, fixed_iters=smooth_iters)[0]
    z1 = S(r)
    c2 = restrict(g, Phi2, r - op(z1))
    z2 = z1 + prolong(g, Phi2, (A2inv @ c2.ravel()).reshape(c2.shape))
    return z2 + S(r - op(z2))


def solve_A(A: np.ndarray, g: CoarseGeometry, Phi2: np.ndarray, A2: np.ndarray, rhs: np.ndarray,
            tol: float = 1e-10, smooth_iters: int = 4, restart: int = 8, maxiter: int = 500):
    """Step 5: A x = rhs by flexible GCR preconditioned with ``vcycle2``."""
    A2inv = np.linalg.inv(level2_dense(A2, g))
    op = lambda c: apply_A(A, g, c)
    B = lambda v: vcycle2(A, g, Phi2, A2inv, v, smooth_iters)
    return fgcr(op, B, rhs, tol=tol, restart=restart, maxiter=maxiter)


def random_coarse_op(g: CoarseGeometry, seed: int, diag: float = 4.0) -> np.ndarray:
    """A random Hermitian 9-point coarse operator on g's coarse lattice (for pins that do
    not need a fine operator): A[a, 0] Hermitian with ``diag`` on the diagonal, the
    forward legs random and each backward leg the adjoint of its partner's forward leg."""
    rng = np.random.default_rng(seed)
    n, Vc = g.nvec, g.Vc
    A = np.zeros((Vc, NLEGS, n, n), dtype=np.complex128)
    G = rng.standard_normal((Vc, n, n)) + 1j * rng.standard_normal((Vc, n, n))
    A[:, 0] = 0.25 * (G + np.conj(np.swapaxes(G, -1, -2))) + diag * np.eye(n)
    idx = np.arange(Vc)
    for mu in range(4):
        F = 0.5 * (rng.standard_normal((Vc, n, n)) + 1j * rng.standard_normal((Vc, n, n)))
        A[:, leg_index(mu, +1)] = F
        fwd = neighbour(idx[:, None].astype(float) * np.ones((1, n)), g, mu, +1)[:, 0].astype(int)
        # the backward leg of site a + mu is the adjoint of site a's forward leg
        A[fwd, leg_index(mu, -1)] = np.conj(np.swapaxes(F, -1, -2))
    return A
