"""Oracle: the Hermitian-indefinite domain-wall operator H = Gamma5 D_dwf.

Section 3 of the paper defines the operator used throughout as
H_dwf = gamma5 R5 D_dwf = Gamma5 D_dwf (Shamir domain wall, i.e. the Cayley
form with c = 0, b = 1) but never writes D_dwf out.  The readings taken here:

* Gamma matrices in the chiral basis, gamma_k = [[0, -i s_k], [i s_k, 0]]
  (k = 1..3, s_k the Pauli matrices) and gamma_4 = [[0, 1], [1, 0]], so that
  gamma5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).  The paper
  fixes no basis; any basis has the same spectrum.
* 4d Wilson part, per fifth coordinate s:
      (D_W psi)(x) = (4 - M5) psi(x)
                     - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                  + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ].
* Fifth-dimension part:
      (D_5 psi)(s) = psi(s) - P_- psi(s + 1) - P_+ psi(s - 1),
  with P_pm = (1 pm gamma5)/2 and the walls psi(Ls) = -mf psi(0),
  psi(-1) = -mf psi(Ls - 1).  This orientation makes Gamma5 D_dwf Hermitian.
* D_dwf = D_W + D_5; Gamma5 = gamma5 R5 with (R5 psi)(s) = psi(Ls - 1 - s),
  so (H psi)(x, s) = gamma5 (D_dwf psi)(x, Ls - 1 - s).
* Periodic boundaries in x, y, z; in t the hop across the boundary carries
  the factor ``bc_t`` (+1 periodic, -1 antiperiodic).  The paper is silent on
  boundaries.  On an extent-2 direction the +mu and -mu neighbours coincide
  and both hops are summed.

Fermion fields have shape ``(..., Lt, Lz, Ly, Lx, Ls, 4, 3)`` (any leading
batch axes); gauge fields ``(4, Lt, Lz, Ly, Lx, 3, 3)``.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------- gamma basis
SIGMA = np.array(
    [
        [[0, 1], [1, 0]],
        [[0, -1j], [1j, 0]],
        [[1, 0], [0, -1]],
    ],
    dtype=np.complex128,
)


def _chiral_gammas() -> np.ndarray:
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    z = np.zeros((2, 2))
    for k in range(3):
        g[k] = np.block([[z, -1j * SIGMA[k]], [1j * SIGMA[k], z]])
    g[3] = np.block([[z, np.eye(2)], [np.eye(2), z]])
    return g


GAMMA = _chiral_gammas()                       # gamma_mu, mu = 0..3 <-> x, y, z, t
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
IDENT4 = np.eye(4, dtype=np.complex128)
P_PLUS = 0.5 * (IDENT4 + GAMMA5)
P_MINUS = 0.5 * (IDENT4 - GAMMA5)

# numpy axis (counted from the end of a fermion array) of direction mu
_F_AXIS = {0: -4, 1: -5, 2: -6, 3: -7}
# numpy axis of direction mu in a single-direction gauge array (Lt, Lz, Ly, Lx, 3, 3)
_G_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


# ------------------------------------------------------------------- helpers
def inner(u: np.ndarray, v: np.ndarray) -> complex:
    """<u, v> = sum conj(u) v over all entries."""
    return complex(np.vdot(u, v))


def norm2(u: np.ndarray) -> float:
    return float(np.vdot(u, u).real)


def spin_mul(M: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix at every site."""
    return np.matmul(M, psi)


def color_mul(Umu: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)(x, s) = U(x) psi(x, s) for a single-direction link field Umu."""
    return np.matmul(psi, np.swapaxes(Umu, -1, -2)[..., None, :, :])


def color_mul_dag(Umu: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U^dag psi)(x, s) = U(x)^dag psi(x, s)."""
    return np.matmul(psi, np.conj(Umu)[..., None, :, :])


def shift_fermion(psi: np.ndarray, mu: int, sign: int, bc_t: int) -> np.ndarray:
    """psi(x + sign*mu) as a field over x; the t-boundary hop picks up bc_t."""
    ax = _F_AXIS[mu]
    out = np.roll(psi, -sign, axis=ax)
    if mu == 3 and bc_t != 1:
        Lt = psi.shape[ax]
        idx = [slice(None)] * psi.ndim
        idx[psi.ndim + ax] = Lt - 1 if sign > 0 else 0
        out[tuple(idx)] *= bc_t
    return out


def shift_links(Umu: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """U_mu(x + sign*mu) as a field over x (links carry no boundary phase)."""
    return np.roll(Umu, -sign, axis=_G_AXIS[mu])


# ------------------------------------------------------------- the operator
def hop(U: np.ndarray, psi: np.ndarray, mu: int, sign: int, bc_t: int) -> np.ndarray:
    """One Wilson hop of D_W (Section 3's kernel, as read in the header; without the -1/2):

    sign=+1: (1 - gamma_mu) U_mu(x) psi(x + mu)
    sign=-1: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
    """
    if sign > 0:
        t = color_mul(U[mu], shift_fermion(psi, mu, +1, bc_t))
        return spin_mul(IDENT4 - GAMMA[mu], t)
    t = color_mul_dag(shift_links(U[mu], mu, -1), shift_fermion(psi, mu, -1, bc_t))
    return spin_mul(IDENT4 + GAMMA[mu], t)


def wilson(U, psi, M5: float, bc_t: int = 1) -> np.ndarray:
    """4d Wilson operator with mass -M5 (the kernel of Section 3's D_dwf, read as in the
    header), applied independently at each s."""
    out = (4.0 - M5) * psi
    for mu in range(4):
        out = out - 0.5 * (hop(U, psi, mu, +1, bc_t) + hop(U, psi, mu, -1, bc_t))
    return out


def d5(psi: np.ndarray, mf: float) -> np.ndarray:
    """Fifth-dimension part of Section 3's D_dwf (read as in the header), with the mass mf
    at the walls (no gauge links in s)."""
    up = np.roll(psi, -1, axis=-3)           # psi(s + 1)
    up[..., -1, :, :] *= -mf                 # psi(Ls) = -mf psi(0)
    dn = np.roll(psi, +1, axis=-3)           # psi(s - 1)
    dn[..., 0, :, :] *= -mf                  # psi(-1) = -mf psi(Ls - 1)
    return psi - spin_mul(P_MINUS, up) - spin_mul(P_PLUS, dn)


def ddwf(U, psi, M5: float, mf: float, bc_t: int = 1) -> np.ndarray:
    """D_dwf = D_W + D_5 (Section 3, the Shamir operator as read in the header)."""
    return wilson(U, psi, M5, bc_t) + d5(psi, mf)


def ddwf_mobius(U, psi, M5: float, mf: float, b5: float, bc_t: int = 1) -> np.ndarray:
    """Moebius domain wall with c5 = 0 (Section 3 names the Shamir operator as the
    Moebius/Cayley form with c = 0, b = 1): the 4d part is scaled by b5,
        (D psi)(s) = (b5 D_W + 1) psi(s) - P_- psi(s + 1) - P_+ psi(s - 1),
    i.e. D = b5 D_W + D_5 (walls as in d5).  b5 = 1 is ddwf."""
    return b5 * wilson(U, psi, M5, bc_t) + d5(psi, mf)


def apply_H_mobius(U, psi, M5: float, mf: float, b5: float, bc_t: int = 1) -> np.ndarray:
    """H = Gamma5 D for the Moebius (c5 = 0) operator (Section 3 names Moebius with c = 0
    beside the Shamir operator)."""
    return gamma5_r5(ddwf_mobius(U, psi, M5, mf, b5, bc_t))


def gamma5_r5(psi: np.ndarray) -> np.ndarray:
    """Gamma5 = gamma5 R5 (Section 3): reflect s -> Ls-1-s and multiply by gamma5."""
    return spin_mul(GAMMA5, psi[..., ::-1, :, :])


def apply_H(U, psi, M5: float, mf: float, bc_t: int = 1) -> np.ndarray:
    """H = Gamma5 D_dwf (Section 3)."""
    return gamma5_r5(ddwf(U, psi, M5, mf, bc_t))


def apply_H_hop(U, psi, mu: int, sign: int, bc_t: int = 1) -> np.ndarray:
    """The part of H made of the single 4d hop reading psi(x + sign*mu):
    Gamma5 applied to -1/2 hop(mu, sign)."""
    return gamma5_r5(-0.5 * hop(U, psi, mu, sign, bc_t))


def apply_D(U, psi, M5, mf, bc_t=1):
    """Alias of ddwf for readability in tests."""
    return ddwf(U, psi, M5, mf, bc_t)


def apply_H_at(U, psi, sites, M5: float, mf: float, bc_t: int = 1) -> np.ndarray:
    """(H psi)(x, s) of Section 3 at a few 5d sites only, written out term by term.

    ``sites``: iterable of (x, y, z, t, s).  Returns an array (len(sites), 4, 3).
    Used to check full-size lattices where a whole-field apply is too slow.
    """
    _, Lt, Lz, Ly, Lx = U.shape[:5]
    Ls = psi.shape[-3]
    ext = (Lx, Ly, Lz, Lt)
    out = []
    for (x, y, z, t, s) in sites:
        sd = Ls - 1 - s                      # H reads D_dwf at the reflected s
        c = [x, y, z, t]

        def f(cc, ss):
            return psi[cc[3], cc[2], cc[1], cc[0], ss]

        d = (4.0 - M5) * f(c, sd)
        for mu in range(4):
            fw = list(c)
            fw[mu] = (c[mu] + 1) % ext[mu]
            bw = list(c)
            bw[mu] = (c[mu] - 1) % ext[mu]
            ph_f = bc_t if (mu == 3 and c[3] == Lt - 1) else 1
            ph_b = bc_t if (mu == 3 and c[3] == 0) else 1
            Uf = U[mu, c[3], c[2], c[1], c[0]]
            Ub = U[mu, bw[3], bw[2], bw[1], bw[0]]
            d = d - 0.5 * ph_f * (IDENT4 - GAMMA[mu]) @ (f(fw, sd) @ Uf.T)
            d = d - 0.5 * ph_b * (IDENT4 + GAMMA[mu]) @ (f(bw, sd) @ np.conj(Ub))
        up = f(c, sd + 1) if sd + 1 < Ls else -mf * f(c, 0)
        dn = f(c, sd - 1) if sd >= 1 else -mf * f(c, Ls - 1)
        d = d + f(c, sd) - P_MINUS @ up - P_PLUS @ dn
        out.append(GAMMA5 @ d)
    return np.array(out)
