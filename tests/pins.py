"""Pins: quantities fixed by mathematics or by the paper, used to check the oracle.

Each function returns an error measure (0 up to rounding when the oracle is
right).  The mutation tests re-use them to show that a planted mistake in the
oracle is caught by at least one pin.
"""
from __future__ import annotations

import numpy as np

import synth


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


# ------------------------------------------------------------ gamma algebra
def gamma_algebra_error(dwf) -> float:
    """Clifford algebra {g_mu, g_nu} = 2 delta, Hermitian gammas, gamma5 = g1 g2 g3 g4
    Hermitian, squares to one and anticommutes with every g_mu; chiral basis
    means gamma5 is diagonal."""
    G = dwf.GAMMA
    I = np.eye(4)
    err = 0.0
    for m in range(4):
        err = max(err, np.abs(G[m] - G[m].conj().T).max())
        for n in range(4):
            ac = G[m] @ G[n] + G[n] @ G[m]
            err = max(err, np.abs(ac - 2 * (m == n) * I).max())
        err = max(err, np.abs(dwf.GAMMA5 @ G[m] + G[m] @ dwf.GAMMA5).max())
    g5 = G[0] @ G[1] @ G[2] @ G[3]
    err = max(err, np.abs(g5 - dwf.GAMMA5).max())
    err = max(err, np.abs(dwf.GAMMA5 @ dwf.GAMMA5 - I).max())
    err = max(err, np.abs(dwf.GAMMA5 - np.diag(np.diag(dwf.GAMMA5))).max())
    return float(err)


# --------------------------------------------------------------- operator
def hermiticity_error(dwf, U, x, y, M5, mf, bc_t=1) -> float:
    """<x, H y> = <H x, y> (H = Gamma5 D_dwf is Hermitian, Section 3)."""
    a = dwf.inner(x, dwf.apply_H(U, y, M5, mf, bc_t))
    b = dwf.inner(dwf.apply_H(U, x, M5, mf, bc_t), y)
    return abs(a - b) / abs(a)


def d5_matrix_s(Ls, mf, Pm, Pp) -> np.ndarray:
    """The fifth-dimension operator as a (Ls*4) x (Ls*4) matrix, index s*4+spin,
    assembled entry by entry from its definition (walls psi(Ls) = -mf psi(0),
    psi(-1) = -mf psi(Ls-1))."""
    M = np.zeros((Ls * 4, Ls * 4), dtype=np.complex128)
    for s in range(Ls):
        M[s * 4:(s + 1) * 4, s * 4:(s + 1) * 4] += np.eye(4)
        up, wup = ((s + 1), 1.0) if s + 1 < Ls else (0, -mf)
        dn, wdn = ((s - 1), 1.0) if s >= 1 else (Ls - 1, -mf)
        M[s * 4:(s + 1) * 4, up * 4:(up + 1) * 4] -= wup * Pm
        M[s * 4:(s + 1) * 4, dn * 4:(dn + 1) * 4] -= wdn * Pp
    return M


def plane_wave_error(dwf, L, Ls, M5, mf, n, chi, bc_t=1, b5=None) -> float:
    """Free field (U = 1): D_dwf [e^{ip.x} chi(s)] = e^{ip.x} [(b(p) + i sum g_mu sin p_mu) chi(s)
    + (D5 chi)(s)], b(p) = -M5 + sum (1 - cos p_mu), p_mu = 2 pi n_mu / L_mu
    (t: (2 n_t + 1) pi / L_t when antiperiodic).  chi: (Ls, 4, 3).  With b5 given, the
    Moebius (c5 = 0) operator: the 4d bracket is multiplied by b5."""
    Lx, Ly, Lz, Lt = L
    p = [2 * np.pi * n[m] / L[m] for m in range(3)]
    p.append((2 * n[3] + (0 if bc_t == 1 else 1)) * np.pi / Lt)
    t, z, y, x = np.indices((Lt, Lz, Ly, Lx))
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    psi = phase[..., None, None, None] * chi[None, None, None, None]
    U = synth.unit_gauge(L)
    got = dwf.ddwf(U, psi, M5, mf, bc_t) if b5 is None else dwf.ddwf_mobius(U, psi, M5, mf, b5, bc_t)
    b = -M5 + sum(1 - np.cos(pm) for pm in p)
    K = b * np.eye(4) + 1j * sum(dwf.GAMMA[m] * np.sin(p[m]) for m in range(4))
    if b5 is not None:
        K = b5 * K
    four = np.einsum("ij,sjc->sic", K, chi)
    D5 = d5_matrix_s(Ls, mf, dwf.P_MINUS, dwf.P_PLUS)
    five = (D5 @ chi.reshape(Ls * 4, 3)).reshape(Ls, 4, 3)
    want = phase[..., None, None, None] * (four + five)[None, None, None, None]
    return relerr(got, want)


def p0_det_error(dwf, Ls, M5, mf) -> float:
    """Free field, zero momentum, one chirality and colour: the Ls x Ls block of
    D_dwf has determinant (1 - M5)^Ls + mf, the combination mf + (1 - M5)^Ls of
    the textbook free domain-wall effective quark mass M5 (2 - M5)(mf + (1 - M5)^Ls)."""
    L = (2, 2, 2, 2)
    U = synth.unit_gauge(L)
    err = 0.0
    for spin in (0, 2):                      # one spin of each chirality
        cols = []
        for s in range(Ls):
            psi = np.zeros(synth.lattice_shape(L) + (Ls, 4, 3), dtype=np.complex128)
            psi[..., s, spin, 0] = 1.0
            out = dwf.ddwf(U, psi, M5, mf)
            cols.append(out[0, 0, 0, 0, :, spin, 0])
        M = np.array(cols).T
        want = (1.0 - M5) ** Ls + mf
        err = max(err, abs(np.linalg.det(M) - want) / abs(want))
    return float(err)


def covariance_error(dwf, U, Om, psi, M5, mf, bc_t=1) -> float:
    """Gauge covariance: D[U^Om](Om psi) = Om D[U] psi with
    U^Om_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag."""
    Ug = np.empty_like(U)
    for mu in range(4):
        Om_f = np.roll(Om, -1, axis=3 - mu)
        Ug[mu] = Om @ U[mu] @ np.conj(np.swapaxes(Om_f, -1, -2))
    Opsi = np.matmul(psi, np.swapaxes(Om, -1, -2)[..., None, :, :])
    lhs = dwf.ddwf(Ug, Opsi, M5, mf, bc_t)
    rhs = np.matmul(dwf.ddwf(U, psi, M5, mf, bc_t), np.swapaxes(Om, -1, -2)[..., None, :, :])
    return relerr(lhs, rhs)


def dense_H_from_stencil(dwf, U, Ls, M5, mf, bc_t=1) -> np.ndarray:
    """Dense matrix of the oracle's H from its action on unit vectors."""
    shp = U.shape[1:5] + (Ls, 4, 3)
    N = int(np.prod(shp))
    E = np.eye(N, dtype=np.complex128).reshape((N,) + shp)
    return dwf.apply_H(U, E, M5, mf, bc_t).reshape(N, N).T


def dense_H_assembled(dwf, U, Ls, M5, mf, bc_t=1) -> np.ndarray:
    """H assembled as a sparse-pattern dense matrix site by site from the
    written-out operator (index ((x4*Ls + s)*4 + spin)*3 + colour), independent
    of the stencil's array rolls."""
    _, Lt, Lz, Ly, Lx = U.shape[:5]
    V4 = Lt * Lz * Ly * Lx
    n5 = Ls * 12
    N = V4 * n5
    D = np.zeros((N, N), dtype=np.complex128)
    G = dwf.GAMMA
    I4 = np.eye(4)
    ext = (Lx, Ly, Lz, Lt)

    def idx(c):
        x, y, z, t = c
        return ((t * Lz + z) * Ly + y) * Lx + x

    D5 = np.kron(d5_matrix_s(Ls, mf, dwf.P_MINUS, dwf.P_PLUS), np.eye(3))
    for t in range(Lt):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    c = (x, y, z, t)
                    i = idx(c)
                    blk = slice(i * n5, (i + 1) * n5)
                    D[blk, blk] += (4.0 - M5) * np.eye(n5) + D5
                    for mu in range(4):
                        f = list(c)
                        f[mu] = (c[mu] + 1) % ext[mu]
                        b = list(c)
                        b[mu] = (c[mu] - 1) % ext[mu]
                        ph_f = bc_t if (mu == 3 and c[3] == Lt - 1) else 1.0
                        ph_b = bc_t if (mu == 3 and c[3] == 0) else 1.0
                        Uf = U[mu, t, z, y, x]
                        Ub = np.conj(U[mu, b[3], b[2], b[1], b[0]]).T
                        jf, jb = idx(f), idx(b)
                        D[blk, jf * n5:(jf + 1) * n5] += -0.5 * ph_f * np.kron(
                            np.eye(Ls), np.kron(I4 - G[mu], Uf))
                        D[blk, jb * n5:(jb + 1) * n5] += -0.5 * ph_b * np.kron(
                            np.eye(Ls), np.kron(I4 + G[mu], Ub))
    R5 = np.eye(Ls)[::-1]
    Gam5 = np.kron(np.eye(V4), np.kron(R5, np.kron(dwf.GAMMA5, np.eye(3))))
    return Gam5 @ D
