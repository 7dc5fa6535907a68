"""Seeded synthetic inputs for the HDCR hot path.

This module draws random numbers and arranges them into lattice fields.  It
holds none of the solver's arithmetic: both the CUDA path and the oracle take
their inputs from here, and neither side imports the other.

Conventions (shared vocabulary, not method arithmetic):

* A 4d lattice is given as ``L = (Lx, Ly, Lz, Lt)``; arrays are stored with
  ``t`` slowest and ``x`` fastest, i.e. numpy shape ``(Lt, Lz, Ly, Lx, ...)``.
* Gauge field ``U``: complex128 array of shape ``(4, Lt, Lz, Ly, Lx, 3, 3)``,
  ``U[mu, t, z, y, x, a, b]`` is the colour matrix element ``U_mu(x)_{ab}`` of
  the link leaving site ``x`` in direction ``mu`` (0..3 = x, y, z, t).
* 5d fermion field ``psi``: complex128 array of shape
  ``(Lt, Lz, Ly, Lx, Ls, 4, 3)`` (site, fifth coordinate s, spin, colour).

The synthetic links follow the recipe U = exp(i*eps*H) with H a Gaussian
traceless Hermitian matrix, which stands in for the dynamical ensemble of the
paper's Section 5 (the ensemble itself is not available here).  "Gaussian
traceless Hermitian" is read in the convention used for HMC momenta:
H = sum_a omega_a lambda_a / 2 over the eight Gell-Mann matrices with
omega_a ~ N(0, 1).  With it eps = 0.5 gives a mean plaquette of about 0.50
and eps = 0.3 about 0.79 (a physical DWF ensemble at a^-1 = 1.73 GeV sits
near 0.59).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "plaquette",
    "gauge_field",
    "random_su3_field",
    "gaussian_fermion",
    "point_sources",
    "device_gaussian",
    "unit_gauge",
    "lattice_shape",
]


def rng(seed: int) -> np.random.Generator:
    """numpy PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def lattice_shape(L) -> tuple:
    """numpy shape (Lt, Lz, Ly, Lx) of a 4d lattice L = (Lx, Ly, Lz, Lt)."""
    Lx, Ly, Lz, Lt = (int(v) for v in L)
    return (Lt, Lz, Ly, Lx)


def _gell_mann_generators() -> np.ndarray:
    """T_a = lambda_a / 2, a = 1..8 (tr T_a T_b = delta_ab / 2)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1.0, 1.0, -2.0]) / np.sqrt(3.0)
    return l / 2


_T = _gell_mann_generators()


def _traceless_hermitian(g: np.random.Generator, n: int) -> np.ndarray:
    """n matrices H = sum_a omega_a T_a with omega_a ~ N(0, 1)."""
    w = g.standard_normal((n, 8))
    return np.einsum("na,aij->nij", w, _T)


def _expm_i_hermitian(H: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for a stack of Hermitian 3x3 matrices via eigh."""
    w, V = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("nab,nb,ncb->nac", V, ph, np.conj(V))
    # one polar re-unitarisation step keeps |U^dag U - 1| at rounding level
    u, _, vh = np.linalg.svd(U)
    U = u @ vh
    det = np.linalg.det(U)
    U = U / (det ** (1.0 / 3.0))[:, None, None]
    return U


def random_su3_field(L, seed: int, eps: float = 1.0, n_links: int | None = None) -> np.ndarray:
    """A field of SU(3) matrices exp(i*eps*H), one per site (shape (Lt,Lz,Ly,Lx,3,3))."""
    shp = lattice_shape(L)
    n = int(np.prod(shp)) if n_links is None else n_links
    g = rng(seed)
    U = _expm_i_hermitian(_traceless_hermitian(g, n), eps)
    return U.reshape(shp + (3, 3))


def gauge_field(L, eps: float, seed: int) -> np.ndarray:
    """Synthetic gauge field U_mu(x) = exp(i*eps*H_mu(x)), H Gaussian traceless Hermitian."""
    shp = lattice_shape(L)
    n = 4 * int(np.prod(shp))
    g = rng(seed)
    U = _expm_i_hermitian(_traceless_hermitian(g, n), eps)
    return np.ascontiguousarray(U.reshape((4,) + shp + (3, 3)))


def unit_gauge(L) -> np.ndarray:
    """Free field: every link the identity."""
    shp = lattice_shape(L)
    U = np.zeros((4,) + shp + (3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_fermion(L, Ls: int, seed: int, count: int | None = None) -> np.ndarray:
    """Gaussian complex 5d fermion field(s), Re and Im ~ N(0,1).

    Shape ``(Lt,Lz,Ly,Lx,Ls,4,3)``, or ``(count, Lt,Lz,Ly,Lx,Ls,4,3)`` when
    ``count`` is given (e.g. the noise vectors that seed the subspace).
    """
    shp = lattice_shape(L) + (int(Ls), 4, 3)
    if count is not None:
        shp = (int(count),) + shp
    g = rng(seed)
    return g.standard_normal(shp) + 1j * g.standard_normal(shp)


def device_gaussian(nfields: int, V5: int, seed: int, device="cuda", dtype=None):
    """Gaussian complex fields drawn on the device (torch's seeded generator of that
    device), Re and Im ~ N(0,1): a tensor (nfields, V5 * 12) of complex128 (or
    ``dtype``).  For lattices too large to draw on the host in reasonable time; the
    entries are independent, so the layout they are read in does not matter.
    Deterministic for a given seed and device type, not equal to gaussian_fermion."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    dt = torch.float64 if dtype is None or dtype == torch.complex128 else torch.float32
    x = torch.randn((int(nfields), int(V5) * 12, 2), generator=g, device=device, dtype=dt)
    return torch.view_as_complex(x)


def point_sources(L, Ls: int, site=(0, 0, 0, 0), s: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at 4d site ``site`` = (x,y,z,t), fifth coordinate s.

    Shape ``(12, Lt,Lz,Ly,Lx,Ls,4,3)``; source ``3*spin+colour`` is a unit
    vector in that spin-colour component.
    """
    shp = lattice_shape(L) + (int(Ls), 4, 3)
    out = np.zeros((12,) + shp, dtype=np.complex128)
    x, y, z, t = site
    for sp in range(4):
        for c in range(3):
            out[3 * sp + c, t, z, y, x, s, sp, c] = 1.0
    return out


def plaquette(U: np.ndarray) -> float:
    """Mean plaquette Re tr(U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag) / 3 of a
    gauge field (a roughness diagnostic of the synthetic inputs)."""
    ax = {0: 3, 1: 2, 2: 1, 3: 0}
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = (U[mu] @ np.roll(U[nu], -1, axis=ax[mu])
                 @ np.conj(np.swapaxes(np.roll(U[mu], -1, axis=ax[nu]), -1, -2))
                 @ np.conj(np.swapaxes(U[nu], -1, -2)))
            tot += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3.0
    return tot / 6.0
