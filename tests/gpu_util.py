"""Helpers for the GPU parity tests: numpy <-> ABI layouts and comparisons.

The layout conversions here are written independently of the library's own
conversion kernels so that a layout bug cannot cancel out.
"""
import numpy as np


def planes(psi: np.ndarray) -> np.ndarray:
    """natural (..., Lt, Lz, Ly, Lx, Ls, 4, 3) -> library layout (..., V4, 12, Ls)."""
    lead = psi.shape[:-7]
    Ls = psi.shape[-3]
    a = psi.reshape(lead + (-1, Ls, 12))
    return np.ascontiguousarray(np.swapaxes(a, -1, -2))


def natural(pl: np.ndarray, L, Ls) -> np.ndarray:
    """library layout (..., V4, 12, Ls) -> natural (..., Lt, Lz, Ly, Lx, Ls, 4, 3).

    An array without the (V4, 12, Ls) trailing shape is read as n such fields."""
    Lx, Ly, Lz, Lt = L
    V4 = Lx * Ly * Lz * Lt
    n = pl.size // (V4 * 12 * Ls)
    if pl.ndim >= 3 and pl.shape[-3:] == (V4, 12, Ls):
        lead = pl.shape[:-3]
    else:
        lead = (n,) if n > 1 else ()
    a = np.swapaxes(pl.reshape(lead + (V4, 12, Ls)), -1, -2)
    return np.ascontiguousarray(a.reshape(lead + (Lt, Lz, Ly, Lx, Ls, 4, 3)))


def links(U: np.ndarray) -> np.ndarray:
    """(4, Lt, Lz, Ly, Lx, 3, 3) -> (4, V4, 3, 3) (same memory order)."""
    return np.ascontiguousarray(U.reshape(4, -1, 3, 3))


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def dev(a: np.ndarray, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return t if dtype is None else t.to(dtype)


def host(t) -> np.ndarray:
    return t.detach().to("cpu").numpy()
