"""Helpers for the GPU parity tests: numpy <-> ABI layouts and comparisons.

The layout conversions here are written independently of the library's own
conversion kernels so that a layout bug cannot cancel out.
"""
import numpy as np


def planes(psi: np.ndarray) -> np.ndarray:
    """natural (..., Lt, Lz, Ly, Lx, Ls, 4, 3) -> planes (..., 12, V5)."""
    lead = psi.shape[:-7]
    a = psi.reshape(lead + (-1, 12))
    return np.ascontiguousarray(np.swapaxes(a, -1, -2))


def natural(pl: np.ndarray, L, Ls) -> np.ndarray:
    """planes (..., 12, V5) -> natural (..., Lt, Lz, Ly, Lx, Ls, 4, 3)."""
    Lx, Ly, Lz, Lt = L
    lead = pl.shape[:-2]
    a = np.swapaxes(pl, -1, -2)
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
