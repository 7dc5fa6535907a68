"""HDCR hot path for GB300: Python binding of libhdcr (arXiv:1611.06944).

Thin layer over the C ABI declared in ``include/hdcr.h``: it checks tensor
shapes, dtypes and devices, passes raw device pointers and the current CUDA
stream, and turns a nonzero status into ``HDCRError``.  PyTorch supplies
device memory and streams only; every step of the method runs in the CUDA
library.  The library is loaded on first use; every call raises ImportError
when it has not been built (there is no CPU fallback).

Tensor layouts (see ``include/hdcr.h``):
  gauge      (4, V4, 3, 3) complex, or any contiguous tensor of that size
  fermion    (..., 12, V5) complex "planes", component c = 3*spin + colour,
             5d site i5 = x4*Ls + s
  natural    (..., Lt, Lz, Ly, Lx, Ls, 4, 3) complex (converted by to_planes)
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib


class _LazyLib:
    """Loads libhdcr.so on first attribute access (ImportError if it is missing)."""

    _handle = None

    def __getattr__(self, name):
        if _LazyLib._handle is None:
            _LazyLib._handle = _lib.load()
        return getattr(_LazyLib._handle, name)


_L = _LazyLib()


def load_library():
    """Load libhdcr.so now (raises ImportError if it has not been built)."""
    return _L.hdcr_version()

__all__ = [
    "HDCRError", "Lattice", "apply_g5dwf", "apply_gamma5_r5", "to_planes", "from_planes",
    "convert", "cdot", "norm2", "cr_solve", "cr_solve_into", "library_path",
]

library_path = _lib.LIB_PATH


class HDCRError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _L.hdcr_last_error().decode(errors="replace")
        super().__init__(f"{what}: {_lib.STATUS_NAMES.get(status, status)} ({msg})")


def _check(status: int, what: str) -> None:
    if status != _lib.HDCR_OK:
        raise HDCRError(status, what)


@dataclass(frozen=True)
class Lattice:
    """4d extents L = (Lx, Ly, Lz, Lt), fifth-dimension extent Ls, time boundary bc_t."""
    L: tuple
    Ls: int
    bc_t: int = 1

    @property
    def V4(self) -> int:
        Lx, Ly, Lz, Lt = self.L
        return Lx * Ly * Lz * Lt

    @property
    def V5(self) -> int:
        return self.V4 * self.Ls

    def c_geom(self) -> _lib.hdcr_geom:
        g = _lib.hdcr_geom()
        for i in range(4):
            g.L[i] = int(self.L[i])
        g.Ls = int(self.Ls)
        g.bc_t = int(self.bc_t)
        return g


def _code(t: torch.Tensor) -> int:
    if t.dtype == torch.complex128:
        return _lib.HDCR_C128
    if t.dtype == torch.complex64:
        return _lib.HDCR_C64
    raise TypeError(f"unsupported dtype {t.dtype}; use complex128 or complex64")


def _dev(t: torch.Tensor, name: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _params(M5: float, mf: float) -> _lib.hdcr_dwf_params:
    return _lib.hdcr_dwf_params(float(M5), float(mf))


def _nfields(lat: Lattice, t: torch.Tensor, name: str) -> int:
    per = 12 * lat.V5
    if t.numel() == 0 or t.numel() % per:
        raise ValueError(f"{name} has {t.numel()} entries, not a multiple of 12*V5 = {per}")
    return t.numel() // per


def apply_g5dwf(lat: Lattice, U: torch.Tensor, psi: torch.Tensor, M5: float, mf: float,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """out = Gamma5 D_dwf psi (Section 3) for every field in psi."""
    if U.dtype != psi.dtype:
        raise TypeError("U and psi must share a dtype")
    if U.numel() != 4 * lat.V4 * 9:
        raise ValueError("U must hold 4*V4*9 complex numbers")
    n = _nfields(lat, psi, "psi")
    out = torch.empty_like(psi) if out is None else out
    g = lat.c_geom()
    p = _params(M5, mf)
    _check(_L.hdcr_apply_g5dwf(C_ref(g), C_ref(p), _dev(U, "U"), _dev(psi, "psi"), _dev(out, "out"),
                               _code(psi), n, _stream(stream)), "apply_g5dwf")
    return out


def apply_gamma5_r5(lat: Lattice, psi: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """out = gamma5 R5 psi."""
    n = _nfields(lat, psi, "psi")
    out = torch.empty_like(psi) if out is None else out
    g = lat.c_geom()
    _check(_L.hdcr_apply_gamma5_r5(C_ref(g), _dev(psi, "psi"), _dev(out, "out"), _code(psi), n,
                                   _stream(stream)), "apply_gamma5_r5")
    return out


def to_planes(lat: Lattice, natural: torch.Tensor, stream=None) -> torch.Tensor:
    """(..., Lt, Lz, Ly, Lx, Ls, 4, 3) -> (..., 12, V5)."""
    n = _nfields(lat, natural, "natural")
    lead = natural.shape[:-7]
    out = torch.empty(lead + (12, lat.V5), dtype=natural.dtype, device=natural.device)
    g = lat.c_geom()
    _check(_L.hdcr_fermion_to_planes(C_ref(g), _dev(natural, "natural"), _dev(out, "out"),
                                     _code(natural), n, _stream(stream)), "to_planes")
    return out


def from_planes(lat: Lattice, planes: torch.Tensor, stream=None) -> torch.Tensor:
    """(..., 12, V5) -> (..., Lt, Lz, Ly, Lx, Ls, 4, 3)."""
    n = _nfields(lat, planes, "planes")
    lead = planes.shape[:-2]
    Lx, Ly, Lz, Lt = lat.L
    out = torch.empty(lead + (Lt, Lz, Ly, Lx, lat.Ls, 4, 3), dtype=planes.dtype, device=planes.device)
    g = lat.c_geom()
    _check(_L.hdcr_fermion_from_planes(C_ref(g), _dev(planes, "planes"), _dev(out, "out"),
                                       _code(planes), n, _stream(stream)), "from_planes")
    return out


def convert(t: torch.Tensor, dtype: torch.dtype, stream=None) -> torch.Tensor:
    """Precision conversion complex128 <-> complex64 in a library kernel."""
    out = torch.empty(t.shape, dtype=dtype, device=t.device)
    _check(_L.hdcr_convert(_dev(t, "in"), _code(t), _dev(out, "out"), _code(out), t.numel(),
                           _stream(stream)), "convert")
    return out


def cdot(u: torch.Tensor, v: torch.Tensor, stream=None) -> complex:
    """<u, v> = sum conj(u) v, FP64 accumulation (synchronises the stream)."""
    if u.dtype != v.dtype or u.numel() != v.numel():
        raise ValueError("u and v must match in dtype and size")
    res = torch.empty(2, dtype=torch.float64, device=u.device)
    _check(_L.hdcr_cdot(_dev(u, "u"), _dev(v, "v"), u.numel(), _code(u), res.data_ptr(),
                        _stream(stream)), "cdot")
    r = res.cpu()
    return complex(float(r[0]), float(r[1]))


def norm2(u: torch.Tensor, stream=None) -> float:
    """sum |u|^2 with FP64 accumulation (synchronises the stream)."""
    res = torch.empty(1, dtype=torch.float64, device=u.device)
    _check(_L.hdcr_norm2(_dev(u, "u"), u.numel(), _code(u), res.data_ptr(), _stream(stream)), "norm2")
    return float(res.cpu()[0])


def cr_solve(lat: Lattice, U: torch.Tensor, b: torch.Tensor, M5: float, mf: float,
             tol: float = 1e-10, max_iter: int = 100000, x0: torch.Tensor | None = None,
             stream=None):
    """Unpreconditioned conjugate residual on H x = b (Section 3). Returns (x, stats dict)."""
    if U.dtype != b.dtype:
        raise TypeError("U and b must share a dtype")
    if _nfields(lat, b, "b") != 1:
        raise ValueError("cr_solve takes one right-hand side")
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    st = _lib.hdcr_solve_stats()
    g = lat.c_geom()
    p = _params(M5, mf)
    _check(_L.hdcr_cr_solve(C_ref(g), C_ref(p), _dev(U, "U"), _dev(b, "b"), _dev(x, "x"), _code(b),
                            float(tol), int(max_iter), C_ref(st), _stream(stream)), "cr_solve")
    return x, st.as_dict()


def cr_solve_into(lat: Lattice, U: torch.Tensor, b: torch.Tensor, x: torch.Tensor, M5: float,
                  mf: float, tol: float = 1e-10, max_iter: int = 100000, stream=None) -> dict:
    """cr_solve with a caller-owned x (initial guess in, iterate out, also when the
    iteration cap is reached and HDCRError(NOT_CONVERGED) is raised)."""
    if U.dtype != b.dtype or x.dtype != b.dtype or x.numel() != b.numel():
        raise TypeError("U, b and x must share a dtype and b, x a size")
    st = _lib.hdcr_solve_stats()
    g = lat.c_geom()
    p = _params(M5, mf)
    _check(_L.hdcr_cr_solve(C_ref(g), C_ref(p), _dev(U, "U"), _dev(b, "b"), _dev(x, "x"), _code(b),
                            float(tol), int(max_iter), C_ref(st), _stream(stream)), "cr_solve")
    return st.as_dict()


def C_ref(obj):
    import ctypes
    return ctypes.byref(obj)
