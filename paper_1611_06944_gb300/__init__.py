"""HDCR hot path for GB300: Python binding of libhdcr (arXiv:1611.06944).

Thin layer over the C ABI declared in ``include/hdcr.h``: it checks tensor
shapes, dtypes and devices, passes raw device pointers and the current CUDA
stream, and turns a nonzero status into ``HDCRError``.  PyTorch supplies
device memory and streams only; every step of the method runs in the CUDA
library.  The library is loaded on first use; every call raises ImportError
when it has not been built (there is no CPU fallback).

Tensor layouts (see ``include/hdcr.h``):
  gauge      (4, V4, 3, 3) complex, or any contiguous tensor of that size
  fermion    (..., V4, 12, Ls) complex "packed": for each 4d site the 12
             components c = 3*spin + colour, each a run over s
  natural    (..., Lt, Lz, Ly, Lx, Ls, 4, 3) complex (converted by pack/unpack)
"""
from __future__ import annotations

import ctypes
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
    "HDCRError", "Lattice", "apply_g5dwf", "apply_gamma5_r5", "pack", "unpack",
    "convert", "cdot", "norm2", "cr_solve", "cr_solve_into", "library_path",
    "Subspace", "build_subspace", "subspace_from_vectors", "restrict", "prolong",
    "CoarseOperator", "build_coarse_op", "apply_coarse", "hdcr_solve",
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


def pack(lat: Lattice, natural: torch.Tensor, stream=None) -> torch.Tensor:
    """(..., Lt, Lz, Ly, Lx, Ls, 4, 3) -> packed (..., V4, 12, Ls)."""
    n = _nfields(lat, natural, "natural")
    lead = natural.shape[:-7]
    out = torch.empty(lead + (lat.V4, 12, lat.Ls), dtype=natural.dtype, device=natural.device)
    g = lat.c_geom()
    _check(_L.hdcr_fermion_pack(C_ref(g), _dev(natural, "natural"), _dev(out, "out"),
                                _code(natural), n, _stream(stream)), "pack")
    return out


def unpack(lat: Lattice, packed: torch.Tensor, stream=None) -> torch.Tensor:
    """packed (..., V4, 12, Ls) -> (..., Lt, Lz, Ly, Lx, Ls, 4, 3)."""
    n = _nfields(lat, packed, "packed")
    if packed.dim() >= 3 and tuple(packed.shape[-3:]) == (lat.V4, 12, lat.Ls):
        lead = tuple(packed.shape[:-3])
    else:
        lead = (n,) if n > 1 else ()
    Lx, Ly, Lz, Lt = lat.L
    out = torch.empty(lead + (Lt, Lz, Ly, Lx, lat.Ls, 4, 3), dtype=packed.dtype, device=packed.device)
    g = lat.c_geom()
    _check(_L.hdcr_fermion_unpack(C_ref(g), _dev(packed, "packed"), _dev(out, "out"),
                                  _code(packed), n, _stream(stream)), "unpack")
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
    return ctypes.byref(obj)


# ------------------------------------------------------------------ two-level
class Subspace:
    """Block-orthonormal subspace basis (Section 4), owned by the library."""

    def __init__(self, handle, lat: Lattice, block, nvec: int, dtype: torch.dtype, device):
        self._h = handle
        self.lat = lat
        self.block = tuple(block)
        self.nvec = nvec
        self.dtype = dtype
        self.device = device
        self.coarse_L = tuple(lat.L[i] // self.block[i] for i in range(4))
        self.Vc = self.coarse_L[0] * self.coarse_L[1] * self.coarse_L[2] * self.coarse_L[3]

    @property
    def handle(self):
        return self._h

    def vectors(self, stream=None) -> torch.Tensor:
        """The nvec basis fields as complex128, packed layout (nvec, V4, 12, Ls)."""
        out = torch.empty((self.nvec, self.lat.V4, 12, self.lat.Ls), dtype=torch.complex128,
                          device=self.device)
        _check(_L.hdcr_subspace_get_vectors(self._h, out.data_ptr(), _stream(stream)), "subspace vectors")
        return out

    def close(self):
        if self._h:
            _L.hdcr_subspace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _block_arr(block):
    arr = (ctypes.c_int * 4)(*[int(b) for b in block])
    return arr


def build_subspace(lat: Lattice, U: torch.Tensor, noise: torch.Tensor, M5: float, mf: float, block,
                   smooth_iters: int = 10, store_dtype: torch.dtype = torch.complex128,
                   stream=None) -> Subspace:
    """Subspace from nvec/2 noise fields (complex128, packed): smoothing by CR on H x = 0,
    Gamma5 chiral split, block orthonormalisation (Section 4)."""
    if U.dtype != torch.complex128 or noise.dtype != torch.complex128:
        raise TypeError("build_subspace takes complex128 links and noise")
    half = _nfields(lat, noise, "noise")
    h = ctypes.c_void_p()
    g = lat.c_geom()
    p = _params(M5, mf)
    code = _lib.HDCR_C128 if store_dtype == torch.complex128 else _lib.HDCR_C64
    _check(_L.hdcr_build_subspace(C_ref(g), C_ref(p), _dev(U, "U"), _dev(noise, "noise"), 2 * half,
                                  _block_arr(block), int(smooth_iters), code, _stream(stream),
                                  ctypes.byref(h)), "build_subspace")
    return Subspace(h, lat, block, 2 * half, store_dtype, U.device)


def subspace_from_vectors(lat: Lattice, block, vectors: torch.Tensor,
                          store_dtype: torch.dtype = torch.complex128, stream=None) -> Subspace:
    """Subspace from given (already split) complex128 fields: block orthonormalisation only."""
    if vectors.dtype != torch.complex128:
        raise TypeError("vectors must be complex128")
    nvec = _nfields(lat, vectors, "vectors")
    h = ctypes.c_void_p()
    g = lat.c_geom()
    code = _lib.HDCR_C128 if store_dtype == torch.complex128 else _lib.HDCR_C64
    _check(_L.hdcr_subspace_from_vectors(C_ref(g), _block_arr(block), nvec, _dev(vectors, "vectors"),
                                         code, _stream(stream), ctypes.byref(h)), "subspace_from_vectors")
    return Subspace(h, lat, block, nvec, store_dtype, vectors.device)


def restrict(sub: Subspace, fine: torch.Tensor, stream=None) -> torch.Tensor:
    """P^dag fine: (nrhs, Vc, nvec) coarse vectors."""
    n = _nfields(sub.lat, fine, "fine")
    out = torch.empty((n, sub.Vc, sub.nvec), dtype=fine.dtype, device=fine.device)
    _check(_L.hdcr_restrict(sub.handle, _dev(fine, "fine"), out.data_ptr(), _code(fine), n,
                            _stream(stream)), "restrict")
    return out


def prolong(sub: Subspace, coarse: torch.Tensor, stream=None) -> torch.Tensor:
    """P coarse: (nrhs, V4, 12, Ls) fine fields."""
    per = sub.Vc * sub.nvec
    if coarse.numel() % per:
        raise ValueError("coarse vectors must hold a multiple of Vc*nvec entries")
    n = coarse.numel() // per
    out = torch.empty((n, sub.lat.V4, 12, sub.lat.Ls), dtype=coarse.dtype, device=coarse.device)
    _check(_L.hdcr_prolong(sub.handle, _dev(coarse, "coarse"), out.data_ptr(), _code(coarse), n,
                           _stream(stream)), "prolong")
    return out


class CoarseOperator:
    """Little Dirac operator (Eq. 4.5) on the coarse lattice; keeps its subspace alive."""

    def __init__(self, handle, sub: Subspace, dtype: torch.dtype, M5: float, mf: float):
        self._h = handle
        self.sub = sub
        self.dtype = dtype
        self.M5 = M5
        self.mf = mf

    @property
    def handle(self):
        return self._h

    def op(self, stream=None) -> torch.Tensor:
        """A as complex128 (Vc, 9, nvec, nvec)."""
        s = self.sub
        out = torch.empty((s.Vc, 9, s.nvec, s.nvec), dtype=torch.complex128, device=s.device)
        _check(_L.hdcr_coarse_get_op(self._h, out.data_ptr(), _stream(stream)), "coarse op")
        return out

    def close(self):
        if self._h:
            _L.hdcr_coarse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_coarse_op(sub: Subspace, U: torch.Tensor, M5: float, mf: float,
                    op_dtype: torch.dtype = torch.complex128, stream=None) -> CoarseOperator:
    """A^{ab}_{jk} = <phi_j^a|H|phi_k^b> for the 9 legs of every coarse site (Eq. 4.5)."""
    if U.dtype != torch.complex128:
        raise TypeError("build_coarse_op takes complex128 links")
    h = ctypes.c_void_p()
    p = _params(M5, mf)
    code = _lib.HDCR_C128 if op_dtype == torch.complex128 else _lib.HDCR_C64
    _check(_L.hdcr_build_coarse_op(sub.handle, C_ref(p), _dev(U, "U"), code, _stream(stream),
                                   ctypes.byref(h)), "build_coarse_op")
    return CoarseOperator(h, sub, op_dtype, M5, mf)


def apply_coarse(co: CoarseOperator, c: torch.Tensor, stream=None) -> torch.Tensor:
    """9-point coarse stencil applied to (nrhs, Vc, nvec) coarse vectors."""
    per = co.sub.Vc * co.sub.nvec
    if c.numel() % per:
        raise ValueError("coarse vectors must hold a multiple of Vc*nvec entries")
    out = torch.empty_like(c)
    _check(_L.hdcr_apply_coarse(co.handle, _dev(c, "c"), _dev(out, "out"), _code(c), c.numel() // per,
                                _stream(stream)), "apply_coarse")
    return out


def hdcr_solve(co: CoarseOperator, U: torch.Tensor, b: torch.Tensor, x0: torch.Tensor | None = None,
               tol: float = 1e-10, max_outer: int = 500, restart: int = 8, smoother_steps: int = 8,
               coarse_tol: float = 1e-4, coarse_max: int = 1000,
               inner_dtype: torch.dtype = torch.complex128, stream=None):
    """H x = b by flexible GCR preconditioned with the two-level V-cycle (Section 4).
    Returns (x, stats dict); raises HDCRError when the solve fails."""
    if U.dtype != torch.complex128 or b.dtype != torch.complex128:
        raise TypeError("hdcr_solve takes complex128 links and source")
    if _nfields(co.sub.lat, b, "b") != 1:
        raise ValueError("hdcr_solve takes one right-hand side")
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    prm = _lib.hdcr_solve_params(float(tol), int(max_outer), int(restart), int(smoother_steps),
                                 float(coarse_tol), int(coarse_max),
                                 _lib.HDCR_C128 if inner_dtype == torch.complex128 else _lib.HDCR_C64)
    st = _lib.hdcr_solve_stats()
    _check(_L.hdcr_solve(co.handle, _dev(U, "U"), _dev(b, "b"), _dev(x, "x"), C_ref(prm), C_ref(st),
                         _stream(stream)), "hdcr_solve")
    return x, st.as_dict()
