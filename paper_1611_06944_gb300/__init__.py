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


def launch_count() -> int:
    """Kernels launched by libhdcr so far in this process."""
    return int(_L.hdcr_launch_count())


def stencil_timer(enable: bool) -> None:
    """Start (reset) or stop event timing of every application of H."""
    _check(_L.hdcr_stencil_timer(1 if enable else 0), "stencil_timer")


def stencil_timer_read(dtype, fused_cheb: bool = False) -> dict:
    """Stencil launches of one precision since the timer started: device ms, launches and
    5d sites of those that carry events, and all launches and sites (``all_*``).
    fused_cheb=True (complex128): the FP64 applications carrying a fused Chebyshev
    smoother step, which the plain complex128 count leaves out."""
    code = _lib.HDCR_TIMER_C128_CHEB if fused_cheb else _dt(dtype)
    ms = ctypes.c_double()
    nl = ctypes.c_longlong()
    ns = ctypes.c_longlong()
    _check(_L.hdcr_stencil_timer_read(code, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(ns)),
           "stencil_timer_read")
    al = ctypes.c_longlong()
    asites = ctypes.c_longlong()
    _check(_L.hdcr_stencil_timer_count(code, ctypes.byref(al), ctypes.byref(asites)), "stencil_timer_count")
    return {"ms": ms.value, "launches": nl.value, "sites": ns.value, "all_launches": al.value,
            "all_sites": asites.value}


def stencil_tune(mode: int = 1, force_variant: int = -1) -> None:
    """FP32 stencil tile autotuner: mode 1 tunes on first use (default), 0 keeps the
    default tile, 2 forgets tuned choices; force_variant >= 0 pins one tile variant."""
    _check(_L.hdcr_stencil_tune(int(mode), int(force_variant)), "stencil_tune")


def stencil_tune_info(lat: "Lattice", nrhs: int = 1, nvariants: int = 16) -> dict:
    """The tile variant tuned for (lat, nrhs) (-1 if none yet) and the microseconds per
    launch the tuner measured for each variant (-1 where it does not fit)."""
    v = ctypes.c_int()
    us = (ctypes.c_float * nvariants)()
    g = lat.c_geom()
    _check(_L.hdcr_stencil_tune_info(ctypes.byref(g), int(nrhs), ctypes.byref(v), us, nvariants),
           "stencil_tune_info")
    return {"variant": v.value, "us": [round(float(x), 2) for x in us]}


def probe_fma_rate(dtype: torch.dtype = torch.complex128, stream=None) -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (FMA = 2 flops): FP64 for
    complex128, FP32 for complex64.  The roofline denominator of the FP64 operator."""
    r = ctypes.c_double()
    _check(_L.hdcr_probe_fma_rate(_dt(dtype), ctypes.byref(r), _stream(stream)), "probe_fma_rate")
    return r.value


def tc_gemm_info() -> dict:
    """Coarse-level tensor-core GEMMs issued so far, and those that fell back to plain FP32."""
    c = ctypes.c_ulonglong()
    f = ctypes.c_ulonglong()
    _check(_L.hdcr_tc_gemm_info(ctypes.byref(c), ctypes.byref(f)), "tc_gemm_info")
    return {"calls": c.value, "fallbacks": f.value}


def load_library():
    """Load libhdcr.so now (raises ImportError if it has not been built)."""
    return _L.hdcr_version()

__all__ = [
    "HDCRError", "Lattice", "probe_fma_rate", "tc_gemm_info", "apply_g5dwf", "apply_gamma5_r5", "pack", "unpack",
    "convert", "cdot", "cdot_noalloc", "norm2", "stencil_tune", "stencil_tune_info",
    "apply_cf_overlap", "cf_cr_solve", "cf_filter", "build_cf_coarse_op", "gamma5_split", "build_cf_subspace", "h16_bytes", "encode_h16", "decode_h16", "apply_g5dwf_h16", "mobius_to_shamir", "cr_solve", "cr_solve_into", "library_path",
    "Subspace", "build_subspace", "subspace_from_vectors", "restrict", "prolong",
    "CoarseOperator", "build_coarse_op", "apply_coarse", "coarse_invert", "coarse_solve_dense",
    "build_level2", "level2_get", "coarse_solve_level2",
    "hdcr_solve", "hdcr_solve_into", "hdcr_solve_multi", "cgne_rb_solve", "gauge_force", "gauge_grad", "HDCRSolve",
    "solve_autograd",
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


def _dev(t: torch.Tensor, name: str, host_ok: bool = False) -> int:
    """Pointer of a contiguous CUDA tensor; with host_ok also of a CPU tensor, for the
    entry points that stage host buffers through the device themselves."""
    if not t.is_cuda and not (host_ok and t.device.type == "cpu"):
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


def _cf_params(beta, R: float) -> _lib.hdcr_cf_params:
    p = _lib.hdcr_cf_params()
    p.ncomp = len(beta) + 1
    for i, b in enumerate(beta):
        p.beta[i] = float(b)
    p.R = float(R)
    return p


def apply_cf_overlap(lat: Lattice, U: torch.Tensor, psi: torch.Tensor, M5: float, beta, R: float,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The continued-fraction overlap operator of Section 3 on len(beta) + 1 components,
    stored as the fifth coordinate (lat.Ls must be len(beta) + 1)."""
    if U.dtype != psi.dtype:
        raise TypeError("U and psi must share a dtype")
    n = _nfields(lat, psi, "psi")
    out = torch.empty_like(psi) if out is None else out
    g = lat.c_geom()
    _check(_L.hdcr_apply_cf_overlap(C_ref(g), float(M5), C_ref(_cf_params(beta, R)), _dev(U, "U"), _dev(psi, "psi"),
                                    _dev(out, "out"), _code(psi), n, _stream(stream)), "apply_cf_overlap")
    return out


def cf_cr_solve(lat: Lattice, U: torch.Tensor, b: torch.Tensor, M5: float, beta, R: float, tol: float = 1e-10,
                max_iter: int = 100000, stream=None):
    """CR on the continued-fraction operator.  Returns (x, stats dict)."""
    x = torch.zeros_like(b)
    st = _lib.hdcr_solve_stats()
    g = lat.c_geom()
    _check(_L.hdcr_cf_cr_solve(C_ref(g), float(M5), C_ref(_cf_params(beta, R)), _dev(U, "U"), _dev(b, "b"),
                               _dev(x, "x"), _code(b), float(tol), int(max_iter), C_ref(st), _stream(stream)),
           "cf_cr_solve")
    return x, st.as_dict()


def h16_bytes(lat: Lattice) -> int:
    """Bytes of one fermion field in FP16 storage: 12 V5 half2 and V5 FP32 site scales."""
    return 52 * lat.V5


def encode_h16(lat: Lattice, psi: torch.Tensor, stream=None) -> torch.Tensor:
    """FP16 storage (half2 per complex number, one FP32 scale per 5d site) of the
    complex128 / complex64 fields psi: a uint8 tensor (nfields, 52 V5)."""
    n = _nfields(lat, psi, "psi")
    out = torch.empty((n, h16_bytes(lat)), dtype=torch.uint8, device=psi.device)
    g = lat.c_geom()
    _check(_L.hdcr_fermion_encode_h16(C_ref(g), _dev(psi, "psi"), _code(psi), _dev(out, "out"), n,
                                      _stream(stream)), "encode_h16")
    return out


def decode_h16(lat: Lattice, buf: torch.Tensor, dtype: torch.dtype = torch.complex64, stream=None) -> torch.Tensor:
    """The fields of an FP16-storage buffer as complex numbers in the library layout."""
    per = h16_bytes(lat)
    if buf.dtype != torch.uint8 or buf.numel() % per:
        raise ValueError(f"an FP16-storage buffer is uint8 with a multiple of {per} bytes")
    n = buf.numel() // per
    out = torch.empty((n, lat.V4, 12, lat.Ls), dtype=dtype, device=buf.device)
    g = lat.c_geom()
    _check(_L.hdcr_fermion_decode_h16(C_ref(g), _dev(buf, "buf"), _dev(out, "out"), _code(out), n,
                                      _stream(stream)), "decode_h16")
    return out if n > 1 else out[0]


def apply_g5dwf_h16(lat: Lattice, U: torch.Tensor, buf: torch.Tensor, M5: float, mf: float,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """H = Gamma5 D_dwf on fields in FP16 storage (FP32 arithmetic, complex64 links)."""
    if U.dtype != torch.complex64:
        raise TypeError("apply_g5dwf_h16 takes complex64 links")
    per = h16_bytes(lat)
    if buf.dtype != torch.uint8 or buf.numel() % per:
        raise ValueError(f"an FP16-storage buffer is uint8 with a multiple of {per} bytes")
    out = torch.empty_like(buf) if out is None else out
    g = lat.c_geom()
    p = _params(M5, mf)
    _check(_L.hdcr_apply_g5dwf(C_ref(g), C_ref(p), _dev(U, "U"), _dev(buf, "buf"), _dev(out, "out"),
                               _lib.HDCR_H16, buf.numel() // per, _stream(stream)), "apply_g5dwf_h16")
    return out


def mobius_to_shamir(U: torch.Tensor, M5: float, mf: float, b5: float, stream=None):
    """The Moebius (c5 = 0) operator b5 D_W + D_5 as this library's Shamir operator:
    returns (b5 U, M5', mf) with M5' = 4 - b5 (4 - M5), the scaled links computed on the
    device.  Pass them to any call in place of (U, M5, mf)."""
    out = torch.empty_like(U)
    p = _params(M5, mf)
    q = _lib.hdcr_dwf_params()
    _check(_L.hdcr_mobius_to_shamir(C_ref(p), float(b5), _dev(U, "U"), _dev(out, "U_out"), _code(U), U.numel(),
                                    C_ref(q), _stream(stream)), "mobius_to_shamir")
    return out, q.M5, q.mf


def apply_gamma5_r5(lat: Lattice, psi: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """out = gamma5 R5 psi."""
    n = _nfields(lat, psi, "psi")
    out = torch.empty_like(psi) if out is None else out
    g = lat.c_geom()
    _check(_L.hdcr_apply_gamma5_r5(C_ref(g), _dev(psi, "psi", True), _dev(out, "out", True), _code(psi), n,
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


def cdot_noalloc(u: torch.Tensor, v: torch.Tensor, stream=None) -> complex:
    """<u, v> like cdot, through the entry point that allocates no device memory
    (its scratch is a fixed array in the library; see hdcr_cdot_noalloc)."""
    if u.dtype != v.dtype or u.numel() != v.numel():
        raise ValueError("u and v must match in dtype and size")
    res = torch.empty(2, dtype=torch.float64, device=u.device)
    _check(_L.hdcr_cdot_noalloc(_dev(u, "u"), _dev(v, "v"), u.numel(), _code(u), res.data_ptr(),
                                _stream(stream)), "cdot_noalloc")
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


def cgne_rb_solve(lat: Lattice, U: torch.Tensor, b: torch.Tensor, M5: float, mf: float, tol: float = 1e-10,
                  max_iter: int = 100000, stream=None):
    """H x = b by red-black (even-odd) preconditioned CGNE, the comparison solver of
    Section 5, in FP64 (every extent even).  Returns (x, stats dict); raises
    HDCRError when the solve fails."""
    if U.dtype != torch.complex128 or b.dtype != torch.complex128:
        raise TypeError("cgne_rb_solve takes complex128 links and source")
    x = torch.empty_like(b)
    g = lat.c_geom()
    p = _params(M5, mf)
    st = _lib.hdcr_solve_stats()
    _check(_L.hdcr_cgne_rb_solve(C_ref(g), C_ref(p), _dev(U, "U"), _dev(b, "b"), _dev(x, "x"), float(tol),
                                 int(max_iter), C_ref(st), _stream(stream)), "cgne_rb_solve")
    return x, st.as_dict()


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


def _dt(d) -> int:
    if isinstance(d, str) and d == "h16":
        return _lib.HDCR_H16
    return _lib.HDCR_C128 if d == torch.complex128 else _lib.HDCR_C64


def build_subspace(lat: Lattice, U: torch.Tensor, noise: torch.Tensor, M5: float, mf: float, block,
                   kind: str = "chebyshev", order: int = 300, lam_cut: float = 0.3, lam_max: float = 8.0,
                   filter_dtype: torch.dtype = torch.complex128,
                   store_dtype: torch.dtype = torch.complex128, stream=None) -> Subspace:
    """Subspace from nvec/2 noise fields (complex128, packed) (Section 4): each is filtered
    towards the low modes of H -- kind "cr" (``order`` CR steps on H x = 0) or
    "chebyshev" (the order-``order`` low-pass filter T(t(H^2)) of Fig. 1) -- then split
    by Gamma5 chirality and block-orthonormalised in FP64."""
    if U.dtype != torch.complex128 or noise.dtype != torch.complex128:
        raise TypeError("build_subspace takes complex128 links and noise")
    half = _nfields(lat, noise, "noise")
    sp = _lib.hdcr_subspace_params()
    sp.nvec = 2 * half
    for i in range(4):
        sp.block[i] = int(block[i])
    sp.kind = {"cr": _lib.HDCR_SUBSPACE_CR_SMOOTH, "chebyshev": _lib.HDCR_SUBSPACE_CHEBYSHEV}[kind]
    sp.order = int(order)
    sp.lam_cut = float(lam_cut)
    sp.lam_max = float(lam_max)
    sp.filter_dtype = _dt(filter_dtype)
    sp.store_dtype = _dt(store_dtype)
    h = ctypes.c_void_p()
    g = lat.c_geom()
    p = _params(M5, mf)
    _check(_L.hdcr_build_subspace(C_ref(g), C_ref(p), _dev(U, "U", True), _dev(noise, "noise", True), C_ref(sp),
                                  _stream(stream), ctypes.byref(h)), "build_subspace")
    return Subspace(h, lat, block, 2 * half, store_dtype, torch.device("cuda", torch.cuda.current_device()))


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
                    op_dtype: torch.dtype = torch.complex128, fast: bool = False, fp32_build: bool = False,
                    stream=None) -> CoarseOperator:
    """A^{ab}_{jk} = <phi_j^a|H|phi_k^b> for the 9 legs of every coarse site (Eq. 4.5).
    fast=True (complex64 only) builds with one pass of TF32 tensor-core products
    (relative error ~1e-3) instead of the three that keep FP32 accuracy.
    fp32_build=True (complex128 only) builds with the FP32-exact tensor-core path
    from the FP32-rounded basis and stores complex128 (relative error ~1e-7): for a
    solve whose coarse correction is the FP32 dense inverse."""
    if U.dtype != torch.complex128:
        raise TypeError("build_coarse_op takes complex128 links")
    if fast and op_dtype != torch.complex64:
        raise ValueError("fast=True builds a complex64 operator")
    if fp32_build and op_dtype != torch.complex128:
        raise ValueError("fp32_build=True builds a complex128 operator")
    h = ctypes.c_void_p()
    p = _params(M5, mf)
    if op_dtype == torch.complex128:
        code = _lib.HDCR_C128_TC if fp32_build else _lib.HDCR_C128
    else:
        code = _lib.HDCR_C64_FAST if fast else _lib.HDCR_C64
    _check(_L.hdcr_build_coarse_op(sub.handle, C_ref(p), _dev(U, "U", True), code, _stream(stream),
                                   ctypes.byref(h)), "build_coarse_op")
    return CoarseOperator(h, sub, op_dtype, M5, mf)


def cf_filter(lat: Lattice, U: torch.Tensor, x: torch.Tensor, M5: float, beta, R: float, kind: str = "cr",
              order: int = 10, lam_cut: float = 0.5, lam_max: float = 8.0, stream=None) -> torch.Tensor:
    """The subspace filter on the continued-fraction operator, in place on the field x
    (lat.Ls = len(beta) + 1 components): kind "cr" (order CR steps on H_cf x = 0) or
    "chebyshev" (the low-pass filter of Fig. 1 on H_cf^2).  Returns x."""
    if _nfields(lat, x, "x") != 1:
        raise ValueError("cf_filter takes one field")
    sp = _lib.hdcr_subspace_params()
    sp.kind = {"cr": _lib.HDCR_SUBSPACE_CR_SMOOTH, "chebyshev": _lib.HDCR_SUBSPACE_CHEBYSHEV}[kind]
    sp.order = int(order)
    sp.lam_cut = float(lam_cut)
    sp.lam_max = float(lam_max)
    g = lat.c_geom()
    _check(_L.hdcr_cf_filter(C_ref(g), float(M5), C_ref(_cf_params(beta, R)), _dev(U, "U"), _dev(x, "x"), _code(x),
                             C_ref(sp), _stream(stream)), "cf_filter")
    return x


def gamma5_split(lat: Lattice, v: torch.Tensor, stream=None):
    """((1 + gamma5)/2 v, (1 - gamma5)/2 v): the 4d chirality of each site and fifth
    coordinate (no R5 reflection) for every field of v."""
    n = _nfields(lat, v, "v")
    plus, minus = torch.empty_like(v), torch.empty_like(v)
    g = lat.c_geom()
    _check(_L.hdcr_gamma5_split(C_ref(g), _dev(v, "v"), _dev(plus, "plus"), _dev(minus, "minus"), _code(v), n,
                                _stream(stream)), "gamma5_split")
    return plus, minus


def build_cf_subspace(lat: Lattice, U: torch.Tensor, noise: torch.Tensor, M5: float, beta, R: float, block,
                      kind: str = "cr", order: int = 20, lam_cut: float = 0.3, lam_max: float = 10.0,
                      stream=None) -> "Subspace":
    """Section 4's subspace for the continued-fraction operator: the nvec/2 complex128
    noise fields (copied) filtered by cf_filter, split by 4d chirality (plus halves
    first, then minus), block-orthonormalised in FP64 (basis stored complex128)."""
    if noise.dtype != torch.complex128:
        raise TypeError("build_cf_subspace takes complex128 noise")
    x = noise.clone()
    for i in range(_nfields(lat, x, "noise")):
        cf_filter(lat, U, x[i], M5, beta, R, kind=kind, order=order, lam_cut=lam_cut, lam_max=lam_max, stream=stream)
    plus, minus = gamma5_split(lat, x, stream=stream)
    return subspace_from_vectors(lat, block, torch.cat([plus, minus]).contiguous(), stream=stream)


def build_cf_coarse_op(sub: Subspace, U: torch.Tensor, M5: float, beta, R: float, stream=None) -> CoarseOperator:
    """The little operator of the continued-fraction operator on the complex128 basis
    ``sub`` (built on its N-component geometry); hdcr_solve with the returned handle
    runs the two-level method on H_cf."""
    if U.dtype != torch.complex128:
        raise TypeError("build_cf_coarse_op takes complex128 links")
    h = ctypes.c_void_p()
    _check(_L.hdcr_cf_build_coarse_op(sub.handle, float(M5), C_ref(_cf_params(beta, R)), _dev(U, "U", True),
                                      _stream(stream), ctypes.byref(h)), "cf_build_coarse_op")
    return CoarseOperator(h, sub, torch.complex128, M5, 0.0)


def apply_coarse(co: CoarseOperator, c: torch.Tensor, stream=None) -> torch.Tensor:
    """9-point coarse stencil applied to (nrhs, Vc, nvec) coarse vectors."""
    per = co.sub.Vc * co.sub.nvec
    if c.numel() % per:
        raise ValueError("coarse vectors must hold a multiple of Vc*nvec entries")
    out = torch.empty_like(c)
    _check(_L.hdcr_apply_coarse(co.handle, _dev(c, "c"), _dev(out, "out"), _code(c), c.numel() // per,
                                _stream(stream)), "apply_coarse")
    return out


def coarse_invert(co: CoarseOperator, stream=None) -> None:
    """Dense FP32 inverse of the coarse operator (Gauss-Jordan with partial pivoting)."""
    _check(_L.hdcr_coarse_invert(co.handle, _stream(stream)), "coarse_invert")


def coarse_solve_dense(co: CoarseOperator, c: torch.Tensor, stream=None) -> torch.Tensor:
    """A^{-1} c with the dense inverse (complex64 coarse vectors)."""
    per = co.sub.Vc * co.sub.nvec
    out = torch.empty_like(c)
    _check(_L.hdcr_coarse_solve_dense(co.handle, _dev(c, "c"), _dev(out, "out"), c.numel() // per,
                                      _stream(stream)), "coarse_solve_dense")
    return out


def build_level2(co: CoarseOperator, noise: torch.Tensor, block, nvec2: int | None = None, smooth_iters: int = 200,
                 cycle_smooth: int = 16, stream=None) -> None:
    """The third level of the coarse solve (Section 4's construction applied to A, the
    recursion of Section 5): level-2 basis from nvec2/2 complex128 coarse noise vectors
    (shape (nvec2/2, Vc, nvec)), blocks of ``block`` coarse sites, A2 and its dense
    inverse, kept in ``co`` for coarse_solver="recursive"."""
    if noise.dtype != torch.complex128:
        raise TypeError("level-2 noise must be complex128")
    per = co.sub.Vc * co.sub.nvec
    half = noise.numel() // per
    if noise.numel() != half * per or half < 1:
        raise ValueError("noise must hold nvec2/2 coarse vectors")
    prm = _lib.hdcr_level2_params()
    prm.nvec2 = int(nvec2 if nvec2 is not None else 2 * half)
    for i in range(4):
        prm.block[i] = int(block[i])
    prm.smooth_iters = int(smooth_iters)
    prm.cycle_smooth = int(cycle_smooth)
    _check(_L.hdcr_coarse_build_level2(co.handle, C_ref(prm), _dev(noise, "noise", True), _stream(stream)),
           "build_level2")


def level2_get(co: CoarseOperator, stream=None):
    """(basis, A2) of the third level as complex128: (nvec2, Vc, nvec) and (Vc2, 9, nvec2, nvec2)."""
    n2 = ctypes.c_int()
    L2 = (ctypes.c_int * 4)()
    _check(_L.hdcr_coarse_level2_info(co.handle, ctypes.byref(n2), L2), "level2_info")
    if n2.value == 0:
        raise ValueError("the coarse operator has no third level")
    Vc2 = L2[0] * L2[1] * L2[2] * L2[3]
    dev = co.sub.device
    vec = torch.empty((n2.value, co.sub.Vc, co.sub.nvec), dtype=torch.complex128, device=dev)
    op = torch.empty((Vc2, 9, n2.value, n2.value), dtype=torch.complex128, device=dev)
    _check(_L.hdcr_coarse_level2_get(co.handle, vec.data_ptr(), op.data_ptr(), _stream(stream)), "level2_get")
    return vec, op


def coarse_solve_level2(co: CoarseOperator, c: torch.Tensor, tol: float = 1e-10, max_iter: int = 500,
                        stream=None):
    """A^{-1} c for one coarse vector (the operator's dtype) by the recursive solver;
    returns (x, iterations)."""
    out = torch.empty_like(c)
    it = ctypes.c_int()
    _check(_L.hdcr_coarse_solve_level2(co.handle, _dev(c, "c"), _dev(out, "out"), float(tol), int(max_iter),
                                       ctypes.byref(it), _stream(stream)), "coarse_solve_level2")
    return out, it.value


def _solve_params(tol, max_outer, restart, smoother, smoother_order, cheb_lo, cheb_hi, coarse_solver,
                  coarse_tol, coarse_max, inner_dtype, cycle="symmetric"):
    prm = _lib.hdcr_solve_params()
    prm.tol = float(tol)
    prm.max_outer = int(max_outer)
    prm.restart = int(restart)
    prm.smoother_kind = {"cr": _lib.HDCR_SMOOTHER_CR, "chebyshev": _lib.HDCR_SMOOTHER_CHEBYSHEV}[smoother]
    prm.smoother_order = int(smoother_order)
    prm.cheb_lo = float(cheb_lo)
    prm.cheb_hi = float(cheb_hi)
    prm.coarse_solver = {"cr": _lib.HDCR_COARSE_CR, "dense": _lib.HDCR_COARSE_DENSE,
                         "recursive": _lib.HDCR_COARSE_RECURSIVE}[coarse_solver]
    prm.coarse_tol = float(coarse_tol)
    prm.coarse_max = int(coarse_max)
    prm.inner_dtype = _dt(inner_dtype)
    prm.cycle = {"symmetric": _lib.HDCR_CYCLE_SYMMETRIC, "post": _lib.HDCR_CYCLE_POST}[cycle]
    return prm


def hdcr_solve_into(co: CoarseOperator, U: torch.Tensor, b: torch.Tensor, x: torch.Tensor,
                    tol: float = 1e-10, max_outer: int = 500, restart: int = 8,
                    smoother: str = "chebyshev", smoother_order: int = 10, cheb_lo: float = 1.0,
                    cheb_hi: float = 64.0, coarse_solver: str = "dense", coarse_tol: float = 1e-4,
                    coarse_max: int = 1000, inner_dtype: torch.dtype = torch.complex128,
                    cycle: str = "symmetric", stream=None) -> dict:
    """hdcr_solve with a caller-owned x (initial guess in, iterate out).  Returns the
    stats dict, including a failed solve's status, without raising."""
    if U.dtype != torch.complex128 or b.dtype != torch.complex128 or x.dtype != torch.complex128:
        raise TypeError("hdcr_solve takes complex128 links, source and solution")
    prm = _solve_params(tol, max_outer, restart, smoother, smoother_order, cheb_lo, cheb_hi,
                        coarse_solver, coarse_tol, coarse_max, inner_dtype, cycle)
    st = _lib.hdcr_solve_stats()
    status = _L.hdcr_solve(co.handle, _dev(U, "U", True), _dev(b, "b", True), _dev(x, "x", True), C_ref(prm),
                           C_ref(st), _stream(stream))
    d = st.as_dict()
    d["status"] = status
    return d


def hdcr_solve(co: CoarseOperator, U: torch.Tensor, b: torch.Tensor, x0: torch.Tensor | None = None,
               tol: float = 1e-10, max_outer: int = 500, restart: int = 8,
               smoother: str = "chebyshev", smoother_order: int = 10, cheb_lo: float = 1.0,
               cheb_hi: float = 64.0, coarse_solver: str = "dense", coarse_tol: float = 1e-4,
               coarse_max: int = 1000, inner_dtype: torch.dtype = torch.complex128, cycle: str = "symmetric",
               stream=None):
    """H x = b by flexible GCR preconditioned with the two-level V-cycle (Section 4).
    smoother "chebyshev" (S = H p(H^2), p ~ 1/y on [cheb_lo, cheb_hi]) or "cr"
    (smoother_order CR steps); coarse_solver "dense" (exact, FP32 inverse), "cr" or
    "recursive" (third level); cycle "symmetric" (smoother before and after the coarse
    correction, Section 4's composite) or "post" (coarse correction, then smoother).
    Returns (x, stats dict); raises HDCRError when the solve fails."""
    if U.dtype != torch.complex128 or b.dtype != torch.complex128:
        raise TypeError("hdcr_solve takes complex128 links and source")
    if _nfields(co.sub.lat, b, "b") != 1:
        raise ValueError("hdcr_solve takes one right-hand side")
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    prm = _solve_params(tol, max_outer, restart, smoother, smoother_order, cheb_lo, cheb_hi,
                        coarse_solver, coarse_tol, coarse_max, inner_dtype, cycle)
    st = _lib.hdcr_solve_stats()
    _check(_L.hdcr_solve(co.handle, _dev(U, "U", True), _dev(b, "b", True), _dev(x, "x", True), C_ref(prm),
                         C_ref(st), _stream(stream)), "hdcr_solve")
    return x, st.as_dict()


# ------------------------------------------------------------------ gradient
def hdcr_solve_multi(co: CoarseOperator, U: torch.Tensor, B: torch.Tensor, x0: torch.Tensor | None = None,
                     tol: float = 1e-10, max_outer: int = 500, restart: int = 8, smoother_order: int = 10,
                     cheb_lo: float = 1.0, cheb_hi: float = 64.0, inner_dtype: torch.dtype = torch.complex128,
                     graph: bool = True, cycle: str = "symmetric", stream=None):
    """H x_r = b_r for the nrhs fields of B at once (the Section 4 solve batched over
    right-hand sides; Chebyshev smoother, dense coarse solve).  graph=True replays the
    V-cycle from a captured CUDA graph.  Returns (X, list of per-rhs stats dicts); raises
    HDCRError when the solve fails."""
    if U.dtype != torch.complex128 or B.dtype != torch.complex128:
        raise TypeError("hdcr_solve_multi takes complex128 links and sources")
    nrhs = _nfields(co.sub.lat, B, "B")
    X = torch.zeros_like(B) if x0 is None else x0.clone()
    prm = _solve_params(tol, max_outer, restart, "chebyshev", smoother_order, cheb_lo, cheb_hi, "dense", 1e-4,
                        1000, inner_dtype, cycle)
    st = (_lib.hdcr_solve_stats * nrhs)()
    _check(_L.hdcr_solve_multi(co.handle, _dev(U, "U"), _dev(B, "B"), _dev(X, "X"), nrhs, C_ref(prm),
                               1 if graph else 0, st, _stream(stream)), "hdcr_solve_multi")
    return X, [st[i].as_dict() for i in range(nrhs)]


def gauge_force(lat: Lattice, x: torch.Tensor, w: torch.Tensor, stream=None) -> torch.Tensor:
    """F_mu(x) with dL = Re sum tr(dU F) for L = Re(eta^dag x), H x = b, w = Gamma5 H^{-1} eta.
    Returns a (4, V4, 3, 3) tensor, F[mu, x4, b, a] = (F_mu(x))_ba."""
    if x.dtype != w.dtype or _nfields(lat, x, "x") != 1 or _nfields(lat, w, "w") != 1:
        raise ValueError("x and w must be single fields of one dtype")
    F = torch.empty((4, lat.V4, 3, 3), dtype=x.dtype, device=x.device)
    g = lat.c_geom()
    _check(_L.hdcr_gauge_force(C_ref(g), _dev(x, "x", True), _dev(w, "w", True), F.data_ptr(), _code(x),
                               _stream(stream)), "gauge_force")
    return F


def gauge_grad(lat: Lattice, x: torch.Tensor, w: torch.Tensor, stream=None) -> torch.Tensor:
    """The gauge force of (x, w) stored as the gradient with respect to the links:
    G[mu, x4, a, b] = conj(F_mu(x)_ba) = dL/dRe U_ab + i dL/dIm U_ab (torch's convention
    for complex gradients).  Returns a (4, V4, 3, 3) tensor of x's dtype."""
    if x.dtype != w.dtype or _nfields(lat, x, "x") != 1 or _nfields(lat, w, "w") != 1:
        raise ValueError("x and w must be single fields of one dtype")
    G = torch.empty((4, lat.V4, 3, 3), dtype=x.dtype, device=x.device)
    g = lat.c_geom()
    _check(_L.hdcr_gauge_grad(C_ref(g), _dev(x, "x"), _dev(w, "w"), G.data_ptr(), _code(x),
                              _stream(stream)), "gauge_grad")
    return G


# default true-residual target of the differentiable solve per input precision: the
# complex64 form returns FP32 fields, for which 1e-7 is below their own rounding
_AUTOGRAD_TOL = {torch.complex128: 1e-10, torch.complex64: 1e-7}


def _autograd_setup(lat, U64, noise, M5, mf, block, filter_kw, dtype):
    """Subspace and coarse operator of the differentiable solve in the precision of
    the inputs (complex64: FP32 filter, basis and coarse operator)."""
    kw = dict(filter_kw)
    if dtype == torch.complex64:
        kw.setdefault("filter_dtype", torch.complex64)
        kw.setdefault("store_dtype", torch.complex64)
    sub = build_subspace(lat, U64, noise, M5, mf, block, **kw)
    co = build_coarse_op(sub, U64, M5, mf, op_dtype=sub.dtype)
    return sub, co


def _autograd_solve(lat, U, rhs, noise, M5, mf, block, filter_kw, solve_kw):
    """H(U) x = rhs with a freshly built subspace and coarse operator, which are freed
    before returning; U and rhs share their dtype (complex128 or complex64) and so
    does x.  The outer flexible GCR runs in FP64 on the upcast inputs; with complex64
    inputs the V-cycle (smoother, basis, coarse operator) runs in FP32."""
    dtype = U.dtype
    U64 = U if dtype == torch.complex128 else convert(U, torch.complex128)
    r64 = rhs.contiguous() if dtype == torch.complex128 else convert(rhs.contiguous(), torch.complex128)
    kw = dict(solve_kw)
    kw.setdefault("tol", _AUTOGRAD_TOL[dtype])
    sub, co = _autograd_setup(lat, U64, noise, M5, mf, block, filter_kw, dtype)
    try:
        x, st = hdcr_solve(co, U64, r64, inner_dtype=sub.dtype, **kw)
    finally:
        co.close()
        sub.close()
    return (x if dtype == torch.complex128 else convert(x, dtype)), st


class HDCRSolve(torch.autograd.Function):
    """x = H(U)^{-1} b by HDCR, differentiable in U and b; U, b and x are complex128
    or complex64 (one dtype for all three).

    Forward: build the subspace and coarse operator from ``noise`` (not
    differentiated: the converged solution does not depend on it), solve, and free
    them: only U, x and the noise are kept for the backward.
    Backward, given g = dL/dx (torch convention): the subspace and coarse operator
    are rebuilt from the same noise, the adjoint solve H y = g runs with the same
    Hermitian operator and coarse space, then dL/db = y and dL/dU is the gauge force
    of (x, Gamma5 y) in gradient layout (``gauge_grad``), both in the input dtype.
    Recomputing costs one more setup per backward and saves keeping the nvec basis
    fields and the coarse operator alive between forward and backward.
    """

    @staticmethod
    def forward(ctx, U, b, lat, noise, M5, mf, block, filter_kw, solve_kw):
        if U.dtype not in _AUTOGRAD_TOL or b.dtype != U.dtype:
            raise TypeError("solve_autograd takes complex128 or complex64 links and source of one dtype")
        x, st = _autograd_solve(lat, U, b, noise, M5, mf, block, filter_kw, solve_kw)
        ctx.lat, ctx.M5, ctx.mf, ctx.block = lat, M5, mf, block
        ctx.filter_kw, ctx.solve_kw = filter_kw, solve_kw
        ctx.save_for_backward(U, x, noise)
        ctx.stats = st
        return x

    @staticmethod
    def backward(ctx, gx):
        U, x, noise = ctx.saved_tensors
        y, st = _autograd_solve(ctx.lat, U, gx.to(U.dtype), noise, ctx.M5, ctx.mf, ctx.block, ctx.filter_kw,
                                ctx.solve_kw)
        ctx.backward_stats = st
        gU = gauge_grad(ctx.lat, x, apply_gamma5_r5(ctx.lat, y))
        return gU, y, None, None, None, None, None, None, None


def solve_autograd(lat: Lattice, U: torch.Tensor, b: torch.Tensor, noise: torch.Tensor, M5: float, mf: float,
                   block, filter_kw: dict | None = None, solve_kw: dict | None = None) -> torch.Tensor:
    """Differentiable HDCR solve: see HDCRSolve.  ``noise`` (nvec/2 complex128 fields)
    seeds the subspace, rebuilt identically in the backward."""
    return HDCRSolve.apply(U, b, lat, noise, M5, mf, tuple(block), filter_kw or {}, solve_kw or {})
