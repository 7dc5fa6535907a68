"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol include/hdcr.h declares, and rejects bad arguments on the host before
touching a GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdcr.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc to build the library")


@pytest.fixture(scope="module")
def lib():
    from paper_1611_06944_gb300 import build as b
    path = b.build()
    from paper_1611_06944_gb300 import _lib
    return _lib.load(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(hdcr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ["hdcr_apply_g5dwf", "hdcr_cr_solve", "hdcr_cdot", "hdcr_norm2"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1611_06944_gb300 import _lib
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in hdcr.h but not exported"
        assert n in _lib.SIGNATURES, f"{n} has no ctypes signature in the binding"
    assert set(_lib.SIGNATURES) == set(names)


def test_binding_constants_match_the_header():
    """Every #define HDCR_* integer of include/hdcr.h that the binding mirrors has the
    same value there (dtype codes, smoother / coarse-solver / cycle kinds)."""
    from paper_1611_06944_gb300 import _lib
    defs = dict(re.findall(r"#define\s+(HDCR_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", open(HEADER).read()))
    mirrored = [n for n in defs if hasattr(_lib, n)]
    assert len(mirrored) >= 12
    for n in mirrored:
        assert getattr(_lib, n) == int(defs[n]), n
    for n in ("HDCR_C128_TC", "HDCR_CYCLE_POST", "HDCR_COARSE_RECURSIVE"):
        assert n in mirrored
    dtypes = [int(defs[n]) for n in ("HDCR_C128", "HDCR_C64", "HDCR_C64_FAST", "HDCR_H16", "HDCR_C128_TC")]
    assert len(set(dtypes)) == len(dtypes)


def test_status_strings(lib):
    assert lib.hdcr_strerror(0) == b"ok"
    assert lib.hdcr_strerror(-2) == b"bad geometry"
    assert lib.hdcr_version() >= 100


def _geom(L=(4, 4, 4, 4), Ls=8, bc=1):
    from paper_1611_06944_gb300 import _lib
    g = _lib.hdcr_geom()
    for i in range(4):
        g.L[i] = L[i]
    g.Ls = Ls
    g.bc_t = bc
    return g


def test_bad_geometry_rejected_on_host(lib):
    from paper_1611_06944_gb300 import _lib
    p = _lib.hdcr_dwf_params(1.8, 0.01)
    fake = ctypes.c_void_p(0x1000)
    fake2 = ctypes.c_void_p(0x2000)
    for bad in [_geom(Ls=1), _geom(L=(0, 4, 4, 4)), _geom(bc=0)]:
        s = lib.hdcr_apply_g5dwf(ctypes.byref(bad), ctypes.byref(p), fake, fake, fake2, 0, 1, None)
        assert s == -2
        assert lib.hdcr_last_error()
    g = _geom()
    assert lib.hdcr_apply_g5dwf(ctypes.byref(g), ctypes.byref(p), None, fake, fake2, 0, 1, None) == -1
    assert lib.hdcr_apply_g5dwf(ctypes.byref(g), ctypes.byref(p), fake, fake, fake, 0, 1, None) == -1
    assert lib.hdcr_apply_g5dwf(ctypes.byref(g), ctypes.byref(p), fake, fake, fake2, 7, 1, None) == -1
    assert lib.hdcr_apply_g5dwf(ctypes.byref(g), ctypes.byref(p), fake, fake, fake2, 0, 0, None) == -1
    st = _lib.hdcr_solve_stats()
    assert lib.hdcr_cr_solve(ctypes.byref(g), ctypes.byref(p), fake, fake, fake2, 0, -1.0, 10,
                             ctypes.byref(st), None) == -1


def test_new_entry_points_reject_bad_arguments_on_host(lib):
    """Argument checks of the autotuner, FP16 storage, the batched and red-black
    solves and the Moebius conversion, all before any CUDA call."""
    from paper_1611_06944_gb300 import _lib
    p = _lib.hdcr_dwf_params(1.8, 0.01)
    q = _lib.hdcr_dwf_params()
    fake = ctypes.c_void_p(0x1000)
    fake2 = ctypes.c_void_p(0x2000)
    odd_ptr = ctypes.c_void_p(0x1008)  # 8-byte but not 16-byte aligned
    st = _lib.hdcr_solve_stats()
    g = _geom()
    # tile autotuner: mode 0..2, force_variant >= -1
    assert lib.hdcr_stencil_tune(3, -1) == -1
    assert lib.hdcr_stencil_tune(1, -2) == -1
    assert lib.hdcr_stencil_tune(1, -1) == 0
    v = ctypes.c_int()
    assert lib.hdcr_stencil_tune_info(ctypes.byref(g), 0, ctypes.byref(v), None, 0) == -1
    # FP16 storage: dtype, distinct aligned buffers; the operator needs an even Ls <= 16
    assert lib.hdcr_fermion_encode_h16(ctypes.byref(g), fake, 5, fake2, 1, None) == -1
    assert lib.hdcr_fermion_encode_h16(ctypes.byref(g), fake, 0, fake, 1, None) == -1
    assert lib.hdcr_fermion_encode_h16(ctypes.byref(g), odd_ptr, 0, fake2, 1, None) == -1
    assert lib.hdcr_fermion_decode_h16(ctypes.byref(g), fake, fake2, 0, 0, None) == -1
    g5 = _geom(Ls=5)
    assert lib.hdcr_apply_g5dwf(ctypes.byref(g5), ctypes.byref(p), fake, fake, fake2, _lib.HDCR_H16, 1, None) == -1
    # red-black CGNE: every extent even, tol > 0
    godd = _geom(L=(4, 3, 4, 4))
    assert lib.hdcr_cgne_rb_solve(ctypes.byref(godd), ctypes.byref(p), fake, fake, fake2, 1e-10, 10,
                                  ctypes.byref(st), None) == -2
    assert lib.hdcr_cgne_rb_solve(ctypes.byref(g), ctypes.byref(p), fake, fake, fake2, 0.0, 10,
                                  ctypes.byref(st), None) == -1
    # Moebius conversion: b5 > 0, a known dtype
    assert lib.hdcr_mobius_to_shamir(ctypes.byref(p), 0.0, fake, fake2, 0, 36, ctypes.byref(q), None) == -1
    assert lib.hdcr_mobius_to_shamir(ctypes.byref(p), 1.5, fake, fake2, 9, 36, ctypes.byref(q), None) == -1
    # batched solve and coarse build: a null handle is refused
    prm = _lib.hdcr_solve_params()
    assert lib.hdcr_solve_multi(None, fake, fake, fake2, 2, ctypes.byref(prm), 1, ctypes.byref(st), None) == -1
    h = ctypes.c_void_p()
    assert lib.hdcr_build_coarse_op(None, ctypes.byref(p), fake, _lib.HDCR_C64_FAST, None, ctypes.byref(h)) == -1


def test_overlap_and_level2_entry_points_reject_bad_arguments_on_host(lib):
    """Argument checks of the continued-fraction calls (component count against Ls,
    positive beta, filter parameters), the 4d chirality split, the third level and the
    solve's cycle and timer codes, all before any CUDA call."""
    from paper_1611_06944_gb300 import _lib
    fake = ctypes.c_void_p(0x1000)
    fake2 = ctypes.c_void_p(0x2000)
    fake3 = ctypes.c_void_p(0x3000)
    st = _lib.hdcr_solve_stats()
    g5 = _geom(Ls=5)
    cf = _lib.hdcr_cf_params()
    cf.ncomp = 5
    for i, b in enumerate((1.3, 0.9, 1.7, 0.6)):
        cf.beta[i] = b
    cf.R = 0.3
    g4 = _geom(Ls=4)
    assert lib.hdcr_apply_cf_overlap(ctypes.byref(g4), 1.8, ctypes.byref(cf), fake, fake2, fake3, 0, 1, None) == -1
    cf.beta[2] = -1.0
    assert lib.hdcr_apply_cf_overlap(ctypes.byref(g5), 1.8, ctypes.byref(cf), fake, fake2, fake3, 0, 1, None) == -1
    cf.beta[2] = 1.7
    assert lib.hdcr_apply_cf_overlap(ctypes.byref(g5), 1.8, ctypes.byref(cf), fake, fake2, fake2, 0, 1, None) == -1
    assert lib.hdcr_cf_cr_solve(ctypes.byref(g5), 1.8, ctypes.byref(cf), fake, fake2, fake3, 0, 0.0, 10,
                                ctypes.byref(st), None) == -1
    sp = _lib.hdcr_subspace_params()
    sp.kind = _lib.HDCR_SUBSPACE_CHEBYSHEV
    sp.order = 10
    sp.lam_cut, sp.lam_max = 0.5, 0.4                   # lam_max must exceed lam_cut
    assert lib.hdcr_cf_filter(ctypes.byref(g5), 1.8, ctypes.byref(cf), fake, fake2, 0, ctypes.byref(sp), None) == -1
    sp.kind = 7
    assert lib.hdcr_cf_filter(ctypes.byref(g5), 1.8, ctypes.byref(cf), fake, fake2, 0, ctypes.byref(sp), None) == -1
    h = ctypes.c_void_p()
    assert lib.hdcr_cf_build_coarse_op(None, 1.8, ctypes.byref(cf), fake, None, ctypes.byref(h)) == -1
    # the chirality split: distinct outputs, a known dtype, at least one field
    assert lib.hdcr_gamma5_split(ctypes.byref(g5), fake, fake2, fake2, 0, 1, None) == -1
    assert lib.hdcr_gamma5_split(ctypes.byref(g5), fake, fake2, fake3, 3, 1, None) == -1
    assert lib.hdcr_gamma5_split(ctypes.byref(g5), fake, fake2, fake3, 0, 0, None) == -1
    # the third level and the solve need a coarse handle
    l2 = _lib.hdcr_level2_params()
    assert lib.hdcr_coarse_build_level2(None, ctypes.byref(l2), fake, None) == -1
    it = ctypes.c_int()
    assert lib.hdcr_coarse_solve_level2(None, fake, fake2, 1e-6, 10, ctypes.byref(it), None) == -1
    prm = _lib.hdcr_solve_params()
    prm.cycle = 5
    assert lib.hdcr_solve(None, fake, fake2, fake3, ctypes.byref(prm), ctypes.byref(st), None) == -1
    # the stencil timer knows FP64, FP32, FP16 storage and the fused FP64 smoother step only
    ms, nl, ns = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
    assert lib.hdcr_stencil_timer_read(_lib.HDCR_TIMER_C128_CHEB, ctypes.byref(ms), ctypes.byref(nl),
                                       ctypes.byref(ns)) == 0
    assert lib.hdcr_stencil_timer_read(7, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(ns)) == -1
