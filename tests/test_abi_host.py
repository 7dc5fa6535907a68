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
