"""The allocation-free inner product hdcr_cdot_noalloc, called through the C ABI.

Callers that may not let the library allocate device memory (a caller that
keeps all device memory in its own pool, a runtime that forbids allocations
after start-up) use this entry point; its scratch is a fixed array inside the
library.  It must give the same result as hdcr_cdot, call after call
(the shared scratch keeps the previous call's contents, so a stale completion
counter or partial sum would show up on the second call), and refuse sizes its
scratch cannot hold.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abi():
    import paper_1611_06944_gb300 as hd
    from paper_1611_06944_gb300 import _lib
    hd.load_library()
    return hd._L, _lib


def _dot(fn, u, v, dtype_code):
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = fn(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), u.numel(), dtype_code,
            ctypes.c_void_p(res.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    r = res.cpu().numpy()
    return complex(r[0], r[1])


@pytest.mark.parametrize("n", [1, 4097, 1_000_003, 12 * 16 ** 4 * 16])
def test_noalloc_matches_cdot_twice(abi, n):
    L, lib = abi
    rng = synth.rng(7000 + n % 97)
    for dtype, code, tol in [(np.complex128, lib.HDCR_C128, 1e-13), (np.complex64, lib.HDCR_C64, 1e-13)]:
        u = torch.from_numpy((rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(dtype)).cuda()
        v = torch.from_numpy((rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(dtype)).cuda()
        want = _dot(L.hdcr_cdot, u, v, code)
        # rounding scale of a sum of n products: sum |u_i| |v_i|
        scale = float((u.abs().double() * v.abs().double()).sum())
        for _ in range(2):                       # two calls in a row share the scratch
            got = _dot(L.hdcr_cdot_noalloc, u, v, code)
            assert abs(got - want) <= tol * scale
        # a different input right after: nothing carries over from the previous call
        got2 = _dot(L.hdcr_cdot_noalloc, v, u, code)
        assert abs(got2 - np.conj(want)) <= tol * scale


def test_noalloc_rejects_sizes_beyond_its_scratch(abi):
    L, lib = abi
    u = torch.zeros(4, dtype=torch.complex128, device="cuda")
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = L.hdcr_cdot_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), 268435456 + 1,
                             lib.HDCR_C128, ctypes.c_void_p(res.data_ptr()), None)
    assert st == -1
    assert b"static scratch" in L.hdcr_last_error()
