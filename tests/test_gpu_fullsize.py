"""The precision form at its full size (24^3 x 48 x 16, eps = 0.5, mf = 0.005; FP32
stencil and V-cycle, coarse operator nvec = 32 built on the tensor cores, FP64
flexible GCR to a true residual of 1e-10), checked by the FP64 oracle on sampled
5d sites: the oracle evaluates H x site by site (Section 3's operator written out
term by term), and the residual b - H x it finds there must be at the solve's
level, while the library's own FP64 residual at those sites must agree with it.
This test holds about 70 GB on the device and runs for about a minute."""
import numpy as np
import pytest

import synth
from oracle import dwf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class _Natural:
    """A library-layout field (V4, 12, Ls) read as oracle.dwf's natural layout:
    psi[t, z, y, x, s] -> (4, 3) spin-colour array, without unpacking the whole field."""

    def __init__(self, lib, L, Ls):
        self.lib = lib
        self.L = L
        Lx, Ly, Lz, Lt = L
        self.shape = (Lt, Lz, Ly, Lx, Ls, 4, 3)

    def __getitem__(self, idx):
        t, z, y, x, s = idx
        Lx, Ly, Lz, Lt = self.L
        x4 = ((t * Lz + z) * Ly + y) * Lx + x
        return self.lib[x4, :, s].reshape(4, 3)


def test_precision_form_fullsize_residual_by_oracle():
    import paper_1611_06944_gb300 as hd
    torch.cuda.empty_cache()  # the library allocates its own workspaces (~150 GB at the peak)
    L, Ls, eps, M5, mf, nvec = (24, 24, 24, 48), 16, 0.5, 1.8, 0.005, 32
    lat = hd.Lattice(L, Ls, 1)
    Uh = synth.gauge_field(L, eps, 1002)
    U = torch.from_numpy(Uh.reshape(4, -1, 3, 3).copy()).cuda()
    b = synth.device_gaussian(1, lat.V5, 2002)[0].reshape(lat.V4, 12, Ls).contiguous()
    noise = synth.device_gaussian(nvec // 2, lat.V5, 3002).reshape(nvec // 2, lat.V4, 12, Ls).contiguous()
    sub = hd.build_subspace(lat, U, noise, M5, mf, (6, 6, 6, 6), kind="chebyshev", order=600, lam_cut=0.1,
                            lam_max=8.0, filter_dtype=torch.complex64, store_dtype=torch.complex64)
    del noise
    co = hd.build_coarse_op(sub, U, M5, mf, op_dtype=torch.complex64, fast=True)
    x, st = hd.hdcr_solve(co, U, b, tol=1e-10, restart=8, max_outer=300, smoother="chebyshev", smoother_order=10,
                          cheb_lo=1.0, cheb_hi=64.0, coarse_solver="dense", inner_dtype=torch.complex64)
    assert st["status"] == 0 and st["true_resid"] <= 1e-10
    # the library's FP64 residual field
    r = (b - hd.apply_g5dwf(lat, U, x, M5, mf)).cpu().numpy()
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    co.close()
    sub.close()
    rng = synth.rng(7100)
    Lx, Ly, Lz, Lt = L
    sites = [(int(rng.integers(Lx)), int(rng.integers(Ly)), int(rng.integers(Lz)), int(rng.integers(Lt)),
              int(rng.integers(Ls))) for _ in range(48)]
    sites += [(0, 0, 0, 0, 0), (Lx - 1, Ly - 1, Lz - 1, Lt - 1, Ls - 1)]  # the corners, where every hop wraps
    Hx = dwf.apply_H_at(Uh, _Natural(xh, L, Ls), sites, M5, mf, 1)
    bn, rn = _Natural(bh, L, Ls), _Natural(r, L, Ls)
    ro = np.array([bn[t, z, y, x_, s] for (x_, y, z, t, s) in sites]) - Hx
    rg = np.array([rn[t, z, y, x_, s] for (x_, y, z, t, s) in sites])
    bs = np.array([bn[t, z, y, x_, s] for (x_, y, z, t, s) in sites])
    # the oracle's residual on the sample is at the solve's level (1e-10 overall; a 50-site
    # sample of a residual spread over the lattice fluctuates by a small factor)
    assert np.linalg.norm(ro) / np.linalg.norm(bs) <= 1e-9
    # and the library's FP64 residual agrees with it to FP64 rounding of H x (|Hx| ~ |b|)
    assert np.linalg.norm(rg - ro) <= 1e-13 * np.linalg.norm(Hx) * 10
