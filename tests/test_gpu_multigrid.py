"""GPU parity of the two-level pieces (Section 4) against the FP64 oracle:
subspace, P^dag / P, the little Dirac operator and its 9-point application,
and the HDCR solve."""
import numpy as np
import pytest

import synth
from oracle import dwf, multigrid as mg
from oracle.krylov import cr
from gpu_util import dev, host, links, natural, planes, relerr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M5 = 1.8


@pytest.fixture(scope="module")
def hd():
    import paper_1611_06944_gb300 as hd
    return hd


def _oracle_sub(L, Ls, block, nvec, eps, mf, seed, iters=10, bc=1):
    g = mg.Geometry(L, Ls, block)
    U = synth.gauge_field(L, eps, seed)
    noise = synth.gaussian_fermion(L, Ls, seed + 1, count=nvec // 2)
    sub = mg.build_subspace(U, noise, g, M5, mf, bc, smooth_iters=iters)
    return g, U, noise, sub


# the tiny 4^4 x 8 workload (2^4 coarse, legs alias) and a ragged block shape
SUBSPACE_CASES = [
    ((4, 4, 4, 4), 8, (2, 2, 2, 2), 8, 0.3, 0.01, 1),
    ((6, 4, 2, 4), 5, (3, 2, 1, 2), 4, 0.5, 0.05, -1),
]


@pytest.mark.parametrize("L,Ls,block,nvec,eps,mf,bc", SUBSPACE_CASES)
def test_build_subspace_matches_oracle(hd, L, Ls, block, nvec, eps, mf, bc):
    g, U, noise, sub = _oracle_sub(L, Ls, block, nvec, eps, mf, 3000, bc=bc)
    lat = hd.Lattice(L, Ls, bc)
    gsub = hd.build_subspace(lat, dev(links(U)), dev(planes(noise)), M5, mf, block, kind="cr", order=10)
    got = natural(host(gsub.vectors()), L, Ls)
    want = mg.from_blocks(g, sub.Phi)
    for k in range(nvec):
        assert relerr(got[k], want[k]) < 1e-10, k


def _gpu_sub_from_oracle(hd, lat, g, sub, dtype=None):
    vec = planes(mg.from_blocks(g, sub.Phi))
    return hd.subspace_from_vectors(lat, g.block, dev(vec),
                                    store_dtype=torch.complex128 if dtype is None else dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_restrict_prolong_match_oracle(hd, dtype):
    L, Ls, block = (4, 6, 4, 4), 4, (2, 3, 2, 2)
    g, U, noise, sub = _oracle_sub(L, Ls, block, 6, 0.5, 0.05, 3100, iters=3)
    lat = hd.Lattice(L, Ls)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    gsub = _gpu_sub_from_oracle(hd, lat, g, sub, tdt)
    v = synth.gaussian_fermion(L, Ls, 3101, count=2)
    vd = dev(planes(v), tdt)
    c = host(hd.restrict(gsub, vd)).astype(np.complex128)
    tol = 1e-13 if dtype == "c128" else 1e-5
    for r in range(2):
        assert relerr(c[r], mg.restrict(sub, v[r])) < tol
    rng = synth.rng(3102)
    cc = rng.standard_normal((g.Vc, 6)) + 1j * rng.standard_normal((g.Vc, 6))
    f = natural(host(hd.prolong(gsub, dev(cc, tdt))).astype(np.complex128), L, Ls)
    assert relerr(f, mg.prolong(sub, cc)) < tol
    # P^dag P = 1: restricting the basis itself gives the identity in every block
    basis = gsub.vectors().to(tdt)
    gram = host(hd.restrict(gsub, basis)).astype(np.complex128)       # (k, a, j)
    assert np.abs(gram - np.eye(6)[:, None, :]).max() < (1e-13 if dtype == "c128" else 1e-5)


COARSE_CASES = [
    ((4, 4, 4, 4), 8, (2, 2, 2, 2), 8, 0.3, 0.01, 1),       # 2^4 coarse: +mu and -mu legs alias
    ((6, 6, 4, 4), 4, (2, 2, 2, 2), 4, 0.5, 0.05, -1),      # extents 3 and 2 mixed
]


@pytest.mark.parametrize("L,Ls,block,nvec,eps,mf,bc", COARSE_CASES)
def test_coarse_op_matches_oracle(hd, L, Ls, block, nvec, eps, mf, bc):
    g, U, noise, sub = _oracle_sub(L, Ls, block, nvec, eps, mf, 3200, iters=4, bc=bc)
    lat = hd.Lattice(L, Ls, bc)
    gsub = _gpu_sub_from_oracle(hd, lat, g, sub)
    A = mg.coarse_op(U, sub, M5, mf, bc)
    co = hd.build_coarse_op(gsub, dev(links(U)), M5, mf)
    assert relerr(host(co.op()), A) < 1e-12
    # the 9-point application
    rng = synth.rng(3201)
    c = rng.standard_normal((g.Vc, nvec)) + 1j * rng.standard_normal((g.Vc, nvec))
    y = host(hd.apply_coarse(co, dev(c)))
    assert relerr(y, mg.coarse_apply(A, g, c)) < 1e-13
    # FP32 build from the same basis
    gsub32 = _gpu_sub_from_oracle(hd, lat, g, sub, torch.complex64)
    co32 = hd.build_coarse_op(gsub32, dev(links(U)), M5, mf, op_dtype=torch.complex64)
    assert relerr(host(co32.op()), A) < 1e-5
    y32 = host(hd.apply_coarse(co32, dev(c, torch.complex64))).astype(np.complex128)
    assert relerr(y32, mg.coarse_apply(A, g, c)) < 1e-5


def test_coarse_op_properties_full_size(hd):
    """16^4 x 16, 4^4 blocks, nvec = 24 (the two-level FP64 workload): properties
    that hold at any size -- Galerkin identity A c = P^dag H P c, Hermitian legs,
    orthonormal blocks."""
    L, Ls, block, nvec = (16, 16, 16, 16), 16, (4, 4, 4, 4), 24
    lat = hd.Lattice(L, Ls)
    U = dev(links(synth.gauge_field(L, 0.5, 3300)))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 3301, count=nvec // 2)))
    sub = hd.build_subspace(lat, U, noise, M5, 0.01, block, kind="chebyshev", order=60,
                            filter_dtype=torch.complex64)
    del noise
    co = hd.build_coarse_op(sub, U, M5, 0.01)
    A = host(co.op())
    gc = mg.Geometry(L, Ls, block)
    idx = np.arange(gc.Vc)
    assert np.abs(A[:, 0] - np.conj(np.swapaxes(A[:, 0], -1, -2))).max() < 1e-12 * np.abs(A).max()
    for mu in range(4):
        nb = mg.coarse_neighbour(idx[:, None], gc, mu, +1)[:, 0]
        d = A[:, mg.leg_index(mu, 1)] - np.conj(np.swapaxes(A[nb, mg.leg_index(mu, -1)], -1, -2))
        assert np.abs(d).max() < 1e-12 * np.abs(A).max()
    rng = synth.rng(3302)
    c = rng.standard_normal((gc.Vc, nvec)) + 1j * rng.standard_normal((gc.Vc, nvec))
    cd = dev(c)
    lhs = host(hd.apply_coarse(co, cd))
    rhs = host(hd.restrict(sub, hd.apply_g5dwf(lat, U, hd.prolong(sub, cd), M5, 0.01)))
    assert relerr(lhs, rhs) < 1e-12
    gram = host(hd.restrict(sub, sub.vectors()))
    assert np.abs(gram - np.eye(nvec)[:, None, :]).max() < 1e-12


def test_subspace_errors(hd):
    L, Ls = (4, 4, 4, 4), 4
    lat = hd.Lattice(L, Ls)
    U = dev(links(synth.gauge_field(L, 0.3, 1)))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 2, count=2)))
    with pytest.raises(hd.HDCRError) as e:
        hd.build_subspace(lat, U, noise, M5, 0.01, (3, 2, 2, 2), kind="cr", order=2)
    assert e.value.status == -2
    with pytest.raises(hd.HDCRError) as e:
        hd.build_subspace(lat, U, noise, M5, 0.01, (4, 2, 2, 2), kind="cr", order=2)  # coarse extent 1
    assert e.value.status == -2
    v = synth.gaussian_fermion(L, Ls, 3, count=1)
    dup = planes(np.concatenate([v, v]))
    with pytest.raises(hd.HDCRError) as e:
        hd.subspace_from_vectors(lat, (2, 2, 2, 2), dev(dup))
    assert e.value.status == -5


@pytest.mark.parametrize("nvec,L,Ls,block", [(24, (4, 4, 4, 4), 4, (2, 2, 2, 2)),
                                             (66, (4, 4, 4, 4), 4, (2, 2, 2, 2)),
                                             (10, (6, 4, 4, 2), 5, (3, 2, 2, 1))])   # ragged block, odd Ls
def test_block_orthonormalisation_matches_oracle(hd, nvec, L, Ls, block):
    """subspace_from_vectors: the GPU's block orthonormalisation (two rounds of
    Cholesky QR per block; modified Gram-Schmidt for blocks whose Cholesky pivot
    collapses and for nvec > 64) against the oracle's modified Gram-Schmidt applied
    twice.  Random vectors, except that in block 0 vector 1 is vector 0 plus 1e-6
    noise (condition ~1e6: Gram-Schmidt) and in block 1 vector 3 is a combination of
    vectors 0..2 plus 1e-3 noise (condition ~1e3: Cholesky QR).  The QR factor with a
    positive real diagonal is unique, so the two agree to the rounding amplified by
    the condition number."""
    g = mg.Geometry(L, Ls, block)
    rng = synth.rng(3300 + nvec)
    shape = (nvec,) + synth.gaussian_fermion(L, Ls, 1).shape
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    bx, by, bz, bt = block
    b0 = (slice(0, bt), slice(0, bz), slice(0, by), slice(0, bx))            # (t, z, y, x) of block 0
    b1 = (slice(0, bt), slice(0, bz), slice(0, by), slice(bx, 2 * bx))       # block 1: the next in x
    noise = rng.standard_normal(v[0][b0].shape) + 1j * rng.standard_normal(v[0][b0].shape)
    v[1][b0] = v[0][b0] + 1e-6 * noise
    v[3][b1] = 0.5 * v[0][b1] - 0.3j * v[1][b1] + 0.7 * v[2][b1] + 1e-3 * noise
    lat = hd.Lattice(L, Ls)
    got = natural(host(hd.subspace_from_vectors(lat, block, dev(planes(v))).vectors()), L, Ls)
    want = mg.from_blocks(g, mg.basis_from_vectors(g, v).Phi)
    for k in range(nvec):
        assert relerr(got[k], want[k]) < 1e-9, k
    # every block orthonormal: <phi_j^a, phi_k^a> = delta_jk
    Gb = np.einsum("jak,lak->ajl", np.conj(mg.to_blocks(g, got)), mg.to_blocks(g, got))
    assert np.abs(Gb - np.eye(nvec)[None]).max() < 1e-12


@pytest.mark.parametrize("fdt", ["c128", "c64"])
def test_chebyshev_filter_subspace_matches_oracle(hd, fdt):
    L, Ls, block, nvec, mf = (4, 4, 4, 4), 8, (2, 2, 2, 2), 4, 0.01
    g = mg.Geometry(L, Ls, block)
    U = synth.gauge_field(L, 0.5, 3400)
    noise = synth.gaussian_fermion(L, Ls, 3401, count=nvec // 2)
    sm = np.stack([mg.chebyshev_filter(U, x0, M5, mf, 1, 0.5, 8.0, 20) for x0 in noise])
    want = mg.from_blocks(g, mg.basis_from_vectors(g, mg.chiral_split(sm)).Phi)
    tdt = torch.complex128 if fdt == "c128" else torch.complex64
    gsub = hd.build_subspace(hd.Lattice(L, Ls), dev(links(U)), dev(planes(noise)), M5, mf, block,
                             kind="chebyshev", order=20, lam_cut=0.5, lam_max=8.0, filter_dtype=tdt)
    got = natural(host(gsub.vectors()), L, Ls)
    tol = 1e-10 if fdt == "c128" else 1e-3
    for k in range(nvec):
        assert relerr(got[k], want[k]) < tol, k


@pytest.mark.parametrize("L,Ls,block,nvec,nrhs", [((6, 6, 4, 4), 4, (2, 2, 2, 2), 4, 2),
                                                   ((8, 8, 8, 8), 4, (2, 2, 2, 2), 8, 1),
                                                   ((8, 8, 8, 8), 4, (2, 2, 2, 2), 8, 3)])
def test_dense_coarse_inverse(hd, L, Ls, block, nvec, nrhs):
    """The FP32 dense inverse of A (Gauss-Jordan in panels of 128 columns, the rank-128
    updates on the tensor cores) applied to one vector (matrix-vector product) and to
    several (one tensor-core GEMM) against numpy's LU solve of the same A; 2048 unknowns
    take 16 panels."""
    mf = 0.05
    g, U, noise, sub = _oracle_sub(L, Ls, block, nvec, 0.5, mf, 3500, iters=4)
    lat = hd.Lattice(L, Ls)
    gsub = _gpu_sub_from_oracle(hd, lat, g, sub, torch.complex64)
    co = hd.build_coarse_op(gsub, dev(links(U)), M5, mf, op_dtype=torch.complex64)
    hd.coarse_invert(co)
    Ad = mg.coarse_dense(host(co.op()), g)
    rng = synth.rng(3501)
    c = rng.standard_normal((nrhs, g.Vc, nvec)) + 1j * rng.standard_normal((nrhs, g.Vc, nvec))
    y = host(hd.coarse_solve_dense(co, dev(c, torch.complex64))).astype(np.complex128).reshape(c.shape)
    cond = np.linalg.cond(Ad)
    for r in range(nrhs):
        want = np.linalg.solve(Ad, c[r].ravel()).reshape(c[r].shape)
        assert relerr(y[r], want) < max(1e-5, cond * 3e-7)


SOLVER_CASES = [
    # (inner dtype, smoother, coarse solver, mf)
    ("c128", "chebyshev", "dense", 0.01),
    ("c64", "chebyshev", "dense", 0.01),
    ("c128", "cr", "cr", 0.1),
]


@pytest.mark.parametrize("inner,smoother,coarse,mf", SOLVER_CASES)
def test_hdcr_solve_tiny_workload(hd, inner, smoother, coarse, mf):
    """4^4 x 8, eps = 0.3, 2^4 blocks, nvec = 8: HDCR to a true residual of 1e-10
    (checked by the oracle) and the same solution as the oracle's CR."""
    L, Ls, block, nvec = (4, 4, 4, 4), 8, (2, 2, 2, 2), 8
    lat = hd.Lattice(L, Ls)
    Uh = synth.gauge_field(L, 0.3, 1000)
    U = dev(links(Uh))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 3001, count=nvec // 2)))
    tdt = torch.complex128 if inner == "c128" else torch.complex64
    sub = hd.build_subspace(lat, U, noise, M5, mf, block, kind="chebyshev", order=100, lam_cut=0.3,
                            store_dtype=tdt)
    co = hd.build_coarse_op(sub, U, M5, mf, op_dtype=tdt)
    b = synth.gaussian_fermion(L, Ls, 2000)
    x, st = hd.hdcr_solve(co, U, dev(planes(b)), tol=1e-10, inner_dtype=tdt, smoother=smoother,
                          smoother_order=10 if smoother == "chebyshev" else 8, coarse_solver=coarse,
                          max_outer=2000, restart=16)
    assert st["status"] == 0 and st["true_resid"] <= 1e-10
    xg = natural(host(x), L, Ls)
    r = b - dwf.apply_H(Uh, xg, M5, mf)
    assert np.sqrt(dwf.norm2(r) / dwf.norm2(b)) <= 1.01e-10
    xo, _ = cr(lambda v: dwf.apply_H(Uh, v, M5, mf), b, tol=1e-12, maxiter=50000)
    assert relerr(xg, xo) < 1e-6
    assert st["coarse_matvecs"] > 0 and st["iters"] > 0


@pytest.mark.parametrize("cycle,coarse", [("symmetric", "dense"), ("post", "dense"), ("symmetric", "cr")])
def test_hdcr_vcycle_matches_oracle_first_iterate(hd, cycle, coarse):
    """With the linear Chebyshev smoother the preconditioner is a fixed linear map (up to
    the FP32 dense coarse inverse), so the first FGCR iterate x1 = a B b, with a the
    least-squares step, agrees with the oracle's V-cycle to the coarse inverse's accuracy
    (both cycles: smoother before and after the coarse correction, or after only).
    With the FP64 coarse CR run to 1e-13 in place of the FP32 inverse the agreement is
    to FP64 rounding, which pins the FP64 smoother (its recurrence steps fused into
    the operator's epilogue) tightly."""
    L, Ls, block, nvec, mf = (4, 4, 4, 4), 8, (2, 2, 2, 2), 8, 0.05
    g, U, noise, sub = _oracle_sub(L, Ls, block, nvec, 0.3, mf, 3600, iters=6)
    lat = hd.Lattice(L, Ls)
    gsub = _gpu_sub_from_oracle(hd, lat, g, sub)
    co = hd.build_coarse_op(gsub, dev(links(U)), M5, mf)
    b = synth.gaussian_fermion(L, Ls, 3601)
    with pytest.raises(hd.HDCRError):
        x1, _ = hd.hdcr_solve(co, dev(links(U)), dev(planes(b)), tol=1e-14, max_outer=1, restart=1)
    xd = dev(np.zeros_like(planes(b)))
    A = mg.coarse_op(U, sub, M5, mf)
    Ad = mg.coarse_dense(A, g)
    p = mg.HDCRParams(M5=M5, mf=mf)
    S = lambda v: mg.chebyshev_smoother(U, v, p)
    Qc = lambda c: np.linalg.solve(Ad, c.ravel()).reshape(c.shape)
    z = mg.vcycle(U, sub, A, b, p, S=S, Qc=Qc, cycle=cycle)
    w = dwf.apply_H(U, z, M5, mf)
    x1 = (np.vdot(w, b) / np.vdot(w, w)) * z
    # the GPU solve with max_outer = 1 leaves its first iterate in x via hdcr_solve_into
    kw = dict(coarse_solver="cr", coarse_tol=1e-13, coarse_max=20000) if coarse == "cr" else {}
    st = hd.hdcr_solve_into(co, dev(links(U)), dev(planes(b)), xd, tol=1e-14, max_outer=1, restart=1,
                            cycle=cycle, **kw)
    assert st["status"] == -3
    assert relerr(natural(host(xd), L, Ls), x1) < (1e-9 if coarse == "cr" else 1e-4)


def test_hdcr_solve_reports_cap(hd):
    L, Ls, block, nvec, mf = (4, 4, 4, 4), 4, (2, 2, 2, 2), 4, 0.01
    lat = hd.Lattice(L, Ls)
    U = dev(links(synth.gauge_field(L, 0.3, 1000)))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, 3001, count=2)))
    sub = hd.build_subspace(lat, U, noise, M5, mf, block, kind="cr", order=10)
    co = hd.build_coarse_op(sub, U, M5, mf)
    b = dev(planes(synth.gaussian_fermion(L, Ls, 2000)))
    with pytest.raises(hd.HDCRError) as e:
        hd.hdcr_solve(co, U, b, tol=1e-12, max_outer=2)
    assert e.value.status == -3


@pytest.mark.parametrize("L,Ls,block,nvec,lam_cut,seeds", [
    ((4, 4, 4, 4), 8, (2, 2, 2, 2), 24, 0.5, (1000, 2000, 3000)),   # the tiny 4^4 x 8 workload, eps = 0.3
    ((8, 8, 8, 8), 8, (4, 4, 4, 4), 24, 0.5, (1100, 2100, 3100)),   # a mid-size lattice, eps = 0.5
])
def test_hdcr_needs_fewer_fine_matvecs_than_cr(hd, L, Ls, block, nvec, lam_cut, seeds):
    """The point of the preconditioner (Section 4): the two-level solve to a true
    residual of 1e-10 applies H fewer times than plain CR to the same tolerance, counting
    every application (the order-10 Chebyshev smoother's, the V-cycle's residuals and
    the outer iteration's).  With fewer basis vectors (8 or 16 on these lattices) the
    coarse space misses low modes and the count exceeds CR's."""
    eps = 0.3 if L == (4, 4, 4, 4) else 0.5
    lat = hd.Lattice(L, Ls)
    U = dev(links(synth.gauge_field(L, eps, seeds[0])))
    b = dev(planes(synth.gaussian_fermion(L, Ls, seeds[1])))
    noise = dev(planes(synth.gaussian_fermion(L, Ls, seeds[2], count=nvec // 2)))
    _, st_cr = hd.cr_solve(lat, U, b, M5, 0.01, tol=1e-10, max_iter=100000)
    sub = hd.build_subspace(lat, U, noise, M5, 0.01, block, kind="chebyshev", order=200, lam_cut=lam_cut)
    co = hd.build_coarse_op(sub, U, M5, 0.01)
    x, st = hd.hdcr_solve(co, U, b, tol=1e-10, max_outer=40, restart=16)
    mv = st["fine_matvecs"] + st["fine_matvecs_lo"]
    print(f"{L} x {Ls}: HDCR {st['iters']} outer iterations, {mv} applications of H; plain CR {st_cr['fine_matvecs']}")
    assert st["status"] == 0 and st["true_resid"] <= 1e-10
    assert mv < st_cr["fine_matvecs"]
