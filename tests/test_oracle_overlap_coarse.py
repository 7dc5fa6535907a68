"""Pins of the oracle's two-level pieces for the continued-fraction operator
(oracle/overlap.py: apply_cf_hop, cf_coarse_op)."""
import numpy as np
import pytest

import synth
from oracle import dwf, multigrid as mg, overlap as ov
from pins import relerr

M5, R = 1.8, 0.3
BETA = [1.3, 0.8, 1.1, 0.6]          # five components


def _field(L, N, seed, count=None):
    return synth.gaussian_fermion(L, N, seed, count=count)


def test_hops_and_local_part_sum_to_the_operator():
    """H_cf = (site-local part) + sum of the eight hop parts; the site-local part is
    what remains on a field supported on one site: it has no neighbours' values."""
    L, N = (4, 4, 2, 4), 5
    U = synth.gauge_field(L, 0.5, 700)
    psi = _field(L, N, 701)
    hops = sum(ov.apply_cf_hop(U, psi, mu, s, BETA) for mu in range(4) for s in (+1, -1))
    local = ov.apply_cf(U, psi, M5, BETA, R) - hops
    # the local part of a field confined to one site stays on that site
    one = np.zeros_like(psi)
    one[1, 0, 2, 3] = psi[1, 0, 2, 3]
    loc1 = ov.apply_cf(U, one, M5, BETA, R) - sum(ov.apply_cf_hop(U, one, mu, s, BETA)
                                                 for mu in range(4) for s in (+1, -1))
    mask = np.zeros(psi.shape[:4], bool)
    mask[1, 0, 2, 3] = True
    assert np.abs(loc1[~mask]).max() < 1e-14
    # and it is linear and site by site the same map (checked on the full field)
    assert relerr(local[1, 0, 2, 3], loc1[1, 0, 2, 3]) < 1e-13
    # with beta -> the hop of component 0 is gamma5 (-1/2) hop of the Wilson kernel
    h = ov.apply_cf_hop(U, psi, 2, -1, BETA)
    want = dwf.spin_mul(dwf.GAMMA5, -0.5 * dwf.hop(U, psi, 2, -1, 1))
    assert relerr(h[..., 0, :, :], want[..., 0, :, :]) < 1e-15
    assert relerr(h[..., 1, :, :], -want[..., 1, :, :]) < 1e-15
    assert relerr(h[..., 4, :, :], BETA[0] * want[..., 4, :, :]) < 1e-15


@pytest.fixture(scope="module")
def small():
    L, N, block, nvec = (6, 6, 6, 6), 3, (2, 2, 2, 2), 4      # 3^4 coarse lattice
    beta = [1.2, 0.7]
    g = mg.Geometry(L, N, block)
    U = synth.gauge_field(L, 0.5, 710)
    v = _field(L, N, 711, count=nvec)
    sub = mg.basis_from_vectors(g, v)
    A = ov.cf_coarse_op(U, sub, M5, beta, R)
    return g, U, sub, A, beta


def test_cf_coarse_op_galerkin(small):
    """A c = P^dag H_cf P c for random coarse vectors: the legs and the neighbour map
    of the 9-point stencil reproduce the operator on the block subspace."""
    g, U, sub, A, beta = small
    rng = synth.rng(712)
    for _ in range(2):
        c = rng.standard_normal((g.Vc, sub.nvec)) + 1j * rng.standard_normal((g.Vc, sub.nvec))
        want = mg.restrict(sub, ov.apply_cf(U, mg.prolong(sub, c), M5, beta, R))
        assert relerr(mg.coarse_apply(A, g, c), want) < 1e-13


def test_cf_coarse_op_is_hermitian_and_nine_point(small):
    """H_cf Hermitian: A^{a,a+mu} = (A^{a+mu,a}_(-mu))^dag and A^{aa} Hermitian; a block
    column beyond the 8 neighbours is zero (brute force: P^dag H_cf applied to one block's
    basis vector)."""
    g, U, sub, A, beta = small
    for a in range(g.Vc):
        assert np.abs(A[a, 0] - A[a, 0].conj().T).max() < 1e-13
    for mu in range(4):
        Ap = A[:, mg.leg_index(mu, +1)]
        Am = A[:, mg.leg_index(mu, -1)]
        Am_shift = mg.coarse_neighbour(Am.reshape(g.Vc, -1), g, mu, +1).reshape(Am.shape)
        assert np.abs(Ap - np.conj(np.transpose(Am_shift, (0, 2, 1)))).max() < 1e-13
    # one basis vector of block 0: its image under P^dag H_cf lives on block 0 and its 8 neighbours
    e = np.zeros((g.Vc, sub.nvec), dtype=complex)
    e[0, 1] = 1.0
    img = mg.restrict(sub, ov.apply_cf(U, mg.prolong(sub, e), M5, beta, R))
    nb = {0}
    for mu in range(4):
        for s in (+1, -1):
            idx = np.arange(g.Vc).reshape(g.coarse_shape())
            nb.add(int(np.roll(idx, -s, axis=3 - mu).reshape(-1)[0]))
    far = [a for a in range(g.Vc) if a not in nb]
    assert len(far) == g.Vc - 9 and np.abs(img[far]).max() < 1e-14
    assert np.abs(img[list(nb)]).max() > 1e-3
