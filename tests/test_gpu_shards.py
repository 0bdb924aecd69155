"""The g-sharded build (xk_setup_shard), through the C ABI, on one GPU.

Every term of Eq. exoccri is a sum over the interpolation points g, so a
partition of [0, N_aux) into slices gives shard builds whose K_{mu i} and
E_x sum to the full build's (Sec. IV.B-D; the multi-GPU run reduces them
with one allreduce).  Here the shards of 2, 3 and 4 uneven slices run one
after another on one GPU and their host sum is compared with the unsharded
oracle at each path's bar: FP64 1e-8 Ha / 1e-7, tensor path 1e-6 Ha / 1e-6.
"""
import numpy as np
import pytest

import oracle
from cellgen import config_spec, load_cell

pytestmark = pytest.mark.gpu

BARS = {"fp64": (1e-8, 1e-7), "f16x3": (1e-6, 1e-6)}


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


def _slices(na, p):
    # uneven slices (the first ones shorter), none on a tile boundary
    w = np.arange(1, p + 1, dtype=float)
    b = np.concatenate([[0], np.round(np.cumsum(w) / w.sum() * na)]).astype(int)
    b[-1] = na
    return list(zip(b[:-1], b[1:]))


def _sharded(xk, c, mode, p):
    Ks, Es, Ee = np.zeros((c.N, c.n)), 0.0, 0.0
    for g0, g1 in _slices(c.idx.size, p):
        h = xk.Handle.shard(c.phi, c.idx, c.V[g0:g1], c.W[g0:g1], g0, g1, c.dV, c.n, mode=mode)
        try:
            K, E = h.build(c.C)
            Ee += h.energy(c.C)
        finally:
            h.release()
        Ks += K
        Es += E
    return Ks, Es, Ee


@pytest.mark.parametrize("mode", ["fp64", "f16x3"])
def test_shards_8centre(xk, cell1, mode):
    c = cell1
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    tol_e, tol_k = BARS[mode]
    for p in (2, 3, 4):
        K, E, Ee = _sharded(xk, c, mode, p)
        assert abs(E - E0) <= tol_e, (mode, p, E - E0)
        assert np.max(np.abs(K - K0)) <= tol_k, (mode, p, np.max(np.abs(K - K0)))
        assert abs(Ee - E0) <= tol_e, (mode, p, Ee - E0)  # the shares of xk_energy


@pytest.mark.parametrize("n_occ,mode", [(100, "f16x3"), (150, "f16x3"), (54, "fp64")])
def test_shards_27centre(xk, n_occ, mode):
    """27-centre cell: n = 100 (the fused pair role), n = 150 (the stored-T
    path), and the FP64 path with n = 54."""
    spec = config_spec(4, k=3)
    spec.n_occ = n_occ
    c = load_cell(spec)
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    tol_e, tol_k = BARS[mode]
    for p in (2, 3):
        K, E, _ = _sharded(xk, c, mode, p)
        assert abs(E - E0) <= tol_e, (n_occ, p, E - E0)
        assert np.max(np.abs(K - K0)) <= tol_k, (n_occ, p, np.max(np.abs(K - K0)))


def test_shard_rejects_full_k_and_ace(xk, cell1):
    """A shard's K is a partial sum: the full K and the ACE factorisation of
    one shard are refused (they belong to the summed K)."""
    c = cell1
    h = xk.Handle.shard(c.phi, c.idx, c.V[:100], c.W[:100], 0, 100, c.dV, c.n, mode="fp64")
    try:
        h.build(c.C)
        for call in (lambda: h.build_full(c.C), lambda: h.ace()):
            with pytest.raises(xk.XKError) as e:
                call()
            assert e.value.code == xk.XK_EINVAL
    finally:
        h.release()
