"""Failure detection inside the tensor-core kernels (XK_F16X3), on the GPU.

Every wait of a kernel's pipeline (a TMA stage, an MMA result, an epilogue
hand-off) is bounded; when a bound runs out the kernel records a code, stops,
waits for its own copies and MMAs, frees its tensor memory and returns, and
the call reports XK_ETIMEDOUT.  These tests shorten the bound of one handle
to a single cycle (xk_set_wait_limit), so that the first wait that is not
already satisfied gives up, and check the status on each route that reports
it (blocking build, energy, serving ticket), and that the same handle then
builds correctly again at the default bound.  Nothing here faults or hangs
the GPU: the kernels return by themselves within the default bound.
"""
import numpy as np
import pytest

from cellgen import config_spec, load_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


def _timeout_then_recover(xk, c):
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        K0, E0 = h.build(c.C)
        h.set_wait_limit(1)
        with pytest.raises(xk.XKError) as e:
            h.build(c.C)
        assert e.value.code == xk.XK_ETIMEDOUT
        with pytest.raises(xk.XKError) as e:
            h.energy(c.C)
        assert e.value.code == xk.XK_ETIMEDOUT
        # serving: the ticket of the build that gave up reports it
        t = h.submit(c.C)
        while True:
            try:
                st, _, _, _ = xk.poll(t, c.N, c.n)
            except xk.XKError as err:
                assert err.code == xk.XK_ETIMEDOUT
                break
            assert st == xk.XK_PENDING
        h.set_wait_limit(0)
        K1, E1 = h.build(c.C)
        t = h.submit(c.C)
        while True:
            st, K2, E2, _ = xk.poll(t, c.N, c.n)
            if st == xk.XK_OK:
                break
    finally:
        h.release()
    assert E1 == E0 and E2 == E0
    assert np.max(np.abs(K1 - K0)) <= 1e-7 and np.max(np.abs(K2 - K0)) <= 1e-7


def test_timeout_pair_and_gemm_kernels(xk, cell1):
    """8-centre cell (n = 16): orbital and line GEMMs and the three-role pair kernel."""
    _timeout_then_recover(xk, cell1)


def test_timeout_fused_role(xk):
    """27-centre cell with n = 100: the fused pair role (S once, M1 and M2)."""
    spec = config_spec(4, k=3)
    spec.n_occ = 100
    _timeout_then_recover(xk, load_cell(spec))


def test_negative_limit_rejected(xk, cell1):
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        with pytest.raises(xk.XKError) as e:
            h.set_wait_limit(-1)
        assert e.value.code == xk.XK_EINVAL
    finally:
        h.release()
