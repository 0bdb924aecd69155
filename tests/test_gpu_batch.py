"""Batches and serving on the tensor-core path (XK_F16X3), through the C ABI.

A batch runs one build of every member (cells of different sizes) as one
CUDA graph with one grouped pair launch.  E_x is summed in a fixed order, so
it equals the member's own xk_build bit for bit; K does too, except for
members with 65 <= n <= 128, whose fused pair role adds M2 tiles into FP32
copies in the order the CTAs finish (K then agrees to rounding, 1e-7).
The same holds for builds of different cells submitted together
(xk_submit / xk_poll): each result is the same alone and in the mix.
"""
import numpy as np
import pytest

from cellgen import CellSpec, Shell, build_cell, config_spec, load_cell

pytestmark = pytest.mark.gpu


TOL_REPEAT_K = 1e-7


def same_build(K, E, Kr, Er, n):
    if 64 < n <= 128:
        return E == Er and np.max(np.abs(K - Kr)) <= TOL_REPEAT_K
    return np.array_equal(K, Kr) and E == Er


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


@pytest.fixture(scope="module")
def cells(cell1):
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    ragged = build_cell(CellSpec("ragged", np.array([[0.1, 0.2, 0.3], [0.6, 0.5, 0.45],
                                                      [0.3, 0.75, 0.8]]), 6.5, 13, sh, 7, 97,
                                 9001))
    out = [cell1, ragged, load_cell(config_spec(4, k=3))]
    for n_occ in (128, 150):  # piece width 128, and the n > 128 path
        spec = config_spec(4, k=3)
        spec.n_occ = n_occ
        out.append(load_cell(spec))
    return out


def test_batch_equals_single_builds(xk, cells):
    hs = [xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3") for c in cells]
    rng = np.random.default_rng(5)
    C2 = [c.C + 0.01 * rng.standard_normal(c.C.shape) for c in cells]
    try:
        ref = [h.build(c.C) for h, c in zip(hs, cells)]
        ref2 = [h.build(C) for h, C in zip(hs, C2)]
        b = xk.Batch(hs)
        try:
            before = xk.kernel_launches()
            for Cs, want in ((C2, ref2), ([c.C for c in cells], ref), (C2, ref2)):
                Ks, Es = b.build(Cs)
                for K, E, (Kr, Er), c in zip(Ks, Es, want, cells):
                    assert same_build(K, E, Kr, Er, c.n), c.spec.name
            assert xk.kernel_launches() > before
        finally:
            b.release()
    finally:
        for h in hs:
            h.release()


def test_batch_rejects_bad_members(xk, cell1):
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    hf = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="fp64")
    try:
        for members in ([h, h], [h, hf]):
            with pytest.raises(xk.XKError) as e:
                xk.Batch(members)
            assert e.value.code == xk.XK_EINVAL
    finally:
        h.release()
        hf.release()


def test_submit_poll_alone_and_mixed(xk, cells):
    """Serving: builds of three cells of different sizes submitted together
    (overlapping on the GPU) give the same results as each built alone."""
    use = [cells[0], cells[2], cells[3], cells[4]]
    hs = [xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3") for c in use]
    try:
        ref = [h.build(c.C) for h, c in zip(hs, use)]
        tickets = []
        for rep in range(2):
            for h, c, r in zip(hs, use, ref):
                tickets.append((h.submit(c.C), c, r))
        for t, c, (Kr, Er) in tickets:
            while True:
                st, K, E, eb = xk.poll(t, c.N, c.n)
                if st == xk.XK_OK:
                    break
            assert same_build(K, E, Kr, Er, c.n)
            # the ticket's error estimate |E_x - E_K| (E_K = -sum K o C): the
            # host's value, and within what the K tolerance (1e-6 per element)
            # allows over the sum of |C|
            assert abs(eb - abs(E + float(np.sum(K * c.C)))) <= 1e-10
            assert eb <= 1e-6 * float(np.sum(np.abs(c.C))) + 1e-6
    finally:
        for h in hs:
            h.release()
