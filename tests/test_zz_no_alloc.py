"""The allocation-free exchange-energy entry point (xk_exchange_energy_noalloc).

Some callers cannot allocate device memory when they call the library -- for
example code inside a CUDA graph capture, or a host whose own pool owns the
device heap.  For them the library offers an E_x reduction whose scratch is a
fixed device array compiled into the library.  This test checks, through the
C ABI and on two calls in a row, that it returns the same E_x as the
ordinary build (which allocates its scratch with the handle), and that it
refuses counts beyond its fixed capacity.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_build(cell1):
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as xk

    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="fp64")
    K, E = h.build(c.C)
    h.release()
    Kd = torch.from_numpy(K).cuda()
    Cd = torch.from_numpy(np.ascontiguousarray(c.C)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        Ed = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        xk.exchange_energy_noalloc(Kd.data_ptr(), Cd.data_ptr(), K.size, Ed.data_ptr(),
                                   stream.cuda_stream)
        stream.synchronize()
        assert abs(float(Ed.item()) - E) <= 1e-12 * abs(E)

    # counts that exercise the reduction: none (E_x = -0), one chunk, several
    # chunks with a ragged last one, the 64-centre cell's N n, and the fixed
    # maximum; each checked against an exactly rounded host sum, twice in a row
    import math
    rng = np.random.default_rng(11)
    for count in (0, 1, 3 * 2048 + 17, 832 * 128, 2048 * 2048):
        a = rng.standard_normal(max(count, 1))
        b = rng.standard_normal(max(count, 1))
        ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        want = -math.fsum((a[:count] * b[:count]).tolist()) if count else 0.0
        scale = math.fsum(np.abs(a[:count] * b[:count]).tolist()) if count else 0.0
        for _ in range(2):
            Ed = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            xk.exchange_energy_noalloc(ad.data_ptr(), bd.data_ptr(), count, Ed.data_ptr(),
                                       stream.cuda_stream)
            stream.synchronize()
            got = float(Ed.item())
            assert abs(got - want) <= 1e-13 * scale, (count, got, want)

    # a count above the fixed capacity is refused before any device work
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(xk.XKError) as err:
        xk.exchange_energy_noalloc(Kd.data_ptr(), Cd.data_ptr(), 2048 * 2048 + 1, Ed.data_ptr(),
                                   stream.cuda_stream)
    assert err.value.code == xk.XK_EINVAL
