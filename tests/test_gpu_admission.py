"""Queued admission on the device: with a budget that holds one handle of the
8-centre cell, a second xk_setup_queued waits in the queue while the first is
live, is admitted when xk_release frees it, and then builds the same K and
E_x bit for bit."""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


@pytest.mark.parametrize("mode", ["fp64", "f16x3"])
def test_queued_handle_admitted_on_release(xk, cell1, monkeypatch, mode):
    c = cell1
    need = xk.footprint(c.Ng, c.N, c.n, c.Naux, mode)
    base, waiting = xk.admit_state()
    assert waiting == 0
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", str(base + int(1.5 * need)))
    h1 = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode=mode)
    K1, E1 = h1.build(c.C)
    got = {}

    def second():
        try:
            got["h"] = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode=mode,
                                 queue_timeout_ms=30000.0)
            got["t"] = time.perf_counter()
        except xk.XKError as e:
            got["err"] = e

    t = threading.Thread(target=second)
    t.start()
    time.sleep(0.3)
    assert t.is_alive() and xk.admit_state()[1] == 1  # waiting behind the live handle
    t_rel = time.perf_counter()
    h1.release()
    t.join(60.0)
    assert "err" not in got, got.get("err")
    assert got["t"] >= t_rel
    h2 = got["h"]
    try:
        K2, E2 = h2.build(c.C)
    finally:
        h2.release()
    assert np.array_equal(K1, K2) and E1 == E2
    assert xk.admit_state() == (base, 0)
