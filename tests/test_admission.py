"""The admission queue of the C++ runtime (xk_setup_queued, xk_admit_*), on
the host: requests wait in arrival order until their bytes fit the budget
(XK_HBM_BUDGET_BYTES less what is admitted), a release admits the waiters,
and a wait that runs out leaves the queue with XK_ETIMEDOUT.  Nothing here
touches a device: with the budget variable set, a request that does not fit
is decided before any device call."""
import ctypes
import threading
import time

import numpy as np
import pytest

import paper_2207_04636_gb300 as xk
from paper_2207_04636_gb300 import build as xkbuild


@pytest.fixture(scope="module")
def L():
    xkbuild.build_library()
    return xk.lib()


def _code(fn):
    try:
        fn()
    except xk.XKError as e:
        return e.code
    return xk.XK_OK


def test_reserve_now_or_refuse(L, monkeypatch):
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", "1000")
    base, waiting = xk.admit_state()
    assert waiting == 0
    a = xk.admit_reserve(600)
    assert xk.admit_state() == (base + 600, 0)
    assert _code(lambda: xk.admit_reserve(600)) == xk.XK_ENOMEM           # now: no room
    t0 = time.perf_counter()
    assert _code(lambda: xk.admit_reserve(600, 30.0)) == xk.XK_ETIMEDOUT  # queued: runs out
    assert time.perf_counter() - t0 >= 0.025
    assert "not admitted" in xk.last_error()
    assert _code(lambda: xk.admit_reserve(1001, 1000.0)) == xk.XK_ENOMEM  # above the cap itself
    assert xk.admit_state() == (base + 600, 0)  # the timed-out request left the queue
    xk.admit_release(a)
    assert xk.admit_state() == (base, 0)
    assert _code(lambda: xk.admit_release(a)) == xk.XK_EINVAL             # unknown token
    tok = ctypes.c_uint64()
    assert L.xk_admit_reserve(10, float("nan"), ctypes.byref(tok)) == xk.XK_EINVAL
    assert L.xk_admit_reserve(10, 0.0, None) == xk.XK_EINVAL
    assert L.xk_admit_state(None, None) == xk.XK_EINVAL


def test_queue_admits_in_arrival_order_on_release(L, monkeypatch):
    """A holds 600 of 1000.  Request 1 (500) cannot fit; request 2 (300) would
    fit but arrived later, so it waits behind 1.  Releasing A admits 1, then 2."""
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", "1000")
    base, _ = xk.admit_state()
    a = xk.admit_reserve(600)
    done = {}

    def req(name, nbytes):
        tok = xk.admit_reserve(nbytes, 10000.0)
        done[name] = (time.perf_counter(), tok)

    t1 = threading.Thread(target=req, args=("first", 500))
    t1.start()
    time.sleep(0.1)
    t2 = threading.Thread(target=req, args=("second", 300))
    t2.start()
    time.sleep(0.2)
    assert not done and xk.admit_state() == (base + 600, 2)
    t_rel = time.perf_counter()
    xk.admit_release(a)
    t1.join(10.0)
    t2.join(10.0)
    assert set(done) == {"first", "second"}
    assert t_rel <= done["first"][0] <= done["second"][0]
    assert xk.admit_state() == (base + 800, 0)
    for _, tok in done.values():
        xk.admit_release(tok)
    assert xk.admit_state() == (base, 0)


def _tables(Ng=64, N=6, n=3, Naux=10, seed=0):
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((Ng, N))
    idx = np.sort(rng.choice(Ng, Naux, replace=False)).astype(np.int32)
    V = rng.standard_normal((Naux, Ng))
    W = rng.standard_normal((Naux, Naux))
    return phi, idx, V, W + W.T


def test_setup_queued_waits_then_times_out(L, monkeypatch):
    """xk_setup_queued: a footprint above the whole budget fails at once; one
    that fits the budget but not beside a reservation waits and times out;
    both before any device call."""
    phi, idx, V, W = _tables()
    need = xk.footprint(64, 6, 3, 10, "f16x3")
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    setup = lambda t: L.xk_setup_queued(64, 6, 3, 10, p(phi), p(idx), p(V), p(W), 0.1, 2, t,  # noqa: E731
                                        ctypes.byref(h))
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", str(need - 1))
    assert setup(1000.0) == xk.XK_ENOMEM
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", str(need + 100))
    a = xk.admit_reserve(200)
    t0 = time.perf_counter()
    assert setup(40.0) == xk.XK_ETIMEDOUT
    assert time.perf_counter() - t0 >= 0.035
    assert not h.value
    assert setup(-1.0) == xk.XK_EINVAL
    assert setup(float("inf")) == xk.XK_EINVAL
    xk.admit_release(a)
    assert xk.admit_state()[1] == 0


def test_head_timeout_admits_the_next(L, monkeypatch):
    """The oldest request (700 of 1000, 600 held) times out and leaves the
    queue; the request behind it (300, which fits beside the 600) is then
    admitted without any release."""
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", "1000")
    base, _ = xk.admit_state()
    a = xk.admit_reserve(600)
    got = {}

    def head():
        got["head"] = _code(lambda: xk.admit_reserve(700, 150.0))

    def second():
        try:
            got["second"] = xk.admit_reserve(300, 5000.0)
            got["t"] = time.perf_counter()
        except xk.XKError as e:
            got["second_err"] = e.code

    t1 = threading.Thread(target=head)
    t1.start()
    time.sleep(0.05)
    t0 = time.perf_counter()
    t2 = threading.Thread(target=second)
    t2.start()
    t1.join(5.0)
    t2.join(5.0)
    assert got["head"] == xk.XK_ETIMEDOUT
    assert "second" in got, got
    assert got["t"] - t0 < 2.0
    xk.admit_release(got["second"])
    xk.admit_release(a)
    assert xk.admit_state() == (base, 0)


def test_concurrent_reserve_release(L, monkeypatch):
    """Sixteen threads reserve and release random amounts against a small
    budget, some waiting and some timing out: no deadlock, no lost bytes."""
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", "1000")
    base, _ = xk.admit_state()
    errors = []

    def worker(seed):
        rng = np.random.default_rng(seed)
        for _ in range(40):
            nbytes = int(rng.integers(1, 400))
            try:
                tok = xk.admit_reserve(nbytes, float(rng.choice([-1.0, 5.0, 200.0])))
            except xk.XKError as e:
                if e.code not in (xk.XK_ENOMEM, xk.XK_ETIMEDOUT):
                    errors.append(e.code)
                continue
            time.sleep(float(rng.uniform(0, 0.002)))
            xk.admit_release(tok)

    ths = [threading.Thread(target=worker, args=(s,)) for s in range(16)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(60.0)
    assert not any(t.is_alive() for t in ths)
    assert not errors
    assert xk.admit_state() == (base, 0)
