"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/xk.h declares, sizes its footprint, and rejects
invalid inputs with XK_EINVAL before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2207_04636_gb300 as xk
from paper_2207_04636_gb300 import build as xkbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    xkbuild.build_library()
    return xk.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "xk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xk_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert {"xk_setup", "xk_build", "xk_submit", "xk_poll", "xk_release", "xk_footprint",
            "xk_last_error", "xk_build_device", "xk_ace", "xk_energy", "xk_build_full", "xk_coulomb", "xk_setup_isdf", "xk_tables", "xk_isdf_points"} <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_footprint(L):
    f2 = xk.footprint(216000, 832, 128, 4000, "fp64")
    # the paper's extra memory cost: the stored potentials V are N_aux x N_g doubles
    assert f2 > 4000 * 216000 * 8
    assert xk.footprint(2 * 216000, 832, 128, 4000, "fp64") > f2
    out = ctypes.c_size_t()
    assert L.xk_footprint(0, 832, 128, 4000, 0, ctypes.byref(out)) == xk.XK_EINVAL
    assert L.xk_footprint(100, 8, 9, 4, 0, ctypes.byref(out)) == xk.XK_EINVAL   # n > N
    assert L.xk_footprint(100, 8, 4, 101, 0, ctypes.byref(out)) == xk.XK_EINVAL  # Naux > Ng
    assert L.xk_footprint(100, 8, 4, 10, 7, ctypes.byref(out)) == xk.XK_EINVAL   # mode


def _tables(Ng=64, N=6, n=3, Naux=10, seed=0):
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((Ng, N))
    idx = np.sort(rng.choice(Ng, Naux, replace=False)).astype(np.int32)
    V = rng.standard_normal((Naux, Ng))
    W = rng.standard_normal((Naux, Naux))
    return phi, idx, V, W + W.T


def _setup(L, phi, idx, V, W, dV=0.1, n=3, mode=0):
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    return L.xk_setup(phi.shape[0], phi.shape[1], n, idx.shape[0], p(phi), p(idx), p(V), p(W),
                      dV, mode, ctypes.byref(h))


def test_setup_rejects_invalid_inputs(L):
    phi, idx, V, W = _tables()
    bad = idx.copy()
    bad[3] = bad[2]
    assert _setup(L, phi, bad, V, W) == xk.XK_EINVAL
    assert "duplicate" in xk.last_error()
    bad = idx.copy()
    bad[-1] = phi.shape[0]
    assert _setup(L, phi, bad, V, W) == xk.XK_EINVAL
    bad = idx.copy()
    bad[0] = -1
    assert _setup(L, phi, bad, V, W) == xk.XK_EINVAL
    Wa = W.copy()
    Wa[0, 1] += 1e-6
    assert _setup(L, phi, idx, V, Wa) == xk.XK_EINVAL
    assert "symmetric" in xk.last_error()
    assert _setup(L, phi, idx, V, W, dV=0.0) == xk.XK_EINVAL
    assert _setup(L, phi, idx, V, W, dV=float("nan")) == xk.XK_EINVAL
    assert _setup(L, phi, idx, V, W, n=7) == xk.XK_EINVAL
    assert _setup(L, phi, idx, V, W, mode=5) == xk.XK_EINVAL
    h = ctypes.c_void_p()
    assert L.xk_setup(64, 6, 3, 10, None, None, None, None, 0.1, 0, ctypes.byref(h)) == xk.XK_EINVAL
    assert L.xk_setup(64, 6, 3, 10, None, None, None, None, 0.1, 0, None) == xk.XK_EINVAL


def test_setup_isdf_rejects_invalid_inputs(L):
    phi, idx, V, W = _tables()
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    # N_g = 64 = 4^3: grid 5 does not match, L must be positive, idx checked as in xk_setup
    assert L.xk_setup_isdf(64, 6, 3, 10, p(phi), p(idx), 5, 1.0, 0, ctypes.byref(h)) == xk.XK_EINVAL
    assert "grid" in xk.last_error()
    assert L.xk_setup_isdf(64, 6, 3, 10, p(phi), p(idx), 4, 0.0, 0, ctypes.byref(h)) == xk.XK_EINVAL
    bad = idx.copy()
    bad[1] = bad[0]
    assert L.xk_setup_isdf(64, 6, 3, 10, p(phi), p(bad), 4, 1.0, 0, ctypes.byref(h)) == xk.XK_EINVAL
    assert L.xk_setup_isdf(64, 6, 3, 10, None, p(idx), 4, 1.0, 0, ctypes.byref(h)) == xk.XK_EINVAL


def test_null_handles_and_tickets(L):
    buf = np.zeros(4)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    assert L.xk_build(None, p, p, p) == xk.XK_EINVAL
    assert L.xk_build_device(None, p, p, p, None) == xk.XK_EINVAL
    assert L.xk_release(None) == xk.XK_EINVAL
    assert L.xk_poll(ctypes.c_uint64(123456789), p, p, None) == xk.XK_EINVAL
    assert "unknown ticket" in xk.last_error()
    t = ctypes.c_uint64()
    assert L.xk_submit(None, p, 0.0, ctypes.byref(t)) == xk.XK_EINVAL
    assert L.xk_ace(None, p, p, None, None) == xk.XK_EINVAL
    assert L.xk_energy(None, p, p) == xk.XK_EINVAL
    assert L.xk_build_full(None, p, p) == xk.XK_EINVAL
    assert L.xk_coulomb(None, 4, 1.0, p, p, p) == xk.XK_EINVAL
    assert L.xk_tables(None, p, None, 0, None, None) == xk.XK_EINVAL
    cnt = ctypes.c_int32()
    assert L.xk_isdf_points(4, 2, None, 2, 1e-14, p, ctypes.byref(cnt)) == xk.XK_EINVAL
    assert L.xk_isdf_points(0, 2, p, 2, 1e-14, p, ctypes.byref(cnt)) == xk.XK_EINVAL
    assert L.xk_isdf_points(2, 2, p, 2, -1.0, p, ctypes.byref(cnt)) == xk.XK_EINVAL
    assert L.xk_energy_device(None, p, p, None) == xk.XK_EINVAL
    b = ctypes.c_void_p()
    assert L.xk_batch_create(None, 0, ctypes.byref(b)) == xk.XK_EINVAL
    assert L.xk_batch_create(None, 1, None) == xk.XK_EINVAL
    assert L.xk_batch_build(None, p, p, p) == xk.XK_EINVAL
    assert L.xk_batch_release(None) == xk.XK_EINVAL
    assert L.xk_set_wait_limit(None, 0) == xk.XK_EINVAL
    assert L.xk_autotune_info(None, None, None) == xk.XK_EINVAL


def test_setup_refused_beyond_budget(L, monkeypatch):
    """Admission by footprint: with XK_HBM_BUDGET_BYTES below the handle's
    footprint, xk_setup returns XK_ENOMEM before any device call (the caller
    may retry once live handles are released)."""
    phi, idx, V, W = _tables()
    need = xk.footprint(phi.shape[0], phi.shape[1], 3, idx.shape[0], "f16x3")
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", str(need - 1))
    assert _setup(L, phi, idx, V, W, mode=2) == xk.XK_ENOMEM
    assert "XK_HBM_BUDGET_BYTES" in xk.last_error()
    monkeypatch.setenv("XK_HBM_BUDGET_BYTES", "0")
    assert _setup(L, phi, idx, V, W, mode=0) == xk.XK_ENOMEM


def test_setup_shard_rejects_bad_slices(L):
    """xk_setup_shard checks its slice [g0, g1) (non-empty, inside [0, N_aux))
    and the symmetry of W on the slice's diagonal block before any device call."""
    phi, idx, V, W = _tables()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    h = ctypes.c_void_p()
    for g0, g1 in ((5, 5), (-1, 4), (6, 11), (7, 3)):
        rows = max(g1 - max(g0, 0), 1)
        Vr = np.ascontiguousarray(V[:rows])
        Wr = np.ascontiguousarray(W[:rows])
        assert L.xk_setup_shard(64, 6, 3, 10, g0, g1, p(phi), p(idx), p(Vr), p(Wr), 0.1, 0,
                                ctypes.byref(h)) == xk.XK_EINVAL, (g0, g1)
    Wr = np.ascontiguousarray(W[2:6])
    Wr[0, 3] += 1e-6  # W[2, 3] != W[3, 2]: the block [2, 6) x [2, 6) is not symmetric
    assert L.xk_setup_shard(64, 6, 3, 10, 2, 6, p(phi), p(idx), p(np.ascontiguousarray(V[2:6])),
                            p(Wr), 0.1, 0, ctypes.byref(h)) == xk.XK_EINVAL
    assert "symmetric" in xk.last_error()
