"""The GPU ISDF set-up (xk_setup_isdf: X_gg, X_gR, the Cholesky fit, the
DFT Poisson solve and W on the device, all FP64) against the oracle's tables
(oracle.isdf_tables), and the exchange built from them against the oracle.

Tolerances: the tables agree to 1e-8 of their largest element (the fit
amplifies rounding by cond(X_gg), 1.7e3 to 1.7e6 on these cells); the
builds keep the FP64 (1e-8 Ha, 1e-7) and tensor-path (1e-6 Ha, 1e-6) bars.
"""
import numpy as np
import pytest

import oracle
from cellgen import CellSpec, Shell, build_cell, config_spec, load_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


def _ragged():
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    return build_cell(CellSpec("ragged", np.array([[0.1, 0.2, 0.3], [0.6, 0.5, 0.45],
                                                    [0.3, 0.75, 0.8]]), 6.5, 13, sh, 7, 97, 9001))


@pytest.mark.parametrize("which", ["cell1", "ragged", "cubic27"])
def test_isdf_tables_and_build_fp64(xk, cell1, which):
    c = {"cell1": lambda: cell1, "ragged": _ragged,
         "cubic27": lambda: load_cell(config_spec(4, k=3))}[which]()
    chi0, V0, W0, ridge0 = oracle.isdf_tables(c.phi, c.idx, c.L, c.grid)
    h = xk.Handle.isdf(c.phi, c.idx, c.grid, c.L, c.n, mode="fp64")
    try:
        rows = [0, c.Naux // 2, c.Naux - 1]
        W, Vr, ridge = h.tables(rows)
        K, E = h.build(c.C)
    finally:
        h.release()
    assert ridge == ridge0 == 0.0
    assert np.max(np.abs(W - W0)) <= 1e-8 * np.max(np.abs(W0))
    assert np.max(np.abs(W - W.T)) == 0.0
    assert np.max(np.abs(Vr - V0[rows])) <= 1e-8 * np.max(np.abs(V0))
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, V0, W0, c.C, c.dV)
    assert abs(E - E0) <= 1e-8, (E, E0)
    assert np.max(np.abs(K - K0)) <= 1e-7


@pytest.mark.parametrize("which", ["cell1", "cubic27"])
def test_isdf_build_f16x3(xk, cell1, which):
    c = cell1 if which == "cell1" else load_cell(config_spec(4, k=3))
    _, V0, W0, _ = oracle.isdf_tables(c.phi, c.idx, c.L, c.grid)
    h = xk.Handle.isdf(c.phi, c.idx, c.grid, c.L, c.n, mode="f16x3")
    try:
        K, E = h.build(c.C)
    finally:
        h.release()
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, V0, W0, c.C, c.dV)
    assert abs(E - E0) <= 1e-6, (E, E0)
    assert np.max(np.abs(K - K0)) <= 1e-6
