"""The oracle on the seeded 8-centre cell against stored values written by
tests/golden/make_golden.py (oracle only): catches drift of the oracle or of
the input generator across machines and versions."""
import json
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_config1_golden(cell1):
    with open(os.path.join(HERE, "golden", "config1.json")) as f:
        g = json.load(f)
    c = cell1
    assert [int(i) for i in c.idx[:16]] == g["idx_head"]
    K, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert abs(E - g["Ex_rps"]) < 1e-9 * abs(g["Ex_rps"])
    assert abs(np.linalg.norm(K) - g["K_fro"]) < 1e-9 * g["K_fro"]
    Ex = oracle.exact_exchange_energy(c.phi, c.C, c.L, c.grid, c.dV)
    assert abs(Ex - g["Ex_exact"]) < 1e-10 * abs(g["Ex_exact"])


def test_generator_without_fit_matches_fitted_inputs():
    """build_cell(fit=False) gives the same basis, coefficients and points as
    the fitted cell and leaves the tables out (for a set-up that forms them
    on the device)."""
    from cellgen import CellSpec, Shell, build_cell
    import numpy as np
    spec = CellSpec("nofit", np.array([[0.1, 0.2, 0.15], [0.55, 0.6, 0.45]]), 5.0, 10,
                    [Shell(0, (0.6,), (1.0,)), Shell(1, (0.9,), (1.0,))], 3, 20, 79)
    a = build_cell(spec)
    b = build_cell(spec, fit=False)
    assert b.V is None and b.W is None
    assert np.array_equal(a.phi, b.phi) and np.array_equal(a.C, b.C)
    assert np.array_equal(a.idx, b.idx) and a.dV == b.dV
