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
