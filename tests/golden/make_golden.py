"""Writes tests/golden/config1.json from the CPU oracle only.

The paper prints no worked example with numbers for these synthetic inputs,
so the stored values are the oracle's own results on the seeded 8-centre
diamond cell (inputs from cellgen), kept to catch drift of the oracle or of
the generator between machines and versions.  Run:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from cellgen import GENERATOR_VERSION, build_cell, config_spec  # noqa: E402


def main():
    c = build_cell(config_spec(1))
    K, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Ex = oracle.exact_exchange_energy(c.phi, c.C, c.L, c.grid, c.dV)
    Kij, _, _, branch = oracle.ace_factor(K, c.C)
    out = {
        "cell": "config 1: 8-centre diamond, L=6.74, N=32, n=16, 24^3 grid, N_aux=256",
        "generator": GENERATOR_VERSION,
        "Ex_rps": E,
        "Ex_exact": Ex,
        "K_fro": float(np.linalg.norm(K)),
        "K_sum": float(K.sum()),
        "Kij_trace": float(np.trace(Kij)),
        "ace_branch": branch,
        "idx_head": [int(i) for i in c.idx[:16]],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
