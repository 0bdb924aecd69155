"""FP64 CPU oracle of the robust-PS occ-RI exchange build (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this package.  It shares no code with the GPU
library (paper_2207_04636_gb300) and never calls it.
"""
from .exx import (orbitals, rps_lines, exx_rps_occri, exx_variant, exx_energy_direct,
                  rps_eri, exx_rps_4index, exx_rps_full, exx_exact_fft, exact_exchange_energy,
                  exchange_energy, ace_factor, coulomb_j)
from .isdf import isdf_tables, select_points
from .poisson import coulomb_potential, kernel_g
