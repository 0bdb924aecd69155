"""Seeded synthetic inputs for the exchange build (geometry, basis on the
grid, occupied coefficients, ISDF points, V and W).  Shared by the tests, the
oracle's checks and the benchmark; holds none of the build's arithmetic."""
from .cells import (Cell, CellSpec, Shell, build_cell, load_cell, config_spec,
                    draw_coefficients, perturb_coefficients, pseudo_scf_sequence, s_orthonormal,
                    potentials, coulomb_kernel_g, basis_on_grid, fit_isdf,
                    select_points_exact, thc_potential, CUBIC_SIZES, GENERATOR_VERSION)
