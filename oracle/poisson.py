"""Grid Coulomb potential for the oracle (FP64, NumPy FFT).

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py; never by the GPU library.

Definition followed (Eq. 2eint, Eq. cou-1 of arXiv 2207.04636): the grid
kernel is v(R - R') = (1/N_g) sum_G exp(-iG.R) (4 pi / G^2) exp(iG.R'), with
the G = 0 term removed (Sec. IV.E), so that the potential of a grid function
f is Pois(f)(R) = sum_R' v(R - R') f(R') = IFFT[(4 pi / G^2) FFT[f]](R) with
NumPy's normalisation (the 1/N_g sits in the inverse transform).

Pinned by tests/test_oracle_pins.py::test_poisson_gaussian_charge against the
analytic Ewald-split potential of a periodic Gaussian charge.
"""
import numpy as np


def kernel_g(L: float, grid: int) -> np.ndarray:
    """4 pi / |G|^2 on the FFT frequency grid of a cubic cell, 0 at G = 0.
    G = 2 pi m / L with m the signed FFT frequency index (only |G|^2 enters,
    so the sign given to the Nyquist frequency does not matter)."""
    m = np.fft.fftfreq(grid) * grid
    g = 2.0 * np.pi * m / L
    g2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    k = np.zeros_like(g2)
    nz = g2 > 0
    k[nz] = 4.0 * np.pi / g2[nz]
    return k


def coulomb_potential(f: np.ndarray, L: float, grid: int) -> np.ndarray:
    """Pois(f) for one grid function (flat, length grid**3) or a stack of
    them (shape (m, grid**3)).  Returns the same shape, real."""
    k = kernel_g(L, grid)
    shp = f.shape
    f3 = f.reshape(-1, grid, grid, grid)
    out = np.fft.ifftn(np.fft.fftn(f3, axes=(1, 2, 3)) * k, axes=(1, 2, 3)).real
    return out.reshape(shp)
