"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test names the statement it checks (arXiv 2207.04636).  None of them
re-types the oracle's own formula: they compare it with an independent route
(the conventional FFT exchange, the literal 4-index integrals, an analytic
Ewald potential, an exact algebraic identity) or with invariances.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from cellgen import (basis_on_grid, build_cell, config_spec, draw_coefficients, fit_isdf,
                     potentials, select_points_exact, thc_potential)
from cellgen.cells import CellSpec, Shell


def _rel(a, b):
    return abs(a - b) / abs(b)


def _geometry(spec):
    rng = np.random.default_rng(spec.seed)
    return spec.frac * spec.L + rng.uniform(-spec.jitter, spec.jitter, size=spec.frac.shape)


@pytest.fixture(scope="module")
def trivial_fit():
    """Config-1 geometry on a 12^3 grid with every grid point an interpolation
    point and chi = I, so V(g, .) is the Coulomb kernel row of point g and W
    its restriction to the points (the exact-limit setting of Sec. IV.C)."""
    spec = config_spec(1)
    grid = 12
    cen = _geometry(spec)
    phi = basis_on_grid(cen, spec.L, grid, spec.shells)
    Ng = phi.shape[0]
    dV = spec.L ** 3 / Ng
    S = dV * phi.T @ phi
    C = draw_coefficients(S, 16, 7)
    idx = np.arange(Ng)
    V = potentials(np.eye(Ng), spec.L, grid)
    return dict(phi=phi, C=C, idx=idx, V=V, W=V.copy(), dV=dV, L=spec.L, grid=grid, S=S)


# ---------------------------------------------------------------- P10 -----

def _ewald_gaussian_potential(d, L, alpha, eta):
    """Potential (G = 0 removed) of the periodic, unit-normalised Gaussian
    charge (alpha/pi)^{3/2} exp(-alpha r^2) at displacements d (m, 3), by
    Ewald splitting with a softer exponent eta < alpha:
      phi(d) = (4 pi/Omega) sum_{G != 0} exp(-G^2/4eta)/G^2 cos(G.d)
               - sum_T [erf(sqrt(eta)|d+T|) - erf(sqrt(alpha)|d+T|)] / |d+T|
               + (pi/Omega)(1/alpha - 1/eta)."""
    omega = L ** 3
    mmax = int(math.ceil(math.sqrt(4 * eta * 40.0) * L / (2 * math.pi))) + 1
    m = np.arange(-mmax, mmax + 1)
    G = 2 * math.pi * np.stack(np.meshgrid(m, m, m, indexing="ij"), -1).reshape(-1, 3) / L
    G2 = np.einsum("ij,ij->i", G, G)
    G, G2 = G[G2 > 0], G2[G2 > 0]
    recip = (4 * math.pi / omega) * (np.cos(d @ G.T) * (np.exp(-G2 / (4 * eta)) / G2)).sum(1)
    tmax = int(math.ceil(6.5 / math.sqrt(eta) / L)) + 1
    t = np.arange(-tmax, tmax + 1)
    T = L * np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    real = np.zeros(d.shape[0])
    for Tv in T:
        r = np.linalg.norm(d + Tv, axis=1)
        real += (erf(math.sqrt(eta) * r) - erf(math.sqrt(alpha) * r)) / r
    return recip - real + (math.pi / omega) * (1 / alpha - 1 / eta)


def test_poisson_gaussian_charge():
    """P10: the grid Poisson solve of Eq. cou-1 reproduces the analytic
    periodic potential of a Gaussian charge (G = 0 removed, Sec. IV.E)."""
    L, grid, alpha, eta = 6.0, 40, 1.2, 0.35
    A = np.array([1.234, 2.71, 3.3])
    x = np.arange(grid) * (L / grid)
    R = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    rho = np.zeros(R.shape[0])
    for tx in range(-2, 3):
        for ty in range(-2, 3):
            for tz in range(-2, 3):
                d = R - A + L * np.array([tx, ty, tz])
                rho += np.exp(-alpha * np.einsum("ij,ij->i", d, d))
    rho *= (alpha / math.pi) ** 1.5
    pot = oracle.coulomb_potential(rho, L, grid)
    sel = np.random.default_rng(3).choice(R.shape[0], 60, replace=False)
    ref = _ewald_gaussian_potential(R[sel] - A, L, alpha, eta)
    assert np.max(np.abs(pot[sel] - ref)) < 1e-8
    # the G = 0 term is absent: the potential has zero mean over the cell
    assert abs(pot.mean()) < 1e-12


# ---------------------------------------------------------------- P1 ------

def test_exact_limit_equals_fft_exchange(trivial_fit):
    """P1: with every grid point an interpolation point and chi = I the three
    robust-PS terms are each exact, so Eq. exoccri equals the conventional
    FFT exchange of Eq. exchange (Sec. IV.C: N_chi = N_g gives the exact result)."""
    f = trivial_fit
    K, E = oracle.exx_rps_occri(f["phi"], f["idx"], f["V"], f["W"], f["C"], f["dV"])
    Kx, Kmx, Ex = oracle.exx_exact_fft(f["phi"], f["C"], f["L"], f["grid"], f["dV"])
    assert _rel(E, Ex) < 1e-11
    assert np.max(np.abs(K - Kmx)) < 1e-11 * np.max(np.abs(Kmx))
    # two independent exact routes agree (N*n solves vs n^2 solves)
    E2 = oracle.exact_exchange_energy(f["phi"], f["C"], f["L"], f["grid"], f["dV"])
    assert _rel(E2, Ex) < 1e-12


# ---------------------------------------------------------------- P2 ------

def test_full_rank_fit_is_exact(cell1):
    """P2: with N_aux equal to the rank of the pair matrix the ISDF fit of
    Eq. isdf has no residual, so robust PS equals exact exchange."""
    c = cell1
    idx = np.sort(select_points_exact(c.phi, 10 ** 6))
    assert idx.size <= c.N * (c.N + 1) // 2
    chi, _ = fit_isdf(c.phi, idx)
    V = potentials(chi, c.L, c.grid)
    W = thc_potential(V, chi)
    K, E = oracle.exx_rps_occri(c.phi, idx, V, W, c.C, c.dV)
    Kx, Kmx, Ex = oracle.exx_exact_fft(c.phi, c.C, c.L, c.grid, c.dV)
    assert _rel(E, Ex) < 1e-9
    assert np.max(np.abs(K - Kmx)) < 1e-8 * np.max(np.abs(Kmx))


# ---------------------------------------------------------------- P3 ------

@pytest.fixture(scope="module")
def tiny():
    spec = CellSpec("tiny", np.array([[0.1, 0.2, 0.15], [0.55, 0.6, 0.45]]), 5.0, 10,
                    [Shell(0, (0.6,), (1.0,)), Shell(1, (0.9,), (1.0,))], 3, 30, 77)
    return build_cell(spec, keep_chi=True)


def test_occri_equals_4index_definition(tiny):
    """P3: the occ-RI contraction order of Eq. exoccri equals the literal
    4-index robust-PS integrals of Eq. rps contracted with D = C C^T."""
    c = tiny
    K, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    K4, Kmui4, E4 = oracle.exx_rps_4index(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert _rel(E, E4) < 1e-12
    assert np.max(np.abs(K - Kmui4)) < 1e-12 * np.max(np.abs(K))


def test_full_k_equals_4index_definition(tiny, cell1):
    """Eq. rpsEx in its step order, with the three terms of Eq. rps, equals
    the literal 4-index integrals contracted with D = C C^T; the result is
    symmetric, and K C is the occ-RI rectangle of Eq. exoccri."""
    c = tiny
    Kf = oracle.exx_rps_full(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    K4, _, _ = oracle.exx_rps_4index(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert np.max(np.abs(Kf - K4)) < 1e-12 * np.max(np.abs(K4))
    c = cell1
    Kf = oracle.exx_rps_full(c.phi, c.idx, c.V, c.W, c.C, c.dV, gblock=100)
    assert np.max(np.abs(Kf - Kf.T)) < 1e-12 * np.max(np.abs(Kf))
    Kmui, _ = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert np.max(np.abs(Kf @ c.C - Kmui)) < 1e-12 * np.max(np.abs(Kmui))


def test_coulomb_equals_4index_definition(tiny):
    """J of the density route (one Poisson solve of rho) equals the literal
    grid integrals (mu nu|lam sig) = dV sum_R rho_{mu nu} Pois(rho_{lam sig})
    (Eq. 2eint, one Poisson solve per pair density) contracted with
    D = C C^T; E_J = tr(C^T J C) = sum_ij (ii|jj) > 0 (the kernel 4 pi / G^2
    is positive)."""
    c = tiny
    J, EJ = oracle.coulomb_j(c.phi, c.C, c.L, c.grid, c.dV)
    N = c.N
    rho = np.einsum("rm,rn->mnr", c.phi, c.phi).reshape(N * N, -1)
    pot = oracle.coulomb_potential(rho, c.L, c.grid)
    eri = c.dV * rho @ pot.T                           # (mu nu | lam sig)
    D = (c.C @ c.C.T).reshape(-1)
    J4 = (eri @ D).reshape(N, N)
    assert np.max(np.abs(J - J4)) < 1e-12 * np.max(np.abs(J4))
    assert np.max(np.abs(J - J.T)) < 1e-12 * np.max(np.abs(J))
    assert abs(EJ - np.trace(c.C.T @ J @ c.C)) < 1e-12 * abs(EJ)
    assert EJ > 0


# ---------------------------------------------------------------- P6 ------

def test_symmetry(tiny, cell1):
    """P6: robust PS restores bra-ket symmetry (Sec. III.B): the 4-index
    integrals and the full K_{mu nu} are symmetric, W is symmetric (Eq.
    thcpot) and K_ij = C^T K_{mu i} is symmetric."""
    c = tiny
    N = c.N
    eri = oracle.rps_eri(c.phi, c.idx, c.V, c.W, c.dV)
    assert np.max(np.abs(eri - eri.T)) < 1e-12 * np.max(np.abs(eri))
    e4 = eri.reshape(N, N, N, N)
    assert np.max(np.abs(e4 - e4.transpose(1, 0, 2, 3))) < 1e-12 * np.max(np.abs(eri))
    K4, _, _ = oracle.exx_rps_4index(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert np.max(np.abs(K4 - K4.T)) < 1e-12 * np.max(np.abs(K4))
    c = cell1
    assert np.array_equal(c.W, c.W.T)
    K, _ = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Kij = c.C.T @ K
    assert np.max(np.abs(Kij - Kij.T)) < 1e-12 * np.max(np.abs(Kij))


def test_ps_alone_is_not_symmetric(tiny):
    """The first line of Eq. rps alone (pseudospectral) is not bra-ket
    symmetric, which is the defect robust PS removes (Sec. III.B)."""
    c = tiny
    N = c.N
    rho = np.einsum("rm,rn->mnr", c.phi, c.phi).reshape(N * N, -1)
    T1 = c.dV * rho[:, c.idx] @ c.V @ rho.T
    assert np.max(np.abs(T1 - T1.T)) > 1e-6 * np.max(np.abs(T1))


# ---------------------------------------------------------------- P7 ------

def test_sign_and_definiteness(cell1):
    """P7: E_x < 0, and the exact grid exchange matrix is positive
    semidefinite because 4 pi / G^2 >= 0 with G = 0 removed."""
    c = cell1
    _, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Kx, _, Ex = oracle.exx_exact_fft(c.phi, c.C, c.L, c.grid, c.dV)
    assert E < 0 and Ex < 0
    w = np.linalg.eigvalsh(0.5 * (Kx + Kx.T))
    assert w.min() > -1e-12 * w.max()


# ---------------------------------------------------------------- P8 ------

def test_closed_form_energy(cell1):
    """P8: contracting Eq. exoccri with C gives
    E_x = -dV (2 sum V o P^2 - sum W o Q^2), P = Psi_g Psi^T, Q = Psi_g Psi_g^T."""
    c = cell1
    _, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Ed = oracle.exx_energy_direct(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert _rel(E, Ed) < 1e-12


# ---------------------------------------------------------------- P9 ------

def test_orbital_rotation(cell1):
    """P9: C -> C U (U orthogonal) maps K_{mu i} -> K_{mu i} U and leaves E_x
    unchanged: the pair kernel sum_i psi_i psi_i is rotation invariant."""
    c = cell1
    U, _ = np.linalg.qr(np.random.default_rng(11).standard_normal((c.n, c.n)))
    K, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Ku, Eu = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C @ U, c.dV)
    assert _rel(Eu, E) < 1e-12
    assert np.max(np.abs(Ku - K @ U)) < 1e-12 * np.max(np.abs(K))


def test_grid_translation(cell1):
    """P9: translating every centre by a grid vector (a cyclic shift of the
    grid in the flat (ix*N2+iy)*N3+iz order, with the points shifted alike)
    leaves K and E_x unchanged."""
    c = cell1
    g = c.grid
    sx, sy, sz = 5, 2, 9

    def roll(a, axis_last):
        shp = a.shape[:-1] + (g, g, g) if axis_last else (g, g, g) + a.shape[1:]
        ax = (-3, -2, -1) if axis_last else (0, 1, 2)
        return np.roll(a.reshape(shp), (sx, sy, sz), axis=ax).reshape(a.shape)

    phi = roll(c.phi, False)
    V = roll(c.V, True)
    ix, iy, iz = np.unravel_index(c.idx, (g, g, g))
    idx = np.ravel_multi_index(((ix + sx) % g, (iy + sy) % g, (iz + sz) % g), (g, g, g))
    K, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Kt, Et = oracle.exx_rps_occri(phi, idx, V, c.W, c.C, c.dV)
    assert _rel(Et, E) < 1e-12
    assert np.max(np.abs(Kt - K)) < 1e-12 * np.max(np.abs(K))


# ---------------------------------------------------------------- P4 ------

def test_rps_error_is_the_dropped_quadratic_term(cell1):
    """P4 (identity form): Sec. III.B writes the exact integral as the three
    robust-PS terms plus one term bilinear in the two fitting errors, which
    robust PS drops.  Hence E_rPS - E_exact = dV sum_ij delta_ij . Pois(delta_ij)
    exactly, with delta_ij(R) = psi_i psi_j (R) - sum_g psi_i psi_j (R_g) chi_g(R);
    it is >= 0 because the kernel is positive semidefinite."""
    c = cell1
    _, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Ex = oracle.exact_exchange_energy(c.phi, c.C, c.L, c.grid, c.dV)
    psi = c.phi @ c.C
    psig = psi[c.idx]
    acc = 0.0
    for i in range(c.n):
        pair = psi[:, i][:, None] * psi                      # (N_g, n)
        fit = (psig[:, i][:, None] * psig).T @ c.chi         # (n, N_g)
        delta = pair.T - fit
        acc += float(np.sum(delta * oracle.coulomb_potential(delta, c.L, c.grid)))
    dropped = c.dV * acc
    assert dropped > 0
    assert abs((E - Ex) - dropped) < 1e-7 * dropped


def test_rps_error_quadratic_thc_linear(trivial_fit):
    """P4 (order form): perturbing an exact fit chi = I by t*eta, the robust-PS
    energy error scales as t^2 (ratio 4 when t doubles) while the THC error
    (third line of Eq. rps alone) scales as t (ratio 2): O(eps^2) vs O(eps)."""
    f = trivial_fit
    Ng = f["phi"].shape[0]
    eta = np.random.default_rng(5).standard_normal((Ng, Ng)) * 1e-2
    Eex = oracle.exact_exchange_energy(f["phi"], f["C"], f["L"], f["grid"], f["dV"])
    err = {}
    for t in (1e-3, 2e-3):
        chi = np.eye(Ng) + t * eta
        V = potentials(chi, f["L"], f["grid"])
        W = thc_potential(V, chi)
        _, E = oracle.exx_rps_occri(f["phi"], f["idx"], V, W, f["C"], f["dV"])
        _, Et = oracle.exx_variant(f["phi"], f["idx"], V, W, f["C"], f["dV"], "thc")
        err[t] = (E - Eex, Et - Eex)
    r_rps = err[2e-3][0] / err[1e-3][0]
    r_thc = err[2e-3][1] / err[1e-3][1]
    assert abs(r_rps - 4.0) < 0.02
    assert abs(r_thc - 2.0) < 0.1


@pytest.fixture(scope="module")
def naux_sweep(cell1):
    c = cell1
    from cellgen.cells import _pair_gram
    X = _pair_gram(c.phi, c.phi)
    piv = select_points_exact(c.phi, 10 ** 6)
    Eex = oracle.exact_exchange_energy(c.phi, c.C, c.L, c.grid, c.dV)
    out = []
    for na in (128, 192, 256, 320, 400):
        idx = np.sort(piv[:na])
        chi, _ = fit_isdf(c.phi, idx)
        V = potentials(chi, c.L, c.grid)
        W = thc_potential(V, chi)
        _, E = oracle.exx_rps_occri(c.phi, idx, V, W, c.C, c.dV)
        tr = np.trace(X)
        res2 = tr - 2 * np.sum(chi * X[idx]) + np.sum(chi * (X[np.ix_(idx, idx)] @ chi))
        out.append((na, math.sqrt(max(res2, 0.0) / tr), E - Eex))
    return out


def test_rps_error_quadratic_in_fit_error(naux_sweep):
    """P4 (sweep form): over least-squares fits with growing N_aux the
    robust-PS error falls as the square of the relative Frobenius residual of
    Eq. isdf (log-log slope in [1.6, 2.6]) and is never negative."""
    eps = np.array([e for _, e, _ in naux_sweep])
    err = np.array([d for _, _, d in naux_sweep])
    assert np.all(err > 0)
    slope = np.polyfit(np.log(eps), np.log(err), 1)[0]
    assert 1.6 <= slope <= 2.6


def test_rps_error_decays_exponentially(naux_sweep):
    """P5: the error falls roughly exponentially with N_aux (Sec. I and V):
    monotone, and log|dE| is close to linear in N_aux (R^2 > 0.8)."""
    na = np.array([n for n, _, _ in naux_sweep], dtype=float)
    le = np.log(np.array([d for _, _, d in naux_sweep]))
    assert np.all(np.diff(le) < 0)
    p = np.polyfit(na, le, 1)
    r2 = 1 - np.sum((le - np.polyval(p, na)) ** 2) / np.sum((le - le.mean()) ** 2)
    assert p[0] < 0 and r2 > 0.8


# ---------------------------------------------------------------- ACE -----

def test_ace_factor(cell1):
    """occ-RI K_ij and its factorisation (Sec. III.C, ACE form): K_ij is
    positive definite here, the Cholesky branch runs, and
    (xi diag(s) xi^T) C reproduces K_{mu i}."""
    c = cell1
    K, _ = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Kij, xi, s, branch = oracle.ace_factor(K, c.C)
    assert branch == "cholesky"
    assert np.max(np.abs((xi * s) @ xi.T @ c.C - K)) < 1e-10 * np.max(np.abs(K))


# ------------------------------------------------------- ISDF set-up -------

def test_isdf_oracle_interpolates_and_fits(cell1):
    """The least-squares fit of Eq. lsqfit interpolates: chi_g(R_g') = delta
    at the interpolation points (the fit's columns at R_g are X_gg^{-1} X_gg);
    with all points of a full-rank selection the fitted pair products are
    exact everywhere; W is symmetric and equals V chi^T; V is the potential
    of chi (the Poisson solver is pinned by P10)."""
    c = cell1
    chi, V, W, ridge = oracle.isdf_tables(c.phi, c.idx, c.L, c.grid)
    assert ridge == 0.0
    assert np.max(np.abs(chi[:, c.idx] - np.eye(c.Naux))) < 1e-8
    assert np.max(np.abs(W - W.T)) == 0.0
    Wr = V @ chi.T
    assert np.max(np.abs(W - Wr)) < 1e-10 * np.max(np.abs(W))
    # full-rank selection: the fit reproduces every pair product rho_mn(R)
    idx = np.sort(select_points_exact(c.phi, 10 ** 6))
    chi2, _, _, _ = oracle.isdf_tables(c.phi, idx, c.L, c.grid)
    rho = np.einsum("rm,rn->rmn", c.phi, c.phi).reshape(c.Ng, -1)
    fit = chi2.T @ rho[idx]
    assert np.max(np.abs(fit - rho)) < 1e-7 * np.max(np.abs(rho))


def test_isdf_oracle_matches_cell_tables(cell1):
    """The generator's tables of the 8-centre cell (its own fit, Poisson and
    W) agree with the oracle's for the same points."""
    c = cell1
    chi, V, W, _ = oracle.isdf_tables(c.phi, c.idx, c.L, c.grid)
    assert np.max(np.abs(V - c.V)) < 1e-9 * np.max(np.abs(c.V))
    assert np.max(np.abs(W - c.W)) < 1e-9 * np.max(np.abs(c.W))


def test_point_selection_oracle(cell1, tiny):
    """The greedy pivoted Cholesky of the pair Gram picks the same points as
    LAPACK's complete-pivoting Cholesky (dpstrf, the generator's route) on
    the 8-centre cell (256 of 13824 points) and on the tiny cell, where the
    rank of the pair products stops it early."""
    from cellgen.cells import _pair_gram, _pivoted_cholesky
    for c, want in ((cell1, 256), (tiny, 30)):
        piv = oracle.select_points(c.phi, want)
        ref = _pivoted_cholesky(_pair_gram(c.phi, c.phi), want)
        assert np.array_equal(piv, ref[:piv.size])
        assert piv.size == min(want, ref.size)
