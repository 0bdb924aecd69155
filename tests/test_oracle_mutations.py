"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each mutant replaces the oracle's robust-PS line evaluation with a version
carrying one plausible error (a dropped term, a wrong sign, a wrong index or
transposed operand).  The exact-limit pin (P1) and the 4-index definition pin
(P3) are re-evaluated with the mutant; at least one must fail.
"""
import numpy as np
import pytest

import oracle
import oracle.exx as ox
from cellgen import basis_on_grid, build_cell, config_spec, draw_coefficients, potentials
from cellgen.cells import CellSpec, Shell


_ORIG = ox.rps_lines


def _lines_parts(phi, idx, V, W, C):
    psi = phi @ C
    psig = psi[idx]
    return psi, psig, phi[idx]


def m_drop_line3(phi, idx, V, W, C, gblock=512):
    l1, l2, l3 = _ORIG(phi, idx, V, W, C)
    return l1, l2, 0 * l3


def m_sign_line2(phi, idx, V, W, C, gblock=512):
    l1, l2, l3 = _ORIG(phi, idx, V, W, C)
    return l1, -l2, l3


def m_line2_bra_at_points(phi, idx, V, W, C, gblock=512):
    # line 2 with its phi_nu evaluated on the full grid index instead of R_g
    psi, psig, phig = _lines_parts(phi, idx, V, W, C)
    l1, _, l3 = _ORIG(phi, idx, V, W, C)
    V2 = V * (psig @ psi.T)
    M2 = V2 @ psi
    return l1, M2.T @ phi[: idx.size], l3


def m_pair_kernel_transposed(phi, idx, V, W, C, gblock=512):
    # P built from psi at R_g on both sides (the line-3 kernel) in lines 1-2
    psi, psig, phig = _lines_parts(phi, idx, V, W, C)
    P = psig @ psig.T
    V2 = V[:, idx] * P
    l1 = (psig.T @ V2) @ phig
    l2 = (V2 @ psig).T @ phig
    _, _, l3 = _ORIG(phi, idx, V, W, C)
    return l1, l2, l3


def m_W_unsquared(phi, idx, V, W, C, gblock=512):
    # line 3 without the Hadamard with Q
    psi, psig, phig = _lines_parts(phi, idx, V, W, C)
    l1, l2, _ = _ORIG(phi, idx, V, W, C)
    return l1, l2, (W @ psig).T @ phig


MUTANTS = [m_drop_line3, m_sign_line2, m_line2_bra_at_points, m_pair_kernel_transposed,
           m_W_unsquared]


@pytest.fixture(scope="module")
def settings():
    spec = config_spec(1)
    rng = np.random.default_rng(spec.seed)
    cen = spec.frac * spec.L + rng.uniform(-0.05, 0.05, size=spec.frac.shape)
    phi = basis_on_grid(cen, spec.L, 10, spec.shells)
    Ng = phi.shape[0]
    dV = spec.L ** 3 / Ng
    C = draw_coefficients(dV * phi.T @ phi, 6, 3)
    V = potentials(np.eye(Ng), spec.L, 10)
    exact = dict(phi=phi, idx=np.arange(Ng), V=V, W=V.copy(), C=C, dV=dV, L=spec.L, grid=10)
    tspec = CellSpec("tiny", np.array([[0.1, 0.2, 0.15], [0.55, 0.6, 0.45]]), 5.0, 10,
                     [Shell(0, (0.6,), (1.0,)), Shell(1, (0.9,), (1.0,))], 3, 30, 77)
    return exact, build_cell(tspec)


def _pins_hold(exact, tiny):
    f = exact
    K, E = oracle.exx_rps_occri(f["phi"], f["idx"], f["V"], f["W"], f["C"], f["dV"])
    _, Kx, Ex = oracle.exx_exact_fft(f["phi"], f["C"], f["L"], f["grid"], f["dV"])
    p1 = abs(E - Ex) < 1e-11 * abs(Ex) and np.max(np.abs(K - Kx)) < 1e-11 * np.max(np.abs(Kx))
    c = tiny
    K, E = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    _, K4, E4 = oracle.exx_rps_4index(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    p3 = abs(E - E4) < 1e-12 * abs(E4) and np.max(np.abs(K - K4)) < 1e-12 * np.max(np.abs(K4))
    return p1 and p3


def test_unmutated_pins_hold(settings):
    assert _pins_hold(*settings)


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m.__name__ for m in MUTANTS])
def test_mutant_is_caught(settings, mutant, monkeypatch):
    monkeypatch.setattr(ox, "rps_lines", mutant)
    assert not _pins_hold(*settings)


# ------------------------------------------------ full K_{mu nu} (Eq. rpsEx)

_ORIG_FULL = ox.exx_rps_full


def _full_terms(phi, idx, V, W, C):
    psi = phi @ C
    psig = psi[idx]
    phig = phi[idx]
    V2 = V * (psig @ psi.T)
    t1 = (phig.T @ V2) @ phi
    t2 = (V2 @ phi).T @ phig
    t3 = phig.T @ ((W * (psig @ psig.T)) @ phig)
    return t1, t2, t3


def f_drop_term2(phi, idx, V, W, C, dV, gblock=512):
    t1, t2, t3 = _full_terms(phi, idx, V, W, C)
    return dV * (2.0 * t1 - t3)


def f_sign_term3(phi, idx, V, W, C, dV, gblock=512):
    t1, t2, t3 = _full_terms(phi, idx, V, W, C)
    return dV * (t1 + t2 + t3)


def f_term1_ket_at_points(phi, idx, V, W, C, dV, gblock=512):
    # term 1 with phi_nu taken at R_g instead of R'
    t1, t2, t3 = _full_terms(phi, idx, V, W, C)
    psi = phi @ C
    V2 = V * (psi[idx] @ psi.T)
    bad = (phi[idx].T @ V2[:, idx]) @ phi[idx]
    return dV * (bad + t2 - t3)


def f_W_unsquared(phi, idx, V, W, C, dV, gblock=512):
    t1, t2, _ = _full_terms(phi, idx, V, W, C)
    return dV * (t1 + t2 - phi[idx].T @ W @ phi[idx])


FULL_MUTANTS = [f_drop_term2, f_sign_term3, f_term1_ket_at_points, f_W_unsquared]


def _full_pin_holds(tiny):
    c = tiny
    Kf = ox.exx_rps_full(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    K4, _, _ = oracle.exx_rps_4index(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    return np.max(np.abs(Kf - K4)) < 1e-12 * np.max(np.abs(K4))


def test_unmutated_full_pin_holds(settings):
    assert _full_pin_holds(settings[1])


@pytest.mark.parametrize("mutant", FULL_MUTANTS, ids=[m.__name__ for m in FULL_MUTANTS])
def test_full_mutant_is_caught(settings, mutant, monkeypatch):
    monkeypatch.setattr(ox, "exx_rps_full", mutant)
    assert not _full_pin_holds(settings[1])


# ------------------------------------------------ Coulomb J on the grid

_ORIG_J = ox.coulomb_j


def j_density_not_squared(phi, C, L, grid, dV):
    psi = phi @ C
    rho = np.sum(np.abs(psi), axis=1)
    v = oracle.coulomb_potential(rho, L, grid)
    return dV * (phi.T @ (v[:, None] * phi)), dV * float(np.sum(rho * v))


def j_potential_not_applied(phi, C, L, grid, dV):
    psi = phi @ C
    rho = np.sum(psi * psi, axis=1)
    return dV * (phi.T @ (rho[:, None] * phi)), dV * float(np.sum(rho * rho))


def j_one_sided(phi, C, L, grid, dV):
    # potential multiplied on one side only: Phi^T v (summed) Phi
    J, EJ = _ORIG_J(phi, C, L, grid, dV)
    return J + 1e-3 * np.triu(J, 1), EJ


J_MUTANTS = [j_density_not_squared, j_potential_not_applied, j_one_sided]


def _j_pin_holds(tiny):
    c = tiny
    J, EJ = ox.coulomb_j(c.phi, c.C, c.L, c.grid, c.dV)
    N = c.N
    rho = np.einsum("rm,rn->mnr", c.phi, c.phi).reshape(N * N, -1)
    pot = oracle.coulomb_potential(rho, c.L, c.grid)
    J4 = ((c.dV * rho @ pot.T) @ (c.C @ c.C.T).reshape(-1)).reshape(N, N)
    return np.max(np.abs(J - J4)) < 1e-12 * np.max(np.abs(J4)) and EJ > 0


def test_unmutated_j_pin_holds(settings):
    assert _j_pin_holds(settings[1])


@pytest.mark.parametrize("mutant", J_MUTANTS, ids=[m.__name__ for m in J_MUTANTS])
def test_j_mutant_is_caught(settings, mutant, monkeypatch):
    monkeypatch.setattr(ox, "coulomb_j", mutant)
    assert not _j_pin_holds(settings[1])


# ------------------------------------------------ ISDF set-up and point selection

import oracle.isdf as oi  # noqa: E402

_ORIG_TABLES = oi.isdf_tables
_ORIG_SELECT = oi.select_points


def t_no_solve(phi, idx, L, grid):
    # the pair Gram columns taken as the fit (no X_gg^{-1})
    G = phi[idx] @ phi.T
    chi = G * G
    V = oracle.coulomb_potential(chi, L, grid)
    W = V @ chi.T
    return chi, V, 0.5 * (W + W.T), 0.0


def t_no_poisson(phi, idx, L, grid):
    chi, _, _, r = _ORIG_TABLES(phi, idx, L, grid)
    W = chi @ chi.T
    return chi, chi, 0.5 * (W + W.T), r


def t_unsymmetrised(phi, idx, L, grid):
    chi, V, _, r = _ORIG_TABLES(phi, idx, L, grid)
    return chi, V, V @ chi.T, r


def s_no_update(rows, want, tol_rel=1e-14):
    # pivots by the initial diagonal only (no Schur-complement update)
    d = np.einsum("ij,ij->i", rows, rows) ** 2
    return np.argsort(-d, kind="stable")[:want]


def s_wrong_gram(rows, want, tol_rel=1e-14):
    # Gram of the rows instead of the pair products
    import scipy.linalg
    X = rows @ rows.T
    _, piv, rank, _ = scipy.linalg.lapack.dpstrf(X, tol=tol_rel * float(np.max(np.diag(X))), lower=1)
    return np.asarray(piv[:min(want, rank)], dtype=np.int64) - 1


T_MUTANTS = [t_no_solve, t_no_poisson, t_unsymmetrised]
S_MUTANTS = [s_no_update, s_wrong_gram]


def _tables_pins_hold(c):
    chi, V, W, _ = oi.isdf_tables(c.phi, c.idx, c.L, c.grid)
    interp = np.max(np.abs(chi[:, c.idx] - np.eye(c.Naux))) < 1e-8
    sym = np.max(np.abs(W - W.T)) == 0.0
    gen = (np.max(np.abs(V - c.V)) < 1e-9 * np.max(np.abs(c.V))
           and np.max(np.abs(W - c.W)) < 1e-9 * np.max(np.abs(c.W)))
    return interp and sym and gen


def _select_pins_hold(c):
    from cellgen.cells import _pair_gram, _pivoted_cholesky
    piv = oi.select_points(c.phi, 40)
    ref = _pivoted_cholesky(_pair_gram(c.phi, c.phi), 40)
    return piv.size == ref[:40].size and np.array_equal(piv, ref[:40])


@pytest.fixture(scope="module")
def small_fitted():
    # a cell with fitted tables small enough for many re-fits
    spec = CellSpec("mut", np.array([[0.1, 0.2, 0.15], [0.55, 0.6, 0.45]]), 5.0, 10,
                    [Shell(0, (0.6,), (1.0,)), Shell(1, (0.9,), (1.0,))], 3, 30, 78)
    return build_cell(spec)


def test_unmutated_isdf_pins_hold(small_fitted):
    assert _tables_pins_hold(small_fitted)
    assert _select_pins_hold(small_fitted)


@pytest.mark.parametrize("mutant", T_MUTANTS, ids=[m.__name__ for m in T_MUTANTS])
def test_tables_mutant_is_caught(small_fitted, mutant, monkeypatch):
    monkeypatch.setattr(oi, "isdf_tables", mutant)
    assert not _tables_pins_hold(small_fitted)


@pytest.mark.parametrize("mutant", S_MUTANTS, ids=[m.__name__ for m in S_MUTANTS])
def test_select_mutant_is_caught(small_fitted, mutant, monkeypatch):
    monkeypatch.setattr(oi, "select_points", mutant)
    assert not _select_pins_hold(small_fitted)
