"""Parity of the tensor-core path (XK_F16X3, through the C ABI) with the CPU oracle.

The path returns E_x from the closed form of Eq. exoccri contracted with C
and K_{mu i} from the split-FP16 tensor-core contractions.  Its error against
the FP64 oracle is held to |dE_x| <= 1e-6 Ha per cell (measured about 4e-8 on
the 64-centre cell) and to max|dK| <= 1e-6 (measured about 1.2e-7).
"""
import numpy as np
import pytest

import oracle
from cellgen import CellSpec, Shell, build_cell, config_spec, load_cell

pytestmark = pytest.mark.gpu

TOL_E, TOL_K = 1e-6, 1e-6
# Handles with 65 <= n <= 128 (128-column pieces) run the fused pair role,
# which adds its M2 tiles into FP32 copies in the order the CTAs finish: two
# builds of the same C agree to rounding in K (and bit for bit in E_x, whose
# per-CTA sums are fixed-order).
TOL_REPEAT_K = 1e-7


def fused(n):
    return 64 < n <= 128


def same_build(K, E, K2, E2, n):
    if fused(n):
        return E == E2 and np.max(np.abs(K - K2)) <= TOL_REPEAT_K
    return np.array_equal(K, K2) and E == E2  # fixed reduction order


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


def _check(xk, c):
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        K, E = h.build(c.C)
        est = h.error_estimate()
        Ee = h.energy(c.C)
        K2, E2 = h.build(c.C)
    finally:
        h.release()
    assert abs(E - E0) <= TOL_E, (E, E0)
    # the per-build estimate |E_x - E_K| (E_K = -sum K o C, formed on the
    # device): it matches the host's value and lies within the K tolerance
    # times sum |C| of the oracle's energy of K
    EK = -float(np.sum(K * c.C))
    assert abs(est - abs(E - EK)) <= 1e-10, (est, E - EK)
    assert abs(EK - E0) <= est + abs(E - E0) + 1e-12
    assert np.max(np.abs(K - K0)) <= TOL_K, np.max(np.abs(K - K0))
    assert same_build(K, E, K2, E2, c.n), (E, E2, np.max(np.abs(K - K2)))
    # E_x alone (xk_energy): the same S products, splits and summation order
    assert Ee == E, (Ee, E)
    return K, E


def test_config1(xk, cell1):
    before = xk.kernel_launches()
    _check(xk, cell1)
    assert xk.kernel_launches() > before


def test_ragged(xk):
    """N = 27, n = 7, N_aux = 97, N_g = 13^3: every tile has a ragged edge."""
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    c = build_cell(CellSpec("ragged", np.array([[0.1, 0.2, 0.3], [0.6, 0.5, 0.45],
                                                 [0.3, 0.75, 0.8]]), 6.5, 13, sh, 7, 97, 9001))
    _check(xk, c)


def test_cubic27(xk):
    """27-centre simple-cubic cell (N = 351, n = 54, N_aux = 1755, N_g = 45^3)."""
    _check(xk, load_cell(config_spec(4, k=3)))


@pytest.mark.parametrize("n_occ", [100, 128])
def test_fused_role(xk, n_occ):
    """65 <= n <= 128 (27-centre cell, N_g = 45^3, N_aux = 1755): the fused
    pair role (S formed once, M1 and M2 from one pass over V).  N_g and N_aux
    leave ragged last tiles (117 of 128 grid points, 27 of 64 interpolation
    points); n = 100 leaves zero columns in the 128-wide pieces."""
    spec = config_spec(4, k=3)
    spec.n_occ = n_occ
    _check(xk, load_cell(spec))


@pytest.mark.parametrize("tiles", [None, "128", "256"])
@pytest.mark.parametrize("n_occ", [150, 200])
def test_large_n(xk, n_occ, tiles, monkeypatch):
    """n > 128 (27-centre cell, N = 351): the pair contractions go through the
    stored T = V o P and three tensor-core GEMMs; n = 150 leaves a ragged
    64-wide piece block and a ragged 128-wide output tile.  With n = 200 on
    27 centres E_x = -117.8 Ha: the three-piece orbitals of the S product keep
    its error far inside 1e-6 Ha (two pieces missed by 4e-6)."""
    # tiles: the back-contraction shape the set-up's autotuner would choose
    # (None), or either shape forced (XK_BACK_TILES), so that both stay tested
    if tiles is not None:
        monkeypatch.setenv("XK_BACK_TILES", tiles)
    spec = config_spec(4, k=3)
    spec.n_occ = n_occ
    _check(xk, load_cell(spec))


def test_back_shape_autotune(xk, monkeypatch):
    """The set-up times the n > 128 back-contractions with 128- and 256-column
    tiles and keeps the faster (256 unless 128 is 3 % faster); XK_BACK_TILES
    fixes the shape without timing."""
    spec = config_spec(4, k=3)
    spec.n_occ = 150
    c = load_cell(spec)
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        info = h.autotune_info()
    finally:
        h.release()
    assert info["ms_128"] > 0 and info["ms_256"] > 0
    want = 128 if info["ms_128"] < 0.97 * info["ms_256"] else 256
    assert info["back_tiles"] == want, info
    monkeypatch.setenv("XK_BACK_TILES", "128")
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        info = h.autotune_info()
    finally:
        h.release()
    assert info["back_tiles"] == 128 and info["ms_128"] == 0 and info["ms_256"] == 0


def _full_cells(cell1):
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    rag = build_cell(CellSpec("ragged", np.array([[0.1, 0.2, 0.3], [0.6, 0.5, 0.45],
                                                   [0.3, 0.75, 0.8]]), 6.5, 13, sh, 7, 97, 9001))
    big = config_spec(4, k=3)
    big.n_occ = 150
    return [cell1, rag, load_cell(config_spec(4, k=3)), load_cell(big)]


def test_full_k(xk, cell1):
    """xk_build_full on the tensor cores against the oracle's K_{mu nu} (Eq.
    rpsEx, three terms of Eq. rps): the 8-centre cell, a ragged cell, the
    27-centre cell with n = 54 and with n = 150 (the n > 128 pieces)."""
    for c in _full_cells(cell1):
        Kf0 = oracle.exx_rps_full(c.phi, c.idx, c.V, c.W, c.C, c.dV)
        h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
        try:
            K, E = h.build(c.C)
            Kf = h.build_full(c.C)
            Kf2 = h.build_full(c.C)
            K2, E2 = h.build(c.C)
        finally:
            h.release()
        err = np.max(np.abs(Kf - Kf0))
        assert err <= TOL_K, (c.spec.name, err)
        assert np.array_equal(Kf, Kf2)
        assert same_build(K, E, K2, E2, c.n)  # the occ-RI build is unaffected


def test_ace_on_tensor_path(xk, cell1):
    """K_ij of the tensor-core build is positive definite and factors; the
    reconstruction (xi diag(s) xi^T) C = K_{mu i} holds up to the asymmetry
    of C^T K_{mu i}, which is of the size of the K error (~1e-7)."""
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    K, _ = h.build(c.C)
    Kij, xi, s, br = h.ace()
    h.release()
    assert br == "cholesky"
    asym = np.max(np.abs(Kij - (c.C.T @ K)))
    assert np.max(np.abs((xi * s) @ xi.T @ c.C - K)) <= 1e-5 * np.max(np.abs(K))
    assert asym <= 1e-5 * np.max(np.abs(Kij))


@pytest.mark.parametrize("n_occ", [None, 100])
def test_ace_on_tensor_path_matches_oracle(xk, cell1, n_occ):
    """Row a11 on the tensor path: xk_ace's K_ij and xi against the oracle's
    ACE factorisation (i) of the same K (the device's FP64 factorisation,
    to rounding) and (ii) of the oracle's own K, within the bounds that the
    measured max|dK| of the build propagates to:
        |dK_ij| <= max_i sum_mu |C_mu,i| max|dK|,
        |dxi|   <= |dK| |L^-1| + |K| |L^-1| cond(K_ij) |dK_ij| / |K_ij|
    (first-order Cholesky perturbation), each with a factor 4 of margin.
    The 8-centre cell (n = 16) and the 27-centre cell with n = 100 (the
    fused pair role)."""
    if n_occ is None:
        c = cell1
    else:
        spec = config_spec(4, k=3)
        spec.n_occ = n_occ
        c = load_cell(spec)
    K0, _ = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        K, _ = h.build(c.C)
        Kij, xi, sg, br = h.ace()
    finally:
        h.release()
    # (i) the same K through the oracle's factorisation
    Kij1, xi1, s1, br1 = oracle.ace_factor(K, c.C)
    assert br == br1 == "cholesky"
    assert np.max(np.abs(Kij - Kij1)) <= 1e-12 * np.max(np.abs(Kij1))
    assert np.max(np.abs(xi - xi1)) <= 1e-9 * np.max(np.abs(xi1))
    # (ii) against the oracle's K, within the propagated K error
    Kij0, xi0, s0, br0 = oracle.ace_factor(K0, c.C)
    dK = np.max(np.abs(K - K0))
    tol_kij = 4.0 * np.max(np.sum(np.abs(c.C), axis=0)) * dK
    assert np.max(np.abs(Kij - Kij0)) <= tol_kij, (np.max(np.abs(Kij - Kij0)), tol_kij)
    Linv = np.linalg.inv(np.linalg.cholesky(Kij0))
    nL = np.linalg.norm(Linv, 2)
    cond = np.linalg.cond(Kij0)
    tol_xi = 4.0 * (dK * c.N * nL + np.max(np.abs(K0)) * c.N * nL * cond
                    * tol_kij / np.linalg.norm(Kij0, 2))
    assert np.max(np.abs(xi - xi0)) <= tol_xi, (np.max(np.abs(xi - xi0)), tol_xi)


@pytest.mark.slow
def test_config2(xk):
    """64-centre supercell (the benchmark workload): E_x within 1e-6 Ha."""
    _check(xk, load_cell(config_spec(2)))


@pytest.mark.slow
def test_config2_scf_steps(xk):
    """The benchmark's pseudo-SCF coefficients (seed 1000, steps 0 to 202):
    |dE_x| <= 1e-6 Ha and max|dK| <= 1e-6 against the FP64 path at every
    sampled step (with two-piece orbital products one of these steps missed
    by 1.4e-6 Ha)."""
    from cellgen import pseudo_scf_sequence
    c = load_cell(config_spec(2))
    Cs = pseudo_scf_sequence(c.S, c.C, 203, 1000)
    hf = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="fp64")
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode="f16x3")
    try:
        for t in (0, 52, 102, 152, 202):
            K0, E0 = hf.build(Cs[t])
            K, E = h.build(Cs[t])
            assert abs(E - E0) <= TOL_E, (t, E - E0)
            assert np.max(np.abs(K - K0)) <= TOL_K, (t, np.max(np.abs(K - K0)))
    finally:
        hf.release()
        h.release()


@pytest.mark.slow
def test_config2_n256(xk):
    """The n > 128 path (stored T = f V o P as FP16 hi/lo, three tensor-core
    GEMMs, three-piece orbitals) at a full-size grid: the 64-centre cell
    (N_g = 60^3, N_aux = 4000) with n = 256, against the FP64 path on the same
    tables (the FP64 path is held to the oracle at 1e-8 Ha on these cells):
    |dE_x| <= 1e-6 Ha, max|dK| <= 1e-6, and the per-build error estimate."""
    from cellgen.cells import draw_coefficients
    c = load_cell(config_spec(2))
    C = draw_coefficients(c.S, 256, 2256)  # 256 S-orthonormal columns on the same tables
    hf = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, 256, mode="fp64")
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, 256, mode="f16x3")
    try:
        K0, E0 = hf.build(C)
        K, E = h.build(C)
        est = h.error_estimate()
        Ee = h.energy(C)
        K2, E2 = h.build(C)
    finally:
        hf.release()
        h.release()
    assert abs(E - E0) <= TOL_E, (E, E0)
    assert np.max(np.abs(K - K0)) <= TOL_K, np.max(np.abs(K - K0))
    assert Ee == E
    assert np.array_equal(K, K2) and E == E2
    assert abs(est - abs(E + float(np.sum(K * C)))) <= 1e-10
