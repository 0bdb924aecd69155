"""Parity of the FP64 GPU path (through the C ABI) with the CPU oracle.

Tolerances are the ones the exchange build is held to in FP64:
|dE_x| <= 1e-8 Ha and max|dK_{mu i}| <= 1e-7.
"""
import numpy as np
import pytest

import oracle
from cellgen import CellSpec, Shell, build_cell, config_spec, load_cell

pytestmark = pytest.mark.gpu

TOL_E, TOL_K = 1e-8, 1e-7


@pytest.fixture(scope="module")
def xk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_04636_gb300 as m
    return m


def _check(xk, c, mode="fp64"):
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode=mode)
    try:
        K, E = h.build(c.C)
        Ee = h.energy(c.C)
    finally:
        h.release()
    assert abs(E - E0) <= TOL_E, (E, E0)
    assert np.max(np.abs(K - K0)) <= TOL_K
    # E_x alone from the closed form -dV (2 sum V o P^2 - sum W o Q^2)
    assert abs(Ee - E0) <= TOL_E, (Ee, E0)
    return K, E


def _spec(name, frac, L, grid, shells, n, naux, seed):
    return CellSpec(name, np.asarray(frac, dtype=float), L, grid, shells, n, naux, seed)


def test_config1_full(xk, cell1):
    """8-centre diamond cell: every element of K_{mu i} and E_x."""
    before = xk.kernel_launches()
    _check(xk, cell1)
    assert xk.kernel_launches() > before


def test_ragged_sizes(xk):
    """Sizes off every tile multiple: N_g = 13^3, N = 3*(1+3+5)=27, n = 7, N_aux = 97."""
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    c = build_cell(_spec("ragged", [[0.1, 0.2, 0.3], [0.6, 0.5, 0.45], [0.3, 0.75, 0.8]], 6.5, 13,
                         sh, 7, 97, 9001))
    _check(xk, c)


@pytest.mark.parametrize("n,naux", [(1, 20), (6, 1), (6, 6)])
def test_degenerate_sizes(xk, n, naux):
    """One occupied orbital, one interpolation point, n = N."""
    sh = [Shell(0, (0.4,), (1.0,)), Shell(0, (1.3,), (1.0,)), Shell(0, (0.2,), (1.0,))]
    c = build_cell(_spec("degen", [[0.2, 0.3, 0.25], [0.7, 0.6, 0.55]], 5.0, 10, sh, n,
                         max(naux, 1), 9100 + n))
    if naux < c.Naux:
        from cellgen import fit_isdf, potentials, thc_potential
        idx = np.sort(c.idx[:naux])
        chi, _ = fit_isdf(c.phi, idx)
        c.V = potentials(chi, c.L, c.grid)
        c.W = thc_potential(c.V, chi)
        c.idx = idx.astype(np.int32)
    _check(xk, c)


def test_deterministic(xk, cell1):
    """Fixed reduction order: two builds are bitwise identical."""
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n)
    K1, E1 = h.build(c.C)
    K2, E2 = h.build(c.C)
    h.release()
    assert np.array_equal(K1, K2) and E1 == E2


def test_build_device_matches(xk, cell1):
    """xk_build_device on torch device buffers equals the host-buffer build."""
    torch = pytest.importorskip("torch")
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n)
    K0, E0 = h.build(c.C)
    Cd = torch.from_numpy(c.C).cuda()
    Kd = torch.empty_like(Cd)
    Ed = torch.empty(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    h.build_device(Cd.data_ptr(), Kd.data_ptr(), Ed.data_ptr(), s.cuda_stream)
    s.synchronize()
    h.release()
    assert np.array_equal(Kd.cpu().numpy(), K0) and float(Ed.item()) == E0


def test_ace_matches_oracle(xk, cell1):
    """occ-RI K_ij and its Cholesky (ACE) factor on the device vs the oracle."""
    c = cell1
    K0, _ = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    Kij0, xi0, s0, br0 = oracle.ace_factor(K0, c.C)
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n)
    h.build(c.C)
    Kij, xi, s, br = h.ace()
    h.release()
    assert br == br0 == "cholesky"
    assert np.max(np.abs(Kij - Kij0)) <= 1e-9 * np.max(np.abs(Kij0))
    assert np.max(np.abs(xi - xi0)) <= 1e-7 * np.max(np.abs(xi0))


@pytest.mark.parametrize("mode", ["fp64", "f16x3"])
def test_energy_leaves_build_state(xk, cell1, mode):
    """xk_energy with other coefficients neither changes the last build's
    K_ij / ACE factor nor its own result when repeated."""
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n, mode=mode)
    h.build(c.C)
    ref = h.ace()
    rng = np.random.default_rng(5)
    C2 = c.C + 0.05 * rng.standard_normal(c.C.shape)
    e1 = h.energy(C2)
    e2 = h.energy(C2)
    after = h.ace()
    _, E2 = h.build(C2)
    h.release()
    assert e1 == e2
    assert abs(e1 - E2) <= (TOL_E if mode == "fp64" else 0.0)
    for a, b in zip(ref[:3], after[:3]):
        assert np.array_equal(a, b)
    assert ref[3] == after[3]


def test_full_k(xk, cell1):
    """xk_build_full (Eq. rpsEx, all three terms of Eq. rps) against the
    oracle's K_{mu nu}; symmetric, and K C is the occ-RI rectangle."""
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    rag = build_cell(_spec("ragged", [[0.1, 0.2, 0.3], [0.6, 0.5, 0.45], [0.3, 0.75, 0.8]], 6.5,
                           13, sh, 7, 97, 9001))
    for c in (cell1, rag):
        Kf0 = oracle.exx_rps_full(c.phi, c.idx, c.V, c.W, c.C, c.dV)
        h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n)
        K, _ = h.build(c.C)
        Kf = h.build_full(c.C)
        h.release()
        assert np.max(np.abs(Kf - Kf0)) <= TOL_K
        assert np.max(np.abs(Kf - Kf.T)) <= 1e-12 * np.max(np.abs(Kf))
        assert np.max(np.abs(Kf @ c.C - K)) <= 1e-10 * np.max(np.abs(K))


def test_coulomb_j(xk, cell1):
    """xk_coulomb (density, DFT-based Poisson solve, J = dV Phi^T diag(v) Phi,
    all FP64) against the oracle's J and E_J; a ragged 13^3 grid too."""
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    rag = build_cell(_spec("ragged", [[0.1, 0.2, 0.3], [0.6, 0.5, 0.45], [0.3, 0.75, 0.8]], 6.5,
                           13, sh, 7, 97, 9001))
    for c in (cell1, rag):
        J0, EJ0 = oracle.coulomb_j(c.phi, c.C, c.L, c.grid, c.dV)
        h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n)
        J, EJ = h.coulomb(c.C, c.grid, c.L)
        J2, EJ2 = h.coulomb(c.C, c.grid, c.L)
        with pytest.raises(xk.XKError):
            h.coulomb(c.C, c.grid + 1, c.L)
        h.release()
        assert np.max(np.abs(J - J0)) <= 1e-10 * np.max(np.abs(J0))
        assert abs(EJ - EJ0) <= 1e-10 * abs(EJ0)
        assert np.array_equal(J, J2) and EJ == EJ2


def test_ace_eigen_branch(xk):
    """A C whose K_ij is indefinite takes the eigen branch; the factor still
    reproduces K_{mu i} on the occupied space: (xi diag(s) xi^T) C = K_{mu i}."""
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,))]
    c = build_cell(_spec("indef", [[0.1, 0.2, 0.3], [0.6, 0.5, 0.45]], 6.0, 12, sh, 4, 30, 9300))
    V, W = -c.V, -c.W  # K -> -K: K_ij is negative definite, Cholesky must fail
    K0, _ = oracle.exx_rps_occri(c.phi, c.idx, V, W, c.C, c.dV)
    _, _, s0, br0 = oracle.ace_factor(K0, c.C)
    h = xk.Handle(c.phi, c.idx, V, W, c.dV, c.n)
    K, _ = h.build(c.C)
    Kij, xi, s, br = h.ace()
    h.release()
    assert br == br0 == "eigen"
    assert np.all(s == -1.0) and np.all(s0 == -1.0)
    assert np.max(np.abs((xi * s) @ xi.T @ c.C - K)) <= 1e-8 * np.max(np.abs(K))


def test_submit_poll_alone_and_mixed(xk, cell1):
    """Serving: builds of two cells of different sizes submitted together give
    the same results as each built alone (bitwise in FP64)."""
    a = cell1
    sh = [Shell(0, (0.35,), (1.0,)), Shell(1, (0.8,), (1.0,)), Shell(2, (1.1,), (1.0,))]
    b = build_cell(_spec("ragged", [[0.1, 0.2, 0.3], [0.6, 0.5, 0.45], [0.3, 0.75, 0.8]], 6.5,
                         13, sh, 7, 97, 9001))
    ha = xk.Handle(a.phi, a.idx, a.V, a.W, a.dV, a.n)
    hb = xk.Handle(b.phi, b.idx, b.V, b.W, b.dV, b.n)
    Ka, Ea = ha.build(a.C)
    Kb, Eb = hb.build(b.C)
    rng = np.random.default_rng(1)
    Ca2 = a.C + 0.01 * rng.standard_normal(a.C.shape)
    Ka2, Ea2 = ha.build(Ca2)
    tickets = [(ha.submit(a.C), a, Ka, Ea), (hb.submit(b.C), b, Kb, Eb),
               (ha.submit(Ca2), a, Ka2, Ea2), (hb.submit(b.C), b, Kb, Eb)]
    for t, c, Kref, Eref in tickets:
        while True:
            st, K, E, eb = xk.poll(t, c.N, c.n)
            if st == xk.XK_OK:
                break
        assert np.array_equal(K, Kref) and E == Eref and eb == 0.0
    ha.release()
    hb.release()


def test_submit_busy_and_deadline(xk, cell1):
    """All four slots in flight -> XK_EBUSY; an expired ticket deadline ->
    XK_ETIMEDOUT from xk_poll (a host-side deadline; the GPU is not stalled)."""
    c = cell1
    h = xk.Handle(c.phi, c.idx, c.V, c.W, c.dV, c.n)
    ts = [h.submit(c.C) for _ in range(4)]
    with pytest.raises(xk.XKError) as e:
        h.submit(c.C)
    assert e.value.code == xk.XK_EBUSY
    for t in ts:
        while xk.poll(t, c.N, c.n)[0] == xk.XK_PENDING:
            pass
    t = h.submit(c.C, deadline_ms=1e-9)
    import time
    time.sleep(0.001)
    try:
        st = xk.poll(t, c.N, c.n)[0]
        assert st in (xk.XK_OK,)   # finished before anyone looked: still fine
    except xk.XKError as err:
        assert err.code == xk.XK_ETIMEDOUT
    h.release()


@pytest.mark.slow
def test_config2_full(xk):
    """64-centre diamond supercell (N=832, n=128, 60^3 grid, N_aux=4000): the
    whole K_{mu i} and E_x against the oracle, at the size the benchmark runs."""
    c = load_cell(config_spec(2))
    _check(xk, c)
