"""CPU oracle of the robust-pseudospectral occ-RI exchange build (FP64).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and
the CPU-baseline / reference legs of bench.py; the GPU library never imports,
links or calls anything here, and nothing here calls the library.

Everything follows arXiv 2207.04636 with one overall factor dV = Omega/N_g on
every robust-PS term (the reading of the paper's 1/Omega, N_g/Omega and
missing prefactors that makes Eq. 2eint the grid form of the Coulomb
integral):

  Psi   = Phi C,  Psi_g = Psi[idx]                       (Eq. rpsEx step 1)
  P     = Psi_g Psi^T          (N_aux x N_g)             (Eq. rpsEx step 2)
  V2    = V o P                                          (Eq. rpsEx step 3)
  line1 = (Psi_g^T V2) Phi                               (Eq. exoccri, 1st line)
  line2 = (V2 Psi)^T Phi_g     (order (a) of Sec. IV.D)  (Eq. exoccri, 2nd line)
  line3 = ((W o (Psi_g Psi_g^T)) Psi_g)^T Phi_g          (Eq. exoccri, 3rd line)
  K_{j nu} = dV (line1 + line2 - line3);  K_{mu i} = K^T (Eq. exoccri, Eq. rps signs)
  E_x   = - sum_{j nu} K_{j nu} C_{nu j}   (closed-shell, D = C C^T, Sec. II.C)

Functions and their pins (tests/test_oracle_pins.py):
  exx_rps_occri     : P1 (exact limit), P2 (full-rank fit), P3 (== 4-index
                      definition), P4 (quadratic error), P5 (decay in N_aux),
                      P6 (symmetry), P7 (E_x < 0), P8 (closed form), P9
                      (invariances)
  exx_rps_4index    : P3, P6 (full K_{mu nu} symmetric)
  exx_rps_full      : == exx_rps_4index's K_{mu nu}; symmetric; K C equals
                      the occ-RI rectangle
  coulomb_j         : == the literal 4-index grid integrals contracted with D;
                      E_J = tr(C^T J C) > 0
  exx_exact_fft     : P1, P2, P7 (K PSD); Poisson pinned by P10
  exx_energy_direct : P8
  ace_factor        : reconstruction and definiteness checks
"""
import math

import numpy as np

from .poisson import coulomb_potential


# --------------------------------------------------------------------------
# robust-PS occ-RI exchange, Eq. exoccri
# --------------------------------------------------------------------------

def orbitals(phi: np.ndarray, C: np.ndarray, idx: np.ndarray):
    """Occupied orbitals on all grid points and at the interpolation points
    (Eq. rpsEx step 1; R_g is a subset of the grid, so Psi_g is a gather)."""
    psi = phi @ C
    return psi, psi[idx]


def rps_lines(phi, idx, V, W, C, gblock: int = 512):
    """The three lines of Eq. exoccri, each an (n x N) array, without dV.

    line1[j,nu] = sum_R' (sum_g psi_j(R_g) V(g,R') P(g,R')) phi_nu(R')
    line2[j,nu] = sum_g  (sum_R psi_j(R)  V(g,R)  P(g,R))  phi_nu(R_g)
    line3[j,nu] = sum_g' (sum_g psi_j(R_g) W(g,g') Q(g,g')) phi_nu(R_g')
    with P(g,R) = sum_i psi_i(R_g) psi_i(R), Q(g,g') = sum_i psi_i(R_g) psi_i(R_g').
    The g index is processed in blocks only to bound memory.
    """
    psi, psig = orbitals(phi, C, idx)
    phig = phi[idx]
    naux, ng = V.shape
    n = C.shape[1]
    M1 = np.zeros((n, ng))            # M1[j,R'] = sum_g psi_j(R_g) V2(g,R')
    M2 = np.zeros((naux, n))          # M2[g,j]  = sum_R V2(g,R) psi_j(R)
    for s in range(0, naux, gblock):
        e = min(s + gblock, naux)
        P = psig[s:e] @ psi.T         # step 2: pair kernel at (R_g, R)
        V2 = V[s:e] * P               # step 3: Hadamard with the stored potentials
        M2[s:e] = V2 @ psi            # line 2, first contraction (over R)
        M1 += psig[s:e].T @ V2        # line 1, first contraction (over R_g)
    line1 = M1 @ phi                  # line 1, contraction over R'
    line2 = M2.T @ phig               # line 2, contraction over R_g
    Q = psig @ psig.T
    M3 = (W * Q) @ psig               # line 3, first contraction (over R_g)
    line3 = M3.T @ phig               # line 3, contraction over R_g'
    return line1, line2, line3


def exchange_energy(Kmui: np.ndarray, C: np.ndarray) -> float:
    """E_x = - sum_{nu,j} K_{nu j} C_{nu j}, summed with math.fsum."""
    return -math.fsum((Kmui * C).ravel().tolist())


def exx_rps_occri(phi, idx, V, W, C, dV, gblock: int = 512):
    """K_{mu i} (N x n) and E_x of the robust-PS occ-RI build (Eq. exoccri)."""
    l1, l2, l3 = rps_lines(phi, idx, V, W, C, gblock)
    K = dV * (l1 + l2 - l3)           # K_{j nu}
    Kmui = np.ascontiguousarray(K.T)
    return Kmui, exchange_energy(Kmui, C)


def exx_variant(phi, idx, V, W, C, dV, which: str):
    """Single-term approximations of Sec. III.B, for the error-order pins:
    'ps'   : first line of Eq. rps only (pseudospectral, not symmetric)
    'sps'  : average of the first two lines (symmetrised pseudospectral)
    'thc'  : third line of Eq. rps only (tensor hypercontraction)."""
    l1, l2, l3 = rps_lines(phi, idx, V, W, C)
    K = {"ps": l1, "sps": 0.5 * (l1 + l2), "thc": l3}[which] * dV
    Kmui = np.ascontiguousarray(K.T)
    return Kmui, exchange_energy(Kmui, C)


def exx_energy_direct(phi, idx, V, W, C, dV, gblock: int = 512) -> float:
    """E_x from contracting Eq. exoccri with C in closed form:
    E_x = -dV (2 sum_{g,R} V(g,R) P(g,R)^2 - sum_{g,g'} W(g,g') Q(g,g')^2)."""
    psi, psig = orbitals(phi, C, idx)
    acc = []
    for s in range(0, V.shape[0], gblock):
        P = psig[s:s + gblock] @ psi.T
        acc.append(float(np.sum(V[s:s + gblock] * P * P)))
    Q = psig @ psig.T
    return -dV * (2.0 * math.fsum(acc) - float(np.sum(W * Q * Q)))


# --------------------------------------------------------------------------
# Full exchange matrix K_{mu nu} with the robust-PS integrals (Eq. rpsEx)
# --------------------------------------------------------------------------

def exx_rps_full(phi, idx, V, W, C, dV, gblock: int = 512):
    """K_{mu nu} (N x N) of Eq. rpsEx with all three terms of Eq. rps, in the
    order of the steps listed after Eq. rpsEx for the first term:
      rho(g,R') = sum_i psi_i(R_g) psi_i(R')  (= P),   V2 = V o rho,
      M_mu(R') = sum_g V2(g,R') phi_mu(R_g),   term1 = sum_R' M_mu(R') phi_nu(R');
    the second term of Eq. rps (rho_{mu lam} at R, rho_{sig nu} at R_g) the
    same way with the roles of R_g and R exchanged, and the third with W and
    Q(g,g') = sum_i psi_i(R_g) psi_i(R_g') between interpolation points:
      K = dV (term1 + term2 - term3)."""
    psi, psig = orbitals(phi, C, idx)
    phig = phi[idx]
    naux, ng = V.shape
    N = phi.shape[1]
    M = np.zeros((N, ng))             # M[mu,R'] = sum_g phi_mu(R_g) V2(g,R')
    M2 = np.zeros((naux, N))          # M2[g,mu] = sum_R V2(g,R) phi_mu(R)
    for s in range(0, naux, gblock):
        e = min(s + gblock, naux)
        rho = psig[s:e] @ psi.T       # step 2
        V2 = V[s:e] * rho             # step 3
        M += phig[s:e].T @ V2         # step 4 (first term)
        M2[s:e] = V2 @ phi            # second term: sum over R first
    term1 = M @ phi                   # step 5: contraction over R'
    term2 = M2.T @ phig               # second term: contraction over R_g
    Q = psig @ psig.T
    term3 = phig.T @ ((W * Q) @ phig)
    return dV * (term1 + term2 - term3)


# --------------------------------------------------------------------------
# Definition check: the robust-PS 4-index integrals, Eq. rps (tiny cells)
# --------------------------------------------------------------------------

def rps_eri(phi, idx, V, W, dV):
    """(mu nu|lam sig) = T1 + T2 - T3 of Eq. rps as an (N^2 x N^2) matrix
    over pair indices (mu nu), (lam sig):
      T1 = dV sum_g sum_R' rho_{mu nu}(R_g) V(g,R') rho_{lam sig}(R')
      T2 = dV sum_R sum_g  rho_{mu nu}(R)  V(g,R)  rho_{lam sig}(R_g)
      T3 = dV sum_g sum_g' rho_{mu nu}(R_g) W(g,g') rho_{lam sig}(R_g')
    with rho_{mu nu}(R) = phi_mu(R) phi_nu(R) (Eq. isdf, diagonal approximation)."""
    N = phi.shape[1]
    rho = np.einsum("rm,rn->mnr", phi, phi).reshape(N * N, -1)    # (N^2, N_g)
    rhog = rho[:, idx]                                            # (N^2, N_aux)
    T1 = rhog @ V @ rho.T
    T2 = rho @ V.T @ rhog.T
    T3 = rhog @ W @ rhog.T
    return dV * (T1 + T2 - T3)


def exx_rps_4index(phi, idx, V, W, C, dV):
    """K_{mu nu} = sum_{lam sig} D_{lam sig} (mu lam|sig nu), D = C C^T, from the
    literal 4-index robust-PS integrals; returns (K_{mu nu}, K_{mu i} = K C, E_x)."""
    N = phi.shape[1]
    eri = rps_eri(phi, idx, V, W, dV).reshape(N, N, N, N)        # (mu lam | sig nu)
    D = C @ C.T
    K = np.einsum("mlsn,ls->mn", eri, D)
    Kmui = K @ C
    return K, Kmui, exchange_energy(Kmui, C)


# --------------------------------------------------------------------------
# Coulomb matrix on the same grid (the comparison partner of Sec. IV.E)
# --------------------------------------------------------------------------

def coulomb_j(phi, C, L, grid, dV):
    """J_{mu nu} = sum_{lam sig} D_{lam sig} (mu nu|lam sig) with D = C C^T and
    the grid integrals of Eq. 2eint: the density rho(R) = sum_i psi_i(R)^2 on
    the grid, its potential Pois(rho) (Eq. cou-1, one FFT pair), then
    J = dV Phi^T diag(Pois(rho)) Phi.  Returns (J, E_J) with
    E_J = sum_{ij} (ii|jj) = dV sum_R rho(R) Pois(rho)(R)."""
    psi = phi @ C
    rho = np.sum(psi * psi, axis=1)
    v = coulomb_potential(rho, L, grid)
    J = dV * (phi.T @ (v[:, None] * phi))
    return J, dV * math.fsum((rho * v).tolist())


# --------------------------------------------------------------------------
# Brute-force exact grid exchange: the conventional FFT route, Eq. exchange
# --------------------------------------------------------------------------

def exx_exact_fft(phi, C, L, grid, dV):
    """K_{mu nu} = dV sum_i sum_R phi_mu(R) psi_i(R) Pois(psi_i phi_nu)(R)
    (Eq. exchange: N*n Poisson solves); returns (K_{mu nu}, K_{mu i} = K C, E_x)."""
    psi = phi @ C
    N, n = C.shape
    K = np.zeros((N, N))
    for i in range(n):
        rho = (psi[:, i][:, None] * phi).T                       # (N, N_g): psi_i phi_nu
        pot = coulomb_potential(rho, L, grid)                     # (N, N_g)
        K += dV * ((phi * psi[:, i][:, None]).T @ pot.T)          # [mu, nu]
    Kmui = K @ C
    return K, Kmui, exchange_energy(Kmui, C)


def exact_exchange_energy(phi, C, L, grid, dV) -> float:
    """E_x = -dV sum_{ij} sum_R psi_i psi_j Pois(psi_i psi_j) with n^2 solves;
    an independent route to the exact energy."""
    psi = phi @ C
    n = C.shape[1]
    acc = []
    for i in range(n):
        rho = psi[:, i][None, :] * psi.T                          # (n, N_g)
        pot = coulomb_potential(rho, L, grid)
        acc.append(float(np.sum(rho * pot)))
    return -dV * math.fsum(acc)


# --------------------------------------------------------------------------
# occ-RI K_ij and its factorisation (ACE form), Sec. III.C
# --------------------------------------------------------------------------

def ace_factor(Kmui: np.ndarray, C: np.ndarray, cutoff: float = 1e-12):
    """K_ij = C^T K_{mu i}, symmetrised; factor K_ij = L L^T by Cholesky when
    it is positive definite, else by eigendecomposition keeping eigenvalues
    with |lambda| > cutoff * max|lambda|.  Returns (K_ij, xi, sign, branch)
    with the ACE vectors xi = K_{mu i} L^{-T} (Cholesky) or
    K_{mu i} U |Lambda|^{-1/2} (eigen), so K ~ xi diag(sign) xi^T on the
    occupied space."""
    Kij = C.T @ Kmui
    Kij = 0.5 * (Kij + Kij.T)
    try:
        Lc = np.linalg.cholesky(Kij)
        xi = np.linalg.solve(Lc, Kmui.T).T
        return Kij, xi, np.ones(Kij.shape[0]), "cholesky"
    except np.linalg.LinAlgError:
        lam, U = np.linalg.eigh(Kij)
        keep = np.abs(lam) > cutoff * np.max(np.abs(lam))
        xi = Kmui @ (U[:, keep] / np.sqrt(np.abs(lam[keep])))
        return Kij, xi, np.sign(lam[keep]), "eigen"
