"""FP64 CPU oracle of the ISDF set-up (test infrastructure only).

Imported by tests/ only; the GPU library never imports or calls it.

Point selection (Sec. III.A): greedy complete-pivoting Cholesky of the pair
Gram X(R, R') = (phi(R) . phi(R'))^2 over candidate points, written
left-looking: at step t the pivot is the largest remaining diagonal (the
first one on ties), its column is X(:, p) minus the contributions of the
earlier columns, and the diagonal drops by the new column squared; it stops
when the largest remaining diagonal is at most tol_rel times the largest
initial one.  In exact arithmetic these are the column pivots of QRCP on the
pair matrix.

Given the basis on the grid and the interpolation points, it forms the
tables the exchange build consumes, in the order of Sec. III.A and Sec. IV.C
of arXiv 2207.04636:

  X_gg  = (Phi_g Phi_g^T) o (Phi_g Phi_g^T)            (Eq. lsqfit, N_aux x N_aux)
  X_gR  = (Phi_g Phi^T) o (Phi_g Phi^T)                 (Eq. lsqfit, N_aux x N_g)
  chi   = X_gg^{-1} X_gR  by a Cholesky factorisation   (the least-squares fit)
  V     = Pois(chi_g) for every g                        (Eq. rpsPot, one FFT pair each)
  W     = V chi^T, symmetrised                           (Eq. thcpot)

If the plain Cholesky factorisation of X_gg fails, a ridge of
1e-14 tr(X_gg) / N_aux is added to its diagonal (and reported).
"""
import numpy as np
import scipy.linalg

from .poisson import coulomb_potential


def isdf_tables(phi: np.ndarray, idx: np.ndarray, L: float, grid: int):
    """(chi, V, W, ridge) for the interpolation points idx."""
    phig = phi[idx]
    Gg = phig @ phig.T
    Xgg = Gg * Gg
    GR = phig @ phi.T
    XgR = GR * GR
    ridge = 0.0
    try:
        cf = scipy.linalg.cho_factor(Xgg, lower=True)
    except np.linalg.LinAlgError:
        ridge = 1e-14 * float(np.trace(Xgg)) / Xgg.shape[0]
        cf = scipy.linalg.cho_factor(Xgg + ridge * np.eye(Xgg.shape[0]), lower=True)
    chi = scipy.linalg.cho_solve(cf, XgR)
    V = coulomb_potential(chi, L, grid)
    W = V @ chi.T
    return chi, V, 0.5 * (W + W.T), ridge


def select_points(rows: np.ndarray, want: int, tol_rel: float = 1e-14) -> np.ndarray:
    """Pivots (indices into rows, in selection order) of the greedy pivoted
    Cholesky of X = (rows rows^T) o (rows rows^T)."""
    m = rows.shape[0]
    d = np.einsum("ij,ij->i", rows, rows) ** 2
    tol = tol_rel * float(d.max())
    Lc = np.zeros((m, want))
    piv = []
    alive = np.ones(m, dtype=bool)
    for t in range(want):
        dm = np.where(alive, d, -np.inf)
        p = int(np.argmax(dm))
        if not dm[p] > tol:
            break
        col = (rows @ rows[p]) ** 2 - Lc[:, :t] @ Lc[p, :t]
        Lc[:, t] = col / np.sqrt(dm[p])
        d = d - Lc[:, t] ** 2
        alive[p] = False
        piv.append(p)
    return np.asarray(piv, dtype=np.int64)
