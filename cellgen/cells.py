"""Seeded synthetic periodic cells: every input of the exchange build.

This module prepares inputs only.  It builds the geometry, evaluates the
periodised Gaussian basis on the uniform grid, draws S-orthonormal occupied
coefficients, selects ISDF interpolation points, fits the ISDF functions and
forms the auxiliary Coulomb tables V and W.  None of the exchange-build
arithmetic (orbital products, V o P, the three robust-PS lines, K, E_x) lives
here; both the CPU oracle and the GPU library consume what this module makes.

Paper conventions followed (arXiv 2207.04636):
  * uniform grid R = n_i a_i / N_i, flat index (ix*N2 + iy)*N3 + iz  (Sec. II.A.2)
  * periodised Gaussians phi_P(r) = sum_T phi(r + T)                  (Sec. II.A.3)
  * Coulomb kernel 4*pi/G^2 with the G = 0 term removed               (Eq. cou, Sec. IV.E)
  * ISDF: pivots of the pair matrix rho_{mu nu, R}, least-squares fit
    X_{g'g} chi_{gR} = X_{g'R} with X = (Phi_g Phi^T) o (Phi_g Phi^T)  (Eq. isdf, Eq. lsqfit)
  * two-stage point selection: per-atom Voronoi candidates, then a
    global pivoting over their union                                  (Sec. IV.C)
  * V(R_g, R) = potential of chi_g (Eq. rpsPot); W(g, g') = sum_R V(g,R) chi_g'(R) (Eq. thcpot)
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
from typing import Optional

import numpy as np
import scipy.fft
import scipy.linalg
import scipy.linalg.lapack

GENERATOR_VERSION = "cellgen-1"

# Diamond conventional cell: FCC sites plus the (1/4,1/4,1/4) basis shift.
_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
DIAMOND_FRAC = np.concatenate([_FCC, _FCC + 0.25])


@dataclasses.dataclass
class Shell:
    """One shell on every centre: angular momentum l (0, 1 or 2), primitive
    exponents and contraction coefficients of normalised primitives."""
    l: int
    exps: tuple
    coefs: tuple


@dataclasses.dataclass
class CellSpec:
    """Recipe of one synthetic cell (lengths in bohr)."""
    name: str
    frac: np.ndarray          # fractional centre coordinates, (ncentre, 3)
    L: float                  # cubic cell edge
    grid: int                 # points per edge, N_g = grid**3
    shells: list              # list[Shell], the same on every centre
    n_occ: int
    n_aux: int
    seed: int
    jitter: float = 0.05
    isdf: str = "auto"        # "exact" | "voronoi" | "auto"

    def key(self) -> str:
        h = hashlib.sha256()
        h.update(GENERATOR_VERSION.encode())
        h.update(np.ascontiguousarray(self.frac, dtype=np.float64).tobytes())
        h.update(repr((self.L, self.grid, [(s.l, tuple(map(float, s.exps)),
                                            tuple(map(float, s.coefs))) for s in self.shells],
                       self.n_occ, self.n_aux, self.seed, self.jitter, self.isdf)).encode())
        return f"{self.name}_{h.hexdigest()[:16]}"


@dataclasses.dataclass
class Cell:
    """A generated cell.  Arrays are float64 / int32 and C-contiguous.

    phi  : (N_g, N) basis values on the grid, row = grid point
    S    : (N, N) grid overlap dV * phi^T phi
    C    : (N, n) occupied coefficients with C^T S C = I
    idx  : (N_aux,) interpolation points as flat grid indices, ascending
    V    : (N_aux, N_g) potentials of the ISDF functions (None when not fitted)
    W    : (N_aux, N_aux) symmetric THC potential (None when not fitted)
    chi  : (N_aux, N_g) ISDF functions, or None when not kept
    """
    spec: CellSpec
    centres: np.ndarray
    dV: float
    phi: np.ndarray
    S: np.ndarray
    C: np.ndarray
    idx: np.ndarray
    V: np.ndarray
    W: np.ndarray
    chi: Optional[np.ndarray]
    ridge: float
    cond_S: float

    @property
    def Ng(self) -> int:
        return self.phi.shape[0]

    @property
    def N(self) -> int:
        return self.phi.shape[1]

    @property
    def n(self) -> int:
        return self.C.shape[1]

    @property
    def Naux(self) -> int:
        return self.idx.shape[0]

    @property
    def L(self) -> float:
        return self.spec.L

    @property
    def grid(self) -> int:
        return self.spec.grid


# --------------------------------------------------------------------------
# Configurations (sizes shaped like the paper's diamond workloads, Sec. V)
# --------------------------------------------------------------------------

def _diamond_frac(reps: int) -> np.ndarray:
    out = []
    for a in range(reps):
        for b in range(reps):
            for c in range(reps):
                out.append((DIAMOND_FRAC + np.array([a, b, c])) / reps)
    return np.concatenate(out)


def _cubic_frac(k: int) -> np.ndarray:
    g = (np.arange(k) + 0.5) / k
    return np.array([[x, y, z] for x in g for y in g for z in g])


def shells13(rng: np.random.Generator) -> list:
    """2s,2p,1d shells (2 + 6 + 5 = 13 functions with real spherical d),
    one log-uniform exponent in [0.15, 3.0] per shell."""
    a = np.exp(rng.uniform(math.log(0.15), math.log(3.0), size=5))
    return [Shell(0, (float(a[0]),), (1.0,)), Shell(0, (float(a[1]),), (1.0,)),
            Shell(1, (float(a[2]),), (1.0,)), Shell(1, (float(a[3]),), (1.0,)),
            Shell(2, (float(a[4]),), (1.0,))]


CUBIC_SIZES = (8, 27, 64, 125, 216)


def config_spec(config: int, instance: int = 0, k: Optional[int] = None) -> CellSpec:
    """The seeded workload configurations.

    1: 8-centre diamond cell, L=6.74, N=32, n=16, 24^3 grid, N_aux=256.
    2: 64-centre 2x2x2 diamond supercell, L=13.48, N=832, n=128, 60^3, N_aux=4000.
    3: 216-centre 3x3x3 diamond supercell, L=20.22, N=2808, n=432, 90^3, N_aux=13500.
    4: simple-cubic k^3 cell (k = 2..6), spacing 3.37, 13 functions and 2
       occupied orbitals per centre, (15k)^3 grid, N_aux = 5N.
    Seed = 1000*config + instance (+ 100*k for config 4).
    """
    seed = 1000 * config + instance
    if config == 1:
        shells = [Shell(0, (0.25, 0.9), (1.0, 1.0)), Shell(1, (0.5,), (1.0,))]
        return CellSpec("diamond8", _diamond_frac(1), 6.74, 24, shells, 16, 256, seed)
    if config in (2, 3):
        reps = 2 if config == 2 else 3
        shells = shells13(np.random.default_rng(seed + 500))
        n_centre = 8 * reps ** 3
        naux = 4000 if config == 2 else 13500
        grid = 60 if config == 2 else 90
        return CellSpec(f"diamond{n_centre}", _diamond_frac(reps), 6.74 * reps, grid,
                        shells, 2 * n_centre, naux, seed)
    if config == 4:
        if k is None:
            raise ValueError("config 4 needs the lattice size k")
        seed = seed + 100 * k
        shells = shells13(np.random.default_rng(seed + 500))
        n_centre = k ** 3
        return CellSpec(f"cubic{n_centre}", _cubic_frac(k), 3.37 * k, 15 * k, shells,
                        2 * n_centre, 5 * 13 * n_centre, seed)
    raise ValueError(f"unknown configuration {config}")


# --------------------------------------------------------------------------
# Basis on the grid (separable periodic lattice sums)
# --------------------------------------------------------------------------

def _periodic_1d(x: np.ndarray, A: float, L: float, alpha: float) -> np.ndarray:
    """g_k(x) = sum_t (x - A + tL)^k exp(-alpha (x - A + tL)^2), k = 0, 1, 2,
    summed over images until the Gaussian is below 1e-18 in the cell."""
    rcut = math.sqrt(math.log(1e18) / alpha)
    tmax = int(math.ceil(rcut / L)) + 1
    out = np.zeros((3, x.size))
    for t in range(-tmax, tmax + 1):
        d = x - A + t * L
        e = np.exp(-alpha * d * d)
        out[0] += e
        out[1] += d * e
        out[2] += d * d * e
    return out


def _outer3(fx, fy, fz) -> np.ndarray:
    return (fx[:, None, None] * fy[None, :, None] * fz[None, None, :]).reshape(-1)


def _gauss_moments(a: float):
    """I_k = int x^(2k) exp(-2 a x^2) dx for k = 0, 1, 2."""
    i0 = math.sqrt(math.pi / (2 * a))
    return i0, i0 / (4 * a), 3 * i0 / (4 * a) ** 2


def _shell_functions(x: np.ndarray, A: np.ndarray, L: float, sh: Shell) -> list:
    """Grid values of the functions of one shell on one centre.  Each
    primitive is normalised in R^3; a contracted s shell is renormalised with
    the analytic primitive overlap (2 sqrt(ab)/(a+b))^(3/2)."""
    nfun = {0: 1, 1: 3, 2: 5}[sh.l]
    acc = [np.zeros(x.size ** 3) for _ in range(nfun)]
    for a, c in zip(sh.exps, sh.coefs):
        g = [_periodic_1d(x, A[ax], L, a) for ax in range(3)]
        g0 = [gi[0] for gi in g]
        g1 = [gi[1] for gi in g]
        g2 = [gi[2] for gi in g]
        i0, i1, i2 = _gauss_moments(a)
        if sh.l == 0:
            acc[0] += (c / math.sqrt(i0 ** 3)) * _outer3(g0[0], g0[1], g0[2])
        elif sh.l == 1:
            nrm = c / math.sqrt(i1 * i0 * i0)
            acc[0] += nrm * _outer3(g1[0], g0[1], g0[2])
            acc[1] += nrm * _outer3(g0[0], g1[1], g0[2])
            acc[2] += nrm * _outer3(g0[0], g0[1], g1[2])
        else:
            n_xy = c / math.sqrt(i1 * i1 * i0)
            n_x2y2 = c / math.sqrt(2 * i2 * i0 * i0 - 2 * i1 * i1 * i0)
            n_z2 = c / math.sqrt(6 * i2 * i0 * i0 - 6 * i1 * i1 * i0)
            acc[0] += n_xy * _outer3(g1[0], g1[1], g0[2])
            acc[1] += n_xy * _outer3(g0[0], g1[1], g1[2])
            acc[2] += n_xy * _outer3(g1[0], g0[1], g1[2])
            acc[3] += n_x2y2 * (_outer3(g2[0], g0[1], g0[2]) - _outer3(g0[0], g2[1], g0[2]))
            acc[4] += n_z2 * (2 * _outer3(g0[0], g0[1], g2[2]) - _outer3(g2[0], g0[1], g0[2])
                              - _outer3(g0[0], g2[1], g0[2]))
    if sh.l == 0 and len(sh.exps) > 1:
        norm2 = 0.0
        for a, ca in zip(sh.exps, sh.coefs):
            for b, cb in zip(sh.exps, sh.coefs):
                norm2 += ca * cb * (2 * math.sqrt(a * b) / (a + b)) ** 1.5
        acc[0] /= math.sqrt(norm2)
    return acc


def basis_on_grid(centres: np.ndarray, L: float, grid: int, shells: list) -> np.ndarray:
    """Phi[R, mu] of the periodised Gaussians (Sec. II.A.3).  The cell is
    cubic and every Cartesian Gaussian factorises over the axes, so the
    lattice sum is taken per axis.  Function order per centre: shells in
    order; p as (x, y, z); d as (xy, yz, xz, x^2-y^2, 3z^2-r^2)."""
    x = np.arange(grid) * (L / grid)
    nfun = sum({0: 1, 1: 3, 2: 5}[s.l] for s in shells) * len(centres)
    phi = np.empty((grid ** 3, nfun))
    col = 0
    for A in centres:
        for sh in shells:
            for f in _shell_functions(x, A, L, sh):
                phi[:, col] = f
                col += 1
    return phi


# --------------------------------------------------------------------------
# Poisson solve on the grid (setup only: potentials of the ISDF functions)
# --------------------------------------------------------------------------

def coulomb_kernel_g(L: float, grid: int) -> np.ndarray:
    """4 pi / |G|^2 on the FFT frequency grid, G = 0 entry set to zero."""
    g1 = 2 * np.pi * np.fft.fftfreq(grid, d=L / grid)
    g2 = g1[:, None, None] ** 2 + g1[None, :, None] ** 2 + g1[None, None, :] ** 2
    with np.errstate(divide="ignore"):
        k = 4 * np.pi / g2
    k[0, 0, 0] = 0.0
    return k


def potentials(rows: np.ndarray, L: float, grid: int, workers: int = -1) -> np.ndarray:
    """sum_R' v(R - R') f(R') for each row f of `rows` (Eq. cou-1):
    the inverse transform of (4 pi / G^2) times the forward transform."""
    k = coulomb_kernel_g(L, grid)
    out = np.empty_like(rows)
    block = 64
    for s in range(0, rows.shape[0], block):
        f = rows[s:s + block].reshape(-1, grid, grid, grid)
        fg = scipy.fft.fftn(f, axes=(1, 2, 3), workers=workers)
        fg *= k
        out[s:s + block] = scipy.fft.ifftn(fg, axes=(1, 2, 3), workers=workers).real.reshape(
            f.shape[0], -1)
    return out


# --------------------------------------------------------------------------
# ISDF setup (Sec. III.A and IV.C)
# --------------------------------------------------------------------------

def _pivoted_cholesky(X: np.ndarray, want: int) -> np.ndarray:
    """Leading pivots of a complete-pivoting Cholesky of the PSD Gram X.
    In exact arithmetic these equal the column pivots of QRCP on the pair
    matrix whose Gram is X (Sec. III.A)."""
    c, piv, rank, info = scipy.linalg.lapack.dpstrf(X, tol=1e-14 * float(np.max(np.diag(X))),
                                                     lower=1)
    if info < 0:
        raise RuntimeError(f"dpstrf failed: info={info}")
    take = min(want, int(rank))
    return np.asarray(piv[:take], dtype=np.int64) - 1


def _pair_gram(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = (A B^T) o (A B^T): the Gram of the pair products (Eq. lsqfit)."""
    G = A @ B.T
    return G * G


def select_points_exact(phi: np.ndarray, n_aux: int) -> np.ndarray:
    """Pivoted Cholesky of the full pair Gram over every grid point."""
    X = _pair_gram(phi, phi)
    return _pivoted_cholesky(X, n_aux)


def select_points_voronoi(phi: np.ndarray, centres: np.ndarray, L: float, grid: int,
                          n_aux: int, per_atom: int) -> np.ndarray:
    """Two-stage selection (Sec. IV.C): per-atom candidates from the grid
    points of each Voronoi cell, then a global pivoting over their union.
    Exact local pair Grams replace the paper's randomised sketch."""
    x = np.arange(grid) * (L / grid)
    pts = np.stack(np.meshgrid(x, x, x, indexing="ij"), axis=-1).reshape(-1, 3)
    best = np.full(pts.shape[0], np.inf)
    owner = np.zeros(pts.shape[0], dtype=np.int64)
    for I, A in enumerate(centres):
        d = pts - A
        d -= L * np.round(d / L)
        r2 = np.einsum("ij,ij->i", d, d)
        m = r2 < best
        best[m] = r2[m]
        owner[m] = I
    cand = []
    for I in range(len(centres)):
        loc = np.nonzero(owner == I)[0]
        piv = _pivoted_cholesky(_pair_gram(phi[loc], phi[loc]), per_atom)
        cand.append(loc[piv])
    cand = np.unique(np.concatenate(cand))
    piv = _pivoted_cholesky(_pair_gram(phi[cand], phi[cand]), n_aux)
    return cand[piv]


def fit_isdf(phi: np.ndarray, idx: np.ndarray, block: int = 16384):
    """chi = X_gg^{-1} X_gR by Cholesky (Eq. lsqfit).  A ridge of
    1e-14 tr(X_gg)/N_aux is added only if the plain factorisation fails."""
    phig = phi[idx]
    Xgg = _pair_gram(phig, phig)
    ridge = 0.0
    try:
        cf = scipy.linalg.cho_factor(Xgg, lower=True)
    except np.linalg.LinAlgError:
        ridge = 1e-14 * float(np.trace(Xgg)) / Xgg.shape[0]
        cf = scipy.linalg.cho_factor(Xgg + ridge * np.eye(Xgg.shape[0]), lower=True)
    chi = np.empty((idx.size, phi.shape[0]))
    for s in range(0, phi.shape[0], block):
        chi[:, s:s + block] = scipy.linalg.cho_solve(cf, _pair_gram(phig, phi[s:s + block]))
    return chi, ridge


def thc_potential(V: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """W(g, g') = sum_R V(g, R) chi_g'(R) (Eq. thcpot), symmetrised; the
    exact W is symmetric because the Coulomb kernel is."""
    W = V @ chi.T
    return 0.5 * (W + W.T)


# --------------------------------------------------------------------------
# Occupied coefficients
# --------------------------------------------------------------------------

def s_orthonormal(S: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """C = S^{-1/2} Q with Q from the QR of Z, so that C^T S C = I."""
    w, U = np.linalg.eigh(S)
    s_mhalf = (U / np.sqrt(w)) @ U.T
    Q, _ = np.linalg.qr(Z)
    return np.ascontiguousarray(s_mhalf @ Q)


def draw_coefficients(S: np.ndarray, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return s_orthonormal(S, rng.standard_normal((S.shape[0], n)))


def perturb_coefficients(S: np.ndarray, C: np.ndarray, seed: int, step: float = 0.05) -> np.ndarray:
    """One pseudo-SCF update C <- S-orthonormalise(C + step * noise)."""
    rng = np.random.default_rng(seed)
    return s_orthonormal(S, C + step * rng.standard_normal(C.shape))


def pseudo_scf_sequence(S: np.ndarray, C0: np.ndarray, count: int, seed: int,
                        step: float = 0.05) -> list:
    """count coefficient matrices of a seeded pseudo-SCF run: C_0 = C0 and
    C_{t+1} = S^{-1/2} qr(S^{1/2} C_t + step * noise).Q, i.e. each step adds
    noise in the orthonormal frame and re-orthonormalises in S."""
    w, U = np.linalg.eigh(S)
    s_half = (U * np.sqrt(w)) @ U.T
    s_mhalf = (U / np.sqrt(w)) @ U.T
    rng = np.random.default_rng(seed)
    out = [np.ascontiguousarray(C0)]
    X = s_half @ C0
    for _ in range(count - 1):
        X, _ = np.linalg.qr(X + step * rng.standard_normal(X.shape))
        out.append(np.ascontiguousarray(s_mhalf @ X))
    return out


# --------------------------------------------------------------------------
# Cell assembly
# --------------------------------------------------------------------------

def build_cell(spec: CellSpec, keep_chi: bool = False, idx: Optional[np.ndarray] = None,
               fit: bool = True) -> Cell:
    """Generate every input of one cell from its spec (deterministic in the seed).
    With fit=False the ISDF fit, V and W are left out (V = W = None): the basis,
    the coefficients and the interpolation points only, for a set-up that forms
    the tables elsewhere."""
    rng = np.random.default_rng(spec.seed)
    jit = rng.uniform(-spec.jitter, spec.jitter, size=spec.frac.shape)
    centres = spec.frac * spec.L + jit
    Ng = spec.grid ** 3
    dV = spec.L ** 3 / Ng
    phi = basis_on_grid(centres, spec.L, spec.grid, spec.shells)
    S = dV * (phi.T @ phi)
    ev = np.linalg.eigvalsh(S)
    cond_S = float(ev[-1] / ev[0])
    if not cond_S < 1e10:
        raise RuntimeError(f"basis is numerically linearly dependent: cond(S)={cond_S:.3e}")
    C = draw_coefficients(S, spec.n_occ, spec.seed + 1)
    if idx is None:
        mode = spec.isdf
        if mode == "auto":
            mode = "exact" if Ng <= 20000 else "voronoi"
        if mode == "exact":
            idx = select_points_exact(phi, spec.n_aux)
        else:
            c = spec.n_aux / phi.shape[1]
            n_i = phi.shape[1] // len(centres)
            idx = select_points_voronoi(phi, centres, spec.L, spec.grid, spec.n_aux,
                                        int(math.ceil(c * n_i)) + 10)
    idx = np.sort(np.asarray(idx, dtype=np.int64))
    if idx.size < spec.n_aux:
        raise RuntimeError(f"only {idx.size} independent interpolation points (< {spec.n_aux})")
    if not fit:
        return Cell(spec, centres, dV, np.ascontiguousarray(phi), S, C, idx.astype(np.int32),
                    None, None, None, 0.0, cond_S)
    chi, ridge = fit_isdf(phi, idx)
    V = potentials(chi, spec.L, spec.grid)
    W = thc_potential(V, chi)
    return Cell(spec, centres, dV, np.ascontiguousarray(phi), S, C,
                idx.astype(np.int32), V, W, chi if keep_chi else None, ridge, cond_S)


def cache_dir() -> str:
    return os.environ.get("XK_CELL_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "xk_cells"))


def load_cell(spec: CellSpec, keep_chi: bool = False, use_cache: bool = True) -> Cell:
    """build_cell with an on-disk cache keyed by the spec and generator version."""
    if not use_cache or keep_chi:
        return build_cell(spec, keep_chi=keep_chi)
    d = os.path.join(cache_dir(), spec.key())
    names = ("centres", "phi", "S", "C", "idx", "V", "W", "meta")
    if all(os.path.exists(os.path.join(d, f + ".npy")) for f in names):
        a = {f: np.load(os.path.join(d, f + ".npy")) for f in names}
        dV, ridge, cond_S = (float(v) for v in a["meta"])
        return Cell(spec, a["centres"], dV, a["phi"], a["S"], a["C"], a["idx"], a["V"],
                    a["W"], None, ridge, cond_S)
    cell = build_cell(spec)
    try:
        os.makedirs(d, exist_ok=True)
        for f in names[:-1]:
            tmp = os.path.join(d, f + ".tmp.npy")
            np.save(tmp, getattr(cell, f))
            os.replace(tmp, os.path.join(d, f + ".npy"))
        np.save(os.path.join(d, "meta.npy"), np.array([cell.dV, cell.ridge, cell.cond_S]))
    except OSError:
        pass
    return cell
