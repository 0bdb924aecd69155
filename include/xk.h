/*
 * xk.h -- C ABI of the GB300 robust-pseudospectral occ-RI exchange build.
 *
 * The library evaluates, for one periodic cell whose auxiliary tables are
 * kept in device memory, the occ-RI exchange rectangle of arXiv 2207.04636,
 * Eq. exoccri (Sec. III.C, with the robust-PS integrals of Eq. rps,
 * Sec. III.B), and the exchange energy:
 *
 *   Psi   = Phi C,  Psi_g = Psi[idx]                     (Eq. rpsEx, step 1)
 *   P     = Psi_g Psi^T,  V2 = V o P                     (Eq. rpsEx, steps 2-3)
 *   line1 = (Psi_g^T V2) Phi                             (Eq. exoccri, line 1)
 *   line2 = (V2 Psi)^T Phi_g   (contraction order (a), Sec. IV.D)
 *   line3 = ((W o (Psi_g Psi_g^T)) Psi_g)^T Phi_g        (Eq. exoccri, line 3)
 *   K_{mu i} = dV (line1 + line2 - line3)^T,   E_x = -sum_{mu,i} K_{mu i} C_{mu i}
 *
 * One factor dV = Omega / N_g multiplies every term (the grid form of the
 * Coulomb integral, Eq. 2eint).  No FFT runs inside a build: V and W are
 * computed once per geometry by the caller (Eq. rpsPot, Eq. thcpot).
 *
 * Entry points: set-up and release (xk_footprint, xk_setup, xk_setup_shard, xk_setup_isdf,
 * xk_isdf_points, xk_tables, xk_release); admission (xk_setup_queued,
 * xk_admit_reserve, xk_admit_release, xk_admit_state); builds (xk_build, xk_build_device,
 * xk_ace); serving (xk_submit, xk_poll) and batches (xk_batch_create,
 * xk_batch_build, xk_batch_release); other products on the same tables
 * (xk_energy, xk_energy_device, xk_build_full, xk_coulomb,
 * xk_exchange_energy_noalloc); diagnostics and control (xk_last_error,
 * xk_kernel_launches, xk_timing_enable, xk_timing_read, xk_set_wait_limit,
 * xk_autotune_info).
 *
 * Conventions for every entry point:
 *   - All matrices are row-major, double precision, densely packed.
 *   - Host pointers are owned by the caller; the library copies what it
 *     needs before returning (xk_setup, xk_build, xk_submit) and never keeps
 *     a caller pointer.  Device pointers (xk_build_device) stay owned by the
 *     caller and must stay valid until the work on the given stream is done.
 *   - Return codes only; nothing throws across this boundary.  On failure
 *     xk_last_error() gives a message for the calling thread.
 *   - Grid points are flat indices (ix*N2 + iy)*N3 + iz of the uniform grid
 *     (Sec. II.A.2); the library only needs Phi and V to agree on them.
 */
#ifndef XK_H
#define XK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xk_handle xk_handle;
typedef uint64_t xk_ticket;

enum {
  XK_OK = 0,
  XK_PENDING = 1,     /* xk_poll: the build is still running              */
  XK_EINVAL = -1,     /* bad shape, null pointer, bad index, bad table     */
  XK_ENOMEM = -2,     /* footprint beyond the admission budget; retry later */
  XK_ETIMEDOUT = -3,  /* a bounded wait or a ticket deadline expired       */
  XK_ECUDA = -4,      /* any other CUDA error (message in xk_last_error)   */
  XK_EBUSY = -5       /* every submission slot of the handle is in use     */
};

enum {
  XK_FP64 = 0,        /* every step in FP64 on the CUDA cores               */
  XK_TF32 = 1,        /* reserved, rejected by xk_setup                      */
  XK_F16X3 = 2        /* bulk contractions on the tcgen05 tensor cores with
                         operands split into FP16 pieces: a fixed-point main
                         piece whose products accumulate exactly in FP32 and
                         an FP16 remainder (three products per pair of
                         operands), FP64 cross-tile sums, FP64 K and E_x.
                         E_x is returned in the closed form
                         -dV (2 sum V o P^2 - sum W o Q^2) (Eq. exoccri
                         contracted with C), accumulated from the pair
                         products.  n <= 128: one fused kernel, P never
                         stored; n > 128: T = V o P stored as FP16 hi/lo
                         (4 N_aux (N_g + N_aux) bytes more) and contracted
                         by three tensor-core GEMMs.                        */
};

/*
 * Device bytes one handle of this shape and mode holds (tables + scratch).
 * This is the paper's extra memory cost O(N_chi N_g) of the stored
 * potentials (Sec. IV, memory column of the cost table), plus scratch.
 * Returns XK_EINVAL on non-positive sizes or an unknown mode.
 */
int xk_footprint(int64_t Ng, int32_t N, int32_t n, int32_t Naux, int mode, size_t* bytes);

/*
 * Copy the per-geometry tables to the current CUDA device and return a
 * handle.  Inputs (host memory, read only, may be freed after return):
 *   basis_on_points  Ng x N      Phi[R, mu] = phi_mu(R)        (Sec. II.A.3)
 *   interp_idx       Naux        grid index of each R_g, each in [0, Ng),
 *                                no duplicates                  (Eq. isdf)
 *   V_aux            Naux x Ng   V(R_g, R), potential of chi_g  (Eq. rpsPot)
 *   W_aux            Naux x Naux W(R_g, R_g'), symmetric        (Eq. thcpot)
 *   dV               Omega / N_g, > 0
 *   mode             XK_FP64 or XK_F16X3
 * Errors: XK_EINVAL (sizes, null pointers, idx out of range or duplicated,
 * W not symmetric to 1e-12 relative, dV <= 0, n > N, Naux > Ng; for
 * XK_F16X3 also basis columns linearly dependent on the grid),
 * XK_ENOMEM (footprint above the admission budget: free device memory less
 * a reserve, or XK_HBM_BUDGET_BYTES when set), XK_ECUDA.
 */
int xk_setup(int64_t Ng, int32_t N, int32_t n, int32_t Naux,
             const double* basis_on_points, const int32_t* interp_idx,
             const double* V_aux, const double* W_aux,
             double dV, int mode, xk_handle** out);

/*
 * A shard of the build for a g-partitioned multi-GPU run (one process per
 * GPU).  Every term of Eq. exoccri is a sum over the interpolation points g
 * (lines 1 and 2 over the g of V o P, line 3 over the g of the rows of
 * W o Q), so the build splits over g-slices with no exchange until the end:
 * the shard holds the rows [g0, g1) of V and of W, the whole basis table and
 * all Naux interpolation points (the orbitals at every point are needed for
 * the g' of W o Q), and each build returns the slice's share of K_{mu i} and
 * of E_x.  The shares of a partition of [0, Naux) sum to the full build's K
 * and E_x: one allreduce of the N x n K and one scalar (Sec. IV.B-D: the
 * paper also keeps the O(n N_chi N) contraction of order (a) local).
 *   interp_idx  Naux, all interpolation points (as in xk_setup)
 *   V_rows      (g1 - g0) x Ng: rows g0 .. g1-1 of V_aux
 *   W_rows      (g1 - g0) x Naux: rows g0 .. g1-1 of W_aux (all columns)
 * Other arguments and the device tables as in xk_setup; the footprint is
 * that of the slice.  A shard handle builds (xk_build, xk_build_device,
 * xk_submit, xk_energy: partial E_x, batches); xk_build_full, xk_ace and
 * xk_tables return XK_EINVAL for it (they need the summed K or all rows).
 * xk_poll's and xk_error_estimate's estimate is that of the share.
 * Errors: as xk_setup, plus XK_EINVAL unless 0 <= g0 < g1 <= Naux; W is
 * checked for symmetry on its block [g0, g1) x [g0, g1).
 */
int xk_setup_shard(int64_t Ng, int32_t N, int32_t n, int32_t Naux, int32_t g0, int32_t g1,
                   const double* basis_on_points, const int32_t* interp_idx,
                   const double* V_rows, const double* W_rows, double dV, int mode,
                   xk_handle** out);

/*
 * Queued admission for serving many SCF runs on one device (each run holds
 * its tables for its lifetime; the paper's SCF loop, Sec. IV.F).  Every
 * handle's footprint (xk_footprint) counts against an admission budget: the
 * device's free memory less a 1 GiB reserve and, when the environment
 * variable XK_HBM_BUDGET_BYTES is set, that many bytes less the footprints of
 * the live handles and reservations (checked first, with no device call).
 * xk_setup and the other set-ups refuse a footprint above the budget at once
 * (XK_ENOMEM).  xk_setup_queued instead waits: requests queue in arrival
 * order, the oldest is admitted as soon as its footprint fits (xk_release and
 * xk_admit_release wake the queue; device memory freed elsewhere is seen
 * within 50 ms), later ones wait behind it, and a request still waiting after
 * timeout_ms milliseconds leaves the queue with XK_ETIMEDOUT.  Arguments
 * otherwise as xk_setup; the calling thread blocks while it waits.
 * Errors: as xk_setup; XK_EINVAL for a negative or non-finite timeout_ms;
 * XK_ENOMEM at once for a footprint above XK_HBM_BUDGET_BYTES itself;
 * XK_ETIMEDOUT when not admitted in time.
 */
int xk_setup_queued(int64_t Ng, int32_t N, int32_t n, int32_t Naux,
                    const double* basis_on_points, const int32_t* interp_idx,
                    const double* V_aux, const double* W_aux, double dV, int mode,
                    double timeout_ms, xk_handle** out);

/*
 * A reservation of `bytes` against the same admission budget (host
 * bookkeeping, no device memory): for memory the caller allocates itself
 * next to the handles.  timeout_ms < 0 admits now or fails with XK_ENOMEM;
 * otherwise the request queues with the set-ups as in xk_setup_queued.
 * Without XK_HBM_BUDGET_BYTES the budget is the current device's free memory
 * less 1 GiB and less the live reservations.  *token identifies the
 * reservation for xk_admit_release, which returns its bytes and wakes the
 * queue.  Errors: XK_EINVAL (NULL token, non-finite timeout, unknown token),
 * XK_ENOMEM, XK_ETIMEDOUT, XK_ECUDA (device query).
 */
int xk_admit_reserve(uint64_t bytes, double timeout_ms, uint64_t* token);
int xk_admit_release(uint64_t token);

/*
 * Bytes currently admitted (live handles, their extra buffers and the
 * reservations) and the number of requests waiting in the admission queue.
 * Errors: XK_EINVAL (NULL argument).
 */
int xk_admit_state(uint64_t* admitted_bytes, uint32_t* waiting);

/*
 * The same set-up with the ISDF tables formed on the device in FP64 from the
 * basis and the interpolation points (Sec. III.A, IV.C): on a cubic cell of
 * side L with grid^3 = N_g points (flat order as above, dV = L^3 / N_g),
 *   X_gg = (Phi_g Phi_g^T) o (Phi_g Phi_g^T),  X_gR = (Phi_g Phi^T) o (Phi_g Phi^T),
 *   chi  = X_gg^{-1} X_gR  (Eq. lsqfit: blocked Cholesky and two blocked solves;
 *          a ridge of 1e-14 tr(X_gg) / N_aux when the plain factorisation fails),
 *   V    = Pois(chi_g) with the grid kernel 4 pi / G^2, G = 0 removed (Eq. rpsPot),
 *   W    = V chi^T, symmetrised (Eq. thcpot),
 * and then the handle as xk_setup would build it from those V and W.  The
 * points interp_idx come from the caller (e.g. xk_isdf_points).  XK_FP64 forms the
 * tables in the handle's own buffers; XK_F16X3 holds FP64 temporaries of
 * about 8 (N_g N + 2 N_aux N_g + 2 N_aux^2) bytes during the call, admitted
 * with the handle.  Errors: as xk_setup, plus XK_EINVAL when grid^3 != N_g,
 * L <= 0 or X_gg is not positive definite even with the ridge.
 */
int xk_setup_isdf(int64_t Ng, int32_t N, int32_t n, int32_t Naux,
                  const double* basis_on_points, const int32_t* interp_idx,
                  int32_t grid, double L, int mode, xk_handle** out);

/*
 * Interpolation points on the GPU (Sec. III.A): the greedy complete-pivoting
 * Cholesky of the pair Gram X(a, b) = (rows_a . rows_b)^2 over m candidate
 * grid points (rows: host, m x N, the basis at the candidates), in FP64.
 * At each step the pivot is the largest remaining diagonal (the first on
 * ties); it stops after `want` pivots or when the largest remaining diagonal
 * is at most tol_rel times the largest initial one (1e-14 is the usual
 * choice).  In exact arithmetic these are the column pivots of QRCP on the
 * pair matrix.  piv_out (host, want) receives the pivots as indices into
 * rows, in selection order; *count the number taken.  A two-stage selection
 * (Sec. IV.C: per-atom candidates, then a global pivoting over their union)
 * is two levels of calls.  Scratch: about 8 (m^2 + m want + m N) bytes of
 * device memory during the call (admission as xk_setup).
 * Errors: XK_EINVAL (null pointers, sizes <= 0, bad tol_rel), XK_ENOMEM,
 * XK_ECUDA.
 */
int xk_isdf_points(int32_t m, int32_t N, const double* rows, int32_t want, double tol_rel,
                   int32_t* piv_out, int32_t* count);

/*
 * Read back tables of an XK_FP64 handle (e.g. those xk_setup_isdf formed):
 * W_out (host, N_aux x N_aux, nullable), the rows rows[0..nrows) of V into
 * V_rows_out (host, nrows x N_g; nrows may be 0), and the ridge added to
 * X_gg (nullable; 0 for xk_setup handles).  Errors: XK_EINVAL (null handle,
 * XK_F16X3 handle, bad rows), XK_ECUDA.
 */
int xk_tables(xk_handle* h, double* W_out, const int32_t* rows, int32_t nrows,
              double* V_rows_out, double* ridge);

/*
 * One exchange build, blocking.  C (host, N x n) are the occupied
 * coefficients; K_out (host, N x n) receives K_{mu i}; Ex (host) receives
 * E_x.  Builds on one handle are serialised.
 * Errors: XK_EINVAL (null pointers), XK_ECUDA.
 */
int xk_build(xk_handle* h, const double* C, double* K_out, double* Ex);

/*
 * The same build on device memory, enqueued on `stream` (a cudaStream_t,
 * NULL = the legacy default stream) and returning at once.  C_dev (N x n),
 * K_dev (N x n) and Ex_dev (1 double) are device pointers owned by the
 * caller.  The handle's scratch is reused, so builds on one handle must not
 * overlap: enqueue them on one stream.  Errors: XK_EINVAL, XK_ECUDA.
 */
int xk_build_device(xk_handle* h, const double* C_dev, double* K_dev, double* Ex_dev,
                    void* stream);

/*
 * The full exchange matrix K_{mu nu} (N x N) with the robust-PS integrals,
 * for the one non-occ-RI build at the end of an SCF run (Eq. rpsEx with all
 * three terms of Eq. rps, Sec. III.B-C):
 *   K = dV (Phi_g^T (V o P) Phi + Phi^T (V o P)^T Phi_g - Phi_g^T (W o Q) Phi_g),
 *   P = Psi_g Psi^T,  Q = Psi_g Psi_g^T,  Psi = Phi C.
 * It is symmetric (to rounding) and K C equals the K_{mu i} of xk_build.
 * The contractions run over the grid first (M = (V o P) Phi, N_aux x N),
 * O(N N_aux N_g) work against the occ-RI build's O(n N_aux N_g).
 * XK_FP64: every product in FP64.  XK_F16X3: V o P and W o Q stored as hi/lo
 * FP16 and contracted on the tensor cores; the first call on a handle
 * allocates about 4 N_aux (N_g + N_aux) bytes of extra device memory (on top
 * of xk_footprint; admitted like xk_setup: XK_ENOMEM when it does not fit).
 * C (host, N x n) is copied; K_out (host, N x N, row-major) receives K.
 * Neither the last build's K_{mu i} nor the state xk_ace reads is touched.
 * Errors: XK_EINVAL (null pointers), XK_ENOMEM, XK_ETIMEDOUT, XK_ECUDA.
 */
int xk_build_full(xk_handle* h, const double* C, double* K_out);

/*
 * Coulomb matrix on the same grid tables (the comparison partner of the
 * exchange build, Sec. IV.E), for a cubic cell of side L with grid^3 = N_g
 * points in the flat order of xk_setup:
 *   rho(R) = sum_i psi_i(R)^2,  v = Pois(rho) (Eq. cou-1: 4 pi / G^2 on the
 *   grid's reciprocal vectors G = 2 pi m / L, G = 0 removed),
 *   J = dV Phi^T diag(v) Phi,   E_J = sum_ij (ii|jj) = dV sum_R rho(R) v(R),
 * with D = C C^T as for E_x (closed shell: E_2e = 2 E_J + E_x).  The Poisson
 * solve is a 3-D DFT done as three passes of 1-D DFTs in FP64 (O(g) per
 * output, no FFT library); everything runs in FP64.  XK_FP64 handles only
 * (the tensor-path handle keeps no FP64 basis table).  The first call
 * allocates about 8 N_g (N + 6) bytes of scratch, admitted like xk_setup.
 * C (host, N x n) is copied; J_out (host, N x N) and E_J (host) receive the
 * results.  Errors: XK_EINVAL (null pointers, XK_F16X3 handle,
 * grid^3 != N_g, L <= 0), XK_ENOMEM, XK_ECUDA.
 */
int xk_coulomb(xk_handle* h, int32_t grid, double L, const double* C, double* J_out,
               double* E_J);

/*
 * The exchange energy alone, without K (a cheap convergence monitor between
 * full builds): Eq. exoccri contracted with C gives the closed form
 *   E_x = -dV (2 sum_{g,R} V(g,R) P(g,R)^2 - sum_{g,g'} W(g,g') Q(g,g')^2),
 *   P = Psi_g Psi^T,  Q = Psi_g Psi_g^T,  Psi = Phi C,
 * (line 1 and line 2 each contribute the V term, line 3 the W term).  Only
 * the orbitals and the pair products run: no second product and no line
 * contraction.  XK_FP64: P and Q in FP64 and the two weighted sums of
 * squares in FP64.  XK_F16X3: the pair kernel's S products and energy sums
 * with the same splits and summation order as xk_build, so for n <= 128 the
 * value equals the E_x of xk_build bit for bit (n > 128: the same T-product
 * energy sums, also bit for bit).  C (host, N x n) is copied; Ex (host)
 * receives E_x.  Neither K nor the state xk_ace reads is touched.
 * Errors: XK_EINVAL (null pointers), XK_ETIMEDOUT (a bounded wait inside a
 * kernel gave up), XK_ECUDA.
 */
int xk_energy(xk_handle* h, const double* C, double* Ex);

/*
 * xk_energy on device memory, enqueued on `stream` (cudaStream_t, NULL =
 * legacy default) and returning at once: C_dev (N x n) and Ex_dev (1 double)
 * are caller-owned device pointers.  Errors: XK_EINVAL, XK_ECUDA.
 */
int xk_energy_device(xk_handle* h, const double* C_dev, double* Ex_dev, void* stream);

/*
 * occ-RI K_ij of the last completed build on this handle and its ACE
 * factorisation (Sec. III.C), computed on the device in FP64:
 * K_ij = C^T K_{mu i} symmetrised; Cholesky K_ij = L L^T when it is positive
 * definite (branch 0, xi = K_{mu i} L^{-T}, K ~ xi xi^T on the occupied
 * space), else a Jacobi eigendecomposition keeping |lambda| > 1e-12 max|lambda|
 * (branch 1, xi = K_{mu i} U |Lambda|^{-1/2}; sign_out gets sign(lambda),
 * zero for dropped columns).  Outputs are host memory: Kij_out n x n,
 * xi_out N x n, sign_out n (nullable), branch (nullable).
 * Errors: XK_EINVAL (no build yet, null pointers), XK_ECUDA.
 */
int xk_ace(xk_handle* h, double* Kij_out, double* xi_out, double* sign_out, int* branch);

/*
 * Serving: enqueue a build and return a ticket at once.  C is copied into a
 * pinned slot before return.  Each handle runs its builds in order on its
 * own stream, so builds of different handles (different SCF runs, cells of
 * different sizes) overlap on the GPU.  deadline_ms > 0 sets how long the
 * ticket may stay pending before xk_poll reports XK_ETIMEDOUT (0 = none).
 * Errors: XK_EINVAL, XK_EBUSY (all slots of the handle in flight), XK_ECUDA.
 */
int xk_submit(xk_handle* h, const double* C, double deadline_ms, xk_ticket* t);

/*
 * Non-blocking completion check.  XK_PENDING while the build runs;
 * XK_OK once done, after copying K_{mu i} (N x n) to K_out and E_x to Ex.
 * err_est (nullable) receives this build's a-posteriori error estimate
 * |E_x - E_K|, where E_K = -sum_{mu,i} K_{mu i} C_{mu i} is the energy of the
 * returned K (computed on the device in FP64, fixed order) and E_x the
 * returned energy.  For XK_FP64 the two are the same number (0).  For
 * XK_F16X3, E_x is the closed form of Eq. exoccri contracted with C,
 * formed from the exact pair products, while K carries the rounding of the
 * split FP16 back-contractions: the gap estimates the error of K on the
 * occupied space (it tracks |E_K - E_x(FP64)| to within the much smaller
 * error of the closed form).  The parity tests hold E_x to 1e-6 Ha and K to
 * 1e-6 against the FP64 path.  A ticket is consumed by the XK_OK,
 * XK_ETIMEDOUT or XK_ECUDA result.  XK_EINVAL for an unknown ticket.
 */
int xk_poll(xk_ticket t, double* K_out, double* Ex, double* err_est);

/*
 * The error estimate of xk_poll for the last build enqueued on the handle by
 * xk_build or xk_build_device (waits for the handle's stream): |E_x - E_K|
 * with E_K = -sum K o C of the returned K; 0 for XK_FP64.  Errors: XK_EINVAL
 * (NULL argument, no build yet), XK_ECUDA.
 */
int xk_error_estimate(xk_handle* h, double* est);

/*
 * What the set-up's autotuner chose for an XK_F16X3 handle (it times its own
 * launches on its own sizes when the handle is created):
 *   info[0]  width of the n > 128 back-contraction tiles, 128 or 256 (0 for
 *            n <= 128); the faster of the two, 256 unless 128 is 3 % faster;
 *            XK_BACK_TILES=128 or 256 in the environment fixes it
 *   info[1]  the K split of M2 (the role-A split for n <= 64)
 *   ms[0..2] set-up timing (ms) of the 128- and 256-column back-contraction
 *            shapes, and of the tuned pair launch for n <= 64 (0 when not timed)
 * info: 2 int32, ms: 3 doubles, caller-owned.  Errors: XK_EINVAL (NULL
 * argument, XK_FP64 handle).
 */
int xk_autotune_info(xk_handle* h, int32_t* info, double* ms);

/*
 * Free every device and host resource of the handle (waits for its work).
 * Tickets of the handle still pending become unknown.  It takes the handle's
 * lock, so it waits for a call already inside the handle, but the caller
 * must not start xk_submit or xk_poll on the handle (or its tickets) while
 * xk_release runs: the handle's memory is gone when it returns.
 */
int xk_release(xk_handle* h);

/*
 * Bound, in SM clock cycles, on every pipeline wait inside the handle's
 * tensor-core kernels (a TMA stage, an MMA result, an epilogue hand-off);
 * 0 restores the default of 2e9 cycles (about one second).  A wait that runs
 * out makes its kernel record a code, stop its loops, wait (with the default
 * bound) for its own TMA copies and MMAs, free its tensor memory and return;
 * the build then reports XK_ETIMEDOUT and the handle stays usable.  Applies
 * to builds enqueued afterwards (a batch keeps the limit its members had
 * when it was created).  No effect on XK_FP64 handles, whose kernels do not
 * wait on one another.  It exists so that the timeout path can be exercised
 * (a tiny limit) and so that a caller can bound a build more tightly than
 * one second per wait.  Errors: XK_EINVAL (NULL handle, negative cycles).
 */
int xk_set_wait_limit(xk_handle* h, int64_t cycles);

/*
 * Batches: one exchange build for each of several handles (cells of
 * different sizes, different SCF runs) as one unit of device work.  The
 * paper builds one cell at a time; a batch is the grouped, launch-bound
 * form of the same per-iteration step (Eq. exoccri for every member).
 *   xk_batch_create   handles: count distinct XK_F16X3 handles on one device;
 *                     the batch keeps pointers to them (release the batch
 *                     before any of its handles).
 *   xk_batch_build    C[i] (host, N_i x n_i) -> K_out[i] (host, N_i x n_i),
 *                     Ex_out[i]; blocking.  The device work of the whole
 *                     batch (every member's orbitals, one grouped pair launch
 *                     over all members with n <= 128, the line steps) is
 *                     captured into a CUDA graph on the first call and
 *                     replayed afterwards; results equal xk_build's bitwise.
 * Errors: XK_EINVAL (NULL pointers, empty or repeated handles, FP64 handles,
 * handles on different devices), XK_ETIMEDOUT, XK_ECUDA.
 */
typedef struct xk_batch xk_batch;
int xk_batch_create(xk_handle* const* handles, int count, xk_batch** out);
int xk_batch_build(xk_batch* b, const double* const* C, double* const* K_out, double* Ex_out);
int xk_batch_release(xk_batch* b);

/* Message of the last failure on the calling thread ("" if none). */
const char* xk_last_error(void);

/*
 * Steps of a build, for xk_timing_read.  XK_STEP_PAIR covers the pair
 * kernel P and the Hadamard with V (Eq. rpsEx, steps 2-3); in the
 * mixed-precision path it also covers M2 and M1, which one fused kernel
 * computes, and XK_STEP_M2 / XK_STEP_M1 stay at zero.
 */
enum {
  XK_STEP_ORBITALS = 0,  /* Psi = Phi C and the gathers at R_g             */
  XK_STEP_PAIR = 1,      /* P = Psi_g Psi^T, V2 = V o P                     */
  XK_STEP_M2 = 2,        /* M2 = V2 Psi                                     */
  XK_STEP_M1 = 3,        /* M1 = Psi_g^T V2                                 */
  XK_STEP_LINE1 = 4,     /* line1 = M1 Phi                                  */
  XK_STEP_LINE2 = 5,     /* line2 = M2^T Phi_g                              */
  XK_STEP_LINE3 = 6,     /* line3 = ((W o Q) Psi_g)^T Phi_g                 */
  XK_STEP_ASSEMBLE = 7,  /* K = dV (line1 + line2 - line3)^T, E_x           */
  XK_NSTEPS = 8
};

/*
 * Step timing with CUDA events on the handle's stream.  enable != 0 turns it
 * on and clears the accumulators; 0 turns it off.  While on, every build
 * records an event pair around each step.  xk_timing_read waits for the
 * handle's stream, then returns the summed device milliseconds of `step`
 * over the builds since enabling and how many builds contributed.
 * Errors: XK_EINVAL (NULL handle, step out of range), XK_ECUDA.
 */
int xk_timing_enable(xk_handle* h, int enable);
int xk_timing_read(xk_handle* h, int step, double* ms, uint64_t* builds);

/*
 * Exchange energy E_x = -sum_t K[t] C[t] over `count` doubles of device
 * memory (K = K_{mu i}, C the occupied coefficients, both N x n, count = N*n),
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream); the
 * result is written to the device double *Ex_dev.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory at the time of the call -- code running inside a CUDA graph
 * capture, or a host that owns the whole device heap through its own pool
 * and forbids libraries to call cudaMalloc.  It allocates nothing: its
 * partial sums live in a fixed file-scope device array of 2048 doubles
 * (16 KiB), which every device that loads the library holds until the
 * process exits, so count may be at most 2048 * 2048 = 4194304 elements;
 * larger counts return XK_EINVAL.  Every call overwrites the partials it
 * reads, so nothing has to be cleared between calls, but all calls share the
 * one array: calls that overlap on the GPU (different streams, different
 * threads) race and must be serialised by the caller, e.g. on one stream.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Errors: XK_EINVAL (NULL pointer, count < 0 or above the maximum), XK_ECUDA.
 */
int xk_exchange_energy_noalloc(const double* K_dev, const double* C_dev, int64_t count,
                               double* Ex_dev, void* stream);

/*
 * Kernel launches issued by the library since load (counts every kernel of
 * every build): lets a caller confirm the device path ran.
 */
uint64_t xk_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* XK_H */
