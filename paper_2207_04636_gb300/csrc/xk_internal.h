// Internal declarations shared by the translation units of libxk.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <string>

namespace xk {

// Kernel launches issued since load (all translation units), and by the
// calling thread (a graph capture counts its own launches with it).
extern std::atomic<uint64_t> g_launches;
inline thread_local uint64_t t_launches = 0;
inline void count_launch(uint64_t k = 1) {
  g_launches.fetch_add(k, std::memory_order_relaxed);
  t_launches += k;
}

// ---------------------------------------------------------------------------
// FP64 SIMT path (xk_fp64.cu)
// ---------------------------------------------------------------------------

// C[M x N] = alpha * op(A) op(B) (o H) + beta * C, row-major.  op(A)[m,k] is
// A[k*lda + m] when transA else A[m*lda + k]; op(B)[k,n] is B[n*ldb + k] when
// transB else B[k*ldb + n].  H (nullable, ldh) multiplies the result
// element-wise (the Hadamard epilogue).  ksplit > 1 splits K: partial sums
// go to `work` (ksplit * M * N doubles) and are summed in split order, so
// the result does not depend on scheduling.
struct DGemm {
  int M, N, K;
  const double* A; long lda; bool transA;
  const double* B; long ldb; bool transB;
  double* C; long ldc;
  double alpha;
  const double* H; long ldh;
  int ksplit;
  double* work;
  bool upperA;  // op(A) is upper triangular: K steps below a row tile are skipped
  double beta;  // C = alpha op(A) op(B) (o H) + beta C (0: C is not read)
};
cudaError_t dgemm(const DGemm& g, cudaStream_t s);
// Split count dgemm picks when DGemm::ksplit == 0 (work needs ksplit*M*N).
int dgemm_ksplit(int M, int N, int K);

// out[r, c] = in[idx[r] * ld_in + c] for r < rows, c < cols (row gather).
cudaError_t gather_rows_f64(const double* in, long ld_in, const int32_t* idx, int rows, int cols,
                            double* out, long ld_out, cudaStream_t s);

// K[mu, i] = dV * (L1[i, mu] + L2[i, mu] - L3[i, mu]); L* are n x N.
cudaError_t assemble_k_f64(const double* L1, const double* L2, const double* L3, int n, int N,
                           double dV, double* K, cudaStream_t s);

// *out = -sum_j a[j] * b[j] over `len` doubles, fixed summation order.
// `work` holds at least reduce_work_elems() doubles.
cudaError_t neg_dot_f64(const double* a, const double* b, long len, double* work, double* out,
                        cudaStream_t s);
size_t reduce_work_elems();

// Coulomb potential of the density of psi (ng x n) on a cubic g^3 grid of
// side L: rho[R] = sum_i psi[R][i]^2, then c0 = IDFT[(4 pi / G^2) DFT[rho]]
// (G = 0 removed; the real part of c0 is the potential).  tw holds
// (cos, sin)(2 pi m / g) for m < g; c1 is scratch of ng complex values.
cudaError_t coulomb_potential_f64(const double* psi, long ng, int n, int g, double L,
                                  const double2* tw, double* rho, double2* c0, double2* c1,
                                  cudaStream_t s);
// Pois applied to nb complex g^3 grids in c0 (result in c0; c1 scratch of the
// same size): 3-D DFT, times 4 pi / G^2 (G = 0 removed), inverse 3-D DFT.
// The kernel is real and even in G, so real and imaginary parts transform
// independently (two real functions per complex grid).
cudaError_t poisson_c2c_f64(double2* c0, double2* c1, long nb, int g, double L,
                            const double2* tw, cudaStream_t s);
// v[R] = Re(c[R]) and out[R][nu] = v[R] phi[R][nu].
cudaError_t potential_rows_f64(const double2* c, const double* phi, long ng, int N, double* v,
                               double* out, cudaStream_t s);
// *out = scale * sum_j a[j] b[j] (fixed order); `work` holds reduce_work_elems() doubles.
cudaError_t dot_f64(const double* a, const double* b, long len, double scale, double* work,
                    double* out, cudaStream_t s);

// K[mu][nu] = dV (Y[mu][nu] + Y[nu][mu] - Z[mu][nu]) for N x N matrices.
cudaError_t assemble_full_f64(const double* Y, const double* Z, int N, double dV, double* K,
                              cudaStream_t s);

// GPU ISDF set-up (xk_isdf.cu), all FP64: from Phi (ng x N) and Phi_g
// (na x N), X_gg into Xgg (na x na, overwritten by its Cholesky factor),
// chi = X_gg^{-1} X_gR (na x ng), V = Pois(chi) on the cubic grid^3 grid of
// side L (na x ng) and W = V chi^T symmetrised (na x na).  `work` holds the
// split-K work of the products (dgemm_ksplit sizes) and at least na doubles.
// A ridge of 1e-14 tr(X_gg)/na is added when the plain factorisation fails
// (*ridge_out); cudaErrorInvalidValue if it still fails.
cudaError_t isdf_tables_f64(const double* phi, long ng, int N, const double* phig, int na,
                            int grid, double L, double* Xgg, double* chi, double* V, double* W,
                            double* work, int* status, double* ridge_out, cudaStream_t s);
// Interpolation points (Sec. III.A) by a greedy complete-pivoting Cholesky of
// X = (F F^T) o (F F^T) for the m candidate rows F (m x N, device): up to
// `want` pivots (indices into F, selection order) into piv (host), stopping
// when the largest remaining diagonal is at most tol_rel times the largest
// initial one; *count = pivots taken.  Holds m^2 + m want doubles of
// stream-ordered scratch during the call.
cudaError_t select_points_f64(const double* F, int m, int N, int want, double tol_rel,
                              int32_t* piv, int* count, cudaStream_t s);
// In-place blocked Cholesky (lower) of the n x n matrix A (lda); *status = 1
// on a non-positive pivot.
cudaError_t cholesky_blocked_f64(double* A, int n, long lda, int* status, cudaStream_t s);
// B (n x ncols, ldb) := (L L^T)^{-1} B with the lower factor L (ldl).
cudaError_t cholesky_solve_f64(const double* L, int n, long ldl, double* B, long ldb, long ncols,
                               cudaStream_t s);

// *out = -dV (2 sum_t V[t] P[t]^2 - sum_t W[t] Q[t]^2) over lenA and lenC
// elements, in a fixed order; `work` holds reduce_work_elems() doubles.
cudaError_t closed_form_ex_f64(const double* V, const double* P, long lenA, const double* W,
                               const double* Q, long lenC, double dV, double* work, double* out,
                               cudaStream_t s);

// A <- (A + A^T) / 2 for an n x n matrix.
cudaError_t symmetrize_f64(double* A, int n, cudaStream_t s);

// In-place Cholesky A = L L^T (lower, n x n, one block).  *status = 0 on
// success, k + 1 if the k-th pivot is not positive.
cudaError_t cholesky_f64(double* A, int n, int* status, cudaStream_t s);

// X <- B L^{-T} for L lower n x n and B rows x n (row-major): solves
// X L^T = B row by row.
cudaError_t trsm_right_lt_f64(const double* L, int n, const double* B, int rows, double* X,
                              cudaStream_t s);

// Cyclic Jacobi eigendecomposition of the symmetric n x n matrix A (one
// block): on return A holds the eigenvalues on its diagonal and U the
// eigenvectors as columns.  Runs at most max_sweeps sweeps; *sweeps gets the
// number used.
cudaError_t jacobi_eig_f64(double* A, double* U, int n, int max_sweeps, int* sweeps,
                           cudaStream_t s);

// X[r, k] = B[r, k] * f(lambda_k) with f = |lambda|^{-1/2} when
// |lambda| > cut * max|lambda| else 0; sign[k] = sign(lambda) or 0.
cudaError_t scale_eigcols_f64(const double* Adiag_src, int n, const double* B, int rows, double cut,
                              double* X, double* sign, cudaStream_t s);

// Allocation-free E_x = -sum K[t] C[t] with partial sums in a fixed
// file-scope device array (xk_noalloc.cu); count <= noalloc_max_count().
int64_t noalloc_max_count();
cudaError_t exchange_energy_noalloc(const double* K, const double* C, int64_t count, double* Ex,
                                    cudaStream_t s);

}  // namespace xk
