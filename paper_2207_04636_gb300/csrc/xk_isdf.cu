// GPU FP64 ISDF set-up (Sec. III.A and IV.C of arXiv 2207.04636): from the
// basis on the grid and the interpolation points, the tables the exchange
// build consumes,
//   X_gg = (Phi_g Phi_g^T) o (Phi_g Phi_g^T),  X_gR = (Phi_g Phi^T) o (Phi_g Phi^T)
//   chi  = X_gg^{-1} X_gR          (Eq. lsqfit; blocked Cholesky, two blocked solves)
//   V    = Pois(chi_g)              (Eq. rpsPot; DFT-based Poisson, two functions per
//                                    complex transform)
//   W    = V chi^T, symmetrised     (Eq. thcpot)
// all in FP64 on the CUDA cores (DFMA-bound on GB300), with a ridge of
// 1e-14 tr(X_gg) / N_aux added to the diagonal when the plain factorisation
// fails.
#include <algorithm>
#include <cmath>
#include <vector>

#include "xk_internal.h"

namespace xk {

namespace {

constexpr int NB = 64;  // panel and block width of the factorisation and the solves

int nblocks(long total) { return (int)std::max<long>(1, std::min<long>((total + 255) / 256, 152L * 16)); }

__global__ void square_kernel(double* __restrict__ a, long rows, long cols, long ld) {
  const long count = rows * cols;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / cols, c = t % cols;
    const double v = a[r * ld + c];
    a[r * ld + c] = v * v;
  }
}

__global__ void add_diag_kernel(double* __restrict__ a, int n, long ld, double d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    a[(long)i * ld + i] += d;
}

__global__ void copy_diag_kernel(const double* __restrict__ a, int n, long ld, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = a[(long)i * ld + i];
}

// In-place Cholesky (lower) of the kb x kb diagonal block at (k, k); one
// block of 256 threads, the block held in shared memory.  A non-positive
// pivot sets *status = 1 (the pivot is replaced by 1 so the loop ends).
__global__ void potrf_block_kernel(double* __restrict__ A, long lda, int k, int kb,
                                   int* __restrict__ status) {
  __shared__ double a[NB][NB + 1];
  for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) {
    const int i = t / kb, j = t % kb;
    a[i][j] = A[(long)(k + i) * lda + k + j];
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (threadIdx.x == 0) {
      double d = a[j][j];
      if (!(d > 0.0)) {
        atomicExch(status, 1);
        d = 1.0;
      }
      a[j][j] = sqrt(d);
    }
    __syncthreads();
    const double piv = a[j][j];
    for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) a[i][j] /= piv;
    __syncthreads();
    // trailing update of the lower triangle: a[i][l] -= a[i][j] a[l][j], j < l <= i
    const int m = kb - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = j + 1 + t / m, l = j + 1 + t % m;
      if (l <= i) a[i][l] -= a[i][j] * a[l][j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) {
    const int i = t / kb, j = t % kb;
    if (j <= i) A[(long)(k + i) * lda + k + j] = a[i][j];
  }
}

// Panel below the diagonal block: row r of A[k+kb:n, k:k+kb] := x with
// x L11^T = row (forward substitution; one thread per row).
__global__ void trsm_panel_kernel(double* __restrict__ A, long lda, int k, int kb, int n) {
  __shared__ double l[NB][NB + 1];
  for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) {
    const int i = t / kb, j = t % kb;
    l[i][j] = j <= i ? A[(long)(k + i) * lda + k + j] : 0.0;
  }
  __syncthreads();
  for (long r = k + kb + blockIdx.x * (long)blockDim.x + threadIdx.x; r < n;
       r += (long)gridDim.x * blockDim.x) {
    double* row = A + r * lda + k;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j < kb) {
        double v = row[j];
#pragma unroll
        for (int p = 0; p < j; ++p) v -= x[p] * l[j][p];
        x[j] = v / l[j][j];
        row[j] = x[j];
      } else {
        x[j] = 0.0;
      }
    }
  }
}

// Column c of B[k:k+kb, :] := L_kk^{-1} column (forward, lower = true) or
// L_kk^{-T} column (backward, lower = false); one thread per column, the
// block of L in shared memory (identity past kb), the column in registers.
template <bool LOWER>
__global__ void trsv_block_kernel(const double* __restrict__ L, long ldl, int k, int kb,
                                  double* __restrict__ B, long ldb, long ncols) {
  __shared__ double l[NB][NB + 1];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int i = t / NB, j = t % NB;
    double v = (i == j) ? 1.0 : 0.0;
    if (i < kb && j < kb && j <= i) v = L[(long)(k + i) * ldl + k + j];
    l[i][j] = v;
  }
  __syncthreads();
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncols;
       c += (long)gridDim.x * blockDim.x) {
    double y[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) y[j] = j < kb ? B[(long)(k + j) * ldb + c] : 0.0;
    if (LOWER) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        double v = y[j];
#pragma unroll
        for (int p = 0; p < j; ++p) v -= l[j][p] * y[p];
        y[j] = v / l[j][j];
      }
    } else {
#pragma unroll
      for (int j = NB - 1; j >= 0; --j) {
        double v = y[j];
#pragma unroll
        for (int p = j + 1; p < NB; ++p) v -= l[p][j] * y[p];
        y[j] = v / l[j][j];
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < kb) B[(long)(k + j) * ldb + c] = y[j];
  }
}

// c[q][R] = f[2q][R] + i f[2q+1][R] for the rows [r0, r0 + nf) of f (ld).
__global__ void pack_pairs_kernel(const double* __restrict__ f, long ld, long r0, int nf, long ng,
                                  double2* __restrict__ c) {
  const long np = (nf + 1) / 2, count = np * ng;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long q = t / ng, R = t % ng;
    const double re = f[(r0 + 2 * q) * ld + R];
    const double im = (2 * q + 1 < nf) ? f[(r0 + 2 * q + 1) * ld + R] : 0.0;
    c[t] = make_double2(re, im);
  }
}

__global__ void unpack_pairs_kernel(const double2* __restrict__ c, long r0, int nf, long ng,
                                    double* __restrict__ out, long ld) {
  const long np = (nf + 1) / 2, count = np * ng;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long q = t / ng, R = t % ng;
    out[(r0 + 2 * q) * ld + R] = c[t].x;
    if (2 * q + 1 < nf) out[(r0 + 2 * q + 1) * ld + R] = c[t].y;
  }
}

// ---------------------------------------------------------------- point selection
// Greedy complete-pivoting Cholesky of X = (F F^T) o (F F^T), left-looking:
// only the diagonal d is kept up to date; each step forms one column.
// State on the device: d[m] (selected rows set to -1), L[m][want],
// sel[0] = steps taken, sel[1] = stopped flag, val[t] = pivot value, tol.

__global__ void diag_init_kernel(const double* __restrict__ X, int m, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    d[i] = X[(long)i * m + i];
}

// Pivot of step t: the largest d (the lowest index on ties); stops when it is
// not above tol (tol = tol_rel * the largest initial diagonal, set at t = 0).
__global__ void __launch_bounds__(1024) pivot_kernel(double* __restrict__ d, int m, int t,
                                                     double tol_rel, int* __restrict__ sel,
                                                     int32_t* __restrict__ piv,
                                                     double* __restrict__ val,
                                                     double* __restrict__ tol) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  if (sel[1]) return;
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double v = d[i];
    if (v > best) { best = v; bidx = i; }  // increasing i: the first maximum is kept
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    // fold the warps' results in warp order (ties keep the lower index)
    double b0 = bv[0];
    int i0 = bi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > b0 || (bv[w] == b0 && bi[w] < i0)) { b0 = bv[w]; i0 = bi[w]; }
    if (t == 0) *tol = tol_rel * b0;
    if (!(b0 > *tol) || i0 >= m) {
      sel[1] = 1;
    } else {
      piv[t] = i0;
      val[t] = b0;
      d[i0] = -1.0;
      sel[0] = t + 1;
    }
  }
}

// Column t: for every unselected row i (one warp per row),
// L[i][t] = (X[i][p] - sum_{s<t} L[i][s] L[p][s]) / sqrt(val[t]) and
// d[i] -= L[i][t]^2; the pivot row gets L[p][t] = sqrt(val[t]).
__global__ void column_kernel(const double* __restrict__ X, int m, int want, int t,
                              const int* __restrict__ sel, const int32_t* __restrict__ piv,
                              const double* __restrict__ val, double* __restrict__ L,
                              double* __restrict__ d) {
  if (sel[1] || sel[0] <= t) return;
  const int p = piv[t];
  const double sp = sqrt(val[t]);
  const int lane = threadIdx.x & 31;
  const long warps = ((long)gridDim.x * blockDim.x) >> 5;
  const double* lp = L + (long)p * want;
  for (long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    if (i == p) {
      if (lane == 0) L[(long)p * want + t] = sp;
      continue;
    }
    if (d[i] < 0.0) continue;  // selected earlier
    const double* li = L + i * want;
    double acc = 0.0;
    for (int q = lane; q < t; q += 32) acc = fma(li[q], lp[q], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double l = (X[i * m + p] - acc) / sp;
      L[i * want + t] = l;
      d[i] -= l * l;
    }
  }
}

}  // namespace

cudaError_t select_points_f64(const double* F, int m, int N, int want, double tol_rel,
                              int32_t* piv, int* count, cudaStream_t s) {
  if (m <= 0 || want <= 0) {
    *count = 0;
    return cudaSuccess;
  }
  want = std::min(want, m);
  void* buf = nullptr;
  const size_t xb = (size_t)m * m * 8, lb = (size_t)m * want * 8;
  const size_t bytes = xb + lb + (size_t)m * 8 + (size_t)want * 8 + 64 + (size_t)want * 4 + 64;
  cudaError_t e = cudaMallocAsync(&buf, bytes, s);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(buf);
  double* X = reinterpret_cast<double*>(b);
  double* L = reinterpret_cast<double*>(b + xb);
  double* d = reinterpret_cast<double*>(b + xb + lb);
  double* val = d + m;
  double* tol = val + want;
  int* sel = reinterpret_cast<int*>(tol + 2);
  int32_t* dpiv = reinterpret_cast<int32_t*>(sel + 4);
  {
    DGemm g{m, m, N, F, N, false, F, N, true, X, m, 1.0, nullptr, 0, 1, nullptr};
    e = dgemm(g, s);
  }
  if (e == cudaSuccess) {
    square_kernel<<<nblocks((long)m * m), 256, 0, s>>>(X, m, m, m);
    diag_init_kernel<<<nblocks(m), 256, 0, s>>>(X, m, d);
    count_launch(2);
    e = cudaMemsetAsync(sel, 0, 16, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(L, 0, lb, s);
  const int cb = std::max(1, std::min(152 * 8, (m + 7) / 8));  // 8 warps (rows) per block
  for (int t = 0; e == cudaSuccess && t < want; ++t) {
    pivot_kernel<<<1, 1024, 0, s>>>(d, m, t, tol_rel, sel, dpiv, val, tol);
    column_kernel<<<cb, 256, 0, s>>>(X, m, want, t, sel, dpiv, val, L, d);
    count_launch(2);
    if ((t & 255) == 255) e = cudaGetLastError();
  }
  int got = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&got, sel, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && got > 0)
    e = cudaMemcpyAsync(piv, dpiv, (size_t)got * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaError_t e2 = cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *count = got;
  return e;
}

cudaError_t cholesky_blocked_f64(double* A, int n, long lda, int* status, cudaStream_t s) {
  for (int k = 0; k < n; k += NB) {
    const int kb = std::min(NB, n - k);
    potrf_block_kernel<<<1, 256, 0, s>>>(A, lda, k, kb, status);
    count_launch();
    if (k + kb < n) {
      const int rest = n - k - kb;
      trsm_panel_kernel<<<std::max(1, std::min(152 * 4, (rest + 127) / 128)), 128, 0, s>>>(A, lda, k, kb, n);
      count_launch();
      // A22 -= L21 L21^T (the whole square; only its lower triangle is used)
      DGemm g{rest, rest, kb, A + (long)(k + kb) * lda + k, lda, false,
              A + (long)(k + kb) * lda + k, lda, true, A + (long)(k + kb) * lda + k + kb, lda,
              -1.0, nullptr, 0, 1, nullptr, false, 1.0};
      cudaError_t e = dgemm(g, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t cholesky_solve_f64(const double* L, int n, long ldl, double* B, long ldb, long ncols,
                               cudaStream_t s) {
  const int cb = nblocks(ncols);
  // forward: L Y = B, block rows in order (left-looking updates)
  for (int k = 0; k < n; k += NB) {
    const int kb = std::min(NB, n - k);
    if (k > 0) {
      DGemm g{kb, (int)ncols, k, L + (long)k * ldl, ldl, false, B, ldb, false, B + (long)k * ldb,
              ldb, -1.0, nullptr, 0, 1, nullptr, false, 1.0};
      cudaError_t e = dgemm(g, s);
      if (e != cudaSuccess) return e;
    }
    trsv_block_kernel<true><<<cb, 256, 0, s>>>(L, ldl, k, kb, B, ldb, ncols);
    count_launch();
  }
  // backward: L^T X = Y, block rows in reverse order
  const int last = ((n - 1) / NB) * NB;
  for (int k = last; k >= 0; k -= NB) {
    const int kb = std::min(NB, n - k);
    if (k + kb < n) {
      // B_k -= L[k+kb:n, k:k+kb]^T X[k+kb:n]
      DGemm g{kb, (int)ncols, n - k - kb, L + (long)(k + kb) * ldl + k, ldl, true,
              B + (long)(k + kb) * ldb, ldb, false, B + (long)k * ldb, ldb, -1.0, nullptr, 0, 1,
              nullptr, false, 1.0};
      cudaError_t e = dgemm(g, s);
      if (e != cudaSuccess) return e;
    }
    trsv_block_kernel<false><<<cb, 256, 0, s>>>(L, ldl, k, kb, B, ldb, ncols);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t isdf_tables_f64(const double* phi, long ng, int N, const double* phig, int na,
                            int grid, double L, double* Xgg, double* chi, double* V, double* W,
                            double* work, int* status, double* ridge_out, cudaStream_t s) {
  cudaError_t e;
  auto gram = [&]() {
    DGemm g{na, na, N, phig, N, false, phig, N, true, Xgg, na, 1.0, nullptr, 0, 0, work};
    cudaError_t r = dgemm(g, s);
    if (r != cudaSuccess) return r;
    square_kernel<<<nblocks((long)na * na), 256, 0, s>>>(Xgg, na, na, na);
    count_launch();
    return cudaGetLastError();
  };
  // X_gR = (Phi_g Phi^T) o (Phi_g Phi^T) into chi
  {
    DGemm g{na, (int)ng, N, phig, N, false, phi, N, true, chi, ng, 1.0, nullptr, 0, 0, work};
    e = dgemm(g, s);
    if (e != cudaSuccess) return e;
    square_kernel<<<nblocks((long)na * ng), 256, 0, s>>>(chi, na, ng, ng);
    count_launch();
  }
  e = gram();
  if (e != cudaSuccess) return e;
  double ridge = 0.0;
  int st = 0;
  e = cudaMemsetAsync(status, 0, 4, s);
  if (e == cudaSuccess) e = cholesky_blocked_f64(Xgg, na, na, status, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (st != 0) {  // the factorisation failed: add the ridge and factor again
    e = gram();
    if (e != cudaSuccess) return e;
    std::vector<double> d(na);
    copy_diag_kernel<<<nblocks(na), 256, 0, s>>>(Xgg, na, na, work);
    count_launch();
    e = cudaMemcpyAsync(d.data(), work, (size_t)na * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    double tr = 0.0;
    for (double v : d) tr += v;
    ridge = 1e-14 * tr / na;
    add_diag_kernel<<<nblocks(na), 256, 0, s>>>(Xgg, na, na, ridge);
    count_launch();
    e = cudaMemsetAsync(status, 0, 4, s);
    if (e == cudaSuccess) e = cholesky_blocked_f64(Xgg, na, na, status, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (st != 0) return cudaErrorInvalidValue;  // X_gg is not positive definite
  }
  if (ridge_out) *ridge_out = ridge;
  // chi = X_gg^{-1} X_gR
  e = cholesky_solve_f64(Xgg, na, na, chi, ng, ng, s);
  if (e != cudaSuccess) return e;
  // V = Pois(chi), two functions per complex transform, in batches
  {
    const long g3 = (long)grid * grid * grid;
    std::vector<double> t(2 * (size_t)grid);
    for (int m = 0; m < grid; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)grid;
      t[2 * m] = std::cos(a);
      t[2 * m + 1] = std::sin(a);
    }
    const int pairs = (int)std::max<long>(1, std::min<long>((na + 1) / 2, (1L << 28) / (g3 * 16)));
    void* buf = nullptr;
    e = cudaMallocAsync(&buf, (size_t)(2 * pairs * g3 + grid) * 16, s);
    if (e != cudaSuccess) return e;
    double2* c0 = static_cast<double2*>(buf);
    double2* c1 = c0 + pairs * g3;
    double2* tw = c1 + pairs * g3;
    e = cudaMemcpyAsync(tw, t.data(), t.size() * 8, cudaMemcpyHostToDevice, s);
    for (long r0 = 0; e == cudaSuccess && r0 < na; r0 += 2L * pairs) {
      const int nf = (int)std::min<long>(2L * pairs, na - r0);
      const long np = (nf + 1) / 2;
      pack_pairs_kernel<<<nblocks(np * g3), 256, 0, s>>>(chi, ng, r0, nf, g3, c0);
      count_launch();
      e = poisson_c2c_f64(c0, c1, np, grid, L, tw, s);
      if (e != cudaSuccess) break;
      unpack_pairs_kernel<<<nblocks(np * g3), 256, 0, s>>>(c0, r0, nf, g3, V, ng);
      count_launch();
      e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e;
  }
  // W = V chi^T, symmetrised
  {
    DGemm g{na, na, (int)ng, V, ng, false, chi, ng, true, W, na, 1.0, nullptr, 0, 0, work};
    e = dgemm(g, s);
    if (e == cudaSuccess) e = symmetrize_f64(W, na, s);
  }
  return e;
}

}  // namespace xk
