// FP64 kernels of the exchange build: a tiled SIMT DGEMM with a Hadamard
// epilogue and deterministic split-K, row gathers, the K assembly, the E_x
// reduction, and the small dense FP64 factorisations of the occ-RI K_ij.
//
// On GB300 FP64 runs on the CUDA cores at a small fraction of the tensor
// rate, so every FP64 contraction here is bound by the DFMA pipe; the tiles
// only need enough register reuse to keep that pipe fed.
#include "xk_internal.h"

#include <algorithm>

namespace xk {

std::atomic<uint64_t> g_launches{0};

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TPB = 256;

template <bool TA, bool TB, bool HAD>
__global__ void __launch_bounds__(TPB) dgemm_kernel(DGemm g, int kchunk) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const long m0 = (long)blockIdx.y * BM, n0 = (long)blockIdx.x * BN;
  const long kend = min((long)g.K, (long)blockIdx.z * kchunk + kchunk);
  // rows m0.. of an upper-triangular op(A) vanish for k < m0
  const long kbeg = g.upperA ? max((long)blockIdx.z * kchunk, m0) : (long)blockIdx.z * kchunk;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (long k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e = 0; e < (BM * BK) / TPB; ++e) {
      const int l = tid + TPB * e;
      int m, k;
      if (TA) { k = l / BM; m = l % BM; } else { m = l / BK; k = l % BK; }
      const long gm = m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < g.M && gk < kend) v = TA ? g.A[gk * g.lda + gm] : g.A[gm * g.lda + gk];
      As[k][m] = v;
    }
#pragma unroll
    for (int e = 0; e < (BN * BK) / TPB; ++e) {
      const int l = tid + TPB * e;
      int n, k;
      if (TB) { n = l / BK; k = l % BK; } else { k = l / BN; n = l % BN; }
      const long gn = n0 + n, gk = k0 + k;
      double v = 0.0;
      if (gn < g.N && gk < kend) v = TB ? g.B[gn * g.ldb + gk] : g.B[gk * g.ldb + gn];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      if (g.ksplit > 1) {
        g.work[((long)blockIdx.z * g.M + m) * g.N + n] = acc[i][j];
      } else {
        double v = g.alpha * acc[i][j];
        if (HAD) v *= g.H[m * g.ldh + n];
        if (g.beta != 0.0) v += g.beta * g.C[m * g.ldc + n];
        g.C[m * g.ldc + n] = v;
      }
    }
  }
}

// C = alpha * sum_z work[z] (o H), z in increasing order.
__global__ void splitk_reduce_kernel(DGemm g) {
  const long total = (long)g.M * g.N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < g.ksplit; ++z) s += g.work[(long)z * total + t];
    const long m = t / g.N, n = t % g.N;
    double v = g.alpha * s;
    if (g.H) v *= g.H[m * g.ldh + n];
    if (g.beta != 0.0) v += g.beta * g.C[m * g.ldc + n];
    g.C[m * g.ldc + n] = v;
  }
}

int choose_ksplit(int M, int N, int K) {
  const long tiles = (long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const long target = 4L * 152;  // about four waves of CTAs over 152 SMs
  if (tiles >= target) return 1;
  long ks = (target + tiles - 1) / tiles;
  ks = std::min<long>(ks, std::max(1, K / 64));
  return (int)std::max<long>(1, std::min<long>(ks, 64));
}

template <bool TA, bool TB>
cudaError_t launch_tt(const DGemm& g, int kchunk, cudaStream_t s) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.ksplit);
  if (g.H && g.ksplit == 1)
    dgemm_kernel<TA, TB, true><<<grid, TPB, 0, s>>>(g, kchunk);
  else
    dgemm_kernel<TA, TB, false><<<grid, TPB, 0, s>>>(g, kchunk);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int dgemm_ksplit(int M, int N, int K) {
  int ks = choose_ksplit(M, N, K);
  int kchunk = (K + ks - 1) / ks;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk <= 0) kchunk = BK;
  return std::max(1, (K + kchunk - 1) / kchunk);
}

cudaError_t dgemm(const DGemm& gin, cudaStream_t s) {
  DGemm g = gin;
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.ksplit <= 0) g.ksplit = choose_ksplit(g.M, g.N, g.K);
  if (g.ksplit > 1 && !g.work) g.ksplit = 1;
  int kchunk = (g.K + g.ksplit - 1) / g.ksplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk <= 0) kchunk = BK;
  g.ksplit = std::max(1, (g.K + kchunk - 1) / kchunk);
  cudaError_t e;
  if (!g.transA && !g.transB) e = launch_tt<false, false>(g, kchunk, s);
  else if (g.transA && !g.transB) e = launch_tt<true, false>(g, kchunk, s);
  else if (!g.transA && g.transB) e = launch_tt<false, true>(g, kchunk, s);
  else e = launch_tt<true, true>(g, kchunk, s);
  if (e != cudaSuccess || g.ksplit == 1) return e;
  const long total = (long)g.M * g.N;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  splitk_reduce_kernel<<<blocks, 256, 0, s>>>(g);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------

__global__ void gather_rows_kernel(const double* __restrict__ in, long ld_in,
                                   const int32_t* __restrict__ idx, int rows, int cols,
                                   double* __restrict__ out, long ld_out) {
  const long total = (long)rows * cols;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / cols, c = t % cols;
    out[r * ld_out + c] = in[(long)idx[r] * ld_in + c];
  }
}

cudaError_t gather_rows_f64(const double* in, long ld_in, const int32_t* idx, int rows, int cols,
                            double* out, long ld_out, cudaStream_t s) {
  const long total = (long)rows * cols;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  gather_rows_kernel<<<blocks, 256, 0, s>>>(in, ld_in, idx, rows, cols, out, ld_out);
  count_launch();
  return cudaGetLastError();
}

__global__ void assemble_k_kernel(const double* __restrict__ L1, const double* __restrict__ L2,
                                  const double* __restrict__ L3, int n, int N, double dV,
                                  double* __restrict__ K) {
  const long total = (long)n * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long mu = t / n, i = t % n;
    const long src = i * N + mu;
    K[t] = dV * ((L1[src] + L2[src]) - L3[src]);
  }
}

cudaError_t assemble_k_f64(const double* L1, const double* L2, const double* L3, int n, int N,
                           double dV, double* K, cudaStream_t s) {
  const long total = (long)n * N;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 8);
  assemble_k_kernel<<<blocks, 256, 0, s>>>(L1, L2, L3, n, N, dV, K);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic two-stage reduction: block b sums the contiguous chunk b in a
// fixed per-thread order and a fixed tree; one block then sums the partials.

constexpr int RED_BLOCKS = 512, RED_TPB = 256;

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  return sh[0];
}

__global__ void dot_stage1(const double* __restrict__ a, const double* __restrict__ b, long len,
                           double* __restrict__ part) {
  __shared__ double sh[RED_TPB];
  const long chunk = (len + gridDim.x - 1) / gridDim.x;
  const long beg = blockIdx.x * chunk, end = min(len, beg + chunk);
  double s = 0.0;
  for (long t = beg + threadIdx.x; t < end; t += blockDim.x) s = fma(a[t], b[t], s);
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void dot_stage2(const double* __restrict__ part, int np, double* out) {
  __shared__ double sh[RED_TPB];
  double s = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) *out = -tot;
}

size_t reduce_work_elems() { return RED_BLOCKS; }

cudaError_t neg_dot_f64(const double* a, const double* b, long len, double* work, double* out,
                        cudaStream_t s) {
  dot_stage1<<<RED_BLOCKS, RED_TPB, 0, s>>>(a, b, len, work);
  dot_stage2<<<1, RED_TPB, 0, s>>>(work, RED_BLOCKS, out);
  count_launch(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coulomb J on the grid: density, Poisson solve by a 3-D DFT written as three
// passes of 1-D DFTs (each output an O(g) sum in FP64; the grids here are
// g <= ~100 per axis, so the O(g^4) total is a few hundred MFLOP), and
// J = dV Phi^T diag(v) Phi.

namespace {
int blocks_of(long total) { return (int)std::max<long>(1, std::min<long>((total + 255) / 256, 152L * 16)); }
}  // namespace

// rho[R] = sum_i psi[R][i]^2, also as a complex grid function (imaginary 0).
__global__ void density_kernel(const double* __restrict__ psi, long ng, int n,
                               double* __restrict__ rho, double2* __restrict__ c) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < ng;
       r += (long)gridDim.x * blockDim.x) {
    const double* row = psi + r * n;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(row[i], row[i], s);
    rho[r] = s;
    c[r] = make_double2(s, 0.0);
  }
}

// One pass of a length-g DFT along `axis` (0 = slowest index) of `count`
// values (whole g^3 grids one after another):
// out[k] = sum_j in[j] exp(sign 2 pi i j k / g), tw[m] = (cos, sin)(2 pi m / g).
__global__ void dft_axis_kernel(const double2* __restrict__ in, double2* __restrict__ out, int g,
                                int axis, const double2* __restrict__ tw, double sign, long count) {
  const long stride = axis == 0 ? (long)g * g : axis == 1 ? g : 1;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const int k = (int)((t / stride) % g);
    const long base = t - (long)k * stride;
    double re = 0.0, im = 0.0;
    int m = 0;  // j k mod g
    for (int j = 0; j < g; ++j) {
      const double2 x = in[base + (long)j * stride];
      const double2 w = tw[m];
      const double ws = sign * w.y;
      re = fma(x.x, w.x, fma(-x.y, ws, re));
      im = fma(x.x, ws, fma(x.y, w.x, im));
      m += k;
      if (m >= g) m -= g;
    }
    out[t] = make_double2(re, im);
  }
}

// f(G) *= scale * 4 pi / |G|^2 with G = 2 pi m / L, m the signed frequency
// index of each axis; the G = 0 term is set to zero.
__global__ void coulomb_multiply_kernel(double2* __restrict__ f, int g, double L, double scale,
                                        long count) {
  const long g3 = (long)g * g * g;
  const double two_pi_over_L = 6.283185307179586 / L;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long u = t % g3;
    const int i0 = (int)(u / ((long)g * g)), i1 = (int)((u / g) % g), i2 = (int)(u % g);
    const int m0 = i0 <= (g - 1) / 2 ? i0 : i0 - g;
    const int m1 = i1 <= (g - 1) / 2 ? i1 : i1 - g;
    const int m2 = i2 <= (g - 1) / 2 ? i2 : i2 - g;
    const double g2 = two_pi_over_L * two_pi_over_L * ((double)m0 * m0 + (double)m1 * m1 + (double)m2 * m2);
    const double k = g2 > 0.0 ? scale * 12.566370614359172 / g2 : 0.0;
    f[t] = make_double2(f[t].x * k, f[t].y * k);
  }
}

// v[R] = Re(c[R]); out[R][nu] = v[R] phi[R][nu].
__global__ void potential_rows_kernel(const double2* __restrict__ c, const double* __restrict__ phi,
                                      long ng, int N, double* __restrict__ v, double* __restrict__ out) {
  const long count = ng * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / N;
    const double vr = c[r].x;
    out[t] = vr * phi[t];
    if (t % N == 0) v[r] = vr;
  }
}

__global__ void dot_scaled_stage2(const double* __restrict__ part, int np, double scale, double* out) {
  __shared__ double sh[RED_TPB];
  double s = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) *out = scale * tot;
}

cudaError_t poisson_c2c_f64(double2* c0, double2* c1, long nb, int g, double L,
                            const double2* tw, cudaStream_t s) {
  const long g3 = (long)g * g * g, count = nb * g3;
  const int b = blocks_of(count);
  dft_axis_kernel<<<b, 256, 0, s>>>(c0, c1, g, 2, tw, -1.0, count);
  dft_axis_kernel<<<b, 256, 0, s>>>(c1, c0, g, 1, tw, -1.0, count);
  dft_axis_kernel<<<b, 256, 0, s>>>(c0, c1, g, 0, tw, -1.0, count);
  coulomb_multiply_kernel<<<b, 256, 0, s>>>(c1, g, L, 1.0 / (double)g3, count);  // 1/N_g: inverse
  dft_axis_kernel<<<b, 256, 0, s>>>(c1, c0, g, 2, tw, 1.0, count);
  dft_axis_kernel<<<b, 256, 0, s>>>(c0, c1, g, 1, tw, 1.0, count);
  dft_axis_kernel<<<b, 256, 0, s>>>(c1, c0, g, 0, tw, 1.0, count);
  count_launch(7);
  return cudaGetLastError();
}

cudaError_t coulomb_potential_f64(const double* psi, long ng, int n, int g, double L,
                                  const double2* tw, double* rho, double2* c0, double2* c1,
                                  cudaStream_t s) {
  density_kernel<<<blocks_of(ng), 256, 0, s>>>(psi, ng, n, rho, c0);
  count_launch();
  return poisson_c2c_f64(c0, c1, 1, g, L, tw, s);
}

cudaError_t potential_rows_f64(const double2* c, const double* phi, long ng, int N, double* v,
                               double* out, cudaStream_t s) {
  potential_rows_kernel<<<blocks_of(ng * N), 256, 0, s>>>(c, phi, ng, N, v, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t dot_f64(const double* a, const double* b, long len, double scale, double* work,
                    double* out, cudaStream_t s) {
  dot_stage1<<<RED_BLOCKS, RED_TPB, 0, s>>>(a, b, len, work);
  dot_scaled_stage2<<<1, RED_TPB, 0, s>>>(work, RED_BLOCKS, scale, out);
  count_launch(2);
  return cudaGetLastError();
}

// Full K: K[mu][nu] = dV (Y[mu][nu] + Y[nu][mu] - Z[mu][nu]) (N x N).
__global__ void assemble_full_kernel(const double* __restrict__ Y, const double* __restrict__ Z,
                                     int N, double dV, double* __restrict__ K) {
  const long count = (long)N * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long mu = t / N, nu = t % N;
    K[t] = dV * ((Y[t] + Y[nu * N + mu]) - Z[t]);
  }
}

cudaError_t assemble_full_f64(const double* Y, const double* Z, int N, double dV, double* K,
                              cudaStream_t s) {
  const long count = (long)N * N;
  const int blocks = (int)std::min<long>((count + 255) / 256, 152L * 16);
  assemble_full_kernel<<<std::max(blocks, 1), 256, 0, s>>>(Y, Z, N, dV, K);
  count_launch();
  return cudaGetLastError();
}

// E_x from its closed form, -dV (2 sum w_A p_A^2 - sum w_C p_C^2) (Eq. exoccri
// contracted with C: line 1 and line 2 each give sum V o P o P, line 3 gives
// sum W o Q o Q).  Stage 1: half of the blocks sum the V term, the other
// half the W term; stage 2 adds the per-block sums in a fixed order.
__global__ void wsq_stage1(const double* __restrict__ wa, const double* __restrict__ pa, long la,
                           const double* __restrict__ wc, const double* __restrict__ pc, long lc,
                           double* __restrict__ part) {
  __shared__ double sh[RED_TPB];
  const int half = gridDim.x / 2;
  const bool c = (int)blockIdx.x >= half;
  const double* w = c ? wc : wa;
  const double* p = c ? pc : pa;
  const long len = c ? lc : la;
  const long blk = c ? blockIdx.x - half : blockIdx.x;
  const long chunk = (len + half - 1) / half;
  const long beg = blk * chunk, end = min(len, beg + chunk);
  double s = 0.0;
  for (long t = beg + threadIdx.x; t < end; t += blockDim.x) s = fma(w[t] * p[t], p[t], s);
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void closed_ex_stage2(const double* __restrict__ part, int half, double dV, double* out) {
  __shared__ double sa[RED_TPB], sc[RED_TPB];
  double a = 0.0, c = 0.0;
  for (int t = threadIdx.x; t < half; t += blockDim.x) {
    a += part[t];
    c += part[half + t];
  }
  sa[threadIdx.x] = a;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sc[threadIdx.x] += sc[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = -dV * (2.0 * sa[0] - sc[0]);
}

cudaError_t closed_form_ex_f64(const double* V, const double* P, long lenA, const double* W,
                               const double* Q, long lenC, double dV, double* work, double* out,
                               cudaStream_t s) {
  wsq_stage1<<<RED_BLOCKS, RED_TPB, 0, s>>>(V, P, lenA, W, Q, lenC, work);
  closed_ex_stage2<<<1, RED_TPB, 0, s>>>(work, RED_BLOCKS / 2, dV, out);
  count_launch(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small dense FP64 factorisations (n <= a few hundred; one block each).

__global__ void symmetrize_kernel(double* A, int n) {
  const long total = (long)n * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long i = t / n, j = t % n;
    if (j > i) {
      const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = v;
      A[j * n + i] = v;
    }
  }
}

cudaError_t symmetrize_f64(double* A, int n, cudaStream_t s) {
  symmetrize_kernel<<<64, 256, 0, s>>>(A, n);
  count_launch();
  return cudaGetLastError();
}

__global__ void cholesky_kernel(double* A, int n, int* status) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[(long)k * n + k];
      if (!(d > 0.0)) fail = k + 1;
      else A[(long)k * n + k] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double piv = A[(long)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(long)i * n + k] /= piv;
    __syncthreads();
    const long rem = n - k - 1;
    for (long t = threadIdx.x; t < rem * rem; t += blockDim.x) {
      const int i = k + 1 + (int)(t / rem), j = k + 1 + (int)(t % rem);
      if (j <= i) A[(long)i * n + j] -= A[(long)i * n + k] * A[(long)j * n + k];
    }
    __syncthreads();
  }
  if (!fail)
    for (long t = threadIdx.x; t < (long)n * n; t += blockDim.x) {
      const int i = (int)(t / n), j = (int)(t % n);
      if (j > i) A[t] = 0.0;
    }
  if (threadIdx.x == 0) *status = fail;
}

cudaError_t cholesky_f64(double* A, int n, int* status, cudaStream_t s) {
  cholesky_kernel<<<1, 1024, 0, s>>>(A, n, status);
  count_launch();
  return cudaGetLastError();
}

__global__ void trsm_kernel(const double* __restrict__ L, int n, const double* __restrict__ B,
                            int rows, double* __restrict__ X) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const double* b = B + (long)r * n;
    double* x = X + (long)r * n;
    for (int k = 0; k < n; ++k) {
      double acc = b[k];
      for (int j = 0; j < k; ++j) acc -= L[(long)k * n + j] * x[j];
      x[k] = acc / L[(long)k * n + k];
    }
  }
}

cudaError_t trsm_right_lt_f64(const double* L, int n, const double* B, int rows, double* X,
                              cudaStream_t s) {
  trsm_kernel<<<(rows + 127) / 128, 128, 0, s>>>(L, n, B, rows, X);
  count_launch();
  return cudaGetLastError();
}

// Cyclic Jacobi: rotations (p, q) in row order; each rotation updates the
// two columns, then the two rows of A and the two columns of U in parallel.
__global__ void jacobi_kernel(double* A, double* U, int n, int max_sweeps, int* sweeps) {
  __shared__ double cs[2];
  __shared__ double off_sh[1024];
  __shared__ int done;
  for (long t = threadIdx.x; t < (long)n * n; t += blockDim.x)
    U[t] = (t / n == t % n) ? 1.0 : 0.0;
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int sw = 0;
  for (; sw < max_sweeps; ++sw) {
    double off = 0.0, tot = 0.0;
    for (long t = threadIdx.x; t < (long)n * n; t += blockDim.x) {
      const double v = A[t] * A[t];
      tot += v;
      if (t / n != t % n) off += v;
    }
    off_sh[threadIdx.x] = off;
    __syncthreads();
    if (threadIdx.x == 0) {
      double o = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) o += off_sh[i];
      off_sh[0] = o;
    }
    __syncthreads();
    const double offn = off_sh[0];
    __syncthreads();
    off_sh[threadIdx.x] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double o = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) o += off_sh[i];
      done = (offn <= 1e-30 * o) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (threadIdx.x == 0) {
          const double apq = A[(long)p * n + q];
          double c = 1.0, s = 0.0;
          if (fabs(apq) > 1e-300) {
            const double theta = (A[(long)q * n + q] - A[(long)p * n + p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double akp = A[(long)k * n + p], akq = A[(long)k * n + q];
            A[(long)k * n + p] = c * akp - s * akq;
            A[(long)k * n + q] = s * akp + c * akq;
            const double ukp = U[(long)k * n + p], ukq = U[(long)k * n + q];
            U[(long)k * n + p] = c * ukp - s * ukq;
            U[(long)k * n + q] = s * ukp + c * ukq;
          }
          __syncthreads();
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double apk = A[(long)p * n + k], aqk = A[(long)q * n + k];
            A[(long)p * n + k] = c * apk - s * aqk;
            A[(long)q * n + k] = s * apk + c * aqk;
          }
          __syncthreads();
          if (threadIdx.x == 0) {
            A[(long)p * n + q] = 0.0;
            A[(long)q * n + p] = 0.0;
          }
        }
        __syncthreads();
      }
  }
  if (threadIdx.x == 0) *sweeps = sw;
}

cudaError_t jacobi_eig_f64(double* A, double* U, int n, int max_sweeps, int* sweeps,
                           cudaStream_t s) {
  jacobi_kernel<<<1, 256, 0, s>>>(A, U, n, max_sweeps, sweeps);
  count_launch();
  return cudaGetLastError();
}

__global__ void scale_eigcols_kernel(const double* __restrict__ A, int n,
                                     const double* __restrict__ B, int rows, double cut,
                                     double* __restrict__ X, double* __restrict__ sign) {
  __shared__ double lmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < n; ++k) m = fmax(m, fabs(A[(long)k * n + k]));
    lmax = m;
  }
  __syncthreads();
  const double thr = cut * lmax;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)rows * n;
       t += (long)gridDim.x * blockDim.x) {
    const int k = (int)(t % n);
    const double lam = A[(long)k * n + k];
    X[t] = fabs(lam) > thr ? B[t] / sqrt(fabs(lam)) : 0.0;
  }
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double lam = A[(long)k * n + k];
      sign[k] = fabs(lam) > thr ? (lam > 0 ? 1.0 : -1.0) : 0.0;
    }
}

cudaError_t scale_eigcols_f64(const double* Adiag_src, int n, const double* B, int rows, double cut,
                              double* X, double* sign, cudaStream_t s) {
  scale_eigcols_kernel<<<64, 256, 0, s>>>(Adiag_src, n, B, rows, cut, X, sign);
  count_launch();
  return cudaGetLastError();
}

}  // namespace xk
