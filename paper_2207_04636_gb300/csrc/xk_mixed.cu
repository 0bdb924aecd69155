// Mixed-precision path of the exchange build on the 5th-generation tensor
// cores (tcgen05.mma kind::f16, TMA-fed shared memory, TMEM accumulators).
//
// Number format.  The FP32 accumulator of tcgen05.mma rounds every addition
// toward zero (the 16 products of one instruction are summed exactly, the
// sum is then truncated into the accumulator).  Truncation is biased, so
// long accumulation chains of ordinary FP16/BF16 splits drift by about half
// an ulp per instruction.  Every operand row is therefore split as
//     x = m + h,   m = q * round(x / q),   h = fp16(x - m),
// with a per-row power-of-two grid q = 2^(ceil(log2 max|row|) - 8), so that
// m is an integer multiple of q with |m / q| <= 256 (exact in FP16).  The
// product of two rows is then
//     A0 = sum m_x m_y        on the grid q_x q_y, exact while K <= 256,
//     A1 = sum m_x h_y + h_x m_y + h_x h_y,
// and A1 is about 2^-9 of A0, so its truncation bias is negligible.  A0 and
// A1 live in separate TMEM accumulators; longer sums are drained every
// <= 256 terms into round-to-nearest FP32 running sums.  The orbital product
// Psi = Phi' Q takes a third piece l = fp16(x - m - h) of both operands (six
// MMA passes): with two, its split error alone moved E_x by up to ~1e-6 Ha.
// The pair-kernel second product (V o P times the orbitals) uses a floating
// hi/lo split of V o P and drains every two tiles.
//
// Build chain (arXiv 2207.04636, Eq. exoccri with contraction order (a) of
// Sec. IV.D):
//   1. Psi = Phi C                            gemm                   (Eq. rpsEx step 1)
//   2. Psi_g = Psi[idx], per-row splits       split + gather
//   3. M2 = (V o (Psi_g Psi^T)) Psi           pair kernel, role A    (steps 2-3, line 2)
//      M1^T = (V^T o (Psi Psi_g^T)) Psi_g     pair kernel, role B    (line 1)
//      M3 = (W o (Psi_g Psi_g^T)) Psi_g       pair kernel, role C    (line 3)
//   4. line1^T = Phi^T M1^T, (line2 - line3)^T = Phi_g^T (M2 - M3)   gemm
//   5. K_{mu i} = dV (line1 + line2 - line3)^T (FP64)
//   6. E_x = -dV (2 sum V o P^2 - sum W o Q^2): the contraction of Eq. exoccri
//      with C in closed form, accumulated from the exact pair products in the
//      pair-kernel epilogues (FP32 per tile, FP64 across tiles).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tc_common.cuh"
#include "xk_internal.h"
#include "xk_mixed.h"

namespace xk {

namespace {

using namespace tc;

// ----------------------------------------------------------------- scales
// Global power-of-two scales (device floats) and maxima (FP32 bit patterns).
enum {
  SC_PHI = 0,   // Phi^T, Phi_g^T (the line contractions)
  SC_C,         // Q^T = (L^T C)^T
  SC_PSI,       // Psi, Psi_g
  SC_F_AB,      // V o P before its split (roles A, B)
  SC_F_C,       // W o Q before its split (role C)
  SC_M1,        // M1
  SC_D23,       // (M2 - M3)^T
  SC_OUT_ORB,   // Psi = acc * this
  SC_OUT_AB,    // M2, M1 = acc * this
  SC_OUT_C,     // M3 = acc * this
  SC_OUT_L1,    // line1 = acc * this
  SC_OUT_L23,   // line2 - line3 = acc * this
  SC_PHIP,      // Phi' = Phi L^{-T} (the orbital contraction)
  SC_FA,        // full K: M_A^T = ((V o P) Phi)^T before its split
  SC_FD,        // full K: (M_A - M_C)^T before its split
  SC_OUT_FA,    // full K: M_A = acc * this
  SC_OUT_FC,    // full K: M_C = ((W o Q) Phi_g) = acc * this
  SC_OUT_FY,    // full K: Phi_g^T M_A = acc * this
  SC_OUT_FZ,    // full K: Phi_g^T (M_A - M_C) = acc * this
  NSC
};
enum { AM_PHI = 0, AM_V, AM_W, AM_PHIP, AM_PHIP_RN, AM_C, AM_QCN, AM_PSI, AM_RN2, AM_M1, AM_D23,
       AM_FA, AM_FD, NAM };

constexpr float kHalfTarget = 16384.0f;  // 2^14: split inputs are scaled to |x| <= 2^14
constexpr float kProdTarget = 32768.0f;  // 2^15: V o P is scaled to |x| <= 2^15

__device__ float pow2_scale(float maxabs, float target) {
  if (!(maxabs > 0.0f) || !isfinite(maxabs)) return 1.0f;
  int e = (int)floorf(log2f(target / maxabs));
  float s = ldexpf(1.0f, e);
  while (s * maxabs > target) s *= 0.5f;
  while (s * 2.0f * maxabs <= target) s *= 2.0f;
  return s;
}

__device__ __forceinline__ float am_get(const unsigned* am, int i) { return __uint_as_float(am[i]); }

// stage 0: C scale; 1: Psi / pair scales; 2: M1, (M2 - M3) scales; 3: full-K scales.
__global__ void scales_kernel(const unsigned* __restrict__ am, float* __restrict__ sc, int stage) {
  if (threadIdx.x != 0) return;
  if (stage == 0) {
    sc[SC_C] = pow2_scale(am_get(am, AM_C), kHalfTarget);
    sc[SC_OUT_ORB] = 1.0f / (sc[SC_PHIP] * sc[SC_C]);
    // |Psi(R,j)| <= |Phi'(R,:)| |Q(:,j)| (Cauchy-Schwarz) bounds the orbital scale
    sc[SC_PSI] = pow2_scale(sqrtf(am_get(am, AM_PHIP_RN)) * sqrtf(am_get(am, AM_QCN)) * 1.0001f,
                            kHalfTarget);
  } else if (stage == 1) {
    const float sp = sc[SC_PSI];
    // |P(g,R)| <= max_R sum_i psi_i(R)^2 (Cauchy-Schwarz), so |V o P| <= max|V| rn2
    const float rn2 = am_get(am, AM_RN2) * sp * sp;
    const float fab = pow2_scale(am_get(am, AM_V) * rn2, kProdTarget);
    const float fc = pow2_scale(am_get(am, AM_W) * rn2, kProdTarget);
    sc[SC_F_AB] = fab;
    sc[SC_F_C] = fc;
    sc[SC_OUT_AB] = 1.0f / (fab * sp * sp * sp);
    sc[SC_OUT_C] = 1.0f / (fc * sp * sp * sp);
    sc[SC_OUT_FA] = 1.0f / (fab * sp * sp * sc[SC_PHI]);
    sc[SC_OUT_FC] = 1.0f / (fc * sp * sp * sc[SC_PHI]);
  } else if (stage == 3) {
    sc[SC_FA] = pow2_scale(am_get(am, AM_FA), kHalfTarget);
    sc[SC_FD] = pow2_scale(am_get(am, AM_FD), kHalfTarget);
    sc[SC_OUT_FY] = 1.0f / (sc[SC_PHI] * sc[SC_FA]);
    sc[SC_OUT_FZ] = 1.0f / (sc[SC_PHI] * sc[SC_FD]);
  } else {
    sc[SC_M1] = pow2_scale(am_get(am, AM_M1), kHalfTarget);
    sc[SC_D23] = pow2_scale(am_get(am, AM_D23), kHalfTarget);
    sc[SC_OUT_L1] = 1.0f / (sc[SC_PHI] * sc[SC_M1]);
    sc[SC_OUT_L23] = 1.0f / (sc[SC_PHI] * sc[SC_D23]);
  }
}

__global__ void set_phi_scale_kernel(const unsigned* __restrict__ am, float* __restrict__ sc) {
  if (threadIdx.x == 0) {
    sc[SC_PHI] = pow2_scale(am_get(am, AM_PHI), kHalfTarget);
    sc[SC_PHIP] = pow2_scale(am_get(am, AM_PHIP), kHalfTarget);
  }
}

__global__ void identity_kernel(double* a, int n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)n * n;
       t += (long)gridDim.x * blockDim.x)
    a[t] = (t / n == t % n) ? 1.0 : 0.0;
}

template <class T>
__global__ void absmax_kernel(const T* __restrict__ a, long rows, long cols, long ld,
                              unsigned* __restrict__ out) {
  float m = 0.0f;
  const long total = rows * cols;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / cols, c = t % cols;
    m = fmaxf(m, fabsf((float)a[r * ld + c]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// max over rows of sum_c a[r][c]^2.
template <class T>
__global__ void rownorm2_max_kernel(const T* __restrict__ a, long rows, int cols, long ld,
                                    unsigned* __restrict__ out) {
  float m = 0.0f;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows;
       r += (long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < cols; ++c) {
      const float v = (float)a[r * ld + c];
      s = fmaf(v, v, s);
    }
    m = fmaxf(m, s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m * 1.0001f));
}

// max over columns of sum_r a[r][c]^2 (one block per column).
__global__ void colnorm2_max_kernel(const double* __restrict__ a, long rows, long ld,
                                    unsigned* __restrict__ out) {
  __shared__ float red[8];
  const long c = blockIdx.x;
  float s = 0.0f;
  for (long r = threadIdx.x; r < rows; r += blockDim.x) {
    const float v = (float)a[r * ld + c];
    s = fmaf(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicMax(out, __float_as_uint(t * 1.0001f));
  }
}

// rowmax[r] = max_c |a[r][c]| and glob = max over all, for long FP32 rows whose
// stride is a multiple of 4 (2-D grid: x = column chunks, y = rows; float4 loads).
__global__ void rowmax2d_kernel(const float* __restrict__ a, long cols, long ld,
                                unsigned* __restrict__ rowmax, unsigned* __restrict__ glob) {
  const long r = blockIdx.y;
  const float4* row = reinterpret_cast<const float4*>(a + r * ld);
  const long n4 = cols / 4;
  float m = 0.0f;
  const long step = (long)gridDim.x * blockDim.x;
  long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  for (; c + 3 * step < n4; c += 4 * step) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = row[c + u * step];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
  }
  for (; c < n4; c += step) {
    const float4 v = row[c];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  if (blockIdx.x == 0)
    for (long t = n4 * 4 + threadIdx.x; t < cols; t += blockDim.x) m = fmaxf(m, fabsf(a[r * ld + t]));
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(rowmax + r, __float_as_uint(m));
    atomicMax(glob, __float_as_uint(m));
  }
}

// Grid of a row whose largest |value| is mx: q = 2^(ceil(log2 mx) - 8), at
// least 2^-24 (the FP16 subnormal step), so |x / q| <= 256.
__device__ __forceinline__ float row_grid(float mx) {
  if (!(mx > 0.0f)) return 1.0f;
  int E;
  const float f = frexpf(mx, &E);  // mx = f 2^E, f in [0.5, 1)
  const int e = (f == 0.5f) ? E - 1 : E;
  return ldexpf(1.0f, max(e - 8, -24));
}

// Row r of dst (one block of 128 threads per row): m, h pieces of
// src[r][c] * G on the row's grid for c < cols; zero for cols <= c < ld_dst.
template <class T>
__global__ void __launch_bounds__(128) split_mh_rows_kernel(
    const T* __restrict__ src, long cols, long ld_src, const float* __restrict__ sc, int gidx,
    __half* __restrict__ mo, __half* __restrict__ ho, __half* __restrict__ lo, long ld_dst) {
  __shared__ float red[4];
  const long r = blockIdx.x;
  const T G = (T)sc[gidx];
  const T* row = src + r * ld_src;
  float mx = 0.0f;
  for (long c = threadIdx.x; c < cols; c += blockDim.x) mx = fmaxf(mx, fabsf((float)(row[c] * G)));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
  // FP32 from here: rounding x to FP32 (2^-24) is far below the FP16 step of h
  const float q = row_grid(mx), qi = 1.0f / q;  // q a power of two: x * qi == x / q
  __half* mrow = mo + r * ld_dst;
  __half* hrow = ho + r * ld_dst;
  for (long c = threadIdx.x; c < ld_dst; c += blockDim.x) {
    __half mh = __float2half(0.0f), hh = __float2half(0.0f), lh = __float2half(0.0f);
    if (c < cols) {
      const float x = (float)(row[c] * G);
      const float m = q * rintf(x * qi);
      mh = __float2half_rn(m);
      hh = __float2half_rn(x - m);
      lh = __float2half_rn((x - m) - __half2float(hh));
    }
    mrow[c] = mh;
    hrow[c] = hh;
    if (lo) lo[r * ld_dst + c] = lh;
  }
}

// As split_mh_rows_kernel with the row maxima (of |src|, unscaled) given, for
// FP32 rows (stride a multiple of 4) into pieces of stride a multiple of 8:
// 2-D grid, x = chunks of 8 columns, y = rows.
__global__ void split_mh_rows_pre_kernel(const float* __restrict__ src, long cols, long ld_src,
                                         const unsigned* __restrict__ rowmax,
                                         const float* __restrict__ sc, int gidx,
                                         __half* __restrict__ mo, __half* __restrict__ ho,
                                         long ld_dst) {
  const long r = blockIdx.y;
  const float G = sc[gidx];
  const float q = row_grid(__uint_as_float(rowmax[r]) * G);
  const float qi = 1.0f / q;  // q is a power of two: x * qi == x / q
  const float* row = src + r * ld_src;
  for (long c8 = blockIdx.x * (long)blockDim.x + threadIdx.x; c8 * 8 < ld_dst;
       c8 += (long)gridDim.x * blockDim.x) {
    const long c = c8 * 8;
    float x[8];
    if (c + 8 <= cols) {
      const float4 v0 = *reinterpret_cast<const float4*>(row + c);
      const float4 v1 = *reinterpret_cast<const float4*>(row + c + 4);
      x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
      x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = (c + j < cols) ? row[c + j] : 0.0f;
    }
    uint32_t mw[4], hw[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const float x0 = x[j] * G, x1 = x[j + 1] * G;
      const float m0 = q * rintf(x0 * qi), m1 = q * rintf(x1 * qi);
      const __half2 hm = __floats2half2_rn(m0, m1);
      const __half2 hh = __floats2half2_rn(x0 - m0, x1 - m1);
      mw[j / 2] = *reinterpret_cast<const uint32_t*>(&hm);
      hw[j / 2] = *reinterpret_cast<const uint32_t*>(&hh);
    }
    *reinterpret_cast<uint4*>(mo + r * ld_dst + c) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
    *reinterpret_cast<uint4*>(ho + r * ld_dst + c) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  }
}

// dst[c][r] (ld_dst) = src[r][c] for r < rows, 0 for rows <= r < ld_dst; all c < cols.
template <class T>
__global__ void transpose_kernel(const T* __restrict__ src, long rows, long cols, long ld_src,
                                 T* __restrict__ dst, long ld_dst) {
  __shared__ T tile[32][33];
  const long r0 = (long)blockIdx.x * 32, c0 = (long)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * ld_src + c] : (T)0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_dst) dst[c * ld_dst + r] = tile[threadIdx.x][i];
  }
}

template <class T>
cudaError_t transpose(const T* src, long rows, long cols, long ld_src, T* dst, long ld_dst,
                      cudaStream_t s) {
  dim3 grid((unsigned)((ld_dst + 31) / 32), (unsigned)((cols + 31) / 32));
  transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, ld_src, dst, ld_dst);
  count_launch();
  return cudaGetLastError();
}

// dst[c][r] (stride ld_dst) = float(src[r][c]) for r < rows, c < cols.
__global__ void transpose_f64_f32_kernel(const double* __restrict__ src, long rows, long cols,
                                         long ld_src, float* __restrict__ dst, long ld_dst) {
  __shared__ float tile[32][33];
  const long r0 = (long)blockIdx.y * 32, c0 = (long)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? (float)src[r * ld_src + c] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ld_dst + r] = tile[threadIdx.x][i];
  }
}

// Per-row pieces of FP32 rows, one warp per row (grid-stride): m, h of
// src[r][c] * G on the row's grid for c < cols, zero for cols <= c < ld_dst
// (a multiple of 8); max_r sum_c src[r][c]^2 folded into rn2 once per block.
__global__ void split_rows_f32_kernel(const float* __restrict__ src, long rows, int cols,
                                      long ld_src, const float* __restrict__ sc, int gidx,
                                      __half* __restrict__ mo, __half* __restrict__ ho,
                                      __half* __restrict__ lo, long ld_dst,
                                      unsigned* __restrict__ rn2) {
  __shared__ float red[32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float G = sc[gidx];
  float wn = 0.0f;
  for (long r = (long)blockIdx.x * nw + wib; r < rows; r += (long)gridDim.x * nw) {
    const float* row = src + r * ld_src;
    float mx = 0.0f, nrm = 0.0f;
    for (int c = lane; c < cols; c += 32) {
      const float v = row[c];
      nrm = fmaf(v, v, nrm);
      mx = fmaxf(mx, fabsf(v * G));
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    wn = fmaxf(wn, nrm);
    const float q = row_grid(mx), qi = 1.0f / q;
    for (long c = (long)lane * 8; c < ld_dst; c += 256) {
      uint32_t mw[4], hw[4], lw[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const float x0 = c + j < cols ? row[c + j] * G : 0.0f;
        const float x1 = c + j + 1 < cols ? row[c + j + 1] * G : 0.0f;
        const float m0 = q * rintf(x0 * qi), m1 = q * rintf(x1 * qi);
        const __half2 hm = __floats2half2_rn(m0, m1);
        const __half2 hh = __floats2half2_rn(x0 - m0, x1 - m1);
        const float2 fh = __half22float2(hh);
        const __half2 hl = __floats2half2_rn((x0 - m0) - fh.x, (x1 - m1) - fh.y);
        mw[j / 2] = *reinterpret_cast<const uint32_t*>(&hm);
        hw[j / 2] = *reinterpret_cast<const uint32_t*>(&hh);
        lw[j / 2] = *reinterpret_cast<const uint32_t*>(&hl);
      }
      *reinterpret_cast<uint4*>(mo + r * ld_dst + c) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
      *reinterpret_cast<uint4*>(ho + r * ld_dst + c) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      if (lo) *reinterpret_cast<uint4*>(lo + r * ld_dst + c) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  }
  if (lane == 0) red[wib] = wn;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) wn = fmaxf(wn, red[w]);
    atomicMax(rn2, __float_as_uint(wn * 1.0001f));
  }
}

__global__ void gather_rows_half_kernel(const __half* __restrict__ src, long ld,
                                        const int32_t* __restrict__ idx, int rows,
                                        __half* __restrict__ dst) {
  const long total = (long)rows * ld;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / ld, c = t % ld;
    dst[t] = src[(long)idx[r] * ld + c];
  }
}

// FP64 [rows][cols] -> FP32 [rows][ld_dst], zero padding.
__global__ void f64_to_f32_kernel(const double* __restrict__ src, long rows, long cols,
                                  float* __restrict__ dst, long ld_dst) {
  const long total = rows * ld_dst;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / ld_dst, c = t % ld_dst;
    dst[t] = c < cols ? (float)src[r * cols + c] : 0.0f;
  }
}

// ------------------------------------------------------------ reductions

// out[t] = sum_s a[s][t] - sum_s b[s][t] in FP64 (b nullable); max |out| -> am_slot.
// Error-free accumulation of FP32 terms into an unevaluated sum hi + lo
// (two-sum), in a fixed order; about 2^-44 relative, on the FP32 pipes.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// a_scale (nullable): a power of two applied to the a terms (exact).
__global__ void reduce_parts_kernel(const float* __restrict__ a, int na, const float* __restrict__ b,
                                    int nb, long count, double* __restrict__ out,
                                    unsigned* __restrict__ am_slot,
                                    const float* __restrict__ a_scale = nullptr) {
  float m = 0.0f;
  const float as = a_scale ? *a_scale : 1.0f;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    float hi = 0.0f, lo = 0.0f;
#pragma unroll 8
    for (int p = 0; p < na; ++p) ff_add(hi, lo, a[(long)p * count + t] * as);
    if (b) {
#pragma unroll 8
      for (int p = 0; p < nb; ++p) ff_add(hi, lo, -b[(long)p * count + t]);
    }
    const double s = (double)hi + (double)lo;
    out[t] = s;
    m = fmaxf(m, fabsf((float)s));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (am_slot && (threadIdx.x & 31) == 0) atomicMax(am_slot, __float_as_uint(m));
}

// K[mu][j] = dV * (sum_s L1[s][mu][j] + sum_s L23[s][mu][j]), FP64.
__global__ void final_k_kernel(const float* __restrict__ L1, int n1, const float* __restrict__ L23,
                               int n23, long count, double dV, double* __restrict__ K) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
#pragma unroll 8
    for (int p = 0; p < n1; ++p) ff_add(h1, l1, L1[(long)p * count + t]);
#pragma unroll 8
    for (int p = 0; p < n23; ++p) ff_add(h2, l2, L23[(long)p * count + t]);
    const double s1 = (double)h1 + (double)l1, s2 = (double)h2 + (double)l2;
    K[t] = dV * (s1 + s2);
  }
}

// E_x = -dV (2 sum_k ea[k] - sum_k ec[k]) / G^4 with G the orbital scale, in
// a fixed summation order (one block of 256 threads).
__global__ void __launch_bounds__(1024) final_ex_kernel(const double* __restrict__ ea, int na_,
                                                       const double* __restrict__ ec, int nc_,
                                                       const float* __restrict__ sc, double dV,
                                                       double* Ex) {
  // one block of 1024 threads; four independent sums per thread keep several
  // loads in flight (the n > 128 path has ~10^5 partials per launch); the
  // order is fixed by the launch shape, so a build repeats bit for bit
  __shared__ double sa[32], sb[32];
  double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
  const int T = blockDim.x;
  int t = threadIdx.x;
  for (; t + 3 * T < na_; t += 4 * T) {
    a[0] += ea[t]; a[1] += ea[t + T]; a[2] += ea[t + 2 * T]; a[3] += ea[t + 3 * T];
  }
  for (; t < na_; t += T) a[0] += ea[t];
  t = threadIdx.x;
  for (; t + 3 * T < nc_; t += 4 * T) {
    b[0] += ec[t]; b[1] += ec[t + T]; b[2] += ec[t + 2 * T]; b[3] += ec[t + 3 * T];
  }
  for (; t < nc_; t += T) b[0] += ec[t];
  double x = (a[0] + a[1]) + (a[2] + a[3]), y = (b[0] + b[1]) + (b[2] + b[3]);
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  const int w = threadIdx.x >> 5, nw = T >> 5;
  if ((threadIdx.x & 31) == 0) { sa[w] = x; sb[w] = y; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, v = 0.0;
    for (int k = 0; k < nw; ++k) { u += sa[k]; v += sb[k]; }
    const double g = (double)sc[SC_PSI];
    const double g4 = (g * g) * (g * g);
    *Ex = -dV * (2.0 * u - v) / g4;
  }
}

// Full K: K[mu][nu] = dV (sum_s Z[s][mu][nu] + sum_s Y[s][nu][mu]), FP64, with
// Z = Phi_g^T (M_A - M_C) and Y = Phi_g^T M_A (two-sum FP32 over the splits).
__global__ void final_kfull_kernel(const float* __restrict__ Z, int nz, const float* __restrict__ Y,
                                   int ny, int N, double dV, double* __restrict__ K) {
  const long count = (long)N * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    const long mu = t / N, nu = t % N;
    float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
    for (int p = 0; p < nz; ++p) ff_add(h1, l1, Z[(long)p * count + t]);
    for (int p = 0; p < ny; ++p) ff_add(h2, l2, Y[(long)p * count + nu * N + mu]);
    K[t] = dV * (((double)h1 + (double)l1) + ((double)h2 + (double)l2));
  }
}

// ============================================================ gemm
// out[split][m][c] = scale * sum_{k in split} A[m][k] B[c][k] for one
// 128 x 128 tile, A and B as per-row (m, h) pieces, K-major, 3-stage TMA
// ring.  A0 (m.m) and A1 (m.h + h.m + h.h) accumulate in one of two TMEM
// sets; every kDrain k-blocks (192 terms) the epilogue adds A0 + A1 of the
// finished set into FP32 registers (round to nearest) while the MMA warp
// moves on to the other set.
// Warps 0-7: epilogue (warp w: rows of lane quadrant w % 4, columns
// 64 (w / 4) .. +63; thread = row); warp 8: TMA producer; warp 9: MMA.

struct GemmArgs {
  int M, Ncols, K, kchunk;
  float* out;
  long ldo;          // row stride of out
  long split_stride; // elements between splits of out
  const float* sc;
  int scale_idx;
  int* status;
  // When pm is set (one N tile, no split): write each output row as per-row
  // (m, h) pieces of (row * sc[piece_idx]) into pm / ph [M][ld_p] instead of
  // out, and fold max_r sum_c row[c]^2 into rn2.
  __half* pm;
  __half* ph;
  long ld_p;
  int piece_idx;
  unsigned* rn2;
  // Operands stored MN-major ([K][M], [K][N]; 64 x 64 TMA boxes) instead of
  // K-major ([M][K], [N][K]; 128 x 64 boxes).
  int a_mn, b_mn;
  int transposed;  // write out[col][row] (stride ldo) instead of out[row][col]
  int kdrain;  // k-blocks per accumulator drain (0: kDrain)
  // Three pieces per operand (K-major only): x = m + h + l, l = fp16(x - m - h);
  // A1 adds m l' + l m' (products below 2^-30 of the row maxima are dropped).
  // Two stages of six 16 KB tiles instead of three of four.
  int pieces3;
  // Logical grid of tiles (x: 128-row M tiles, y: 128-column N tiles, z: K
  // splits); the launch has at most one CTA per SM and each CTA walks the
  // tiles blockIdx.x, blockIdx.x + gridDim.x, ... (x fastest).
  int tiles_x, tiles_y, tiles_z;
  long long wait;  // pipeline-wait limit in SM cycles (0: the default)
};

constexpr int G_STAGES = 3;
constexpr int G_STAGE_BYTES = 4 * 16384;
constexpr int G_SMEM = G_STAGES * G_STAGE_BYTES + 1024;
constexpr int kDrain = 3;
constexpr int kGemmEpi = 8;                      // epilogue warps (4 lane quadrants x 2 column halves)
constexpr int kGemmTma = kGemmEpi, kGemmMma = kGemmEpi + 1;
constexpr int kGemmThreads = 32 * (kGemmEpi + 2);

// kShort: the launch shortened its pipeline-wait limit (a separate
// instantiation, so the default one keeps the plain bounded wait).
template <bool kShort>
__device__ __forceinline__ void gemm_body(const CUtensorMap* pAm, const CUtensorMap* pAh,
                                          const CUtensorMap* pBm, const CUtensorMap* pBh,
                                          const CUtensorMap* pAl, const CUtensorMap* pBl,
                                          const GemmArgs& g) {
  extern __shared__ uint8_t g_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(g_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[G_STAGES], empty[G_STAGES], set_ready[2], set_free[2], drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = g.tiles_x * g.tiles_y * g.tiles_z;
  const int kd = g.kdrain > 0 ? g.kdrain : kDrain;
  // tile t -> (M tile, N tile, K split) and its number of 64-wide k-blocks
  auto tile_at = [&](int t, int& bx, int& by, int& bz) {
    bx = t % g.tiles_x;
    by = (t / g.tiles_x) % g.tiles_y;
    bz = t / (g.tiles_x * g.tiles_y);
  };
  auto kblocks = [&](int bz) {
    const int kb0 = bz * g.kchunk, ke = min(g.K, kb0 + g.kchunk);
    return ke > kb0 ? (ke - kb0 + 63) / 64 : 0;
  };
  const bool p3 = g.pieces3 != 0;
  const long long lw = kShort ? wait_limit(g.wait) : kWaitCycles;
  const int ns = p3 ? 2 : G_STAGES;                       // stages
  const int sbytes = p3 ? 6 * 16384 : G_STAGE_BYTES;      // bytes per stage

  if (tid == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&set_ready[s], 1);
      mbar_init(&set_free[s], kGemmEpi);  // one arrival per epilogue warp
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kGemmMma) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == kGemmTma && lane == 0) {
    prefetch_tmap(pAm); prefetch_tmap(pAh); prefetch_tmap(pBm); prefetch_tmap(pBh);
    int last_parity[G_STAGES] = {-1, -1, -1};
    int it = 0;  // k-blocks issued by this CTA over all its tiles
    for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
    int bx, by, bz;
    tile_at(tile, bx, by, bz);
    const int m0 = bx * 128, n0 = by * 128, kbeg = bz * g.kchunk, nkb = kblocks(bz);
    for (int kb = 0; kb < nkb && !abort_flag; ++kb, ++it) {
      const int s = it % ns, use = it / ns;
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, lw)) {
        atomicExch(g.status, 11); abort_flag = 1; break;
      }
      uint8_t* st = sm + s * sbytes;
      mbar_expect_tx(&full[s], sbytes);
      const int kc = kbeg + kb * 64;
      if (p3) {  // A m, h, l at 0, 16, 32 KB; B m, h, l at 48, 64, 80 KB
        tma_load_2d(st, pAm, &full[s], kc, m0);
        tma_load_2d(st + 16384, pAh, &full[s], kc, m0);
        tma_load_2d(st + 32768, pAl, &full[s], kc, m0);
        tma_load_2d(st + 49152, pBm, &full[s], kc, n0);
        tma_load_2d(st + 65536, pBh, &full[s], kc, n0);
        tma_load_2d(st + 81920, pBl, &full[s], kc, n0);
        last_parity[s] = use & 1;
        continue;
      }
      if (!g.a_mn) {
        tma_load_2d(st, pAm, &full[s], kc, m0);
        tma_load_2d(st + 16384, pAh, &full[s], kc, m0);
      } else {  // [64 K rows][64 M] boxes, M halves 8 KB apart
        tma_load_2d(st, pAm, &full[s], m0, kc);
        tma_load_2d(st + 8192, pAm, &full[s], m0 + 64, kc);
        tma_load_2d(st + 16384, pAh, &full[s], m0, kc);
        tma_load_2d(st + 24576, pAh, &full[s], m0 + 64, kc);
      }
      if (!g.b_mn) {
        tma_load_2d(st + 32768, pBm, &full[s], kc, n0);
        tma_load_2d(st + 49152, pBh, &full[s], kc, n0);
      } else {
        tma_load_2d(st + 32768, pBm, &full[s], n0, kc);
        tma_load_2d(st + 40960, pBm, &full[s], n0 + 64, kc);
        tma_load_2d(st + 49152, pBh, &full[s], n0, kc);
        tma_load_2d(st + 57344, pBh, &full[s], n0 + 64, kc);
      }
      last_parity[s] = use & 1;
    }
    }
    for (int s = 0; s < ns; ++s)
      if (last_parity[s] >= 0) mbar_wait(&full[s], last_parity[s]);
  } else if (warp == kGemmMma) {
    // whole warp runs the loop; one elected lane issues each MMA and commit
    const uint32_t idesc = idesc_f16(128, 128, false, g.a_mn != 0, g.b_mn != 0);
    // K-major tiles step 32 B per K = 16; MN-major tiles step 16 rows (2 KB)
    // and keep their two 64-wide halves 8 KB apart (LBO)
    const uint64_t dkm = sdesc_sw128(smem_u32(sm), 16, 1024);
    const uint64_t dmn = sdesc_sw128(smem_u32(sm), 8192, 1024);
    const uint64_t da0 = g.a_mn ? dmn : dkm, db0 = g.b_mn ? dmn : dkm;
    const uint32_t ast = g.a_mn ? 128 : 2, bst = g.b_mn ? 128 : 2;
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(g.status, code); abort_flag = 1; }
      __syncwarp();
    };
    // it: k-blocks over all tiles (stage ring); G0: the tile's first drain group
    // over all tiles (accumulator sets alternate across tile boundaries too)
    int it = 0, G0 = 0;
    bool good = true;
    for (int tile = blockIdx.x; good && tile < ntiles; tile += gridDim.x) {
    int bx, by, bz;
    tile_at(tile, bx, by, bz);
    const int nkb = kblocks(bz);
    for (int kb = 0; kb < nkb; ++kb, ++it) {
      if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) { good = false; break; }
      const int s = it % ns, grp = G0 + kb / kd, set = grp & 1;
      const bool first = (kb % kd) == 0;
      const bool last = (kb % kd) == kd - 1 || kb == nkb - 1;
      if (first && grp >= 2 && !mbar_wait_warp(&set_free[set], ((grp >> 1) - 1) & 1, lw)) {
        fail(14); good = false; break;
      }
      if (!mbar_wait_warp(&full[s], (it / ns) & 1, lw)) { fail(12); good = false; break; }
      tc_fence_after();
      if (p3) {
        const uint64_t dam = dkm + s * (uint64_t)(sbytes >> 4), dah = dam + 1024, dal = dam + 2048;
        const uint64_t dbm = dam + 3072, dbh = dam + 4096, dbl = dam + 5120;
        const uint32_t t0 = tbase + set * 256, t1 = t0 + 128;
        const uint32_t a0 = first ? 0u : 1u;
        mma_ss_run4(t0, dam, dbm, 2, 2, idesc, a0);
        mma_ss_run4(t1, dam, dbh, 2, 2, idesc, a0);
        mma_ss_run4(t1, dah, dbm, 2, 2, idesc, 1u);
        mma_ss_run4(t1, dah, dbh, 2, 2, idesc, 1u);
        mma_ss_run4(t1, dam, dbl, 2, 2, idesc, 1u);
        mma_ss_run4(t1, dal, dbm, 2, 2, idesc, 1u);
        if (elect_one()) {
          mma_commit(&empty[s]);
          if (last) mma_commit(&set_ready[set]);
        }
        __syncwarp();
        continue;
      }
      // stage s: A m-piece at +0, A h at +16 KB, B m at +32 KB, B h at +48 KB; the
      // descriptor address field counts 16-byte units (1024 per 16 KB, 2 per K step)
      const uint64_t dam = da0 + s * (G_STAGE_BYTES >> 4), dah = dam + 1024;
      const uint64_t dbm = db0 + s * (G_STAGE_BYTES >> 4) + 2048, dbh = dbm + 1024;
      const uint32_t t0 = tbase + set * 256, t1 = t0 + 128;
      const uint32_t a0 = first ? 0u : 1u;
      mma_ss_run4(t0, dam, dbm, ast, bst, idesc, a0);
      mma_ss_run4(t1, dam, dbh, ast, bst, idesc, a0);
      mma_ss_run4(t1, dah, dbm, ast, bst, idesc, 1u);
      mma_ss_run4(t1, dah, dbh, ast, bst, idesc, 1u);
      if (elect_one()) {
        mma_commit(&empty[s]);
        if (last) mma_commit(&set_ready[set]);
      }
      __syncwarp();
    }
    G0 += (nkb + kd - 1) / kd;
    }
    if (elect_one()) mma_commit(&drain);
    __syncwarp();
    mbar_wait_warp(&drain, 0);
  } else if (warp < kGemmEpi) {
    // warp w: TMEM lane quadrant w % 4 (rows), column half w / 4 (64 columns)
    const int quad = warp & 3, half = warp >> 2;
    const int r = quad * 32 + lane;
    const int cb = 64 * half;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    __shared__ float prow_mx[2][128], prow_nrm[2][128];
    // Every epilogue warp walks all of the CTA's tiles (after a failed wait
    // without waiting further), so the named barriers below match up.
    int G0 = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int bx, by, bz;
    tile_at(tile, bx, by, bz);
    const int m0 = bx * 128, n0 = by * 128;
    const int ngroups = (kblocks(bz) + kd - 1) / kd;
    float run[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) run[c] = 0.0f;
    bool ok = true;
    for (int gi = 0; gi < ngroups; ++gi) {
      const int grp = G0 + gi, set = grp & 1;
      if (__shfl_sync(0xffffffffu, (int)abort_flag, 0) || !mbar_wait_warp(&set_ready[set], (grp >> 1) & 1, lw)) {
        ok = false;
        if (lane == 0 && !abort_flag) { atomicExch(g.status, 13); abort_flag = 1; }
        __syncwarp();
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        uint32_t a0[16], a1[16];
        tmem_ld16(tbase + lane_off + set * 256 + cb + c, a0);
        tmem_ld16(tbase + lane_off + set * 256 + 128 + cb + c, a1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) run[c + j] += __uint_as_float(a0[j]) + __uint_as_float(a1[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&set_free[set]);
    }
    G0 += ngroups;
    ok = ok && !abort_flag;
    const float scale = g.sc[g.scale_idx];
    if (g.pm) {
      // orbital rows: values, row norm, per-row grid (over both column halves), pieces
      float mx = 0.0f, nrm = 0.0f;
      const float G = g.sc[g.piece_idx];
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        const float v = (ok && cb + c < g.Ncols) ? run[c] * scale : 0.0f;
        run[c] = v;
        nrm = fmaf(v, v, nrm);
        mx = fmaxf(mx, fabsf(v * G));
      }
      prow_mx[half][r] = mx;
      prow_nrm[half][r] = nrm;
      asm volatile("bar.sync 1, %0;" ::"n"(32 * kGemmEpi) : "memory");
      mx = fmaxf(prow_mx[0][r], prow_mx[1][r]);
      nrm = prow_nrm[0][r] + prow_nrm[1][r];
      asm volatile("bar.sync 1, %0;" ::"n"(32 * kGemmEpi) : "memory");  // rewritten by the next tile
      if (half == 0) {
        float wn = (m0 + r < g.M) ? nrm : 0.0f;
        for (int o = 16; o > 0; o >>= 1) wn = fmaxf(wn, __shfl_xor_sync(0xffffffffu, wn, o));
        if (lane == 0) atomicMax(g.rn2, __float_as_uint(wn * 1.0001f));
      }
      if (m0 + r < g.M) {
        const float q = row_grid(mx), qi = 1.0f / q;  // q a power of two: x * qi == x / q
        __half* mrow = g.pm + (long)(m0 + r) * g.ld_p + cb;
        __half* hrow = g.ph + (long)(m0 + r) * g.ld_p + cb;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 8) {
          if (cb + c0 >= g.ld_p) break;
          uint32_t mw[4], hw[4];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const float x0 = run[c0 + j] * G, x1 = run[c0 + j + 1] * G;
            const float m0v = q * rintf(x0 * qi), m1v = q * rintf(x1 * qi);
            const __half2 hm = __floats2half2_rn(m0v, m1v);
            const __half2 hh = __floats2half2_rn(x0 - m0v, x1 - m1v);
            mw[j / 2] = *reinterpret_cast<const uint32_t*>(&hm);
            hw[j / 2] = *reinterpret_cast<const uint32_t*>(&hh);
          }
          *reinterpret_cast<uint4*>(mrow + c0) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
          *reinterpret_cast<uint4*>(hrow + c0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        }
      }
    } else if (g.transposed) {
      const long row = (long)m0 + r;
      if (row < g.M) {
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int col = n0 + cb + c;
          if (col < g.Ncols) g.out[(long)col * g.ldo + row] = ok ? run[c] * scale : 0.0f;
        }
      }
    } else if (m0 + r < g.M) {
      float* orow = g.out + (long)bz * g.split_stride + (long)(m0 + r) * g.ldo;
      if (((g.ldo | g.split_stride) & 3) == 0) {  // 16-byte row segments
#pragma unroll
        for (int c = 0; c < 64; c += 4) {
          const int col = n0 + cb + c;
          if (col + 4 <= g.Ncols) {
            *reinterpret_cast<float4*>(orow + col) =
                ok ? make_float4(run[c] * scale, run[c + 1] * scale, run[c + 2] * scale,
                                 run[c + 3] * scale)
                   : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (col + j < g.Ncols) orow[col + j] = ok ? run[c + j] * scale : 0.0f;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int col = n0 + cb + c;
          if (col < g.Ncols) orow[col] = ok ? run[c] * scale : 0.0f;
        }
      }
    }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kGemmMma) tmem_dealloc(tbase, 512);
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap mAm, const __grid_constant__ CUtensorMap mAh,
                const __grid_constant__ CUtensorMap mBm, const __grid_constant__ CUtensorMap mBh,
                const __grid_constant__ CUtensorMap mAl, const __grid_constant__ CUtensorMap mBl,
                GemmArgs g) {
  if (g.wait > 0 && g.wait < kWaitCycles)
    gemm_body<true>(&mAm, &mAh, &mBm, &mBh, &mAl, &mBl, g);
  else
    gemm_body<false>(&mAm, &mAh, &mBm, &mBh, &mAl, &mBl, g);
}

// SMs of the current device (cached per device).
int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 152;
  }
  return cached[dev];
}

// gemm_kernel over the logical grid `tiles` with at most one CTA per SM.
void launch_gemm(const CUtensorMap& mAm, const CUtensorMap& mAh, const CUtensorMap& mBm,
                 const CUtensorMap& mBh, const CUtensorMap& mAl, const CUtensorMap& mBl, GemmArgs g,
                 dim3 tiles, cudaStream_t s, long long wait = 0) {
  g.wait = wait;
  g.tiles_x = (int)tiles.x;
  g.tiles_y = (int)tiles.y;
  g.tiles_z = (int)tiles.z;
  const long total = (long)tiles.x * tiles.y * tiles.z;
  const unsigned ctas = (unsigned)std::max<long>(1, std::min<long>(total, sm_count()));
  gemm_kernel<<<ctas, kGemmThreads, G_SMEM, s>>>(mAm, mAh, mBm, mBh, mAl, mBl, g);
}

// ============================================================ wide gemm
// The same contraction as gemm_kernel over 128 x 256 output tiles (for the
// n > 128 back-contractions M2 = T_A Psi, M3 = T_C Psi_g, M1^T = T_A^T
// Psi_g): each 96 KB stage of operands (A m, h [128][64]; B m, h [256][64]
// or [64][4 x 64]) feeds twice the MMA work of a 128 x 128 stage, so the
// TMA ring needs 47 instead of 64 bytes per tensor-core cycle.  A0 and A1
// fill the 512 columns of tensor memory (one set): the MMA warp waits for the
// drain of each 192-term group before it starts the next, and 16 epilogue
// warps (lane quadrant w % 4, 64 columns (w / 4)) keep that drain short.
// Output: plain (splits) or transposed, as in gemm_kernel.
constexpr int GW_STAGES = 2;
constexpr int GW_STAGE_BYTES = 2 * 16384 + 2 * 32768;
constexpr int GW_SMEM = GW_STAGES * GW_STAGE_BYTES + 1024;
constexpr int kWideEpi = 16;
constexpr int kWideTma = kWideEpi, kWideMma = kWideEpi + 1;
constexpr int kWideThreads = 32 * (kWideEpi + 2);

// kP3: three pieces per operand (K-major only; the n > 128 orbital product):
// 32-wide K blocks with the 64-byte swizzle, stages of A m, h, l [128][32]
// and B m, h, l [256][32] (72 KB, three stages), six products per K step
// (A1 adds m.l' + l.m'), a drain every 6 K blocks (192 terms).
template <bool kShort, bool kP3>
__device__ __forceinline__ void gemm_wide_body(const CUtensorMap* pAm, const CUtensorMap* pAh,
                                               const CUtensorMap* pBm, const CUtensorMap* pBh,
                                               const CUtensorMap* pAl, const CUtensorMap* pBl,
                                               const GemmArgs& g) {
  extern __shared__ uint8_t gw_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gw_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[3], empty[3], set_ready, set_free, drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = g.tiles_x * g.tiles_y * g.tiles_z;
  auto tile_at = [&](int t, int& bx, int& by, int& bz) {
    bx = t % g.tiles_x;
    by = (t / g.tiles_x) % g.tiles_y;
    bz = t / (g.tiles_x * g.tiles_y);
  };
  constexpr int KB = kP3 ? 32 : 64;                  // K per block
  constexpr int kd = kP3 ? 2 * kDrain : kDrain;      // blocks per drain (192 terms)
  auto kblocks = [&](int bz) {
    const int kb0 = bz * g.kchunk, ke = min(g.K, kb0 + g.kchunk);
    return ke > kb0 ? (ke - kb0 + KB - 1) / KB : 0;
  };
  const long long lw = kShort ? wait_limit(g.wait) : kWaitCycles;
  constexpr int ns = kP3 ? 3 : GW_STAGES;
  constexpr int sbytes = kP3 ? 3 * 8192 + 3 * 16384 : GW_STAGE_BYTES;

  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&set_ready, 1);
    mbar_init(&set_free, kWideEpi);  // one arrival per epilogue warp
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kWideMma) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == kWideTma && lane == 0) {
    prefetch_tmap(pAm); prefetch_tmap(pAh); prefetch_tmap(pBm); prefetch_tmap(pBh);
    int last_parity[3] = {-1, -1, -1};
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
      int bx, by, bz;
      tile_at(tile, bx, by, bz);
      const int m0 = bx * 128, n0 = by * 256, kbeg = bz * g.kchunk, nkb = kblocks(bz);
      for (int kb = 0; kb < nkb && !abort_flag; ++kb, ++it) {
        const int s = it % ns, use = it / ns;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, lw)) {
          atomicExch(g.status, 31); abort_flag = 1; break;
        }
        uint8_t* st = sm + s * sbytes;  // A m +0, A h +16 KB, B m +32 KB, B h +64 KB
        mbar_expect_tx(&full[s], sbytes);
        const int kc = kbeg + kb * KB;
        if constexpr (kP3) {  // A m, h, l at 0, 8, 16 KB; B m, h, l at 24, 40, 56 KB
          tma_load_2d(st, pAm, &full[s], kc, m0);
          tma_load_2d(st + 8192, pAh, &full[s], kc, m0);
          tma_load_2d(st + 16384, pAl, &full[s], kc, m0);
          tma_load_2d(st + 24576, pBm, &full[s], kc, n0);
          tma_load_2d(st + 40960, pBh, &full[s], kc, n0);
          tma_load_2d(st + 57344, pBl, &full[s], kc, n0);
          last_parity[s] = use & 1;
          continue;
        }
        if (!g.a_mn) {
          tma_load_2d(st, pAm, &full[s], kc, m0);
          tma_load_2d(st + 16384, pAh, &full[s], kc, m0);
        } else {  // [64 K rows][64 M] boxes, M halves 8 KB apart
          tma_load_2d(st, pAm, &full[s], m0, kc);
          tma_load_2d(st + 8192, pAm, &full[s], m0 + 64, kc);
          tma_load_2d(st + 16384, pAh, &full[s], m0, kc);
          tma_load_2d(st + 24576, pAh, &full[s], m0 + 64, kc);
        }
        if (!g.b_mn) {  // [256 N rows][64 K] boxes
          tma_load_2d(st + 32768, pBm, &full[s], kc, n0);
          tma_load_2d(st + 65536, pBh, &full[s], kc, n0);
        } else {  // [64 K rows][64 N] boxes, four N blocks 8 KB apart
          for (int q = 0; q < 4; ++q) {
            tma_load_2d(st + 32768 + 8192 * q, pBm, &full[s], n0 + 64 * q, kc);
            tma_load_2d(st + 65536 + 8192 * q, pBh, &full[s], n0 + 64 * q, kc);
          }
        }
        last_parity[s] = use & 1;
      }
    }
    for (int s = 0; s < ns; ++s)
      if (last_parity[s] >= 0) mbar_wait(&full[s], last_parity[s]);
  } else if (warp == kWideMma) {
    const uint32_t idesc = idesc_f16(128, 256, false, g.a_mn != 0, g.b_mn != 0);
    const uint64_t dkm = sdesc_sw128(smem_u32(sm), 16, 1024);
    const uint64_t dmn = sdesc_sw128(smem_u32(sm), 8192, 1024);
    const uint64_t da0 = g.a_mn ? dmn : dkm, db0 = g.b_mn ? dmn : dkm;
    const uint32_t ast = g.a_mn ? 128 : 2, bst = g.b_mn ? 128 : 2;
    const uint64_t d64 = sdesc_sw64(smem_u32(sm), 16, 512);  // three-piece K-major tiles
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(g.status, code); abort_flag = 1; }
      __syncwarp();
    };
    int it = 0, G = 0;  // G: drain groups issued over all tiles
    bool good = true;
    for (int tile = blockIdx.x; good && tile < ntiles; tile += gridDim.x) {
      int bx, by, bz;
      tile_at(tile, bx, by, bz);
      const int nkb = kblocks(bz);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) { good = false; break; }
        const int s = it % ns;
        const bool first = (kb % kd) == 0;
        const bool last = (kb % kd) == kd - 1 || kb == nkb - 1;
        // one accumulator set: group G starts once the epilogue drained group G - 1
        if (first && G >= 1 && !mbar_wait_warp(&set_free, (G - 1) & 1, lw)) {
          fail(34); good = false; break;
        }
        if (!mbar_wait_warp(&full[s], (it / ns) & 1, lw)) { fail(32); good = false; break; }
        tc_fence_after();
        const uint32_t t0 = tbase, t1 = tbase + 256;
        const uint32_t a0 = first ? 0u : 1u;
        if constexpr (kP3) {
          // descriptor address field in 16-byte units: 512 per 8 KB
          const uint64_t am = d64 + (uint64_t)((s * sbytes) >> 4), ah = am + 512, al = am + 1024;
          const uint64_t bm = am + 1536, bh = bm + 1024, bl = bm + 2048;
          mma_ss_run2(t0, am, bm, 2, 2, idesc, a0);
          mma_ss_run2(t1, am, bh, 2, 2, idesc, a0);
          mma_ss_run2(t1, ah, bm, 2, 2, idesc, 1u);
          mma_ss_run2(t1, ah, bh, 2, 2, idesc, 1u);
          mma_ss_run2(t1, am, bl, 2, 2, idesc, 1u);
          mma_ss_run2(t1, al, bm, 2, 2, idesc, 1u);
        } else {
          const uint64_t dam = da0 + s * (GW_STAGE_BYTES >> 4), dah = dam + 1024;
          const uint64_t dbm = db0 + s * (GW_STAGE_BYTES >> 4) + 2048, dbh = dbm + 2048;
          mma_ss_run4(t0, dam, dbm, ast, bst, idesc, a0);
          mma_ss_run4(t1, dam, dbh, ast, bst, idesc, a0);
          mma_ss_run4(t1, dah, dbm, ast, bst, idesc, 1u);
          mma_ss_run4(t1, dah, dbh, ast, bst, idesc, 1u);
        }
        if (elect_one()) {
          mma_commit(&empty[s]);
          if (last) mma_commit(&set_ready);
        }
        __syncwarp();
        if (last) ++G;
      }
    }
    if (elect_one()) mma_commit(&drain);
    __syncwarp();
    mbar_wait_warp(&drain, 0);
  } else if (warp < kWideEpi) {
    const int quad = warp & 3, qc = warp >> 2;
    const int r = quad * 32 + lane;
    const int cb = 64 * qc;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    int G = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      int bx, by, bz;
      tile_at(tile, bx, by, bz);
      const int m0 = bx * 128, n0 = by * 256;
      const int ngroups = (kblocks(bz) + kd - 1) / kd;
      float run[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) run[c] = 0.0f;
      bool ok = true;
      for (int gi = 0; gi < ngroups; ++gi, ++G) {
        if (__shfl_sync(0xffffffffu, (int)abort_flag, 0) || !mbar_wait_warp(&set_ready, G & 1, lw)) {
          ok = false;
          if (lane == 0 && !abort_flag) { atomicExch(g.status, 33); abort_flag = 1; }
          __syncwarp();
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < 64; c += 8) {
          uint32_t a0[8], a1[8];
          tmem_ld8(tbase + lane_off + cb + c, a0);
          tmem_ld8(tbase + lane_off + 256 + cb + c, a1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) run[c + j] += __uint_as_float(a0[j]) + __uint_as_float(a1[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&set_free);
      }
      ok = ok && !abort_flag;
      const float scale = g.sc[g.scale_idx];
      const long row = (long)m0 + r;
      if (row < g.M) {
        if (g.transposed) {
#pragma unroll
          for (int c = 0; c < 64; ++c) {
            const int col = n0 + cb + c;
            if (col < g.Ncols) g.out[(long)col * g.ldo + row] = ok ? run[c] * scale : 0.0f;
          }
        } else {
          float* orow = g.out + (long)bz * g.split_stride + row * g.ldo;
          if (((g.ldo | g.split_stride) & 3) == 0) {
#pragma unroll
            for (int c = 0; c < 64; c += 4) {
              const int col = n0 + cb + c;
              if (col + 4 <= g.Ncols) {
                *reinterpret_cast<float4*>(orow + col) =
                    ok ? make_float4(run[c] * scale, run[c + 1] * scale, run[c + 2] * scale,
                                     run[c + 3] * scale)
                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
              } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  if (col + j < g.Ncols) orow[col + j] = ok ? run[c + j] * scale : 0.0f;
              }
            }
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) {
              const int col = n0 + cb + c;
              if (col < g.Ncols) orow[col] = ok ? run[c] * scale : 0.0f;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kWideMma) tmem_dealloc(tbase, 512);
}

__global__ void __launch_bounds__(kWideThreads, 1)
    gemm_wide_kernel(const __grid_constant__ CUtensorMap mAm, const __grid_constant__ CUtensorMap mAh,
                     const __grid_constant__ CUtensorMap mBm, const __grid_constant__ CUtensorMap mBh,
                     GemmArgs g) {
  if (g.wait > 0 && g.wait < kWaitCycles)
    gemm_wide_body<true, false>(&mAm, &mAh, &mBm, &mBh, &mAm, &mBm, g);
  else
    gemm_wide_body<false, false>(&mAm, &mAh, &mBm, &mBh, &mAm, &mBm, g);
}

// Three pieces per operand, K-major, [128][32] / [256][32] boxes with the
// 64-byte swizzle (the n > 128 orbital product).
__global__ void __launch_bounds__(kWideThreads, 1)
    gemm_wide3_kernel(const __grid_constant__ CUtensorMap mAm, const __grid_constant__ CUtensorMap mAh,
                      const __grid_constant__ CUtensorMap mAl, const __grid_constant__ CUtensorMap mBm,
                      const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                      GemmArgs g) {
  if (g.wait > 0 && g.wait < kWaitCycles)
    gemm_wide_body<true, true>(&mAm, &mAh, &mBm, &mBh, &mAl, &mBl, g);
  else
    gemm_wide_body<false, true>(&mAm, &mAh, &mBm, &mBh, &mAl, &mBl, g);
}

constexpr int GW3_SMEM = 3 * (3 * 8192 + 3 * 16384) + 1024;

void launch_gemm_wide3(const CUtensorMap& mAm, const CUtensorMap& mAh, const CUtensorMap& mAl,
                       const CUtensorMap& mBm, const CUtensorMap& mBh, const CUtensorMap& mBl,
                       GemmArgs g, dim3 tiles, cudaStream_t s, long long wait = 0) {
  g.wait = wait;
  g.tiles_x = (int)tiles.x;
  g.tiles_y = (int)tiles.y;
  g.tiles_z = (int)tiles.z;
  const long total = (long)tiles.x * tiles.y * tiles.z;
  const unsigned ctas = (unsigned)std::max<long>(1, std::min<long>(total, sm_count()));
  gemm_wide3_kernel<<<ctas, kWideThreads, GW3_SMEM, s>>>(mAm, mAh, mAl, mBm, mBh, mBl, g);
}

// gemm_wide_kernel over tiles (x: 128-row M tiles, y: 256-column N tiles,
// z: K splits) with at most one CTA per SM.
void launch_gemm_wide(const CUtensorMap& mAm, const CUtensorMap& mAh, const CUtensorMap& mBm,
                      const CUtensorMap& mBh, GemmArgs g, dim3 tiles, cudaStream_t s,
                      long long wait = 0) {
  g.wait = wait;
  g.tiles_x = (int)tiles.x;
  g.tiles_y = (int)tiles.y;
  g.tiles_z = (int)tiles.z;
  const long total = (long)tiles.x * tiles.y * tiles.z;
  const unsigned ctas = (unsigned)std::max<long>(1, std::min<long>(total, sm_count()));
  gemm_wide_kernel<<<ctas, kWideThreads, GW_SMEM, s>>>(mAm, mAh, mBm, mBh, g);
}

// ============================================================ T products
// One 128 x 128 tile of T = f V' o S, S = A B^T over K = the pieces' width
// (n rounded up to 64): A (rows: the slice's interpolation points) and B
// (rows: grid points, or every interpolation point for T_C) as per-row FP16
// pieces (m, h[, l]), K-major, streamed by TMA in 32-wide K blocks with the
// 64-byte swizzle (one box per operand spans its pieces).  A0 = m.m' and A1 = the cross terms (m.h' + h.m' + h.h'
// [+ m.l' + l.m']) accumulate in one of two tensor-memory sets, drained
// every 6 K blocks (192 terms) into FP32 sums held in registers, as in
// gemm_body.  The epilogue takes the V' tile (FP32, four [128][32] boxes)
// from shared memory, where it loads it by TMA as soon as the previous
// tile's T has left shared memory.  Each thread (one row, 64
// columns) forms V' o S, the energy term V' S^2 and the FP16 hi/lo split of
// f V' S, writes the split in place of the V' boxes its column half has read,
// and one thread per half stores the four [128][32] FP16 boxes with TMA and
// writes the half's energy partial.  V' and T thus cross between HBM and the
// SM in whole lines, no thread waits on a global load or store, and the two
// column halves run without synchronising with each other.
// Warps 0-7: epilogue (warp w: rows 32 (w % 4) .. +31, columns 64 (w / 4)
// .. +63); warp 8: TMA producer; warp 9: MMA.

struct TprodMaps {
  CUtensorMap a, b;        // A and B over (K, rows, piece): [piece][128][32] boxes, 64-byte swizzle
  CUtensorMap v;           // V' FP32 [M][Ncols]: [128][32] boxes, 128-byte swizzle
  CUtensorMap th, tl;      // T hi / lo FP16 [M][ld]: [128][32] boxes, 64-byte swizzle
};

struct TprodArgs {
  int M, Ncols, K;  // rows of A, rows of B (columns of T), K (a multiple of 32)
  const float* sc;
  int f_idx;
  double* epart;    // [2 (by * tiles_x + bx) + column half]: sum V' S^2; nullable
  int store;        // write T (hi, lo) through the maps th, tl
  int ld_t;         // columns of T's rows (the maps' extent): boxes past it are not stored
  int pieces3;      // three pieces per operand (else two)
  int tiles_x, tiles_y;
  int* status;
  long long wait;   // pipeline-wait limit in SM cycles (0: the default)
};

constexpr int TP_KB = 32;                    // K per block
constexpr int TP_BOX = 128 * TP_KB * 2;      // one [128][32] FP16 box: 8 KB
constexpr int TP_RING = 6 * TP_BOX * 3;      // 3 stages of 6 boxes (or 4 stages of 4)
constexpr int TP_VBUF = 128 * 128 * 4;       // the V' tile, rewritten as T hi / lo
constexpr int TP_SMEM = TP_RING + TP_VBUF + 1024;
constexpr int TP_DRAIN = 6;                  // K blocks per accumulator drain (192 terms)

template <bool kShort>
__device__ __forceinline__ void tprod_body(const TprodMaps& mp, const TprodArgs& g) {
  extern __shared__ uint8_t tp_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tp_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* vbuf = sm + TP_RING;
  __shared__ uint64_t full[4], empty[4], set_ready[2], set_free[2], drain, vfull[2];
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  __shared__ double ered[kGemmEpi];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = g.tiles_x * g.tiles_y;
  const int npc = g.pieces3 ? 3 : 2;      // pieces per operand
  const int ns = g.pieces3 ? 3 : 4;       // stages
  const int sbytes = 2 * npc * TP_BOX;    // bytes per stage
  const int nkb = g.K / TP_KB;            // K blocks per tile
  const int ngroups = (nkb + TP_DRAIN - 1) / TP_DRAIN;
  const long long lw = kShort ? wait_limit(g.wait) : kWaitCycles;

  if (tid == 0) {
    for (int s = 0; s < 4; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&set_ready[s], 1);
      mbar_init(&set_free[s], kGemmEpi);  // one arrival per epilogue warp
      mbar_init(&vfull[s], 1);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kGemmMma) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == kGemmTma && lane == 0) {
    prefetch_tmap(&mp.a);
    prefetch_tmap(&mp.b);
    prefetch_tmap(&mp.v);
    int last_parity[4] = {-1, -1, -1, -1};
    int it = 0;  // K blocks issued by this CTA over all its tiles
    for (int tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
      const int m0 = (tile % g.tiles_x) * 128, n0 = (tile / g.tiles_x) * 128;
      for (int kb = 0; kb < nkb && !abort_flag; ++kb, ++it) {
        const int s = it % ns, use = it / ns;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, lw)) {
          atomicExch(g.status, 21); abort_flag = 1; break;
        }
        uint8_t* st = sm + s * sbytes;  // A pieces at p * 8 KB, B pieces at (npc + p) * 8 KB
        mbar_expect_tx(&full[s], sbytes);
        const int kc = kb * TP_KB;
        tma_load_3d(st, &mp.a, &full[s], kc, m0, 0);  // every piece in one box
        tma_load_3d(st + npc * TP_BOX, &mp.b, &full[s], kc, n0, 0);
        last_parity[s] = use & 1;
      }
    }
    for (int s = 0; s < ns; ++s)
      if (last_parity[s] >= 0) mbar_wait(&full[s], last_parity[s]);
  } else if (warp == kGemmMma) {
    const uint32_t idesc = idesc_f16(128, 128, false, false, false);
    const uint64_t d0 = sdesc_sw64(smem_u32(sm), 16, 512);
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(g.status, code); abort_flag = 1; }
      __syncwarp();
    };
    int it = 0, G0 = 0;
    bool good = true;
    for (int tile = blockIdx.x; good && tile < ntiles; tile += gridDim.x) {
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) { good = false; break; }
        const int s = it % ns, grp = G0 + kb / TP_DRAIN, set = grp & 1;
        const bool first = (kb % TP_DRAIN) == 0;
        const bool last = (kb % TP_DRAIN) == TP_DRAIN - 1 || kb == nkb - 1;
        if (first && grp >= 2 && !mbar_wait_warp(&set_free[set], ((grp >> 1) - 1) & 1, lw)) {
          fail(24); good = false; break;
        }
        if (!mbar_wait_warp(&full[s], (it / ns) & 1, lw)) { fail(22); good = false; break; }
        tc_fence_after();
        // descriptor address field in 16-byte units: 512 per 8 KB box, 2 per K step
        const uint64_t am = d0 + (uint64_t)((s * sbytes) >> 4), ah = am + 512, al = am + 1024;
        const uint64_t bm = am + 512 * npc, bh = bm + 512, bl = bm + 1024;
        const uint32_t t0 = tbase + set * 256, t1 = t0 + 128;
        const uint32_t a0 = first ? 0u : 1u;
        mma_ss_run2(t0, am, bm, 2, 2, idesc, a0);
        mma_ss_run2(t1, am, bh, 2, 2, idesc, a0);
        mma_ss_run2(t1, ah, bm, 2, 2, idesc, 1u);
        mma_ss_run2(t1, ah, bh, 2, 2, idesc, 1u);
        if (npc == 3) {
          mma_ss_run2(t1, am, bl, 2, 2, idesc, 1u);
          mma_ss_run2(t1, al, bm, 2, 2, idesc, 1u);
        }
        if (elect_one()) {
          mma_commit(&empty[s]);
          if (last) mma_commit(&set_ready[set]);
        }
        __syncwarp();
      }
      G0 += ngroups;
    }
    if (elect_one()) mma_commit(&drain);
    __syncwarp();
    mbar_wait_warp(&drain, 0);
  } else if (warp < kGemmEpi) {
    const int quad = warp & 3, half = warp >> 2;
    const int r = quad * 32 + lane;
    const int cb = 64 * half;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    const bool leader = quad == 0 && lane == 0;  // issues the half's V' loads and T stores
    uint8_t* vb = vbuf + half * 32768;           // V' boxes of columns cb .. cb + 63
    const float f = g.sc[g.f_idx];
    auto load_v = [&](int tile) {
      const int m0 = (tile % g.tiles_x) * 128, n0 = (tile / g.tiles_x) * 128;
      mbar_expect_tx(&vfull[half], 32768);
      tma_load_2d(vb, &mp.v, &vfull[half], n0 + cb, m0);
      tma_load_2d(vb + 16384, &mp.v, &vfull[half], n0 + cb + 32, m0);
    };
    if (leader && (int)blockIdx.x < ntiles) load_v(blockIdx.x);
    int G0 = 0, j = 0, vlost = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int bx = tile % g.tiles_x, by = tile / g.tiles_x;
      const int m0 = bx * 128, n0 = by * 128;
      float run[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) run[c] = 0.0f;
      bool ok = true;
      for (int gi = 0; gi < ngroups; ++gi) {
        const int grp = G0 + gi, set = grp & 1;
        if (__shfl_sync(0xffffffffu, (int)abort_flag, 0) || !mbar_wait_warp(&set_ready[set], (grp >> 1) & 1, lw)) {
          ok = false;
          if (lane == 0 && !abort_flag) { atomicExch(g.status, 23); abort_flag = 1; }
          __syncwarp();
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
          uint32_t a0[16], a1[16];
          tmem_ld16(tbase + lane_off + set * 256 + cb + c, a0);
          tmem_ld16(tbase + lane_off + set * 256 + 128 + cb + c, a1);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 16; ++q) run[c + q] += __uint_as_float(a0[q]) + __uint_as_float(a1[q]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&set_free[set]);
      }
      G0 += ngroups;
      // the V' boxes of this tile (issued when the previous tile's T had been read out)
      if (!mbar_wait_warp(&vfull[half], j & 1, lw)) {
        ok = false;
        vlost = 1;
        if (lane == 0) { atomicExch(g.status, 25); abort_flag = 1; }
      }
      ok = ok && !abort_flag;
      // row r of the two [128][32] FP32 boxes: 16-byte chunk c sits at c ^ (r % 8)
      float v[64];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 x = *reinterpret_cast<const float4*>(vb + b * 16384 + r * 128 + 16 * (c ^ (r & 7)));
          v[b * 32 + c * 4 + 0] = x.x; v[b * 32 + c * 4 + 1] = x.y;
          v[b * 32 + c * 4 + 2] = x.z; v[b * 32 + c * 4 + 3] = x.w;
        }
      asm volatile("bar.sync %0, 128;" ::"r"(2 + half) : "memory");  // the half's V' is read
      double esum = 0.0;
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 8) {
        uint32_t hw[4], lw4[4];
        float e = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          const float s0 = ok ? run[c0 + q] : 0.0f, s1 = ok ? run[c0 + q + 1] : 0.0f;
          const float p0 = v[c0 + q] * s0, p1 = v[c0 + q + 1] * s1;
          e = fmaf(p0, s0, e);
          e = fmaf(p1, s1, e);
          const float t0 = p0 * f, t1 = p1 * f;
          const __half2 h01 = __floats2half2_rn(t0, t1);
          const float2 b01 = __half22float2(h01);
          const __half2 l01 = __floats2half2_rn(t0 - b01.x, t1 - b01.y);
          hw[q / 2] = *reinterpret_cast<const uint32_t*>(&h01);
          lw4[q / 2] = *reinterpret_cast<const uint32_t*>(&l01);
        }
        esum += (double)e;
        if (g.store) {
          // box c0 / 32 of the half: hi [128][32] at +0, lo at +8 KB; row r is
          // 64 B and its 16-byte chunk c sits at c ^ ((r / 2) % 4)
          uint8_t* bb = vb + (c0 >> 5) * 16384 + r * 64 + 16 * (((c0 & 31) >> 3) ^ ((r >> 1) & 3));
          *reinterpret_cast<uint4*>(bb) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(bb + 8192) = make_uint4(lw4[0], lw4[1], lw4[2], lw4[3]);
        }
      }
      if (g.epart) {
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
        if (lane == 0) ered[warp] = esum;  // read by the leader after the barrier below
      }
      if (g.store) fence_async_smem();
      asm volatile("bar.sync %0, 128;" ::"r"(2 + half) : "memory");  // the half's T is written
      if (leader) {
        if (g.epart)  // per tile and column half, in a fixed order
          g.epart[2 * ((long)by * g.tiles_x + bx) + half] =
              ((ered[4 * half] + ered[4 * half + 1]) + ered[4 * half + 2]) + ered[4 * half + 3];
        if (g.store) {
          for (int b = 0; b < 2; ++b) {
            const int x = n0 + cb + 32 * b;
            if (x >= g.ld_t) break;
            tma_store_2d(&mp.th, vb + b * 16384, x, m0);
            tma_store_2d(&mp.tl, vb + b * 16384 + 8192, x, m0);
          }
          bulk_commit();
          bulk_wait_read();
        }
        if (tile + (int)gridDim.x < ntiles) load_v(tile + gridDim.x);
      }
    }
    if (leader) {
      bulk_wait_all();
      // a V' load whose wait ran out may still be in flight: let it land
      if (vlost && j > 0) mbar_wait(&vfull[half], (j - 1) & 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kGemmMma) tmem_dealloc(tbase, 512);
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    tprod_kernel(const __grid_constant__ TprodMaps mp, TprodArgs g) {
  if (g.wait > 0 && g.wait < kWaitCycles)
    tprod_body<true>(mp, g);
  else
    tprod_body<false>(mp, g);
}

// tprod_kernel over tiles_x x tiles_y tiles with at most one CTA per SM.
void launch_tprod(const TprodMaps& mp, TprodArgs g, cudaStream_t s, long long wait = 0) {
  g.wait = wait;
  const long total = (long)g.tiles_x * g.tiles_y;
  const unsigned ctas = (unsigned)std::max<long>(1, std::min<long>(total, sm_count()));
  tprod_kernel<<<ctas, kGemmThreads, TP_SMEM, s>>>(mp, g);
}

// ============================================================ pair kernel
// For one X tile of 128 rows and a range of Y rows (tiles of 64):
//   S = X Y^T as A0 (m.m, exact) + A1 (cross terms)       K = NP
//   T = V' o S;  e += sum_y T S  (the closed-form energy term, optional)
//   U = f T as floating hi/lo;  acc[x][j] += sum_y U[x][y] Y[y][j]
// X: per-row (m, h) pieces, copied once per CTA into tensor memory (A operand
// of S); Y: per-row (m, h) pieces [rows][NP], K-major, streamed by TMA and
// reused as the MN-major B operand of the second product; V': FP32 [X rows][Y
// cols] tiles streamed by TMA beside Y.  U is written by the epilogue into
// tensor memory and is the A operand of the second product, so shared memory
// carries only the TMA streams, the MMA operand reads and the V' reads.
// Tensor memory: X pieces [0, NP), S = A0 [128, 192) + A1 [192, 256),
// U buffers [256, 320) and [320, 384) (hi 32 + lo 32 columns each),
// second-product accumulator [384, 384 + NP).  16 epilogue warps: warp w
// serves lanes 32 (w % 4) .. +31 and a quarter (w / 4) of the S, U and
// accumulator columns; the accumulator drains every kAccDrain tiles into
// round-to-nearest FP32 sums held in registers.

struct PairArgs {
  int X, Y, ychunk, n;
  const __half* xm;  // X pieces [X rows][ldx]
  const __half* xh;
  long ldx;
  const float* sc;
  int f_idx, out_idx;
  float* out;
  long ldo;
  long part_stride;
  int transposed;  // 0: out[part][x][j]; 1: out[j][x] (single part)
  double* epart;   // nullable: per-CTA sum_y V' S^2 (scaled by G^4)
  int* status;
  // Fused role only (fused_body): V'^T [X rows][ldvt] read through L2 by the
  // epilogue, and the M2 side product reduced into FP32 copies
  // m2acc[copy][y][j] (copy = X tile % ncopy, copies m2_copy_stride apart).
  const float* vt;
  long ldvt;
  float* m2acc;
  int ncopy;
  long m2_copy_stride;
  long long wait;  // pipeline-wait limit in SM cycles (0: the default)
};

// One role of a pair launch (host record; copied into the launch parameters).
struct PairRole {
  CUtensorMap ym, yh, v;  // Y pieces (m, h) and the V' tiles
  CUtensorMap xm, xh;     // fused role: X pieces as [128][64] boxes (the X^T operand)
  int kind;               // 0: pair_body (one back-contraction); 1: fused_body
  PairArgs a;
  int gx;     // the role's own grid is gx x (nblk / gx)
  int nblk;
  int tiles;  // Y tiles per block (longest roles are placed first)
};

constexpr int kAccDrain = 2;                   // tiles per second-product drain
constexpr int kStages = 3;                     // TMA stages of (Y pieces, V')
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kPairThreads = kEpiThreads + 64; // + TMA producer warp + MMA warp

// One launch runs several roles (the three contractions of one build, or
// those of many builds grouped together): the roles' blocks are concatenated
// in the grid, and their tensor maps and arguments are kernel parameters.
// Long roles go first, so the short ones fill the tail of the grid.
template <int NP>
struct PairCfg {
  static constexpr int Y_BYTES = 64 * NP * 2;  // one piece of a 64-row tile
  static constexpr int V_BYTES = 128 * 64 * 4;  // V' tile: two [128][32] FP32 boxes
  static constexpr int STAGE = 2 * Y_BYTES + V_BYTES;
  static constexpr int SMEM = kStages * STAGE + 1024;
  static constexpr uint32_t T_XM = 0, T_XH = NP / 2, T_S0 = 128, T_S1 = 192, T_U = 256,
                            T_ACC = 384;
  static constexpr int AC = NP / 4;            // accumulator columns per epilogue warp
};

// X tile -> tensor memory, by the epilogue warps (lane = row; warp w / 4
// picks the piece (m, h) and the half of its NP / 2 columns; fp16 pairs as in
// memory).  Rows past the end of X are zero.
template <int NP>
__device__ __forceinline__ void load_x_tile(const PairArgs& a, int x0, uint32_t tbase, int warp,
                                            int lane) {
  using C = PairCfg<NP>;
  const int quad = warp & 3, c = warp >> 2;
  const int piece = c >> 1, part = c & 1;
  const int r = quad * 32 + lane;
  const long x = (long)x0 + r;
  const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
  const uint4* src = reinterpret_cast<const uint4*>((piece ? a.xh : a.xm) + x * a.ldx + part * (NP / 2));
  uint32_t w[C::AC];
#pragma unroll
  for (int v = 0; v < C::AC / 4; ++v) {
    const uint4 q = (x < a.X) ? src[v] : make_uint4(0u, 0u, 0u, 0u);
    w[4 * v] = q.x; w[4 * v + 1] = q.y; w[4 * v + 2] = q.z; w[4 * v + 3] = q.w;
  }
  const uint32_t col = (piece ? C::T_XH : C::T_XM) + part * C::AC;
  if constexpr (C::AC == 32) tmem_st32(tbase + lane_off + col, w);
  else tmem_st16(tbase + lane_off + col, w);
  tmem_wait_st();
}

// TMA producer (one thread): T stages of (Y pieces m, h; the [128][64] V'
// tile) through the kStages ring; gives up (status 21) when a stage is not
// released within the bounded wait, then waits for its own copies in flight.
template <int NP>
__device__ __forceinline__ void produce_tiles(const CUtensorMap* mYm, const CUtensorMap* mYh,
                                              const CUtensorMap* mV, uint8_t* sm, uint64_t* full,
                                              uint64_t* empty, int T, int y0, int x0,
                                              volatile int& abort_flag, int* status, long long lw) {
  using C = PairCfg<NP>;
  constexpr int NKB = NP / 64;
  prefetch_tmap(mYm); prefetch_tmap(mYh); prefetch_tmap(mV);
  int last_parity[kStages];
  for (int s = 0; s < kStages; ++s) last_parity[s] = -1;
  for (int t = 0; t < T && !abort_flag; ++t) {
    const int s = t % kStages, use = t / kStages;
    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, lw)) {
      atomicExch(status, 21); abort_flag = 1; break;
    }
    uint8_t* st = sm + s * C::STAGE;
    mbar_expect_tx(&full[s], C::STAGE);
    const int yr = y0 + t * 64;
    for (int kb = 0; kb < NKB; ++kb) {
      tma_load_2d(st + kb * 8192, mYm, &full[s], kb * 64, yr);
      tma_load_2d(st + C::Y_BYTES + kb * 8192, mYh, &full[s], kb * 64, yr);
    }
    tma_load_2d(st + 2 * C::Y_BYTES, mV, &full[s], yr, x0);
    tma_load_2d(st + 2 * C::Y_BYTES + 16384, mV, &full[s], yr + 32, x0);
    last_parity[s] = use & 1;
  }
  for (int s = 0; s < kStages; ++s)
    if (last_parity[s] >= 0) mbar_wait(&full[s], last_parity[s]);
}

// The kernel body: one X tile against a range of Y tiles for one role.
template <int NP, bool kShort>
__device__ __forceinline__ void pair_body(const CUtensorMap* mYm, const CUtensorMap* mYh,
                                          const CUtensorMap* mV, const PairArgs& a, int bx, int by,
                                          int gx) {
  using C = PairCfg<NP>;
  extern __shared__ uint8_t p_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[kStages], empty[kStages], s_full, s_free, u_full[2], u_free[2], acc_ready,
      acc_free, drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  __shared__ double ered[kEpiWarps];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int prod_warp = kEpiWarps, mma_warp = kEpiWarps + 1;
  const int x0 = bx * 128;
  const int y0 = by * a.ychunk;
  const int y1 = min(a.Y, y0 + a.ychunk);
  const int T = y1 > y0 ? (y1 - y0 + 63) / 64 : 0;
  const long long lw = kShort ? wait_limit(a.wait) : kWaitCycles;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&s_full, 1);
    mbar_init(&s_free, kEpiWarps);  // epilogue barriers: one arrival per warp
    for (int b = 0; b < 2; ++b) {
      mbar_init(&u_full[b], kEpiWarps);
      mbar_init(&u_free[b], 1);
    }
    mbar_init(&acc_ready, 1);
    mbar_init(&acc_free, kEpiWarps);
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == mma_warp) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp < kEpiWarps) load_x_tile<NP>(a, x0, tbase, warp, lane);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == prod_warp && lane == 0) {
    produce_tiles<NP>(mYm, mYh, mV, sm, full, empty, T, y0, x0, abort_flag, a.status, lw);
  } else if (warp == mma_warp) {
    // ---------------- MMA issuer: the whole warp runs the loop (warp-uniform
    // descriptors and waits); one elected lane issues each MMA and commit.
    const uint32_t id_s = idesc_f16(128, 64, false, false, false);
    const uint32_t id_acc = idesc_f16(128, NP, false, false, true);
    // Descriptors start from one base; the address field counts 16-byte units,
    // so tile offsets add as immediates.
    const uint64_t dy0 = sdesc_sw128(smem_u32(sm), 16, 1024);
    const uint64_t dy0mn = sdesc_sw128(smem_u32(sm), 8192, 1024);
    constexpr uint64_t kStage16 = C::STAGE >> 4, kYh16 = C::Y_BYTES >> 4;
    const uint32_t txm = tbase + C::T_XM, txh = tbase + C::T_XH;
    const uint32_t ts0 = tbase + C::T_S0, ts1 = tbase + C::T_S1, tacc = tbase + C::T_ACC;
    auto aborted = [&]() { return __shfl_sync(0xffffffffu, (int)abort_flag, 0) != 0; };
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(a.status, code); abort_flag = 1; }
      __syncwarp();
    };
    bool good = T > 0;
    auto issue_acc = [&](int u) -> bool {
      const int s = u % kStages, b = u & 1, grp = u / kAccDrain;
      const bool first = (u % kAccDrain) == 0;
      const bool last = (u % kAccDrain) == kAccDrain - 1 || u == T - 1;
      if (first && grp > 0 && !mbar_wait_warp(&acc_free, (grp - 1) & 1, lw)) return false;
      if (!mbar_wait_warp(&u_full[b], (u >> 1) & 1, lw)) return false;
      tc_fence_after();
      const uint64_t bym = dy0mn + s * kStage16, byh = bym + kYh16;
      const uint32_t tuh = tbase + C::T_U + b * 64, tul = tuh + 32;
      // K step kk: 16 Y rows = 8 TMEM columns of U, 2048 bytes of the MN-major Y tile
      mma_ts_run4_mn(tacc, tuh, bym, id_acc, first ? 0u : 1u);
      mma_ts_run4_mn(tacc, tuh, byh, id_acc, 1u);
      mma_ts_run4_mn(tacc, tul, bym, id_acc, 1u);
      if (elect_one()) {
        mma_commit(&empty[s]);
        mma_commit(&u_free[b]);
        if (last) mma_commit(&acc_ready);
      }
      __syncwarp();
      return true;
    };
    for (int t = 0; good && t < T && !aborted(); ++t) {
      const int s = t % kStages, use = t / kStages;
      if (!mbar_wait_warp(&full[s], use & 1, lw)) { fail(23); good = false; break; }
      if (t > 0 && !mbar_wait_warp(&s_free, (t - 1) & 1, lw)) { fail(24); good = false; break; }
      tc_fence_after();
      const uint64_t dym = dy0 + s * kStage16, dyh = dym + kYh16;
      // K step kk: 8 TMEM columns of X; Y tile offset (kk/4)*8192 + (kk%4)*32 bytes
      if constexpr (NP == 128) {
        mma_ts_run8_kmajor(ts0, txm, dym, id_s, 0u);
        mma_ts_run8_kmajor(ts1, txm, dyh, id_s, 0u);
        mma_ts_run8_kmajor(ts1, txh, dym, id_s, 1u);
        mma_ts_run8_kmajor(ts1, txh, dyh, id_s, 1u);
      } else {
        mma_ts_run4_kmajor(ts0, txm, dym, id_s, 0u);
        mma_ts_run4_kmajor(ts1, txm, dyh, id_s, 0u);
        mma_ts_run4_kmajor(ts1, txh, dym, id_s, 1u);
        mma_ts_run4_kmajor(ts1, txh, dyh, id_s, 1u);
      }
      if (elect_one()) mma_commit(&s_full);
      __syncwarp();
      if (t > 0 && !issue_acc(t - 1)) { fail(25); good = false; break; }
    }
    if (good && T > 0 && !issue_acc(T - 1)) fail(26);
    if (elect_one()) mma_commit(&drain);
    __syncwarp();
    mbar_wait_warp(&drain, 0);
  } else if (warp < kEpiWarps) {
    // ---------------- epilogue: warp w % 4 = TMEM lane quadrant (rows),
    // w / 4 = quarter of the columns
    const int quad = warp & 3, c = warp >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    const long x = (long)x0 + r;
    const bool xok = x < a.X;
    const float f = a.sc[a.f_idx];
    const bool want_e = a.epart != nullptr;
    const uint32_t t_s0 = tbase + lane_off + C::T_S0 + 16 * c, t_s1 = t_s0 + (C::T_S1 - C::T_S0);
    const uint32_t t_u = tbase + lane_off + C::T_U + 8 * c;
    const uint32_t t_acc = tbase + lane_off + C::T_ACC + C::AC * c;
    // V' of this thread's 16 columns: box c / 2 of the stage, 16-byte chunks
    // 4 (c % 2) .. +3 of row r (128-byte swizzle: chunk q sits at q ^ (r % 8))
    const int vbox_off = 2 * C::Y_BYTES + (c >> 1) * 16384 + r * 128;
    const int sw = r & 7, q0 = (c & 1) * 4;
    float run[C::AC];
#pragma unroll
    for (int j = 0; j < C::AC; ++j) run[j] = 0.0f;
    double esum = 0.0;
    bool ok = T > 0;
    // waits and the abort test are warp-uniform: the tensor-memory loads and
    // stores below are warp-collective
    auto aborted = [&]() { return __shfl_sync(0xffffffffu, (int)abort_flag, 0) != 0; };
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(a.status, code); abort_flag = 1; }
      __syncwarp();
    };
    // Per tile: read S(t) and release it first, so that the next S product is
    // queued while this warp drains the accumulator (group ending at t - 1)
    // and forms U(t).
    for (int t = 0; t <= T && !aborted(); ++t) {
      const int b = t & 1;
      float sv[16];
      if (t < T) {
        if (!mbar_wait_warp(&s_full, t & 1, lw)) { fail(27); ok = false; break; }
        tc_fence_after();
        uint32_t u0[16], u1[16];
        tmem_ld16(t_s0, u0);
        tmem_ld16(t_s1, u1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) sv[j] = __uint_as_float(u0[j]) + __uint_as_float(u1[j]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_free);
      }
      // drain the second-product accumulator into the running sums after each group
      if (t > 0 && (((t - 1) % kAccDrain) == kAccDrain - 1 || t == T)) {
        const int grp = (t - 1) / kAccDrain;
        if (!mbar_wait_warp(&acc_ready, grp & 1, lw)) { fail(29); ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < C::AC; h += 16) {  // 16 columns at a time (register budget)
          uint32_t ua[16];
          tmem_ld16(t_acc + h, ua);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) run[h + j] += __uint_as_float(ua[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_free);
      }
      if (t == T) break;
      uint32_t hi[8], lo[8];
      float etile = 0.0f;
      const uint8_t* vrow = sm + (t % kStages) * C::STAGE + vbox_off;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float vv[2];
        {
          const float4 v4 = *reinterpret_cast<const float4*>(vrow + (((q0 + (q >> 1)) ^ sw) << 4));
          vv[0] = (q & 1) ? v4.z : v4.x;
          vv[1] = (q & 1) ? v4.w : v4.y;
        }
        const float p0 = vv[0] * sv[2 * q], p1 = vv[1] * sv[2 * q + 1];
        if (want_e) {
          etile = fmaf(p0, sv[2 * q], etile);
          etile = fmaf(p1, sv[2 * q + 1], etile);
        }
        const float t0 = p0 * f, t1 = p1 * f;
        const __half2 h01 = __floats2half2_rn(t0, t1);
        const float2 b01 = __half22float2(h01);
        const __half2 l01 = __floats2half2_rn(t0 - b01.x, t1 - b01.y);
        hi[q] = *reinterpret_cast<const uint32_t*>(&h01);
        lo[q] = *reinterpret_cast<const uint32_t*>(&l01);
      }
      esum += (double)etile;
      if (t >= 2 && !mbar_wait_warp(&u_free[b], ((t - 2) >> 1) & 1, lw)) { fail(28); ok = false; break; }
      tc_fence_after();
      tmem_st8(t_u + b * 64, hi);
      tmem_st8(t_u + b * 64 + 32, lo);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&u_full[b]);
    }
    ok = ok && !aborted();
    // ---------------- write the running sums
    const float os = a.sc[a.out_idx];
    if (xok) {
#pragma unroll
      for (int j = 0; j < C::AC; ++j) {
        const int col = C::AC * c + j;
        if (col >= a.n) continue;
        const float v = ok ? run[j] * os : 0.0f;
        if (a.transposed)
          a.out[(long)col * a.ldo + x] = v;
        else
          a.out[(long)by * a.part_stride + x * a.ldo + col] = v;
      }
    }
    if (want_e) {
      double e = (ok && xok) ? esum : 0.0;
      for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
      if (lane == 0) ered[warp] = e;
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < kEpiWarps; ++i) sum += ered[i];
        a.epart[(long)by * gx + bx] = sum;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == mma_warp) tmem_dealloc(tbase, 512);
}

// ============================================================ fused pair kernel
// Both back-contractions of Eq. exoccri from one pass over V (n <= 128, the
// 128-column piece layout).  One CTA takes 128 grid points R (X = Psi rows)
// against every interpolation tile g (Y = Psi_g rows, 64 per tile):
//   S^T = X Y^T                    four split passes (A0 exact, A1 cross terms)
//   U^T = f V^T' o S^T             floating hi/lo FP16; e += sum V' S^2
//   M1^T[R][j] += sum_g U^T Y      TS MMAs (U in tensor memory), drained every
//                                  kAccDrain tiles into FP32 registers: M1
//                                  is complete in the CTA (written [j][R])
//   M2[g][j]   += sum_R U^T X      SS MMAs (A = X^T, B = U^T, both MN-major
//                                  in shared memory), drained every tile and
//                                  added with red.global.add.f32 into the
//                                  copy (X tile % ncopy) of M2
// so S is formed once per pair and V is read once (its transposed FP32 copy).
// Tensor memory: X pieces [0, 128), S = A0 [128, 192) + A1 [192, 256),
// U [256, 320) (hi 32 + lo 32), M2 tile [320, 384), M1^T accumulator
// [384, 512).  Shared memory: Y ring and V'^T ring (2 stages of 32 KB each),
// X^T pieces (64 KB), U^T pieces (32 KB).  Per tile the epilogue reads S,
// forms U from the staged V' tile, writes U once the previous tile's products
// have read it, then drains the M1^T group and the previous M2 tile; the
// reductions of that M2 tile into L2 come last, off the path to the next U.
// The M2 copies are FP32 sums whose order depends on the CTA schedule: K_{mu i}
// is reproducible to rounding, not bit for bit (E_x is: its per-CTA sums are
// fixed-order).
constexpr int kFusedStages = 2;
struct FusedCfg {
  static constexpr int NP = 128;
  static constexpr int Y_BYTES = 64 * NP * 2;          // one piece of a 64-row Y tile
  static constexpr int Y_STAGE = 2 * Y_BYTES;          // (m, h)
  static constexpr int V_STAGE = 128 * 64 * 4;         // V'^T tile: two [128][32] FP32 boxes
  static constexpr int OFF_V = kFusedStages * Y_STAGE;
  static constexpr int OFF_X = OFF_V + kFusedStages * V_STAGE;  // X^T pieces: m [0, 32K), h [32K, 64K)
  static constexpr int OFF_U = OFF_X + 4 * 16384;      // U^T pieces: hi [0, 16K), lo [16K, 32K)
  static constexpr int SMEM = OFF_U + 2 * 16384 + 1024;
  static constexpr uint32_t T_XM = 0, T_XH = 64, T_S0 = 128, T_S1 = 192, T_U = 256, T_M2 = 320,
                            T_ACC = 384;
  static constexpr int AC = NP / 4;                    // M1^T columns per epilogue warp
};
static_assert(FusedCfg::SMEM >= PairCfg<128>::SMEM, "one launch size covers both bodies");

__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

template <bool kShort>
__device__ __forceinline__ void fused_body(const CUtensorMap* mYm, const CUtensorMap* mYh,
                                           const CUtensorMap* mV, const CUtensorMap* mXm,
                                           const CUtensorMap* mXh, const PairArgs& a, int bx) {
  using C = FusedCfg;
  constexpr int NP = C::NP;
  extern __shared__ uint8_t p_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t y_full[kFusedStages], y_empty[kFusedStages], v_full[kFusedStages],
      v_empty[kFusedStages], xfull, s_full, s_free, u_full, u_free, acc_ready, acc_free, m2_ready,
      m2_free, drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  __shared__ double ered[kEpiWarps];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int prod_warp = kEpiWarps, mma_warp = kEpiWarps + 1;
  const int x0 = bx * 128;
  const int T = a.Y > 0 ? (a.Y + 63) / 64 : 0;
  const long long lw = kShort ? wait_limit(a.wait) : kWaitCycles;

  if (tid == 0) {
    for (int s = 0; s < kFusedStages; ++s) {
      mbar_init(&y_full[s], 1);
      mbar_init(&y_empty[s], 1);
      mbar_init(&v_full[s], 1);
      mbar_init(&v_empty[s], kEpiWarps);
    }
    mbar_init(&xfull, 1);
    mbar_init(&s_full, 1);
    mbar_init(&s_free, kEpiWarps);
    mbar_init(&u_full, kEpiWarps);
    mbar_init(&u_free, 1);
    mbar_init(&acc_ready, 1);
    mbar_init(&acc_free, kEpiWarps);
    mbar_init(&m2_ready, 1);
    mbar_init(&m2_free, kEpiWarps);
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == mma_warp) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp < kEpiWarps) load_x_tile<NP>(a, x0, tbase, warp, lane);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == prod_warp && lane == 0) {
    // ---------------- TMA producer: X^T pieces once, then per tile the Y
    // pieces (released by the MMA warp) and the V'^T tile (released by the
    // epilogue) through their own rings
    prefetch_tmap(mYm); prefetch_tmap(mYh); prefetch_tmap(mV); prefetch_tmap(mXm); prefetch_tmap(mXh);
    mbar_expect_tx(&xfull, 4 * 16384);
    tma_load_2d(sm + C::OFF_X, mXm, &xfull, 0, x0);
    tma_load_2d(sm + C::OFF_X + 16384, mXm, &xfull, 64, x0);
    tma_load_2d(sm + C::OFF_X + 32768, mXh, &xfull, 0, x0);
    tma_load_2d(sm + C::OFF_X + 49152, mXh, &xfull, 64, x0);
    int ylast[kFusedStages], vlast[kFusedStages];
    for (int s = 0; s < kFusedStages; ++s) ylast[s] = vlast[s] = -1;
    for (int t = 0; t < T && !abort_flag; ++t) {
      const int s = t % kFusedStages, use = t / kFusedStages;
      const int yr = t * 64;
      if (use > 0 && !mbar_wait(&y_empty[s], (use - 1) & 1, lw)) {
        atomicExch(a.status, 41); abort_flag = 1; break;
      }
      uint8_t* st = sm + s * C::Y_STAGE;
      mbar_expect_tx(&y_full[s], C::Y_STAGE);
      tma_load_2d(st, mYm, &y_full[s], 0, yr);
      tma_load_2d(st + 8192, mYm, &y_full[s], 64, yr);
      tma_load_2d(st + C::Y_BYTES, mYh, &y_full[s], 0, yr);
      tma_load_2d(st + C::Y_BYTES + 8192, mYh, &y_full[s], 64, yr);
      ylast[s] = use & 1;
      if (use > 0 && !mbar_wait(&v_empty[s], (use - 1) & 1, lw)) {
        atomicExch(a.status, 42); abort_flag = 1; break;
      }
      uint8_t* sv = sm + C::OFF_V + s * C::V_STAGE;
      mbar_expect_tx(&v_full[s], C::V_STAGE);
      tma_load_2d(sv, mV, &v_full[s], yr, x0);
      tma_load_2d(sv + 16384, mV, &v_full[s], yr + 32, x0);
      vlast[s] = use & 1;
    }
    mbar_wait(&xfull, 0);
    for (int s = 0; s < kFusedStages; ++s) {
      if (ylast[s] >= 0) mbar_wait(&y_full[s], ylast[s]);
      if (vlast[s] >= 0) mbar_wait(&v_full[s], vlast[s]);
    }
  } else if (warp == mma_warp) {
    // ---------------- MMA issuer (whole warp in the loop, one elected lane issues)
    const uint32_t id_s = idesc_f16(128, 64, false, false, false);
    const uint32_t id_m1 = idesc_f16(128, NP, false, false, true);
    const uint32_t id_m2 = idesc_f16(128, 64, false, true, true);
    const uint64_t dy0 = sdesc_sw128(smem_u32(sm), 16, 1024);
    const uint64_t dy0mn = sdesc_sw128(smem_u32(sm), 8192, 1024);
    // X^T: [128 R][64 j] column blocks 16 KB apart (LBO); U^T: one [128 R][64 g] block
    const uint64_t dxm = sdesc_sw128(smem_u32(sm + C::OFF_X), 16384, 1024), dxh = dxm + (32768 >> 4);
    const uint64_t duh = sdesc_sw128(smem_u32(sm + C::OFF_U), 16384, 1024), dul = duh + (16384 >> 4);
    constexpr uint64_t kStage16 = C::Y_STAGE >> 4, kYh16 = C::Y_BYTES >> 4;
    const uint32_t txm = tbase + C::T_XM, txh = tbase + C::T_XH;
    const uint32_t ts0 = tbase + C::T_S0, ts1 = tbase + C::T_S1, tacc = tbase + C::T_ACC;
    const uint32_t tm2 = tbase + C::T_M2, tuh = tbase + C::T_U, tul = tuh + 32;
    auto aborted = [&]() { return __shfl_sync(0xffffffffu, (int)abort_flag, 0) != 0; };
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(a.status, code); abort_flag = 1; }
      __syncwarp();
    };
    bool good = T > 0;
    if (good && !mbar_wait_warp(&xfull, 0, lw)) { fail(43); good = false; }
    // the products of tile u: M1^T (TS, U from tensor memory, Y MN-major) and
    // M2 (SS, X^T and U^T MN-major)
    auto issue_products = [&](int u) -> bool {
      const int s = u % kFusedStages, grp = u / kAccDrain;
      const bool first = (u % kAccDrain) == 0;
      const bool last = (u % kAccDrain) == kAccDrain - 1 || u == T - 1;
      if (first && grp > 0 && !mbar_wait_warp(&acc_free, (grp - 1) & 1, lw)) return false;
      if (!mbar_wait_warp(&u_full, u & 1, lw)) return false;
      tc_fence_after();
      const uint64_t bym = dy0mn + s * kStage16;
      // passes (U_hi, Y_m), (U_hi, Y_h), (U_lo, Y_m); a runtime loop over the
      // passes keeps one pass's operands live at a time
#pragma unroll 1
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t ta = pass == 2 ? tul : tuh;
        const uint64_t db = pass == 1 ? bym + kYh16 : bym;
        mma_ts_run4_mn(tacc, ta, db, id_m1, (first && pass == 0) ? 0u : 1u);
      }
      if (elect_one()) {
        mma_commit(&y_empty[s]);
        if (last) mma_commit(&acc_ready);
      }
      __syncwarp();
      if (u > 0 && !mbar_wait_warp(&m2_free, (u - 1) & 1, lw)) return false;
      tc_fence_after();
      // passes (X_m, U_hi), (X_h, U_hi), (X_m, U_lo); K step kk: 16 R rows =
      // 2048 bytes of both MN-major operands
#pragma unroll 1
      for (int pass = 0; pass < 3; ++pass) {
        const uint64_t da = pass == 1 ? dxh : dxm;
        const uint64_t db = pass == 2 ? dul : duh;
        mma_ss_run8_mn(tm2, da, db, id_m2, pass > 0 ? 1u : 0u);
      }
      if (elect_one()) {
        mma_commit(&u_free);
        mma_commit(&m2_ready);
      }
      __syncwarp();
      return true;
    };
    for (int t = 0; good && t < T && !aborted(); ++t) {
      const int s = t % kFusedStages, use = t / kFusedStages;
      if (!mbar_wait_warp(&y_full[s], use & 1, lw)) { fail(44); good = false; break; }
      if (t > 0 && !mbar_wait_warp(&s_free, (t - 1) & 1, lw)) { fail(45); good = false; break; }
      tc_fence_after();
      const uint64_t dym = dy0 + s * kStage16, dyh = dym + kYh16;
      // passes m.m' -> A0, then m.h', h.m', h.h' -> A1 (the pair kernel's order)
#pragma unroll 1
      for (int pass = 0; pass < 4; ++pass) {
        const uint32_t td = pass == 0 ? ts0 : ts1;
        const uint32_t ta = pass < 2 ? txm : txh;
        const uint64_t db = (pass & 1) ? dyh : dym;
        static_assert(NP / 16 == 8, "one run of eight K steps per pass");
        mma_ts_run8_kmajor(td, ta, db, id_s, pass >= 2 ? 1u : 0u);
      }
      if (elect_one()) mma_commit(&s_full);
      __syncwarp();
      if (t > 0 && !issue_products(t - 1)) { fail(46); good = false; break; }
    }
    if (good && T > 0 && !issue_products(T - 1)) fail(47);
    if (elect_one()) mma_commit(&drain);
    __syncwarp();
    mbar_wait_warp(&drain, 0);
  } else if (warp < kEpiWarps) {
    // ---------------- epilogue: warp w % 4 = TMEM lane quadrant, w / 4 = quarter
    // of the S / U columns (16 g), of the M1^T columns (32 j) and of the M2
    // tile columns (16 g)
    const int quad = warp & 3, c = warp >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    const long x = (long)x0 + r;
    const bool xok = x < a.X;
    const float f = a.sc[a.f_idx];
    const bool want_e = a.epart != nullptr;
    const uint32_t t_s0 = tbase + lane_off + C::T_S0 + 16 * c, t_s1 = t_s0 + (C::T_S1 - C::T_S0);
    const uint32_t t_u = tbase + lane_off + C::T_U + 8 * c;
    const uint32_t t_acc = tbase + lane_off + C::T_ACC + C::AC * c;
    const uint32_t t_m2 = tbase + lane_off + C::T_M2 + 16 * c;
    // V'^T of this thread's 16 columns: box c / 2 of the stage, 16-byte chunks
    // 4 (c % 2) .. +3 of row r (128-byte swizzle: chunk q sits at q ^ (r % 8));
    // U^T row r of the MN-major B operand: chunks 2c, 2c + 1 at (q ^ (r % 8))
    const int vbox_off = C::OFF_V + (c >> 1) * 16384 + r * 128;
    const int sw = r & 7, q0 = (c & 1) * 4;
    uint8_t* urow = sm + C::OFF_U + r * 128;
    const int uc0 = ((2 * c) ^ sw) << 4, uc1 = ((2 * c + 1) ^ sw) << 4;
    float run[C::AC];
#pragma unroll
    for (int j = 0; j < C::AC; ++j) run[j] = 0.0f;
    double esum = 0.0;
    bool ok = T > 0;
    auto aborted = [&]() { return __shfl_sync(0xffffffffu, (int)abort_flag, 0) != 0; };
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(a.status, code); abort_flag = 1; }
      __syncwarp();
    };
    // M1^T group ending at tile u -> running sums
    auto drain_m1 = [&](int u) -> bool {
      if (!mbar_wait_warp(&acc_ready, (u / kAccDrain) & 1, lw)) return false;
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < C::AC; h += 16) {
        uint32_t ua[16];
        tmem_ld16(t_acc + h, ua);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) run[h + j] += __uint_as_float(ua[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_free);
      return true;
    };
    // M2 tile u -> its copy (lane = j: 32 consecutive floats per g row)
    auto drain_m2 = [&](int u) -> bool {
      if (!mbar_wait_warp(&m2_ready, u & 1, lw)) return false;
      tc_fence_after();
      uint32_t mv[16];
      tmem_ld16(t_m2, mv);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&m2_free);
      // accumulator units (the FP64 reduction of the copies applies the scale)
      if (r < a.n) {
        const int g0 = u * 64 + 16 * c;
        float* dst = a.m2acc + (long)(bx % a.ncopy) * a.m2_copy_stride + (long)g0 * a.n + r;
        if (g0 + 16 <= a.Y) {
#pragma unroll
          for (int k = 0; k < 16; ++k, dst += a.n) red_add_f32(dst, __uint_as_float(mv[k]));
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k, dst += a.n)
            if (g0 + k < a.Y) red_add_f32(dst, __uint_as_float(mv[k]));
        }
      }
      return true;
    };
    for (int t = 0; t < T && !aborted(); ++t) {
      const int s = t % kFusedStages;
      float sv[16];
      if (!mbar_wait_warp(&s_full, t & 1, lw)) { fail(48); ok = false; break; }
      tc_fence_after();
      {
        uint32_t u0[16], u1[16];
        tmem_ld16(t_s0, u0);
        tmem_ld16(t_s1, u1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) sv[j] = __uint_as_float(u0[j]) + __uint_as_float(u1[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_free);
      // U(t) from the staged V'^T tile
      if (!mbar_wait_warp(&v_full[s], (t / kFusedStages) & 1, lw)) { fail(49); ok = false; break; }
      uint32_t hi[8], lo[8];
      float etile = 0.0f;
      const uint8_t* vrow = sm + s * C::V_STAGE + vbox_off;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float vv[2];
        {
          const float4 v4 = *reinterpret_cast<const float4*>(vrow + (((q0 + (q >> 1)) ^ sw) << 4));
          vv[0] = (q & 1) ? v4.z : v4.x;
          vv[1] = (q & 1) ? v4.w : v4.y;
        }
        const float p0 = vv[0] * sv[2 * q], p1 = vv[1] * sv[2 * q + 1];
        if (want_e) {
          etile = fmaf(p0, sv[2 * q], etile);
          etile = fmaf(p1, sv[2 * q + 1], etile);
        }
        const float t0 = p0 * f, t1 = p1 * f;
        const __half2 h01 = __floats2half2_rn(t0, t1);
        const float2 b01 = __half22float2(h01);
        const __half2 l01 = __floats2half2_rn(t0 - b01.x, t1 - b01.y);
        hi[q] = *reinterpret_cast<const uint32_t*>(&h01);
        lo[q] = *reinterpret_cast<const uint32_t*>(&l01);
      }
      esum += (double)etile;
      __syncwarp();
      if (lane == 0) mbar_arrive(&v_empty[s]);
      // U(t) replaces U(t - 1) once both products of t - 1 have read it
      if (t > 0 && !mbar_wait_warp(&u_free, (t - 1) & 1, lw)) { fail(50); ok = false; break; }
      tc_fence_after();
      tmem_st8(t_u, hi);
      tmem_st8(t_u + 32, lo);
      *reinterpret_cast<uint4*>(urow + uc0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(urow + uc1) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
      *reinterpret_cast<uint4*>(urow + 16384 + uc0) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      *reinterpret_cast<uint4*>(urow + 16384 + uc1) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
      tmem_wait_st();
      fence_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&u_full);
      // the M1^T group that ended at t - 1, then M2(t - 1) and its reductions
      if (t > 0 && ((t - 1) % kAccDrain) == kAccDrain - 1 && !drain_m1(t - 1)) {
        fail(51); ok = false; break;
      }
      if (t > 0 && !drain_m2(t - 1)) { fail(52); ok = false; break; }
    }
    ok = ok && !aborted();
    // the last M1^T group (ending at T - 1) and the last M2 tile
    if (ok && T > 0 && !drain_m1(T - 1)) { fail(53); ok = false; }
    if (ok && T > 0 && !drain_m2(T - 1)) { fail(54); ok = false; }
    // ---------------- M1 (complete in this CTA): written [j][R]
    if (xok) {
      const float os = a.sc[a.out_idx];
#pragma unroll
      for (int j = 0; j < C::AC; ++j) {
        const int col = C::AC * c + j;
        if (col < a.n) a.out[(long)col * a.ldo + x] = ok ? run[j] * os : 0.0f;
      }
    }
    if (want_e) {
      double e = (ok && xok) ? esum : 0.0;
      for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
      if (lane == 0) ered[warp] = e;
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < kEpiWarps; ++i) sum += ered[i];
        a.epart[bx] = sum;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == mma_warp) tmem_dealloc(tbase, 512);
}

// The three roles of one build; arguments and tensor maps in parameter space
// (selected with constant indices, so they stay operands of the instructions).
struct PairJob3 {
  CUtensorMap ym[3], yh[3], v[3];
  PairArgs a[3];
  int gx[3], nblk[3];
};

template <int NP>
__global__ void __launch_bounds__(kPairThreads, 1) pair_kernel(const __grid_constant__ PairJob3 job) {
  int ri = 0, blk = blockIdx.x;
  if (blk >= job.nblk[0]) {
    blk -= job.nblk[0];
    ri = 1;
    if (blk >= job.nblk[1]) { blk -= job.nblk[1]; ri = 2; }
  }
  const CUtensorMap* mYm = ri == 0 ? &job.ym[0] : ri == 1 ? &job.ym[1] : &job.ym[2];
  const CUtensorMap* mYh = ri == 0 ? &job.yh[0] : ri == 1 ? &job.yh[1] : &job.yh[2];
  const CUtensorMap* mV = ri == 0 ? &job.v[0] : ri == 1 ? &job.v[1] : &job.v[2];
  const PairArgs& a = ri == 0 ? job.a[0] : ri == 1 ? job.a[1] : job.a[2];
  const int gx = ri == 0 ? job.gx[0] : ri == 1 ? job.gx[1] : job.gx[2];
  if (short_wait(a.wait))
    pair_body<NP, true>(mYm, mYh, mV, a, blk % gx, blk / gx, gx);
  else
    pair_body<NP, false>(mYm, mYh, mV, a, blk % gx, blk / gx, gx);
}

// Up to kGroupRoles roles of several builds in one launch, all in parameter
// space (a grouped batch is split into launches of at most this many roles).
constexpr int kGroupRoles = 16;
struct PairJobN {
  CUtensorMap ym[kGroupRoles], yh[kGroupRoles], v[kGroupRoles], xm[kGroupRoles], xh[kGroupRoles];
  PairArgs a[kGroupRoles];
  int gx[kGroupRoles], first[kGroupRoles], kind[kGroupRoles];
  int nroles;
};

// Roles of kind 1 (NP = 128 only) run the fused body: one block per X tile.
template <int NP>
__global__ void __launch_bounds__(kPairThreads, 1)
    pair_kernel_group(const __grid_constant__ PairJobN job) {
  int ri = 0;
  while (ri + 1 < job.nroles && (int)blockIdx.x >= job.first[ri + 1]) ++ri;
  const int gx = job.gx[ri], blk = (int)blockIdx.x - job.first[ri];
  if constexpr (NP == 128) {
    if (job.kind[ri] == 1) {
      if (short_wait(job.a[ri].wait))
        fused_body<true>(&job.ym[ri], &job.yh[ri], &job.v[ri], &job.xm[ri], &job.xh[ri], job.a[ri], blk);
      else
        fused_body<false>(&job.ym[ri], &job.yh[ri], &job.v[ri], &job.xm[ri], &job.xh[ri], job.a[ri], blk);
      return;
    }
  }
  if (short_wait(job.a[ri].wait))
    pair_body<NP, true>(&job.ym[ri], &job.yh[ri], &job.v[ri], job.a[ri], blk % gx, blk / gx, gx);
  else
    pair_body<NP, false>(&job.ym[ri], &job.yh[ri], &job.v[ri], job.a[ri], blk % gx, blk / gx, gx);
}

// ============================================================ energy-only pair kernel
// E_x without K (the closed form of E_x contracted from Eq. exoccri):
// for one X tile of 128 rows and a range of Y tiles,
//   S = X Y^T   (the four split passes of the pair kernel, same order)
//   e += sum_y V' o S o S
// and no second product.  S is double-buffered in tensor memory (buffer b:
// A0 at 128 + 128 b, A1 at 192 + 128 b), so the S product of the next tile
// runs while the epilogue reads V'.  A stage of (Y pieces, V') is released
// by one MMA commit (the S product has read Y) plus one arrival per epilogue
// warp (V' has been read).  The per-tile and per-CTA sums are formed exactly
// as in the pair kernel: with the same split of the Y range the energy
// equals that of the full build bit for bit.

struct EnergyJob {
  CUtensorMap ym[2], yh[2], v[2];
  PairArgs a[2];
  int gx[2], nblk[2];
};

template <int NP, bool kShort>
__device__ __forceinline__ void energy_body(const CUtensorMap* mYm, const CUtensorMap* mYh,
                                            const CUtensorMap* mV, const PairArgs& a, int bx,
                                            int by, int gx) {
  using C = PairCfg<NP>;
  extern __shared__ uint8_t p_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[kStages], empty[kStages], s_full[2], s_free[2], drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  __shared__ double ered[kEpiWarps];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int prod_warp = kEpiWarps, mma_warp = kEpiWarps + 1;
  const int x0 = bx * 128;
  const int y0 = by * a.ychunk;
  const int y1 = min(a.Y, y0 + a.ychunk);
  const int T = y1 > y0 ? (y1 - y0 + 63) / 64 : 0;
  const long long lw = kShort ? wait_limit(a.wait) : kWaitCycles;
  constexpr uint32_t T_SB = 128;  // first S buffer; the second follows 128 columns on

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + kEpiWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&s_full[b], 1);
      mbar_init(&s_free[b], kEpiWarps);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == mma_warp) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp < kEpiWarps) load_x_tile<NP>(a, x0, tbase, warp, lane);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == prod_warp && lane == 0) {
    produce_tiles<NP>(mYm, mYh, mV, sm, full, empty, T, y0, x0, abort_flag, a.status, lw);
  } else if (warp == mma_warp) {
    const uint32_t id_s = idesc_f16(128, 64, false, false, false);
    const uint64_t dy0 = sdesc_sw128(smem_u32(sm), 16, 1024);
    constexpr uint64_t kStage16 = C::STAGE >> 4, kYh16 = C::Y_BYTES >> 4;
    const uint32_t txm = tbase + C::T_XM, txh = tbase + C::T_XH;
    auto aborted = [&]() { return __shfl_sync(0xffffffffu, (int)abort_flag, 0) != 0; };
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(a.status, code); abort_flag = 1; }
      __syncwarp();
    };
    for (int t = 0; t < T && !aborted(); ++t) {
      const int s = t % kStages, use = t / kStages, b = t & 1;
      if (!mbar_wait_warp(&full[s], use & 1, lw)) { fail(31); break; }
      if (t >= 2 && !mbar_wait_warp(&s_free[b], ((t - 2) >> 1) & 1, lw)) { fail(32); break; }
      tc_fence_after();
      const uint64_t dym = dy0 + s * kStage16, dyh = dym + kYh16;
      const uint32_t ts0 = tbase + T_SB + 128 * b, ts1 = ts0 + 64;
      // passes m.m' -> A0, then m.h', h.m', h.h' -> A1 (a runtime loop over
      // the passes keeps the descriptors of one pass live at a time)
#pragma unroll 1
      for (int pass = 0; pass < 4; ++pass) {
        const uint32_t td = pass == 0 ? ts0 : ts1;
        const uint32_t ta = pass < 2 ? txm : txh;
        const uint64_t db = (pass & 1) ? dyh : dym;
        if constexpr (NP == 128)
          mma_ts_run8_kmajor(td, ta, db, id_s, pass >= 2 ? 1u : 0u);
        else
          mma_ts_run4_kmajor(td, ta, db, id_s, pass >= 2 ? 1u : 0u);
      }
      if (elect_one()) {
        mma_commit(&s_full[b]);
        mma_commit(&empty[s]);
      }
      __syncwarp();
    }
    if (elect_one()) mma_commit(&drain);
    __syncwarp();
    mbar_wait_warp(&drain, 0);
  } else if (warp < kEpiWarps) {
    const int quad = warp & 3, c = warp >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
    const long x = (long)x0 + r;
    const bool xok = x < a.X;
    const int vbox_off = 2 * C::Y_BYTES + (c >> 1) * 16384 + r * 128;
    const int sw = r & 7, q0 = (c & 1) * 4;
    double esum = 0.0;
    bool ok = T > 0;
    auto aborted = [&]() { return __shfl_sync(0xffffffffu, (int)abort_flag, 0) != 0; };
    auto fail = [&](int code) {
      if (lane == 0) { atomicExch(a.status, code); abort_flag = 1; }
      __syncwarp();
    };
    for (int t = 0; t < T && !aborted(); ++t) {
      const int b = t & 1;
      if (!mbar_wait_warp(&s_full[b], (t >> 1) & 1, lw)) { fail(33); ok = false; break; }
      tc_fence_after();
      float sv[16];
      {
        const uint32_t t_s0 = tbase + lane_off + T_SB + 128 * b + 16 * c;
        uint32_t u0[16], u1[16];
        tmem_ld16(t_s0, u0);
        tmem_ld16(t_s0 + 64, u1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) sv[j] = __uint_as_float(u0[j]) + __uint_as_float(u1[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_free[b]);
      float etile = 0.0f;
      const uint8_t* vrow = sm + (t % kStages) * C::STAGE + vbox_off;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v4 = *reinterpret_cast<const float4*>(vrow + (((q0 + (q >> 1)) ^ sw) << 4));
        const float v0 = (q & 1) ? v4.z : v4.x, v1 = (q & 1) ? v4.w : v4.y;
        const float p0 = v0 * sv[2 * q], p1 = v1 * sv[2 * q + 1];
        etile = fmaf(p0, sv[2 * q], etile);
        etile = fmaf(p1, sv[2 * q + 1], etile);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[t % kStages]);
      esum += (double)etile;
    }
    ok = ok && !aborted();
    double e = (ok && xok) ? esum : 0.0;
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) ered[warp] = e;
    asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
    if (tid == 0) {
      double sum = 0.0;
      for (int i = 0; i < kEpiWarps; ++i) sum += ered[i];
      a.epart[(long)by * gx + bx] = sum;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == mma_warp) tmem_dealloc(tbase, 512);
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads, 1) energy_kernel(const __grid_constant__ EnergyJob job) {
  const int ri = (int)blockIdx.x >= job.nblk[0] ? 1 : 0;
  const int blk = (int)blockIdx.x - (ri ? job.nblk[0] : 0);
  const int gx = ri ? job.gx[1] : job.gx[0];
  if (short_wait(ri ? job.a[1].wait : job.a[0].wait))
    energy_body<NP, true>(ri ? &job.ym[1] : &job.ym[0], ri ? &job.yh[1] : &job.yh[0],
                  ri ? &job.v[1] : &job.v[0], ri ? job.a[1] : job.a[0], blk % gx, blk / gx, gx);
  else
    energy_body<NP, false>(ri ? &job.ym[1] : &job.ym[0], ri ? &job.yh[1] : &job.yh[0],
                  ri ? &job.v[1] : &job.v[0], ri ? job.a[1] : job.a[0], blk % gx, blk / gx, gx);
}

// ------------------------------------------------------------- host side

// Launches the roles (sorted, longest first) in chunks of at most kGroupRoles.
void launch_pair_roles(const std::vector<PairRole>& rs, int np, cudaStream_t s) {
  for (size_t c0 = 0; c0 < rs.size(); c0 += kGroupRoles) {
    PairJobN job;
    int blocks = 0, k = 0;
    for (size_t i = c0; i < rs.size() && k < kGroupRoles; ++i, ++k) {
      job.ym[k] = rs[i].ym; job.yh[k] = rs[i].yh; job.v[k] = rs[i].v;
      job.xm[k] = rs[i].xm; job.xh[k] = rs[i].xh; job.kind[k] = rs[i].kind;
      job.a[k] = rs[i].a; job.gx[k] = rs[i].gx; job.first[k] = blocks;
      blocks += rs[i].nblk;
    }
    job.nroles = k;
    if (np == 64)
      pair_kernel_group<64><<<blocks, kPairThreads, PairCfg<64>::SMEM, s>>>(job);
    else
      pair_kernel_group<128><<<blocks, kPairThreads, FusedCfg::SMEM, s>>>(job);
    count_launch();
  }
}

void launch_pair3(const PairRole* r, int np, cudaStream_t s) {
  PairJob3 job;
  for (int k = 0; k < 3; ++k) {
    job.ym[k] = r[k].ym; job.yh[k] = r[k].yh; job.v[k] = r[k].v;
    job.a[k] = r[k].a; job.gx[k] = r[k].gx; job.nblk[k] = r[k].nblk;
  }
  const unsigned blocks = (unsigned)(r[0].nblk + r[1].nblk + r[2].nblk);
  if (np == 64)
    pair_kernel<64><<<blocks, kPairThreads, PairCfg<64>::SMEM, s>>>(job);
  else
    pair_kernel<128><<<blocks, kPairThreads, PairCfg<128>::SMEM, s>>>(job);
  count_launch();
}

// Energy-only launch of two roles (the V role and the W role of a build).
void launch_energy2(const PairRole& ra, const PairRole& rc, int np, cudaStream_t s) {
  EnergyJob job;
  const PairRole* r[2] = {&ra, &rc};
  for (int k = 0; k < 2; ++k) {
    job.ym[k] = r[k]->ym; job.yh[k] = r[k]->yh; job.v[k] = r[k]->v;
    job.a[k] = r[k]->a; job.gx[k] = r[k]->gx; job.nblk[k] = r[k]->nblk;
  }
  const unsigned blocks = (unsigned)(ra.nblk + rc.nblk);
  if (np == 64)
    energy_kernel<64><<<blocks, kPairThreads, PairCfg<64>::SMEM, s>>>(job);
  else
    energy_kernel<128><<<blocks, kPairThreads, PairCfg<128>::SMEM, s>>>(job);
  count_launch();
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode() {
  if (g_encode) return cudaSuccess;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// 2-D map of a row-major [rows][ld] array, box [box_rows][box_cols], 128-B
// swizzle by default; cols > 0 limits the map to the first cols columns of
// each row (a box reaching past them reads zeros, a store there is dropped).
cudaError_t make_map(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize, long rows,
                     long ld, int box_rows, int box_cols,
                     CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B, long cols = 0) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols > 0 ? cols : ld), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * esize};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3-D map of `pieces` row-major [rows][ld] arrays piece_stride elements apart:
// a box [pieces][box_rows][box_cols] brings the same tile of every piece.
cudaError_t make_map3(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize, long rows,
                      long ld, int pieces, long piece_stride, int box_rows, int box_cols,
                      CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(pieces)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * esize,
                           static_cast<cuuint64_t>(piece_stride) * esize};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows),
                       static_cast<cuuint32_t>(pieces)};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

long rup(long a, long b) { return (a + b - 1) / b * b; }
int blocks_for(long total, int tpb = 256) {
  return (int)std::max<long>(1, std::min<long>((total + tpb - 1) / tpb, 152L * 16));
}

template <class T>
cudaError_t split_rows(const T* src, long rows, long cols, long ld_src, const float* sc, int gidx,
                       __half* mo, __half* ho, long ld_dst, cudaStream_t s, __half* lo = nullptr) {
  if (rows <= 0) return cudaSuccess;
  split_mh_rows_kernel<T><<<(unsigned)rows, 128, 0, s>>>(src, cols, ld_src, sc, gidx, mo, ho, lo, ld_dst);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

struct MixedState {
  int64_t Ng = 0;
  // Naux: the interpolation points whose rows of V and W this state holds
  // (a slice [g0, g0 + Naux) of NaT points; the whole set unless sharded).
  // The orbitals are gathered at all NaT points (psigA); psig is the view of
  // the slice's rows.
  int N = 0, n = 0, Naux = 0, np = 0, NaT = 0, g0 = 0;
  long Np = 0, Ng8 = 0, Na8 = 0, Ng4 = 0, Na4 = 0, NaT4 = 0, NaT8 = 0;
  double dV = 0.0;
  std::vector<void*> allocs;
  __half *phi_m = nullptr, *phi_h = nullptr, *phiT_m = nullptr, *phiT_h = nullptr,
         *phigT_m = nullptr, *phigT_h = nullptr;
  float *V32 = nullptr, *VT32 = nullptr, *W32 = nullptr;
  int32_t* idx = nullptr;
  __half *CT_m = nullptr, *CT_h = nullptr, *psi_m = nullptr, *psi_h = nullptr, *psig_m = nullptr,
         *psig_h = nullptr, *M1_m = nullptr, *M1_h = nullptr, *D23T_m = nullptr,
         *D23T_h = nullptr;
  float *M2p = nullptr, *M3p = nullptr, *M1 = nullptr, *L1p = nullptr, *L23p = nullptr,
        *sc = nullptr;
  double *D23 = nullptr, *CT64 = nullptr, *D23T64 = nullptr, *red = nullptr, *EpA = nullptr,
         *EpC = nullptr, *Lf = nullptr, *Q64 = nullptr, *dwork = nullptr;
  unsigned* am = nullptr;
  unsigned* rowmax = nullptr;
  int* status = nullptr;
  int xa = 1, partsA = 1, partsC = 1, splitsL1 = 1, splitsL23 = 1;
  int ychunkA = 64, ychunkC = 64;
  // n > 128: shape of the back-contraction tiles (true: 128 x 256, gemm_wide_kernel;
  // false: 128 x 128, gemm_kernel) and the splits of each (index 0: 128 x 128)
  bool wide = true;
  int partsA_s[2] = {1, 1}, partsC_s[2] = {1, 1}, ychunkA_s[2] = {64, 64}, ychunkC_s[2] = {64, 64};
  float shape_ms[2] = {0.0f, 0.0f};  // the set-up's timing of each shape (ms)
  // n > 128: the pair contractions run through a stored T = f V o P (hi/lo
  // FP16, [N_aux][N_g] and [N_aux][N_aux]) and three GEMMs over it
  bool large = false;
  int nt = 1;
  long epA = 1, epC = 1;
  __half *TA_h = nullptr, *TA_l = nullptr, *TC_h = nullptr, *TC_l = nullptr;
  // third pieces: of Psi and Psi_g for n > 128 (the S product), of Phi' and Q
  // for every n (the orbital product)
  __half *psi_l = nullptr, *psig_l = nullptr, *phi_l = nullptr, *CT_l = nullptr;
  __half *psigA_m = nullptr, *psigA_h = nullptr, *psigA_l = nullptr;  // all NaT points
  CUtensorMap m_psigA64_m, m_psigA64_h;
  CUtensorMap m_TA_h, m_TA_l, m_TAmn_h, m_TAmn_l, m_TC_h, m_TC_l,
      m_phi_l, m_CT_l;
  // The T-product launches (tprod_kernel): T_A = f_AB V o (Psi_g Psi^T) and
  // T_C = f_C W o (Psi_g Psi_g^T); set up with T_A, T_C (n > 128: at
  // creation; otherwise with the full-K scratch)
  TprodMaps tpA, tpC;
  // n > 128, orbital product on 128 x 256 tiles: Phi' and Q^T pieces as
  // [128][32] / [256][32] boxes with the 64-byte swizzle
  CUtensorMap m_phi32_m, m_phi32_h, m_phi32_l, m_CT32_m, m_CT32_h, m_CT32_l;
  // Full K_{mu nu} (mixed_enqueue_full): scratch allocated on first use
  bool full_ready = false;
  int splitsF = 1, splitsFC = 1, splitsY = 1, kchunkF = 64, kchunkFC = 64, kchunkY = 64;
  float *MpA = nullptr, *MpC = nullptr, *Yp = nullptr, *Zp = nullptr;
  double *DA = nullptr, *DD = nullptr, *DAT64 = nullptr, *DDT64 = nullptr;
  __half *DAT_m = nullptr, *DAT_h = nullptr, *DDT_m = nullptr, *DDT_h = nullptr;
  CUtensorMap m_DAT_m, m_DAT_h, m_DDT_m, m_DDT_h;
  // n <= 128: the roles of the pair launch.  64-column pieces: A (M2), B (M1),
  // C (M3); 128-column pieces (`fused`): roles[0] is the fused role (M1 and
  // M2 from one pass over V, M2 reduced into kM2Copies copies held in M2p),
  // roles[2] is C, and erole is the energy-only form of the fused role.
  PairRole roles[3];
  bool fused = false;
  PairRole erole;
  long long wait_cycles = 0;  // pipeline-wait limit of the handle's kernels (0: the default)
  float tuned_ms = 0.0f;  // pair launch time of the split the autotuner kept
  int kchunkL1 = 64, kchunkL23 = 64;
  CUtensorMap m_phi_m, m_phi_h, m_CT_m, m_CT_h, m_psi128_m, m_psi128_h, m_psi64_m, m_psi64_h,
      m_psig64_m, m_psig64_h, m_VA, m_VB, m_VC, m_phiT_m, m_phiT_h,
      m_M1_m, m_M1_h, m_phigT_m, m_phigT_h, m_D23T_m, m_D23T_h;
};

cudaError_t make_tprod_maps(MixedState* m);
cudaError_t autotune_back_shape(MixedState* m, cudaStream_t s);

namespace {

template <class T>
cudaError_t alloc(MixedState* m, T** p, size_t elems) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(elems, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  m->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

struct Plan {
  long Np, Ng8, Na8, Ng4, Na4, NaT4, NaT8;
  int np, xa, partsA, partsC, splitsL1, splitsL23, kchunkL1, kchunkL23, ychunkA, ychunkC;
  bool large;
  bool fused;      // 128-column pieces, n <= 128: the fused role replaces roles A and B
  int nt;
  long epA, epC;
  int partsA_max;  // largest role-A split the autotuner may pick (buffer sizes)
  int partsC_max;  // largest role-C split (buffer sizes)
  // n > 128: splits of M2 and M3 for 128 x 128 tiles (partsA / partsC are those
  // of the 128 x 256 tiles); the handle times both shapes at set-up
  int partsA_n = 1, partsC_n = 1, ychunkA_n = 64, ychunkC_n = 64;
};

// FP32 copies of M2 the fused role reduces into (X tile % kM2Copies): each
// copy sums a fraction of the X tiles, and the copies are summed in FP64.
constexpr int kM2Copies = 8;

// Role-A splits the autotuner tries for n <= 128: the X tiles times the
// split fill about 2, 3, 4, 6 or 8 waves of CTAs over the 152 SMs.
std::vector<int> tune_candidates(int64_t Ng, int xa) {
  std::vector<int> c;
  const int cap = (int)std::max<int64_t>(1, (Ng + 63) / 64);
  for (int w : {2, 3, 4, 6, 8}) {
    const int parts = std::max(1, std::min(cap, (w * 152 + xa / 2) / xa));
    const int chunk = (int)(((Ng + parts - 1) / parts + 63) / 64 * 64);
    const int real = (int)((Ng + chunk - 1) / chunk);
    if (std::find(c.begin(), c.end(), real) == c.end()) c.push_back(real);
  }
  return c;
}

// Naux: the held slice of interpolation points; NaT: all of them (the g'
// range of the W term).
Plan make_plan(int64_t Ng, int N, int n, int Naux, int NaT) {
  Plan p;
  p.NaT4 = rup(NaT, 4);
  p.NaT8 = rup(NaT, 8);
  p.np = (int)rup(n, 64);
  p.Np = rup(N, 64);
  p.Ng8 = rup(Ng, 8);
  p.Na8 = rup(Naux, 8);
  p.Ng4 = rup(Ng, 4);
  p.Na4 = rup(Naux, 4);
  p.xa = (Naux + 127) / 128;
  p.large = p.np > 128;
  p.fused = p.np == 128;
  p.nt = (n + 127) / 128;
  if (!p.large) {
    // roles A and C: X = g tiles; split Y so the grid is about four waves of 152 SMs
    p.partsA = std::max(1, std::min<int>(608 / p.xa, (int)((Ng + 63) / 64)));
    p.ychunkA = (int)rup((Ng + p.partsA - 1) / p.partsA, 64);
    p.partsA = (int)((Ng + p.ychunkA - 1) / p.ychunkA);
    p.partsC = std::max(1, std::min<int>(608 / p.xa, (NaT + 63) / 64));
    p.ychunkC = (int)rup((NaT + p.partsC - 1) / p.partsC, 64);
    p.partsC = (NaT + p.ychunkC - 1) / p.ychunkC;
    p.partsA_max = p.partsA;
    for (int c : tune_candidates(Ng, p.xa)) p.partsA_max = std::max(p.partsA_max, c);
    p.partsC_max = p.partsC;
    p.epA = (long)p.partsA_max * p.xa;
    p.epC = (long)p.partsC * p.xa;
    if (p.fused) {  // one CTA per 128 grid points over every g; M2 in kM2Copies copies
      p.partsA = p.partsA_max = kM2Copies;
      p.ychunkA = (int)rup(Naux, 64);
      p.epA = (Ng + 127) / 128;
    }
  } else {
    // M2 = T_A Psi and M3 = T_C Psi_g: K split to about four waves of the
    // 128 x 256 tiles (xa x n / 256) and, for the other shape the autotuner
    // tries, of 128 x 128 tiles (xa x n / 128)
    auto split = [&](int tiles, long K, long kmin, int cap, int& chunk) {
      int sp = std::max(1, std::min<int>(cap / tiles, (int)((K + kmin - 1) / kmin)));
      chunk = (int)rup((K + sp - 1) / sp, 64);
      return (int)((K + chunk - 1) / chunk);
    };
    const int tw = p.xa * ((n + 255) / 256), tn = p.xa * p.nt;
    p.partsA = split(tw, Ng, 4096, 608, p.ychunkA);
    p.partsC = split(tw, NaT, 1024, 304, p.ychunkC);
    p.partsA_n = split(tn, Ng, 4096, 608, p.ychunkA_n);
    p.partsC_n = split(tn, NaT, 1024, 304, p.ychunkC_n);
    // energy partials of the T products: one per tile and column half
    p.epA = 2L * p.xa * ((Ng + 127) / 128);
    p.epC = 2L * p.xa * ((NaT + 127) / 128);
    p.partsA_max = std::max(p.partsA, p.partsA_n);
    p.partsC_max = std::max(p.partsC, p.partsC_n);
  }
  // line GEMMs: (N / 128) x (n / 128) tiles (n / 256 for n > 128, which runs
  // them on 128 x 256 tiles) x K splits of >= 1024; split counts round down,
  // so the tiles fill whole waves of CTAs (a wave plus one tile would run a
  // whole extra tile time)
  const int tiles = ((N + 127) / 128) * (p.large ? (n + 255) / 256 : (n + 127) / 128);
  p.splitsL1 = std::max(1, std::min<int>((int)((Ng + 1023) / 1024), 608 / tiles));
  p.kchunkL1 = (int)rup((Ng + p.splitsL1 - 1) / p.splitsL1, 64);
  p.splitsL1 = (int)((Ng + p.kchunkL1 - 1) / p.kchunkL1);
  p.splitsL23 = std::max(1, std::min<int>((Naux + 511) / 512, 304 / tiles));
  p.kchunkL23 = (int)rup((Naux + p.splitsL23 - 1) / p.splitsL23, 64);
  p.splitsL23 = (Naux + p.kchunkL23 - 1) / p.kchunkL23;
  return p;
}

// Split of Q = L^T C into K steps of 16: the product is bound by the FP64
// pipe, and one 64 x 64 x 16 step per CTA spreads the triangle's uneven row
// work evenly over the SMs.
int q_ksplit(int N) { return std::max(1, std::min(64, (N + 15) / 16)); }

// K splits of the full-K contractions: M_A = T_A Phi (K = N_g), M_C = T_C
// Phi_g (K = N_aux) over (N_aux / 128) x (N / 128) tiles, and Phi_g^T M
// (K = N_aux) over (N / 128)^2 tiles: about four waves, K chunks >= 1024.
struct FullPlan {
  int splitsF, kchunkF, splitsFC, kchunkFC, splitsY, kchunkY;
};

FullPlan make_full_plan(int64_t Ng, int N, int Naux) {
  const int xa = (Naux + 127) / 128, tn = (N + 127) / 128;
  auto split = [](long K, int tiles, int& kchunk) {
    int sp = (int)std::max<long>(1, std::min<long>((K + 1023) / 1024, 608 / tiles));
    kchunk = (int)rup((K + sp - 1) / sp, 64);
    return (int)((K + kchunk - 1) / kchunk);
  };
  FullPlan f;
  f.splitsF = split(Ng, xa * tn, f.kchunkF);
  f.splitsFC = split(Naux, xa * tn, f.kchunkFC);
  f.splitsY = split(Naux, tn * tn, f.kchunkY);
  return f;
}

// Split-K work of the FP64 contractions of the set-up and of Q = L^T C.
// Device staging for the set-up (two buffers): Phi and its layouts, W, and V
// in row chunks of at most N rows.
size_t stage_elems(int64_t Ng, int N, int Naux, long Ng8) {
  const size_t ng = Ng, na = Naux;
  return std::max({ng * N + 2 * (size_t)N * N, (size_t)N * Ng8, na * na, ng * std::min<size_t>(na, N),
                   na * (size_t)N});
}

size_t dwork_elems(int64_t Ng, int N, int n) {
  auto w = [](int M, int Nc, int K) {
    const int ks = dgemm_ksplit(M, Nc, K);
    return ks > 1 ? (size_t)ks * M * Nc : (size_t)1;
  };
  return std::max({w(N, N, (int)Ng), (size_t)q_ksplit(N) * N * n, w((int)Ng, N, N), (size_t)1});
}

}  // namespace

size_t mixed_footprint(int64_t Ng, int N, int n, int Naux, int NaT) {
  const Plan p = make_plan(Ng, N, n, Naux, NaT);
  const size_t ng = Ng, na = Naux, nat = NaT;
  size_t b = 0;
  b += 2 * ng * p.Np * 2 + 2 * (size_t)N * p.Ng8 * 2 + 2 * (size_t)N * p.Na8 * 2;  // Phi pieces
  b += (p.fused ? 0 : na * p.Ng4 * 4) + (p.large ? 0 : ng * p.Na4 * 4) + na * p.NaT4 * 4 + nat * 4;  // V, V^T, W, idx
  if (p.large)  // T, third pieces
    b += 2 * na * p.Ng8 * 2 + 2 * na * p.NaT8 * 2 + (ng + nat) * p.np * 2;
  b += (ng + n) * p.Np * 2;  // third pieces of Phi' and Q
  b += 2 * (size_t)n * p.Np * 2 + (size_t)n * p.Np * 8 + 2 * ng * p.np * 2 + 2 * nat * p.np * 2;
  b += (size_t)p.partsA_max * na * n * 4 + (size_t)p.partsC_max * na * n * 4 + (size_t)n * p.Ng4 * 4;
  b += na * n * 8 + (size_t)n * p.Na8 * 8 + 2 * (size_t)n * p.Ng8 * 2 + 2 * (size_t)n * p.Na8 * 2;
  b += (size_t)p.splitsL1 * N * n * 4 + (size_t)p.splitsL23 * N * n * 4;
  b += (size_t)(p.epA + p.epC) * 8;
  b += (size_t)N * N * 8 + (size_t)N * n * 8 + dwork_elems(Ng, N, n) * 8;
  b += 2 * stage_elems(Ng, N, NaT, p.Ng8) * 8;
  return b + 64 * 1024;
}

size_t mixed_full_footprint(int64_t Ng, int N, int n, int Naux) {
  const Plan p = make_plan(Ng, N, n, Naux, Naux);
  const FullPlan f = make_full_plan(Ng, N, Naux);
  const size_t na = Naux, nN = N;
  size_t b = p.large ? 0 : 2 * na * p.Ng8 * 2 + 2 * na * p.Na8 * 2;  // T_A, T_C (hi, lo)
  if (p.fused) b += na * p.Ng4 * 4;  // V in FP32 [g][R] (the fused build keeps only V^T)
  b += (size_t)(f.splitsF + f.splitsFC) * na * nN * 4;                // M_A, M_C partial sums
  b += 2 * na * nN * 8 + 2 * nN * p.Na8 * 8;                         // M_A, M_A - M_C, transposed
  b += 4 * nN * p.Na8 * 2;                                           // their pieces
  b += 2 * (size_t)f.splitsY * nN * nN * 4;                          // Phi_g^T M partial sums
  return b + 64 * 1024;
}

// Role A with its Y range split into `parts` chunks of whole 64-row tiles.
void set_split_a(MixedState* m, int parts) {
  const long ng = m->Ng, na = m->Naux;
  m->ychunkA = (int)rup((ng + parts - 1) / parts, 64);
  m->partsA = (int)((ng + m->ychunkA - 1) / m->ychunkA);
  m->epA = (long)m->partsA * m->xa;
  PairRole& r = m->roles[0];
  r.a = PairArgs{(int)na, (int)ng, m->ychunkA, m->n, m->psig_m, m->psig_h, m->np, m->sc, SC_F_AB,
                 SC_OUT_AB, m->M2p, m->n, (long)(na * m->n), 0, m->EpA, m->status};
  r.gx = m->xa;
  r.nblk = m->xa * m->partsA;
  r.tiles = m->ychunkA / 64;
}

__global__ void fill_pieces_kernel(__half* a, long count, uint32_t seed) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)t * 2654435761u ^ seed;
    h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
    a[t] = __float2half_rn(((float)(h & 0xffff) / 32768.0f - 1.0f) * 0.0625f);
  }
}

__global__ void set_tune_scales_kernel(float* sc) {
  if (threadIdx.x == 0) {
    sc[SC_F_AB] = 1.0f; sc[SC_F_C] = 1.0f; sc[SC_OUT_AB] = 1.0f; sc[SC_OUT_C] = 1.0f;
  }
}

// Autotuner of the pair launch's role-A split: with pseudo-random orbital
// pieces (full switching activity, like real data) and the handle's own V
// and W, time one pair launch per candidate split (best of two) and keep the
// fastest; the heuristic split stays unless another is 3 % faster.  The
// choice fixes the summation order of the role-A partial sums: results are
// bitwise repeatable for the handle, and agree within the stated tolerance
// between handles that chose differently.
cudaError_t autotune_split_a(MixedState* m, cudaStream_t s) {
  const std::vector<int> cands = tune_candidates(m->Ng, m->xa);
  const long ng = m->Ng, na = m->Naux;
  fill_pieces_kernel<<<blocks_for(ng * m->np), 256, 0, s>>>(m->psi_m, ng * m->np, 1u);
  fill_pieces_kernel<<<blocks_for(ng * m->np), 256, 0, s>>>(m->psi_h, ng * m->np, 2u);
  fill_pieces_kernel<<<blocks_for(na * m->np), 256, 0, s>>>(m->psig_m, na * m->np, 3u);
  fill_pieces_kernel<<<blocks_for(na * m->np), 256, 0, s>>>(m->psig_h, na * m->np, 4u);
  set_tune_scales_kernel<<<1, 32, 0, s>>>(m->sc);
  count_launch(5);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const int base = m->partsA;
  int best = base;
  float best_ms = 0.0f, base_ms = 0.0f;
  launch_pair3(m->roles, m->np, s);  // warm-up
  for (int c : cands) {
    set_split_a(m, c);
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, s);
      launch_pair3(m->roles, m->np, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      ms = std::min(ms, t);
    }
    if (e != cudaSuccess) break;
    if (m->partsA == base) base_ms = ms;
    if (best_ms == 0.0f || ms < best_ms) { best_ms = ms; best = m->partsA; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess && base_ms > 0.0f && best_ms > 0.97f * base_ms) best = base;
  set_split_a(m, best);
  m->tuned_ms = best_ms;
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, 16, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t mixed_create(int64_t Ng, int N, int n, int NaT, int g0, int g1, const double* phi,
                         const int32_t* idx, const double* V, const double* W, double dV,
                         cudaStream_t s, MixedState** out) {
  *out = nullptr;
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  const int Naux = g1 - g0;
  const Plan p = make_plan(Ng, N, n, Naux, NaT);
  e = cudaFuncSetAttribute(pair_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pair_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<128>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pair_kernel_group<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pair_kernel_group<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, FusedCfg::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(energy_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(energy_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<128>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tprod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TP_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GW_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_wide3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GW3_SMEM);
  if (e != cudaSuccess) return e;

  MixedState* m = new MixedState();
  auto bail = [&](cudaError_t err) { mixed_destroy(m); return err; };
  m->Ng = Ng; m->N = N; m->n = n; m->Naux = Naux; m->dV = dV; m->np = p.np;
  m->NaT = NaT; m->g0 = g0; m->NaT4 = p.NaT4; m->NaT8 = p.NaT8;
  m->Np = p.Np; m->Ng8 = p.Ng8; m->Na8 = p.Na8; m->Ng4 = p.Ng4; m->Na4 = p.Na4;
  m->xa = p.xa; m->partsA = p.partsA; m->partsC = p.partsC;
  m->ychunkA = p.ychunkA; m->ychunkC = p.ychunkC;
  m->partsA_s[0] = p.partsA_n; m->partsC_s[0] = p.partsC_n;
  m->ychunkA_s[0] = p.ychunkA_n; m->ychunkC_s[0] = p.ychunkC_n;
  m->partsA_s[1] = p.partsA; m->partsC_s[1] = p.partsC;
  m->ychunkA_s[1] = p.ychunkA; m->ychunkC_s[1] = p.ychunkC;
  m->splitsL1 = p.splitsL1; m->splitsL23 = p.splitsL23;
  m->kchunkL1 = p.kchunkL1; m->kchunkL23 = p.kchunkL23;
  m->large = p.large; m->fused = p.fused; m->nt = p.nt; m->epA = p.epA; m->epC = p.epC;
  const size_t ng = Ng, na = Naux, nat = NaT;
#define MX(ptr, elems)                          \
  do {                                          \
    cudaError_t e_ = alloc(m, &(ptr), (elems)); \
    if (e_ != cudaSuccess) return bail(e_);     \
  } while (0)
  MX(m->phi_m, ng * p.Np); MX(m->phi_h, ng * p.Np);
  MX(m->phiT_m, (size_t)N * p.Ng8); MX(m->phiT_h, (size_t)N * p.Ng8);
  MX(m->phigT_m, (size_t)N * p.Na8); MX(m->phigT_h, (size_t)N * p.Na8);
  if (!p.fused) MX(m->V32, na * p.Ng4);
  MX(m->W32, na * p.NaT4);
  if (!p.large) MX(m->VT32, ng * p.Na4);
  if (p.large) {
    MX(m->TA_h, na * p.Ng8); MX(m->TA_l, na * p.Ng8);
    MX(m->TC_h, na * p.NaT8); MX(m->TC_l, na * p.NaT8);
  }
  // third pieces of Phi' and Q for every n: with two pieces the orbital split
  // alone moves E_x by up to ~1e-6 Ha on the 64-centre cell
  MX(m->phi_l, ng * p.Np); MX(m->CT_l, (size_t)n * p.Np);
  MX(m->idx, nat);
  MX(m->CT_m, (size_t)n * p.Np); MX(m->CT_h, (size_t)n * p.Np); MX(m->CT64, (size_t)n * p.Np);
  // the pieces m, h[, l] of Psi and of Psi at all NaT points, each set in one
  // block with a fixed piece stride (one TMA box can span the pieces)
  {
    const size_t npc = p.large ? 3 : 2, ps = ng * p.np, pa = nat * p.np;
    MX(m->psi_m, npc * ps);
    m->psi_h = m->psi_m + ps;
    MX(m->psigA_m, npc * pa);
    m->psigA_h = m->psigA_m + pa;
    if (p.large) {
      m->psi_l = m->psi_m + 2 * ps;
      m->psigA_l = m->psigA_m + 2 * pa;
      m->psig_l = m->psigA_l + (size_t)g0 * p.np;
    }
  }
  m->psig_m = m->psigA_m + (size_t)g0 * p.np;  // the slice's rows
  m->psig_h = m->psigA_h + (size_t)g0 * p.np;
  MX(m->M2p, (size_t)p.partsA_max * na * n); MX(m->M3p, (size_t)p.partsC_max * na * n);
  MX(m->M1, (size_t)n * p.Ng4);
  MX(m->D23, na * n); MX(m->D23T64, (size_t)n * p.Na8);
  MX(m->M1_m, (size_t)n * p.Ng8); MX(m->M1_h, (size_t)n * p.Ng8);
  MX(m->D23T_m, (size_t)n * p.Na8); MX(m->D23T_h, (size_t)n * p.Na8);
  MX(m->L1p, (size_t)p.splitsL1 * N * n); MX(m->L23p, (size_t)p.splitsL23 * N * n);
  MX(m->EpA, (size_t)p.epA); MX(m->EpC, (size_t)p.epC);
  MX(m->sc, NSC); MX(m->am, NAM); MX(m->status, 4); MX(m->rowmax, (size_t)n);
  MX(m->red, reduce_work_elems());
  MX(m->Lf, (size_t)N * N); MX(m->Q64, (size_t)N * n);
  MX(m->dwork, dwork_elems(Ng, N, n));
#undef MX
  double *stage = nullptr, *stage2 = nullptr;
  {
    const size_t elems = stage_elems(Ng, N, NaT, p.Ng8);
    void* q = nullptr;
    e = cudaMalloc(&q, elems * 8);
    if (e != cudaSuccess) return bail(e);
    stage = static_cast<double*>(q);
    e = cudaMalloc(&q, elems * 8);
    if (e != cudaSuccess) { cudaFree(stage); return bail(e); }
    stage2 = static_cast<double*>(q);
  }
  auto fin = [&](cudaError_t err) {
    cudaFree(stage);
    cudaFree(stage2);
    return err == cudaSuccess ? cudaSuccess : bail(err);
  };
  e = cudaMemsetAsync(m->am, 0, NAM * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->sc, 0, NSC * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, 16, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->idx, idx, nat * 4, cudaMemcpyHostToDevice, s);
  // Phi pieces in three layouts: Phi [R][mu], Phi^T [mu][R], Phi_g^T [mu][g]
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, phi, ng * N * 8, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return fin(e);
  // Orthonormalised basis on the grid: Phi^T Phi = L L^T (Cholesky, FP64) and
  // Phi' = Phi L^{-T}.  Each build forms Psi = Phi' (L^T C), which equals
  // Phi C exactly but contracts two matrices with orthonormal columns, so
  // the split arithmetic is not amplified by the conditioning of the basis.
  {
    DGemm g{N, N, (int)ng, stage, N, true, stage, N, false, m->Lf, N, 1.0, nullptr, 0, 0, m->dwork};
    e = dgemm(g, s);
    if (e == cudaSuccess) e = cholesky_f64(m->Lf, N, m->status, s);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, m->status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && st != 0) e = cudaErrorInvalidValue;  // basis dependent on the grid
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, 16, s);
    if (e != cudaSuccess) return fin(e);
    // stage2 (N x N) <- L^{-T} by solving X L^T = I, then Phi' = Phi L^{-T}
    identity_kernel<<<64, 256, 0, s>>>(stage2 + (size_t)N * N, N);
    count_launch();
    e = trsm_right_lt_f64(m->Lf, N, stage2 + (size_t)N * N, N, stage2, s);
    if (e != cudaSuccess) return fin(e);
    DGemm g2{(int)ng, N, N, stage, N, false, stage2, N, false, stage2 + 2 * (size_t)N * N, N, 1.0,
             nullptr, 0, 0, m->dwork};
    e = dgemm(g2, s);
    if (e != cudaSuccess) return fin(e);
    double* phip = stage2 + 2 * (size_t)N * N;
    absmax_kernel<double><<<blocks_for(ng * N), 256, 0, s>>>(phip, ng, N, N, m->am + AM_PHIP);
    rownorm2_max_kernel<double><<<blocks_for(ng), 256, 0, s>>>(phip, ng, N, N, m->am + AM_PHIP_RN);
    absmax_kernel<double><<<blocks_for(ng * N), 256, 0, s>>>(stage, ng, N, N, m->am + AM_PHI);
    set_phi_scale_kernel<<<1, 32, 0, s>>>(m->am, m->sc);
    count_launch(4);
    e = split_rows<double>(phip, ng, N, N, m->sc, SC_PHIP, m->phi_m, m->phi_h, p.Np, s, m->phi_l);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fin(e);
  }
  e = transpose<double>(stage, ng, N, N, stage2, p.Ng8, s);
  if (e == cudaSuccess) e = split_rows<double>(stage2, N, p.Ng8, p.Ng8, m->sc, SC_PHI, m->phiT_m, m->phiT_h, p.Ng8, s);
  if (e == cudaSuccess) e = gather_rows_f64(stage, N, m->idx + g0, Naux, N, stage2, N, s);
  if (e == cudaSuccess) e = transpose<double>(stage2, na, N, N, stage, p.Na8, s);
  if (e == cudaSuccess) e = split_rows<double>(stage, N, p.Na8, p.Na8, m->sc, SC_PHI, m->phigT_m, m->phigT_h, p.Na8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fin(e);
  // V (and, for n <= 128, V^T) in FP32, converted in chunks of rows; max |V|
  // and max |W| bound the product scales
  if (m->VT32) e = cudaMemsetAsync(m->VT32, 0, ng * p.Na4 * 4, s);
  {
    const long chunk = std::max<long>(1, std::min<long>((long)na, N));
    for (long r0 = 0; r0 < (long)na && e == cudaSuccess; r0 += chunk) {
      const long rows = std::min<long>(chunk, (long)na - r0);
      e = cudaMemcpyAsync(stage, V + (size_t)r0 * ng, rows * ng * 8, cudaMemcpyDefault, s);
      if (e != cudaSuccess) break;
      absmax_kernel<double><<<blocks_for(rows * ng), 256, 0, s>>>(stage, rows, ng, ng, m->am + AM_V);
      count_launch();
      if (m->V32) {
        f64_to_f32_kernel<<<blocks_for(rows * p.Ng4), 256, 0, s>>>(stage, rows, ng, m->V32 + r0 * p.Ng4, p.Ng4);
        count_launch();
      }
      if (m->VT32) {  // V^T [g][R]
        dim3 grid((unsigned)((ng + 31) / 32), (unsigned)((rows + 31) / 32));
        transpose_f64_f32_kernel<<<grid, dim3(32, 8), 0, s>>>(stage, rows, ng, ng, m->VT32 + r0, p.Na4);
        count_launch();
      }
      e = cudaStreamSynchronize(s);  // the next chunk reuses the staging buffer
    }
  }
  // W: the slice's rows, all NaT columns
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, W, na * nat * 8, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return fin(e);
  absmax_kernel<double><<<blocks_for(na * nat), 256, 0, s>>>(stage, na, nat, nat, m->am + AM_W);
  f64_to_f32_kernel<<<blocks_for(na * p.NaT4), 256, 0, s>>>(stage, na, nat, m->W32, p.NaT4);
  count_launch(2);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fin(e);

  const auto F16 = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const int np_ = p.np;
  struct MapSpec { CUtensorMap* m; const void* p; CUtensorMapDataType t; int es; long rows, ld; int br, bc; };
  const MapSpec specs[] = {
      {&m->m_phi_m, m->phi_m, F16, 2, (long)ng, p.Np, 128, 64},
      {&m->m_phi_h, m->phi_h, F16, 2, (long)ng, p.Np, 128, 64},
      {&m->m_CT_m, m->CT_m, F16, 2, n, p.Np, 128, 64},
      {&m->m_CT_h, m->CT_h, F16, 2, n, p.Np, 128, 64},
      {&m->m_phi_l, m->phi_l, F16, 2, (long)ng, p.Np, 128, 64},
      {&m->m_CT_l, m->CT_l, F16, 2, n, p.Np, 128, 64},
      {&m->m_psi128_m, m->psi_m, F16, 2, (long)ng, np_, 128, 64},
      {&m->m_psi128_h, m->psi_h, F16, 2, (long)ng, np_, 128, 64},
      {&m->m_psi64_m, m->psi_m, F16, 2, (long)ng, np_, 64, 64},
      {&m->m_psi64_h, m->psi_h, F16, 2, (long)ng, np_, 64, 64},
      {&m->m_psig64_m, m->psig_m, F16, 2, (long)na, np_, 64, 64},
      {&m->m_psig64_h, m->psig_h, F16, 2, (long)na, np_, 64, 64},
      {&m->m_psigA64_m, m->psigA_m, F16, 2, (long)nat, np_, 64, 64},
      {&m->m_psigA64_h, m->psigA_h, F16, 2, (long)nat, np_, 64, 64},
      {&m->m_phiT_m, m->phiT_m, F16, 2, N, p.Ng8, 128, 64},
      {&m->m_phiT_h, m->phiT_h, F16, 2, N, p.Ng8, 128, 64},
      // the line GEMMs' B operands: [256][64] boxes for the 128 x 256 tiles (n > 128)
      {&m->m_M1_m, m->M1_m, F16, 2, n, p.Ng8, p.large ? 256 : 128, 64},
      {&m->m_M1_h, m->M1_h, F16, 2, n, p.Ng8, p.large ? 256 : 128, 64},
      {&m->m_phigT_m, m->phigT_m, F16, 2, N, p.Na8, 128, 64},
      {&m->m_phigT_h, m->phigT_h, F16, 2, N, p.Na8, 128, 64},
      {&m->m_D23T_m, m->D23T_m, F16, 2, n, p.Na8, p.large ? 256 : 128, 64},
      {&m->m_D23T_h, m->D23T_h, F16, 2, n, p.Na8, p.large ? 256 : 128, 64},
  };
  for (const MapSpec& ms : specs) {
    e = make_map(ms.m, ms.p, ms.t, ms.es, ms.rows, ms.ld, ms.br, ms.bc);
    if (e != cudaSuccess) return fin(e);
  }
  if (p.large) {  // T_A, T_C as K-major [rows][K] and T_A as MN-major [K = R][M = g]
    const MapSpec tspecs[] = {
        {&m->m_TA_h, m->TA_h, F16, 2, (long)na, p.Ng8, 128, 64},
        {&m->m_TA_l, m->TA_l, F16, 2, (long)na, p.Ng8, 128, 64},
        {&m->m_TAmn_h, m->TA_h, F16, 2, (long)na, p.Ng8, 64, 64},
        {&m->m_TAmn_l, m->TA_l, F16, 2, (long)na, p.Ng8, 64, 64},
        {&m->m_TC_h, m->TC_h, F16, 2, (long)na, p.NaT8, 128, 64},
        {&m->m_TC_l, m->TC_l, F16, 2, (long)na, p.NaT8, 128, 64},
    };
    for (const MapSpec& ms : tspecs) {
      e = make_map(ms.m, ms.p, ms.t, ms.es, ms.rows, ms.ld, ms.br, ms.bc);
      if (e != cudaSuccess) return fin(e);
    }
  }
  {  // V' tiles [X rows][Y cols] in FP32: [128][32] boxes, 128-byte swizzle
    const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (m->V32) e = make_map(&m->m_VA, m->V32, F32, 4, (long)na, p.Ng4, 128, 32);
    if (e == cudaSuccess && m->VT32) e = make_map(&m->m_VB, m->VT32, F32, 4, (long)ng, p.Na4, 128, 32);
    if (e == cudaSuccess) e = make_map(&m->m_VC, m->W32, F32, 4, (long)na, p.NaT4, 128, 32);
    if (e == cudaSuccess && p.large) e = make_tprod_maps(m);
    if (e == cudaSuccess && p.large) {
      const auto S64 = CU_TENSOR_MAP_SWIZZLE_64B;
      const struct { CUtensorMap* mp; const __half* ptr; long rows; int br; } w3[] = {
          {&m->m_phi32_m, m->phi_m, (long)ng, 128}, {&m->m_phi32_h, m->phi_h, (long)ng, 128},
          {&m->m_phi32_l, m->phi_l, (long)ng, 128}, {&m->m_CT32_m, m->CT_m, (long)n, 256},
          {&m->m_CT32_h, m->CT_h, (long)n, 256}, {&m->m_CT32_l, m->CT_l, (long)n, 256}};
      for (const auto& q : w3)
        if (e == cudaSuccess) e = make_map(q.mp, q.ptr, F16, 2, q.rows, p.Np, q.br, 32, S64);
    }
    if (e != cudaSuccess) return fin(e);
  }
  if (!p.large) {
    // role A: M2[g][j] = sum_R (V o P)[g][R] Psi[R][j], and sum V o P^2
    // role B: M1[j][R] = sum_g (V^T o P^T)[R][g] Psi_g[g][j], written transposed
    // role C: M3[g][j] = sum_g' (W o Q)[g][g'] Psi_g[g'][j], and sum W o Q^2
    // (128-column pieces: the fused role computes A and B in one pass)
    PairRole* r = m->roles;
    const int gB = (int)((ng + 127) / 128);
    for (int k = 0; k < 3; ++k) r[k].kind = 0;
    if (m->fused) {
      r[0].ym = m->m_psig64_m; r[0].yh = m->m_psig64_h; r[0].v = m->m_VB;
      r[0].xm = m->m_psi128_m; r[0].xh = m->m_psi128_h; r[0].kind = 1;
      r[0].a = PairArgs{(int)ng, (int)na, (int)rup(na, 64), n, m->psi_m, m->psi_h, np_, m->sc,
                        SC_F_AB, SC_OUT_AB, m->M1, m->Ng4, 0, 1, m->EpA, m->status,
                        m->VT32, p.Na4, m->M2p, kM2Copies, (long)(na * n)};
      r[0].gx = gB; r[0].nblk = gB; r[0].tiles = (int)(rup(na, 64) / 64);
      r[1] = r[0];
      r[1].nblk = 0;  // unused: the fused role covers role B
      // energy only: the fused role's S products and sums, in the same order
      m->erole = r[0];
      m->erole.kind = 0;
      m->erole.a = PairArgs{(int)ng, (int)na, (int)rup(na, 64), n, m->psi_m, m->psi_h, np_, m->sc,
                            SC_F_AB, SC_OUT_AB, nullptr, 0, 0, 1, m->EpA, m->status};
    } else {
      r[0].ym = m->m_psi64_m; r[0].yh = m->m_psi64_h; r[0].v = m->m_VA;
      set_split_a(m, m->partsA);
      r[1].ym = m->m_psig64_m; r[1].yh = m->m_psig64_h; r[1].v = m->m_VB;
      r[1].a = PairArgs{(int)ng, (int)na, (int)rup(na, 64), n, m->psi_m, m->psi_h, np_, m->sc,
                        SC_F_AB, SC_OUT_AB, m->M1, m->Ng4, 0, 1, nullptr, m->status};
      r[1].gx = gB; r[1].nblk = gB; r[1].tiles = (int)(rup(na, 64) / 64);
    }
    // role C: X = the slice's points, Y = all NaT points (the g' of W)
    r[2].ym = m->m_psigA64_m; r[2].yh = m->m_psigA64_h; r[2].v = m->m_VC;
    r[2].a = PairArgs{(int)na, (int)nat, m->ychunkC, n, m->psig_m, m->psig_h, np_, m->sc, SC_F_C,
                      SC_OUT_C, m->M3p, n, (long)(na * n), 0, m->EpC, m->status};
    r[2].gx = m->xa; r[2].nblk = m->xa * m->partsC; r[2].tiles = m->ychunkC / 64;
    if (!m->fused) {
      e = autotune_split_a(m, s);
      if (e != cudaSuccess) return fin(e);
    }
  } else {
    e = autotune_back_shape(m, s);
    if (e != cudaSuccess) return fin(e);
  }
  fin(cudaSuccess);
  *out = m;
  return cudaSuccess;
}

void mixed_destroy(MixedState* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

cudaError_t mixed_enqueue_pre(MixedState* m, const double* C, cudaStream_t s, const StepHook& hook) {
  const long ng = m->Ng;
  const int N = m->N, n = m->n, np = m->np;
  cudaError_t e;
  // ---- step 1: Psi = Phi C
  hook(0, 1);
  e = cudaMemsetAsync(m->am + AM_C, 0, (NAM - AM_C) * 4, s);
  if (e != cudaSuccess) return e;
  {
    // L^T is upper triangular: each row tile of Q only needs K >= its first row
    DGemm g{N, n, N, m->Lf, N, true, C, n, false, m->Q64, n, 1.0, nullptr, 0, q_ksplit(N), m->dwork,
            true};
    e = dgemm(g, s);
    if (e != cudaSuccess) return e;
  }
  absmax_kernel<double><<<blocks_for((long)N * n), 256, 0, s>>>(m->Q64, N, n, n, m->am + AM_C);
  colnorm2_max_kernel<<<n, 256, 0, s>>>(m->Q64, N, n, m->am + AM_QCN);
  scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 0);
  count_launch(3);
  e = transpose<double>(m->Q64, N, n, n, m->CT64, m->Np, s);  // Q^T [j][mu], zero for mu >= N
  if (e == cudaSuccess)
    e = split_rows<double>(m->CT64, n, m->Np, m->Np, m->sc, SC_C, m->CT_m, m->CT_h, m->Np, s, m->CT_l);
  if (e != cudaSuccess) return e;
  if (!m->large) {  // Psi = Phi' Q (three pieces each), written directly as per-row pieces
    GemmArgs g{(int)ng, n, N, (int)m->Np, nullptr, 0, 0, m->sc, SC_OUT_ORB, m->status,
               m->psi_m, m->psi_h, np, SC_PSI, m->am + AM_RN2};
    g.pieces3 = 1;
    launch_gemm(m->m_phi_m, m->m_phi_h, m->m_CT_m, m->m_CT_h, m->m_phi_l, m->m_CT_l, g,
                dim3((unsigned)((ng + 127) / 128), 1, 1), s, m->wait_cycles);
  } else {  // n > 128: Psi in FP32 (the M1 buffer, free until step 3), then per-row pieces
    GemmArgs g{};
    g.M = (int)ng; g.Ncols = n; g.K = N; g.kchunk = (int)m->Np;
    g.out = m->M1; g.ldo = n; g.sc = m->sc; g.scale_idx = SC_OUT_ORB; g.status = m->status;
    // three pieces (the orbital split error would dominate E_x at this n), on
    // 128 x 256 tiles
    launch_gemm_wide3(m->m_phi32_m, m->m_phi32_h, m->m_phi32_l, m->m_CT32_m, m->m_CT32_h,
                      m->m_CT32_l, g, dim3((unsigned)((ng + 127) / 128), (unsigned)((n + 255) / 256), 1),
                      s, m->wait_cycles);
    split_rows_f32_kernel<<<152 * 4, 256, 0, s>>>(m->M1, ng, n, n, m->sc, SC_PSI, m->psi_m,
                                                  m->psi_h, m->psi_l, np, m->am + AM_RN2);
    count_launch();
  }
  scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 1);
  const long nat = m->NaT;  // the orbitals at every interpolation point (psig is the slice's view)
  gather_rows_half_kernel<<<blocks_for(nat * np), 256, 0, s>>>(m->psi_m, np, m->idx, (int)nat, m->psigA_m);
  gather_rows_half_kernel<<<blocks_for(nat * np), 256, 0, s>>>(m->psi_h, np, m->idx, (int)nat, m->psigA_h);
  count_launch(4);
  if (m->psi_l) {
    gather_rows_half_kernel<<<blocks_for(nat * np), 256, 0, s>>>(m->psi_l, np, m->idx, (int)nat, m->psigA_l);
    count_launch();
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(0, 0);
  return cudaSuccess;
}

// The two T products (S = Psi_g Psi^T and Psi_g Psi_g^T; three pieces each
// for n > 128, two for n <= 128): T = f V' o S and f W' o S as hi/lo FP16
// when `store`, and the energy sums sum V' o S^2, sum W' o S^2 when `energy`
// (n > 128 only: the per-tile sums fill EpA / EpC).
// Tensor maps of the two T-product launches: A = the slice's Psi_g pieces,
// B = Psi (T_A) or the pieces at all NaT points (T_C), in [128][32] boxes with
// the 64-byte swizzle; V and W limited to their N_g and NaT columns (the
// padding of a last tile reads zeros, so T is zero there); T_A and T_C hi/lo
// as store targets over their padded rows.
cudaError_t make_tprod_maps(MixedState* m) {
  const auto F16 = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const auto S64 = CU_TENSOR_MAP_SWIZZLE_64B;
  const long ng = m->Ng, na = m->Naux, nat = m->NaT, np = m->np;
  const int npc = m->large ? 3 : 2;  // pieces; psig is a view of psigA: the same piece stride
  cudaError_t e = make_map3(&m->tpA.a, m->psig_m, F16, 2, na, np, npc, nat * np, 128, 32, S64);
  if (e == cudaSuccess) e = make_map3(&m->tpA.b, m->psi_m, F16, 2, ng, np, npc, ng * np, 128, 32, S64);
  if (e == cudaSuccess) e = make_map3(&m->tpC.b, m->psigA_m, F16, 2, nat, np, npc, nat * np, 128, 32, S64);
  m->tpC.a = m->tpA.a;
  if (e == cudaSuccess)
    e = make_map(&m->tpA.v, m->V32, F32, 4, na, m->Ng4, 128, 32, CU_TENSOR_MAP_SWIZZLE_128B, ng);
  if (e == cudaSuccess)
    e = make_map(&m->tpC.v, m->W32, F32, 4, na, m->NaT4, 128, 32, CU_TENSOR_MAP_SWIZZLE_128B, nat);
  if (e == cudaSuccess) e = make_map(&m->tpA.th, m->TA_h, F16, 2, na, m->Ng8, 128, 32, S64);
  if (e == cudaSuccess) e = make_map(&m->tpA.tl, m->TA_l, F16, 2, na, m->Ng8, 128, 32, S64);
  if (e == cudaSuccess) e = make_map(&m->tpC.th, m->TC_h, F16, 2, na, m->NaT8, 128, 32, S64);
  if (e == cudaSuccess) e = make_map(&m->tpC.tl, m->TC_l, F16, 2, na, m->NaT8, 128, 32, S64);
  return e;
}

void enqueue_t_products(MixedState* m, cudaStream_t s, bool store, bool energy) {
  const long ng = m->Ng, na = m->Naux;
  TprodArgs t{};
  t.M = (int)na; t.Ncols = (int)ng; t.K = m->np; t.sc = m->sc; t.f_idx = SC_F_AB;
  t.epart = energy ? m->EpA : nullptr; t.store = store ? 1 : 0; t.pieces3 = m->large ? 1 : 0;
  t.ld_t = (int)m->Ng8;
  t.tiles_x = m->xa; t.tiles_y = (int)((ng + 127) / 128); t.status = m->status;
  launch_tprod(m->tpA, t, s, m->wait_cycles);
  TprodArgs tc = t;  // rows: the slice's points; columns: all NaT points
  tc.Ncols = m->NaT; tc.f_idx = SC_F_C; tc.epart = energy ? m->EpC : nullptr;
  tc.ld_t = (int)m->NaT8;
  tc.tiles_y = (m->NaT + 127) / 128;
  launch_tprod(m->tpC, tc, s, m->wait_cycles);
  count_launch(2);
}

cudaError_t mixed_full_prepare(MixedState* m) {
  if (m->full_ready) return cudaSuccess;
  if (m->NaT != m->Naux) return cudaErrorNotSupported;  // a slice has no full K of its own
  const long ng = m->Ng, na = m->Naux;
  const int N = m->N;
  const FullPlan f = make_full_plan(ng, N, (int)na);
  m->splitsF = f.splitsF; m->kchunkF = f.kchunkF;
  m->splitsFC = f.splitsFC; m->kchunkFC = f.kchunkFC;
  m->splitsY = f.splitsY; m->kchunkY = f.kchunkY;
  cudaError_t e = cudaSuccess;
#define FX(ptr, elems)                      \
  do {                                      \
    e = alloc(m, &(ptr), (elems));          \
    if (e != cudaSuccess) return e;         \
  } while (0)
  if (!m->V32) {  // the fused build keeps only V^T: form V [g][R] from it
    FX(m->V32, (size_t)na * m->Ng4);
    e = transpose<float>(m->VT32, ng, na, m->Na4, m->V32, m->Ng4, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e == cudaSuccess)
      e = make_map(&m->m_VA, m->V32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, na, m->Ng4, 128, 32);
    if (e != cudaSuccess) return e;
  }
  if (!m->large) {
    FX(m->TA_h, na * m->Ng8); FX(m->TA_l, na * m->Ng8);
    FX(m->TC_h, na * m->Na8); FX(m->TC_l, na * m->Na8);
  }
  FX(m->MpA, (size_t)f.splitsF * na * N); FX(m->MpC, (size_t)f.splitsFC * na * N);
  FX(m->DA, na * N); FX(m->DD, na * N);
  FX(m->DAT64, (size_t)N * m->Na8); FX(m->DDT64, (size_t)N * m->Na8);
  FX(m->DAT_m, (size_t)N * m->Na8); FX(m->DAT_h, (size_t)N * m->Na8);
  FX(m->DDT_m, (size_t)N * m->Na8); FX(m->DDT_h, (size_t)N * m->Na8);
  FX(m->Yp, (size_t)f.splitsY * N * N); FX(m->Zp, (size_t)f.splitsY * N * N);
#undef FX
  const auto F16 = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  if (!m->large) {
    e = make_map(&m->m_TA_h, m->TA_h, F16, 2, na, m->Ng8, 128, 64);
    if (e == cudaSuccess) e = make_map(&m->m_TA_l, m->TA_l, F16, 2, na, m->Ng8, 128, 64);
    if (e == cudaSuccess) e = make_map(&m->m_TC_h, m->TC_h, F16, 2, na, m->Na8, 128, 64);
    if (e == cudaSuccess) e = make_map(&m->m_TC_l, m->TC_l, F16, 2, na, m->Na8, 128, 64);
    if (e == cudaSuccess) e = make_tprod_maps(m);
    if (e != cudaSuccess) return e;
  }
  e = make_map(&m->m_DAT_m, m->DAT_m, F16, 2, N, m->Na8, 128, 64);
  if (e == cudaSuccess) e = make_map(&m->m_DAT_h, m->DAT_h, F16, 2, N, m->Na8, 128, 64);
  if (e == cudaSuccess) e = make_map(&m->m_DDT_m, m->DDT_m, F16, 2, N, m->Na8, 128, 64);
  if (e == cudaSuccess) e = make_map(&m->m_DDT_h, m->DDT_h, F16, 2, N, m->Na8, 128, 64);
  if (e != cudaSuccess) return e;
  m->full_ready = true;
  return cudaSuccess;
}

// Full K_{mu nu} = dV (Phi_g^T M_A + M_A^T Phi_g - Phi_g^T M_C) with
// M_A = (V o P) Phi and M_C = (W o Q) Phi_g: the three terms of Eq. rps in
// Eq. rpsEx, contracted over the grid first (N_aux N_g N + N_aux N^2 flops
// instead of the listed N N_g N_aux + N_g N^2).
cudaError_t mixed_enqueue_full(MixedState* m, const double* C, double* Kf, cudaStream_t s,
                               const StepHook& hook) {
  if (!m->full_ready) return cudaErrorNotReady;
  const long ng = m->Ng, na = m->Naux;
  const int N = m->N;
  cudaError_t e = mixed_enqueue_pre(m, C, s, hook);
  if (e != cudaSuccess) return e;
  hook(1, 1);
  enqueue_t_products(m, s, true, false);
  const unsigned tn = (unsigned)((N + 127) / 128);
  {  // M_A = T_A Phi (A = T_A [g][R] hi/lo, B = Phi^T pieces [nu][R])
    GemmArgs g{};
    g.M = (int)na; g.Ncols = N; g.K = (int)ng; g.kchunk = m->kchunkF; g.out = m->MpA; g.ldo = N;
    g.split_stride = na * N; g.sc = m->sc; g.scale_idx = SC_OUT_FA; g.status = m->status;
    launch_gemm(m->m_TA_h, m->m_TA_l, m->m_phiT_m, m->m_phiT_h, m->m_TA_h, m->m_phiT_m, g,
                dim3((unsigned)m->xa, tn, (unsigned)m->splitsF), s, m->wait_cycles);
    // M_C = T_C Phi_g (A = T_C [g][g'], B = Phi_g^T pieces [nu][g'])
    GemmArgs gc = g;
    gc.K = (int)na; gc.kchunk = m->kchunkFC; gc.out = m->MpC; gc.scale_idx = SC_OUT_FC;
    launch_gemm(m->m_TC_h, m->m_TC_l, m->m_phigT_m, m->m_phigT_h, m->m_TC_h, m->m_phigT_m, gc,
                dim3((unsigned)m->xa, tn, (unsigned)m->splitsFC), s, m->wait_cycles);
  }
  const long cnt = na * N;
  reduce_parts_kernel<<<blocks_for(cnt), 256, 0, s>>>(m->MpA, m->splitsF, nullptr, 0, cnt, m->DA,
                                                      m->am + AM_FA);
  reduce_parts_kernel<<<blocks_for(cnt), 256, 0, s>>>(m->MpA, m->splitsF, m->MpC, m->splitsFC, cnt,
                                                      m->DD, m->am + AM_FD);
  scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 3);
  count_launch(3);
  e = transpose<double>(m->DA, na, N, N, m->DAT64, m->Na8, s);
  if (e == cudaSuccess) e = transpose<double>(m->DD, na, N, N, m->DDT64, m->Na8, s);
  if (e == cudaSuccess)
    e = split_rows<double>(m->DAT64, N, m->Na8, m->Na8, m->sc, SC_FA, m->DAT_m, m->DAT_h, m->Na8, s);
  if (e == cudaSuccess)
    e = split_rows<double>(m->DDT64, N, m->Na8, m->Na8, m->sc, SC_FD, m->DDT_m, m->DDT_h, m->Na8, s);
  if (e != cudaSuccess) return e;
  {  // Y = Phi_g^T M_A and Z = Phi_g^T (M_A - M_C): A = Phi_g^T pieces, B = M^T pieces
    GemmArgs g{};
    g.M = N; g.Ncols = N; g.K = (int)na; g.kchunk = m->kchunkY; g.out = m->Yp; g.ldo = N;
    g.split_stride = (long)N * N; g.sc = m->sc; g.scale_idx = SC_OUT_FY; g.status = m->status;
    launch_gemm(m->m_phigT_m, m->m_phigT_h, m->m_DAT_m, m->m_DAT_h, m->m_phigT_m, m->m_DAT_m, g,
                dim3(tn, tn, (unsigned)m->splitsY), s, m->wait_cycles);
    GemmArgs gz = g;
    gz.out = m->Zp; gz.scale_idx = SC_OUT_FZ;
    launch_gemm(m->m_phigT_m, m->m_phigT_h, m->m_DDT_m, m->m_DDT_h, m->m_phigT_m, m->m_DDT_m, gz,
                dim3(tn, tn, (unsigned)m->splitsY), s, m->wait_cycles);
    count_launch(4);
  }
  final_kfull_kernel<<<blocks_for((long)N * N), 256, 0, s>>>(m->Zp, m->splitsY, m->Yp, m->splitsY,
                                                             N, m->dV, Kf);
  count_launch();
  e = cudaGetLastError();
  hook(1, 0);
  return e;
}

cudaError_t mixed_enqueue_energy(MixedState* m, const double* C, double* Ex, cudaStream_t s,
                                 const StepHook& hook) {
  cudaError_t e = mixed_enqueue_pre(m, C, s, hook);
  if (e != cudaSuccess) return e;
  hook(1, 1);
  if (m->large)
    enqueue_t_products(m, s, false, true);
  else
    launch_energy2(m->fused ? m->erole : m->roles[0], m->roles[2], m->np, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(1, 0);
  hook(7, 1);
  final_ex_kernel<<<1, 1024, 0, s>>>(m->EpA, (int)m->epA, m->EpC, (int)m->epC, m->sc, m->dV, Ex);
  count_launch();
  e = cudaGetLastError();
  hook(7, 0);
  return e;
}

// n > 128: M2 = T_A Psi, M3 = T_C Psi_g and M1^T = T_A^T Psi_g (written
// transposed) over the stored T, on 128 x 256 tiles (wide) or 128 x 128
// tiles, with the splits of that shape (m->partsA, m->partsC, chunks).
void enqueue_back_contractions(MixedState* m, cudaStream_t s, bool wide) {
  const long ng = m->Ng, na = m->Naux;
  const int n = m->n;
  GemmArgs g2{};
  g2.M = (int)na; g2.Ncols = n; g2.K = (int)ng; g2.kchunk = m->ychunkA; g2.out = m->M2p;
  g2.ldo = n; g2.split_stride = na * n; g2.sc = m->sc; g2.scale_idx = SC_OUT_AB;
  g2.status = m->status; g2.b_mn = 1;
  GemmArgs g3 = g2;
  g3.K = m->NaT; g3.kchunk = m->ychunkC; g3.out = m->M3p; g3.scale_idx = SC_OUT_C;
  GemmArgs g1{};
  g1.M = (int)ng; g1.Ncols = n; g1.K = (int)na; g1.kchunk = (int)rup(na, 64); g1.out = m->M1;
  g1.ldo = m->Ng4; g1.sc = m->sc; g1.scale_idx = SC_OUT_AB; g1.status = m->status;
  g1.a_mn = 1; g1.b_mn = 1; g1.transposed = 1;
  const unsigned gx1 = (unsigned)((ng + 127) / 128);
  if (wide) {
    const unsigned ntw = (unsigned)((n + 255) / 256);
    launch_gemm_wide(m->m_TA_h, m->m_TA_l, m->m_psi64_m, m->m_psi64_h, g2,
                     dim3((unsigned)m->xa, ntw, (unsigned)m->partsA), s, m->wait_cycles);
    launch_gemm_wide(m->m_TC_h, m->m_TC_l, m->m_psigA64_m, m->m_psigA64_h, g3,
                     dim3((unsigned)m->xa, ntw, (unsigned)m->partsC), s, m->wait_cycles);
    launch_gemm_wide(m->m_TAmn_h, m->m_TAmn_l, m->m_psig64_m, m->m_psig64_h, g1,
                     dim3(gx1, ntw, 1), s, m->wait_cycles);
  } else {
    const unsigned nt = (unsigned)m->nt;
    launch_gemm(m->m_TA_h, m->m_TA_l, m->m_psi64_m, m->m_psi64_h, m->m_TA_h, m->m_psi64_m, g2,
                dim3((unsigned)m->xa, nt, (unsigned)m->partsA), s, m->wait_cycles);
    launch_gemm(m->m_TC_h, m->m_TC_l, m->m_psigA64_m, m->m_psigA64_h, m->m_TC_h, m->m_psigA64_m,
                g3, dim3((unsigned)m->xa, nt, (unsigned)m->partsC), s, m->wait_cycles);
    launch_gemm(m->m_TAmn_h, m->m_TAmn_l, m->m_psig64_m, m->m_psig64_h, m->m_TAmn_h,
                m->m_psig64_m, g1, dim3(gx1, nt, 1), s, m->wait_cycles);
  }
  count_launch(3);
}

// Sets the back-contraction shape of an n > 128 handle and its splits.
void set_back_shape(MixedState* m, bool wide) {
  const int k = wide ? 1 : 0;
  m->wide = wide;
  m->partsA = m->partsA_s[k]; m->partsC = m->partsC_s[k];
  m->ychunkA = m->ychunkA_s[k]; m->ychunkC = m->ychunkC_s[k];
}

// Autotuner of the n > 128 back-contractions: times the three GEMMs with each
// tile shape (and its own whole-wave split) on zeroed operands, best of two
// launches each, and keeps the faster; 128 x 256 stays unless 128 x 128 is 3 %
// faster.  XK_BACK_TILES=128 or 256 in the environment fixes the shape (tests).
cudaError_t autotune_back_shape(MixedState* m, cudaStream_t s) {
  if (const char* env = std::getenv("XK_BACK_TILES")) {
    set_back_shape(m, std::atoi(env) != 128);
    return cudaSuccess;
  }
  const long ng = m->Ng, na = m->Naux, nat = m->NaT;
  cudaError_t e = cudaMemsetAsync(m->TA_h, 0, (size_t)na * m->Ng8 * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->TA_l, 0, (size_t)na * m->Ng8 * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->TC_h, 0, (size_t)na * m->NaT8 * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->TC_l, 0, (size_t)na * m->NaT8 * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->psi_m, 0, (size_t)3 * ng * m->np * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->psigA_m, 0, (size_t)3 * nat * m->np * 2, s);
  if (e == cudaSuccess) set_tune_scales_kernel<<<1, 32, 0, s>>>(m->sc);
  count_launch();
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    set_back_shape(m, k == 1);
    enqueue_back_contractions(m, s, m->wide);  // warm-up
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, s);
      enqueue_back_contractions(m, s, m->wide);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      ms = std::min(ms, t);
    }
    m->shape_ms[k] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_back_shape(m, !(e == cudaSuccess && m->shape_ms[0] < 0.97f * m->shape_ms[1]));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, 16, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t mixed_enqueue_pair(MixedState* m, cudaStream_t s, const StepHook& hook) {
  const long na = m->Naux;
  const int n = m->n, np = m->np;
  cudaError_t e;
  // ---- steps 2-3: the three fused pair contractions
  hook(1, 1);
  if (m->large) {
    // n > 128: T_A = f_AB V o (Psi_g Psi^T) and T_C = f_C W o (Psi_g Psi_g^T)
    // as hi/lo FP16 with their energy sums, then M2 = T_A Psi, M3 = T_C Psi_g
    // and M1^T = T_A^T Psi_g (written transposed) on the tensor cores.
    enqueue_t_products(m, s, true, true);
    enqueue_back_contractions(m, s, m->wide);
  } else if (m->fused) {
    // M1 and M2 from one pass over V^T (M2 reduced into the copies), and M3
    e = cudaMemsetAsync(m->M2p, 0, (size_t)kM2Copies * na * n * 4, s);
    if (e != cudaSuccess) return e;
    launch_pair_roles({m->roles[0], m->roles[2]}, np, s);
  } else {
    launch_pair3(m->roles, np, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(1, 0);
  return cudaSuccess;
}

cudaError_t mixed_enqueue_post(MixedState* m, double* K, double* Ex, cudaStream_t s,
                               const StepHook& hook) {
  const long ng = m->Ng, na = m->Naux;
  const int N = m->N, n = m->n;
  cudaError_t e;
  // ---- step 4: line1^T = Phi^T M1^T and (line2 - line3)^T = Phi_g^T (M2 - M3)
  hook(4, 1);
  // the fused role's M2 copies hold accumulator units: scaled here (exact, 2^k)
  reduce_parts_kernel<<<blocks_for(na * n), 256, 0, s>>>(m->M2p, m->partsA, m->M3p, m->partsC,
                                                         na * n, m->D23, m->am + AM_D23,
                                                         m->fused ? m->sc + SC_OUT_AB : nullptr);
  e = cudaMemsetAsync(m->rowmax, 0, (size_t)n * 4, s);
  if (e != cudaSuccess) return e;
  {
    const unsigned chunks = (unsigned)std::min<long>(16, (ng + 1023) / 1024);
    rowmax2d_kernel<<<dim3(chunks, n), 256, 0, s>>>(m->M1, ng, m->Ng4, m->rowmax, m->am + AM_M1);
    scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 2);
    const unsigned schunks = (unsigned)std::min<long>(64, (m->Ng8 / 8 + 255) / 256);
    split_mh_rows_pre_kernel<<<dim3(schunks, n), 256, 0, s>>>(
        m->M1, ng, m->Ng4, m->rowmax, m->sc, SC_M1, m->M1_m, m->M1_h, m->Ng8);
  }
  count_launch(4);
  e = transpose<double>(m->D23, na, n, n, m->D23T64, m->Na8, s);
  if (e == cudaSuccess) e = split_rows<double>(m->D23T64, n, m->Na8, m->Na8, m->sc, SC_D23, m->D23T_m, m->D23T_h, m->Na8, s);
  if (e != cudaSuccess) return e;
  {
    GemmArgs g{N, n, (int)ng, m->kchunkL1, m->L1p, n, (long)N * n, m->sc, SC_OUT_L1, m->status,
               nullptr, nullptr, 0, 0, nullptr};
    if (m->large)
      launch_gemm_wide(m->m_phiT_m, m->m_phiT_h, m->m_M1_m, m->m_M1_h, g,
                       dim3((unsigned)((N + 127) / 128), (unsigned)((n + 255) / 256), (unsigned)m->splitsL1),
                       s, m->wait_cycles);
    else
      launch_gemm(m->m_phiT_m, m->m_phiT_h, m->m_M1_m, m->m_M1_h, m->m_phiT_m, m->m_M1_m, g,
                  dim3((unsigned)((N + 127) / 128), (unsigned)((n + 127) / 128), (unsigned)m->splitsL1), s, m->wait_cycles);
  }
  {
    GemmArgs g{N, n, (int)na, m->kchunkL23, m->L23p, n, (long)N * n, m->sc, SC_OUT_L23, m->status,
               nullptr, nullptr, 0, 0, nullptr};
    if (m->large)
      launch_gemm_wide(m->m_phigT_m, m->m_phigT_h, m->m_D23T_m, m->m_D23T_h, g,
                       dim3((unsigned)((N + 127) / 128), (unsigned)((n + 255) / 256), (unsigned)m->splitsL23),
                       s, m->wait_cycles);
    else
      launch_gemm(m->m_phigT_m, m->m_phigT_h, m->m_D23T_m, m->m_D23T_h, m->m_phigT_m, m->m_D23T_m, g,
                  dim3((unsigned)((N + 127) / 128), (unsigned)((n + 127) / 128), (unsigned)m->splitsL23), s, m->wait_cycles);
  }
  count_launch(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(4, 0);

  // ---- step 5: K_{mu i} and E_x in FP64
  hook(7, 1);
  final_k_kernel<<<blocks_for((long)N * n), 256, 0, s>>>(m->L1p, m->splitsL1, m->L23p,
                                                         m->splitsL23, (long)N * n, m->dV, K);
  final_ex_kernel<<<1, 1024, 0, s>>>(m->EpA, (int)m->epA, m->EpC, (int)m->epC, m->sc, m->dV, Ex);
  count_launch(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(7, 0);
  return cudaSuccess;
}

cudaError_t mixed_enqueue(MixedState* m, const double* C, double* K, double* Ex, cudaStream_t s,
                          const StepHook& hook) {
  cudaError_t e = mixed_enqueue_pre(m, C, s, hook);
  if (e == cudaSuccess) e = mixed_enqueue_pair(m, s, hook);
  if (e == cudaSuccess) e = mixed_enqueue_post(m, K, Ex, s, hook);
  return e;
}

// ---- grouped pair launches over several handles (n <= 128 members)
struct PairGroup {
  int np[2] = {64, 128};
  std::vector<PairRole> roles[2];
  std::vector<MixedState*> large;  // members with n > 128 run their own pair step
  std::vector<MixedState*> fused;  // members whose M2 copies are cleared before the launch
};

cudaError_t mixed_group_create(MixedState* const* ms, int count, PairGroup** out) {
  PairGroup* g = new PairGroup();
  for (int t = 0; t < 2; ++t) {
    for (int i = 0; i < count; ++i)
      if (!ms[i]->large && ms[i]->np == g->np[t])
        for (int k = 0; k < 3; ++k)
          if (ms[i]->roles[k].nblk > 0) g->roles[t].push_back(ms[i]->roles[k]);
    std::stable_sort(g->roles[t].begin(), g->roles[t].end(),
                     [](const PairRole& x, const PairRole& y) { return x.tiles > y.tiles; });
  }
  for (int i = 0; i < count; ++i) {
    if (ms[i]->large) g->large.push_back(ms[i]);
    if (ms[i]->fused) g->fused.push_back(ms[i]);
  }
  *out = g;
  return cudaSuccess;
}

cudaError_t mixed_group_enqueue_pair(PairGroup* g, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (MixedState* m : g->fused)
    if (e == cudaSuccess)
      e = cudaMemsetAsync(m->M2p, 0, (size_t)kM2Copies * m->Naux * m->n * 4, s);
  if (e != cudaSuccess) return e;
  for (int t = 0; t < 2; ++t) launch_pair_roles(g->roles[t], g->np[t], s);
  e = cudaGetLastError();
  StepHook none{nullptr, nullptr};
  for (MixedState* m : g->large)
    if (e == cudaSuccess) e = mixed_enqueue_pair(m, s, none);
  return e;
}

void mixed_group_destroy(PairGroup* g) { delete g; }

void mixed_set_wait_limit(MixedState* m, long long cycles) {
  m->wait_cycles = cycles > 0 ? cycles : 0;
  for (PairRole& r : m->roles) r.a.wait = m->wait_cycles;
  m->erole.a.wait = m->wait_cycles;
}

int* mixed_status_ptr(MixedState* m) { return m->status; }

void mixed_autotune_info(const MixedState* m, int* info, double* ms) {
  info[0] = m->large ? (m->wide ? 256 : 128) : 0;
  info[1] = m->partsA;
  ms[0] = m->shape_ms[0];
  ms[1] = m->shape_ms[1];
  ms[2] = m->tuned_ms;
}

}  // namespace xk
