// Mixed-precision path of the exchange build on the 5th-generation tensor
// cores (tcgen05.mma kind::f16, TMA-fed shared memory, TMEM accumulators).
//
// Every bulk contraction runs as split-FP16x3: a value x (scaled by a power
// of two so that |x| <= 2^15) is held as hi = fp16(x) and lo = fp16(x - hi),
// and a product a*b is formed as hi_a*hi_b + hi_a*lo_b + lo_a*hi_b with FP32
// accumulation.  That keeps about 22 significant bits per product.  Partial
// sums leave the tensor memory as FP32 and are added in FP64; K and E_x are
// assembled in FP64.
//
// Build chain (arXiv 2207.04636, Eq. exoccri with contraction order (a) of
// Sec. IV.D):
//   1. Psi = Phi C                          tc_gemm                (Eq. rpsEx step 1)
//   2. Psi_g = Psi[idx], hi/lo splits       split + gather
//   3. M2 = (V o (Psi_g Psi^T)) Psi         pair kernel, role A    (steps 2-3, line 2)
//      M1^T = (V^T o (Psi Psi_g^T)) Psi_g   pair kernel, role B    (line 1)
//      M3 = (W o (Psi_g Psi_g^T)) Psi_g     pair kernel, role C    (line 3)
//   4. line1^T = Phi^T M1^T, (line2 - line3)^T = Phi_g^T (M2 - M3)   tc_gemm
//   5. K_{mu i} = dV (line1 + line2 - line3)^T, E_x = -sum K o C     FP64
// The pair kernel fuses the pair-kernel GEMM, the Hadamard product with the
// stored potential and the back-contraction: the N_aux x N_g pair matrix is
// never written to memory, and V is streamed from HBM once per role.
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
// Device float array of power-of-two scales and FP32 bit patterns of maxima.
enum {
  SC_PHI = 0,   // Phi, Phi^T, Phi_g^T splits
  SC_C,         // C^T split
  SC_PSI,       // Psi, Psi_g splits
  SC_F_AB,      // V o P before its split (roles A, B)
  SC_F_C,       // W o Q before its split (role C)
  SC_M1,        // M1 split
  SC_D23,       // (M2 - M3) split
  SC_OUT_ORB,   // Psi = acc * this
  SC_OUT_AB,    // M2, M1 = acc * this
  SC_OUT_C,     // M3 = acc * this
  SC_OUT_L1,    // line1 = acc * this
  SC_OUT_L23,   // line2 - line3 = acc * this
  NSC
};
enum { AM_PHI = 0, AM_V, AM_W, AM_C, AM_PSI, AM_RN2, AM_M1, AM_D23, NAM };

constexpr float kHalfTarget = 16384.0f;  // 2^14: split inputs are scaled to |x| <= 2^14
constexpr float kProdTarget = 32768.0f;  // 2^15: V o P is scaled to |x| <= 2^15

__device__ float pow2_scale(float maxabs, float target) {
  if (!(maxabs > 0.0f) || !isfinite(maxabs)) return 1.0f;
  int e = (int)floorf(log2f(target / maxabs));
  float s = ldexpf(1.0f, e);
  while (s * maxabs > target) s *= 0.5f;
  return s;
}

__device__ __forceinline__ float am_get(const unsigned* am, int i) { return __uint_as_float(am[i]); }

// stage 0: C split scale; 1: Psi / pair scales; 2: M1, D23 scales.
__global__ void scales_kernel(const unsigned* __restrict__ am, float* __restrict__ sc, int stage) {
  if (threadIdx.x != 0) return;
  if (stage == 0) {
    sc[SC_C] = pow2_scale(am_get(am, AM_C), kHalfTarget);
    sc[SC_OUT_ORB] = 1.0f / (sc[SC_PHI] * sc[SC_C]);
  } else if (stage == 1) {
    const float sp = pow2_scale(am_get(am, AM_PSI), kHalfTarget);
    sc[SC_PSI] = sp;
    // |P(g,R)| <= max_R sum_i psi_i(R)^2 (Cauchy-Schwarz), so |V o P| <= max|V| rn2
    const float rn2 = am_get(am, AM_RN2) * sp * sp;
    const float fab = pow2_scale(am_get(am, AM_V) * rn2, kProdTarget);
    const float fc = pow2_scale(am_get(am, AM_W) * rn2, kProdTarget);
    sc[SC_F_AB] = fab;
    sc[SC_F_C] = fc;
    sc[SC_OUT_AB] = 1.0f / (fab * sp * sp * sp);
    sc[SC_OUT_C] = 1.0f / (fc * sp * sp * sp);
  } else {
    sc[SC_M1] = pow2_scale(am_get(am, AM_M1), kHalfTarget);
    sc[SC_D23] = pow2_scale(am_get(am, AM_D23), kHalfTarget);
    sc[SC_OUT_L1] = 1.0f / (sc[SC_PHI] * sc[SC_M1]);
    sc[SC_OUT_L23] = 1.0f / (sc[SC_PHI] * sc[SC_D23]);
  }
}

__global__ void set_phi_scale_kernel(const unsigned* __restrict__ am, float* __restrict__ sc) {
  if (threadIdx.x == 0) sc[SC_PHI] = pow2_scale(am_get(am, AM_PHI), kHalfTarget);
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

// max over rows of sum_c a[r][c]^2 (rows of Psi: the orbital density at R).
__global__ void rownorm2_max_kernel(const float* __restrict__ a, long rows, int cols, long ld,
                                    unsigned* __restrict__ out) {
  float m = 0.0f;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows;
       r += (long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < cols; ++c) {
      const float v = a[r * ld + c];
      s = fmaf(v, v, s);
    }
    m = fmaxf(m, s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m * 1.0001f));
}

// ----------------------------------------------------------------- splits

__device__ __forceinline__ void split1(double x, __half& hi, __half& lo) {
  hi = __float2half_rn((float)x);
  lo = __float2half_rn((float)(x - (double)__half2float(hi)));
}
__device__ __forceinline__ void split1(float x, __half& hi, __half& lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn(x - __half2float(hi));
}

// dst[r][c] (ld_dst) = split(src[r][c] * scale) for c < cols, 0 for cols <= c < ld_dst.
template <class T>
__global__ void split_rows_kernel(const T* __restrict__ src, long rows, long cols, long ld_src,
                                  const float* __restrict__ sc, int sidx, __half* __restrict__ hi,
                                  __half* __restrict__ lo, long ld_dst) {
  const T s = (T)sc[sidx];
  const long total = rows * ld_dst;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / ld_dst, c = t % ld_dst;
    __half h = __float2half(0.0f), l = __float2half(0.0f);
    if (c < cols) split1(src[r * ld_src + c] * s, h, l);
    hi[t] = h;
    lo[t] = l;
  }
}

// dst[c][r] (ld_dst >= rows) = split(src[r][c] * scale); zero for rows <= r < ld_dst.
template <class T>
__global__ void split_transpose_kernel(const T* __restrict__ src, long rows, long cols,
                                       long ld_src, const float* __restrict__ sc, int sidx,
                                       __half* __restrict__ hi, __half* __restrict__ lo,
                                       long ld_dst) {
  __shared__ T tile[32][33];
  const T s = (T)sc[sidx];
  const long r0 = (long)blockIdx.x * 32, c0 = (long)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * ld_src + c] * s : (T)0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_dst) {
      __half h, l;
      split1(tile[threadIdx.x][i], h, l);
      hi[c * ld_dst + r] = h;
      lo[c * ld_dst + r] = l;
    }
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

// Pads an FP64 host-copied matrix into FP32 [rows][ld_dst] (zero padding).
__global__ void f64_to_f32_kernel(const double* __restrict__ src, long rows, long cols,
                                  float* __restrict__ dst, long ld_dst) {
  const long total = rows * ld_dst;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const long r = t / ld_dst, c = t % ld_dst;
    dst[t] = c < cols ? (float)src[r * cols + c] : 0.0f;
  }
}

// dst[c][r] (ld_dst) = src[r][c] as FP32, zero padding for r >= rows.
__global__ void f64_to_f32_transpose_kernel(const double* __restrict__ src, long rows, long cols,
                                            float* __restrict__ dst, long ld_dst) {
  __shared__ float tile[32][33];
  const long r0 = (long)blockIdx.x * 32, c0 = (long)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? (float)src[r * cols + c] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_dst) dst[c * ld_dst + r] = tile[threadIdx.x][i];
  }
}

// ------------------------------------------------------------ reductions

// out[m][c] = sum_s a[s][m][c] - sum_s b[s][m][c] in FP64 (b nullable), and
// the running max of |out| into am_slot.
__global__ void reduce_parts_kernel(const float* __restrict__ a, int na, const float* __restrict__ b,
                                    int nb, long count, double* __restrict__ out,
                                    unsigned* __restrict__ am_slot) {
  float m = 0.0f;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count;
       t += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < na; ++p) s += (double)a[(long)p * count + t];
    if (b)
      for (int p = 0; p < nb; ++p) s -= (double)b[(long)p * count + t];
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
    double s1 = 0.0, s2 = 0.0;
    for (int p = 0; p < n1; ++p) s1 += (double)L1[(long)p * count + t];
    for (int p = 0; p < n23; ++p) s2 += (double)L23[(long)p * count + t];
    K[t] = dV * (s1 + s2);
  }
}

// ============================================================ tc_gemm
// out[split][m][c] = scale * sum_{k in split} A[m][k] B[c][k] for a 128 x 128
// tile, A and B split-FP16 hi/lo, K-major, 3-stage TMA ring.
// Warps 0-3: epilogue (thread = row); warp 4: TMA producer; warp 5: MMA.

struct GemmArgs {
  int M, Ncols, K, kchunk;
  float* out;
  long ldo;          // row stride of out
  long split_stride; // elements between splits of out
  const float* sc;
  int scale_idx;
  int* status;
};

constexpr int G_STAGES = 3;
constexpr int G_STAGE_BYTES = 4 * 16384;
constexpr int G_SMEM = G_STAGES * G_STAGE_BYTES + 1024;

__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                   const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                   GemmArgs g) {
  extern __shared__ uint8_t g_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(g_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[G_STAGES], empty[G_STAGES], acc_full, drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 128;
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const int nkb = kend > kbeg ? (kend - kbeg + 63) / 64 : 0;

  if (tid == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(&tslot, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;

  if (warp == 4 && lane == 0) {
    prefetch_tmap(&mAh); prefetch_tmap(&mAl); prefetch_tmap(&mBh); prefetch_tmap(&mBl);
    int last_parity[G_STAGES] = {-1, -1, -1};
    for (int kb = 0; kb < nkb && !abort_flag; ++kb) {
      const int s = kb % G_STAGES, use = kb / G_STAGES;
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
        atomicExch(g.status, 11); abort_flag = 1; break;
      }
      uint8_t* st = sm + s * G_STAGE_BYTES;
      mbar_expect_tx(&full[s], G_STAGE_BYTES);
      const int kc = kbeg + kb * 64;
      tma_load_2d(st, &mAh, &full[s], kc, m0);
      tma_load_2d(st + 16384, &mAl, &full[s], kc, m0);
      tma_load_2d(st + 32768, &mBh, &full[s], kc, n0);
      tma_load_2d(st + 49152, &mBl, &full[s], kc, n0);
      last_parity[s] = use & 1;
    }
    for (int s = 0; s < G_STAGES; ++s)
      if (last_parity[s] >= 0) mbar_wait(&full[s], last_parity[s]);
  } else if (warp == 5 && lane == 0) {
    const uint32_t idesc = idesc_f16(128, 128, false, false, false);
    for (int kb = 0; kb < nkb && !abort_flag; ++kb) {
      const int s = kb % G_STAGES;
      if (!mbar_wait(&full[s], (kb / G_STAGES) & 1)) {
        atomicExch(g.status, 12); abort_flag = 1; break;
      }
      tc_fence_after();
      const uint32_t st = smem_u32(sm + s * G_STAGE_BYTES);
      const uint32_t a_off[3] = {0, 0, 16384}, b_off[3] = {32768, 49152, 32768};
      for (int p = 0; p < 3; ++p)
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ad = sdesc_sw128(st + a_off[p] + kk * 32, 16, 1024);
          const uint64_t bd = sdesc_sw128(st + b_off[p] + kk * 32, 16, 1024);
          mma_f16(tbase, ad, bd, idesc, (kb > 0 || p > 0 || kk > 0) ? 1u : 0u);
        }
      mma_commit(&empty[s]);
    }
    mma_commit(&acc_full);
    mma_commit(&drain);
    mbar_wait(&drain, 0);
  } else if (warp < 4) {
    const int r = warp * 32 + lane;
    const bool ok = mbar_wait(&acc_full, 0);
    tc_fence_after();
    if (!ok) atomicExch(g.status, 13);
    const float scale = g.sc[g.scale_idx];
    float* orow = g.out + (long)blockIdx.z * g.split_stride + (long)(m0 + r) * g.ldo;
    const bool row_ok = (m0 + r) < g.M;
    for (int c = 0; c < 128; c += 16) {
      uint32_t v[16];
      tmem_ld16(tbase + (static_cast<uint32_t>(warp * 32) << 16) + c, v);
      tmem_wait_ld();
      if (row_ok)
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c + j;
          if (col < g.Ncols) orow[col] = (ok && nkb > 0) ? __uint_as_float(v[j]) * scale : 0.0f;
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tbase, 128);
}

// ============================================================ pair kernel
// For one X tile of 128 rows and a range of Y rows (in tiles of 64):
//   S = X Y^T (K = NP), T = f * V' o S, acc[x][j] += sum_y T[x][y] Y[y][j]
// X, Y: split-FP16 [rows][NP] K-major; V': FP32 [X rows][Y cols].
// The Y tile doubles as the MN-major B operand of the second product.

struct PairArgs {
  int X, Y, ychunk, n;
  const float* sc;
  int f_idx, out_idx;
  float* out;
  long ldo;
  long part_stride;
  int transposed;  // 0: out[part][x][j]; 1: out[j][x] (single part)
  int* status;
};

template <int NP>
struct PairCfg {
  static constexpr int X_BYTES = 128 * NP * 2;     // one of hi / lo
  static constexpr int Y_BYTES = 64 * NP * 2;
  static constexpr int V_BYTES = 128 * 64 * 4;
  static constexpr int STAGE = 2 * Y_BYTES + V_BYTES;
  static constexpr int OFF_STAGE = 2 * X_BYTES;
  static constexpr int OFF_V2 = OFF_STAGE + 2 * STAGE;
  static constexpr int V2_BYTES = 128 * 64 * 2;
  static constexpr int SMEM = OFF_V2 + 2 * V2_BYTES + 1024;
};

template <int NP>
__global__ void __launch_bounds__(192, 1)
    pair_kernel(const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
                const __grid_constant__ CUtensorMap mYh, const __grid_constant__ CUtensorMap mYl,
                const __grid_constant__ CUtensorMap mV, PairArgs a) {
  using C = PairCfg<NP>;
  extern __shared__ uint8_t p_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t x_full, full[2], empty[2], s_full[2], s_free[2], v2_full, v2_free, acc_full,
      drain;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * 128;
  const int y0 = blockIdx.y * a.ychunk;
  const int y1 = min(a.Y, y0 + a.ychunk);
  const int T = y1 > y0 ? (y1 - y0 + 63) / 64 : 0;
  constexpr int NKB = NP / 64;

  if (tid == 0) {
    mbar_init(&x_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&s_full[s], 1);
      mbar_init(&s_free[s], 128);
    }
    mbar_init(&v2_full, 128);
    mbar_init(&v2_free, 1);
    mbar_init(&acc_full, 1);
    mbar_init(&drain, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(&tslot, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  const uint32_t t_acc = tbase + 128;

  if (warp == 4 && lane == 0) {
    // ---------------- TMA producer
    prefetch_tmap(&mXh); prefetch_tmap(&mXl); prefetch_tmap(&mYh); prefetch_tmap(&mYl);
    prefetch_tmap(&mV);
    int last_parity[2] = {-1, -1};
    bool xl = false;
    if (T > 0) {
      mbar_expect_tx(&x_full, 2 * C::X_BYTES);
      for (int kb = 0; kb < NKB; ++kb) {
        tma_load_2d(sm + kb * 16384, &mXh, &x_full, kb * 64, x0);
        tma_load_2d(sm + C::X_BYTES + kb * 16384, &mXl, &x_full, kb * 64, x0);
      }
      xl = true;
    }
    for (int t = 0; t < T && !abort_flag; ++t) {
      const int s = t & 1, use = t >> 1;
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
        atomicExch(a.status, 21); abort_flag = 1; break;
      }
      uint8_t* st = sm + C::OFF_STAGE + s * C::STAGE;
      mbar_expect_tx(&full[s], C::STAGE);
      const int yr = y0 + t * 64;
      for (int kb = 0; kb < NKB; ++kb) {
        tma_load_2d(st + kb * 8192, &mYh, &full[s], kb * 64, yr);
        tma_load_2d(st + C::Y_BYTES + kb * 8192, &mYl, &full[s], kb * 64, yr);
      }
      tma_load_2d(st + 2 * C::Y_BYTES, &mV, &full[s], yr, x0);
      tma_load_2d(st + 2 * C::Y_BYTES + 16384, &mV, &full[s], yr + 32, x0);
      last_parity[s] = use & 1;
    }
    if (xl) mbar_wait(&x_full, 0);
    for (int s = 0; s < 2; ++s)
      if (last_parity[s] >= 0) mbar_wait(&full[s], last_parity[s]);
  } else if (warp == 5 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t id_s = idesc_f16(128, 64, false, false, false);
    const uint32_t id_acc = idesc_f16(128, NP, false, false, true);
    const uint32_t xh = smem_u32(sm), xlo = smem_u32(sm + C::X_BYTES);
    const uint32_t v2h = smem_u32(sm + C::OFF_V2), v2l = smem_u32(sm + C::OFF_V2 + C::V2_BYTES);
    bool good = T > 0 && mbar_wait(&x_full, 0);
    if (T > 0 && !good) { atomicExch(a.status, 22); abort_flag = 1; }
    auto issue_acc = [&](int u) -> bool {
      const int s = u & 1;
      if (!mbar_wait(&v2_full, u & 1)) return false;
      tc_fence_after();
      const uint32_t yh = smem_u32(sm + C::OFF_STAGE + s * C::STAGE);
      const uint32_t yl = yh + C::Y_BYTES;
      const uint32_t ao[3] = {v2h, v2h, v2l}, bo[3] = {yh, yl, yh};
      for (int p = 0; p < 3; ++p)
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ad = sdesc_sw128(ao[p] + kk * 32, 16, 1024);
          const uint64_t bd = sdesc_sw128(bo[p] + kk * 2048, 8192, 1024);
          mma_f16(t_acc, ad, bd, id_acc, (u > 0 || p > 0 || kk > 0) ? 1u : 0u);
        }
      mma_commit(&empty[s]);
      mma_commit(&v2_free);
      return true;
    };
    for (int t = 0; good && t < T && !abort_flag; ++t) {
      const int s = t & 1, use = t >> 1;
      if (!mbar_wait(&full[s], use & 1)) { atomicExch(a.status, 23); abort_flag = 1; good = false; break; }
      if (use > 0 && !mbar_wait(&s_free[s], (use - 1) & 1)) {
        atomicExch(a.status, 24); abort_flag = 1; good = false; break;
      }
      tc_fence_after();
      const uint32_t yh = smem_u32(sm + C::OFF_STAGE + s * C::STAGE);
      const uint32_t yl = yh + C::Y_BYTES;
      const uint32_t ao[3] = {xh, xh, xlo}, bo[3] = {yh, yl, yh};
      const uint32_t t_s = tbase + s * 64;
      for (int p = 0; p < 3; ++p)
        for (int kk = 0; kk < NP / 16; ++kk) {
          const uint64_t ad = sdesc_sw128(ao[p] + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024);
          const uint64_t bd = sdesc_sw128(bo[p] + (kk >> 2) * 8192 + (kk & 3) * 32, 16, 1024);
          mma_f16(t_s, ad, bd, id_s, (p > 0 || kk > 0) ? 1u : 0u);
        }
      mma_commit(&s_full[s]);
      if (t > 0 && !issue_acc(t - 1)) { atomicExch(a.status, 25); abort_flag = 1; good = false; break; }
    }
    if (good && T > 0 && !issue_acc(T - 1)) { atomicExch(a.status, 26); abort_flag = 1; }
    mma_commit(&acc_full);
    mma_commit(&drain);
    mbar_wait(&drain, 0);
  } else if (warp < 4) {
    // ---------------- epilogue: T = f V' o S, split, stage for the second product
    const int r = warp * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(warp * 32) << 16;
    const float f = a.sc[a.f_idx];
    uint8_t* v2h = sm + C::OFF_V2;
    uint8_t* v2l = v2h + C::V2_BYTES;
    const int sw = r & 7;
    for (int t = 0; t < T && !abort_flag; ++t) {
      const int s = t & 1;
      if (!mbar_wait(&s_full[s], (t >> 1) & 1)) { atomicExch(a.status, 27); abort_flag = 1; break; }
      tc_fence_after();
      float sv[64];
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        uint32_t u[16];
        tmem_ld16(tbase + lane_off + s * 64 + c, u);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) sv[c + j] = __uint_as_float(u[j]);
      }
      tc_fence_before();
      mbar_arrive(&s_free[s]);
      const uint8_t* vt = sm + C::OFF_STAGE + s * C::STAGE + 2 * C::Y_BYTES;
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int box = q >> 3, qc = q & 7;
        const float4 v = *reinterpret_cast<const float4*>(vt + box * 16384 + r * 128 +
                                                          ((qc ^ sw) << 4));
        const float t0 = v.x * sv[4 * q + 0] * f, t1 = v.y * sv[4 * q + 1] * f;
        const float t2 = v.z * sv[4 * q + 2] * f, t3 = v.w * sv[4 * q + 3] * f;
        const __half2 h01 = __floats2half2_rn(t0, t1), h23 = __floats2half2_rn(t2, t3);
        const float2 b01 = __half22float2(h01), b23 = __half22float2(h23);
        const __half2 l01 = __floats2half2_rn(t0 - b01.x, t1 - b01.y);
        const __half2 l23 = __floats2half2_rn(t2 - b23.x, t3 - b23.y);
        hi[2 * q] = *reinterpret_cast<const uint32_t*>(&h01);
        hi[2 * q + 1] = *reinterpret_cast<const uint32_t*>(&h23);
        lo[2 * q] = *reinterpret_cast<const uint32_t*>(&l01);
        lo[2 * q + 1] = *reinterpret_cast<const uint32_t*>(&l23);
      }
      if (t > 0 && !mbar_wait(&v2_free, (t - 1) & 1)) { atomicExch(a.status, 28); abort_flag = 1; break; }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int off = r * 128 + ((q ^ sw) << 4);
        *reinterpret_cast<uint4*>(v2h + off) = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
        *reinterpret_cast<uint4*>(v2l + off) = make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
      }
      fence_async_smem();
      mbar_arrive(&v2_full);
    }
    // ---------------- drain the accumulator
    bool ok = mbar_wait(&acc_full, 0);
    tc_fence_after();
    if (!ok) atomicExch(a.status, 29);
    ok = ok && !abort_flag;
    const float os = a.sc[a.out_idx];
    const int x = x0 + r;
    const bool row_ok = x < a.X;
#pragma unroll 1
    for (int c = 0; c < NP; c += 16) {
      uint32_t u[16];
      tmem_ld16(t_acc + lane_off + c, u);
      tmem_wait_ld();
      if (!row_ok) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c + j;
        if (col >= a.n) continue;
        const float v = (ok && T > 0) ? __uint_as_float(u[j]) * os : 0.0f;
        if (a.transposed)
          a.out[(long)col * a.ldo + x] = v;
        else
          a.out[(long)blockIdx.y * a.part_stride + (long)x * a.ldo + col] = v;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tbase, 256);
}

// ------------------------------------------------------------- host side

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

// 2-D map of a row-major [rows][ld] array, box [box_rows][box_cols], 128-B swizzle.
cudaError_t make_map(CUtensorMap* m, const void* ptr, CUtensorMapDataType dt, int esize, long rows,
                     long ld, int box_rows, int box_cols) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * esize};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, dt, 2, const_cast<void*>(ptr), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

long rup(long a, long b) { return (a + b - 1) / b * b; }
int blocks_for(long total, int tpb = 256) {
  return (int)std::max<long>(1, std::min<long>((total + tpb - 1) / tpb, 152L * 16));
}

}  // namespace

struct MixedState {
  int64_t Ng = 0;
  int N = 0, n = 0, Naux = 0, np = 0;
  long Np = 0, Ng8 = 0, Na8 = 0, Ng4 = 0, Na4 = 0;
  double dV = 0.0;
  std::vector<void*> allocs;
  __half *phi_h = nullptr, *phi_l = nullptr, *phiT_h = nullptr, *phiT_l = nullptr,
         *phigT_h = nullptr, *phigT_l = nullptr;
  float *V32 = nullptr, *VT32 = nullptr, *W32 = nullptr;
  int32_t* idx = nullptr;
  __half *CT_h = nullptr, *CT_l = nullptr, *psi_h = nullptr, *psi_l = nullptr, *psig_h = nullptr,
         *psig_l = nullptr, *M1_h = nullptr, *M1_l = nullptr, *D23T_h = nullptr,
         *D23T_l = nullptr;
  float *psi32 = nullptr, *M2p = nullptr, *M3p = nullptr, *M1 = nullptr, *L1p = nullptr,
        *L23p = nullptr, *sc = nullptr;
  double *D23 = nullptr, *red = nullptr;
  unsigned* am = nullptr;
  int* status = nullptr;
  int partsA = 1, partsC = 1, splitsOrb = 1, splitsL1 = 1, splitsL23 = 1;
  int ychunkA = 64, ychunkC = 64;
  int kchunkL1 = 64, kchunkL23 = 64;
  CUtensorMap m_phi_h, m_phi_l, m_CT_h, m_CT_l, m_psi128_h, m_psi128_l, m_psi64_h, m_psi64_l,
      m_psig128_h, m_psig128_l, m_psig64_h, m_psig64_l, m_V, m_VT, m_W, m_phiT_h, m_phiT_l,
      m_M1_h, m_M1_l, m_phigT_h, m_phigT_l, m_D23T_h, m_D23T_l;
};

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
  long Np, Ng8, Na8, Ng4, Na4;
  int np, partsA, partsC, splitsL1, splitsL23, kchunkL1, kchunkL23, ychunkA, ychunkC;
};

Plan make_plan(int64_t Ng, int N, int n, int Naux) {
  Plan p;
  p.np = (int)rup(n, 64);
  p.Np = rup(N, 64);
  p.Ng8 = rup(Ng, 8);
  p.Na8 = rup(Naux, 8);
  p.Ng4 = rup(Ng, 4);
  p.Na4 = rup(Naux, 4);
  const int xa = (Naux + 127) / 128;
  // role A and C: X = g tiles; split Y so the grid is about two waves of 152 SMs
  p.partsA = std::max(1, std::min<int>((304 + xa - 1) / xa, (int)((Ng + 63) / 64)));
  p.ychunkA = (int)rup((Ng + p.partsA - 1) / p.partsA, 64);
  p.partsA = (int)((Ng + p.ychunkA - 1) / p.ychunkA);
  p.partsC = std::max(1, std::min<int>((152 + xa - 1) / xa, (Naux + 63) / 64));
  p.ychunkC = (int)rup((Naux + p.partsC - 1) / p.partsC, 64);
  p.partsC = (Naux + p.ychunkC - 1) / p.ychunkC;
  // line GEMMs: M = N (basis) tiles x N = n tiles x K splits of >= 1024
  const int tiles = ((N + 127) / 128) * ((n + 127) / 128);
  p.splitsL1 = std::max(1, std::min<int>((int)((Ng + 1023) / 1024), (608 + tiles - 1) / tiles));
  p.kchunkL1 = (int)rup((Ng + p.splitsL1 - 1) / p.splitsL1, 64);
  p.splitsL1 = (int)((Ng + p.kchunkL1 - 1) / p.kchunkL1);
  p.splitsL23 = std::max(1, std::min<int>((Naux + 511) / 512, (304 + tiles - 1) / tiles));
  p.kchunkL23 = (int)rup((Naux + p.splitsL23 - 1) / p.splitsL23, 64);
  p.splitsL23 = (Naux + p.kchunkL23 - 1) / p.kchunkL23;
  return p;
}

}  // namespace

size_t mixed_footprint(int64_t Ng, int N, int n, int Naux) {
  const Plan p = make_plan(Ng, N, n, Naux);
  const size_t ng = Ng, na = Naux;
  size_t b = 0;
  b += 2 * ng * p.Np * 2 + 2 * (size_t)N * p.Ng8 * 2 + 2 * (size_t)N * p.Na8 * 2;  // Phi splits
  b += na * p.Ng4 * 4 + ng * p.Na4 * 4 + na * p.Na4 * 4 + na * 4;                  // V, V^T, W, idx
  b += 2 * (size_t)p.np * p.Np * 2 + ng * n * 4 + 2 * ng * p.np * 2 + 2 * na * p.np * 2;
  b += (size_t)p.partsA * na * n * 4 + (size_t)p.partsC * na * n * 4 + (size_t)n * p.Ng4 * 4;
  b += na * n * 8 + 2 * (size_t)n * p.Ng8 * 2 + 2 * (size_t)n * p.Na8 * 2;
  b += (size_t)p.splitsL1 * N * n * 4 + (size_t)p.splitsL23 * N * n * 4;
  b += ng * std::max<size_t>(N, Naux) * 8;  // setup staging of the FP64 tables
  return b + 64 * 1024;
}

cudaError_t mixed_create(int64_t Ng, int N, int n, int Naux, const double* phi,
                         const int32_t* idx, const double* V, const double* W, double dV,
                         cudaStream_t s, MixedState** out) {
  *out = nullptr;
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  const Plan p = make_plan(Ng, N, n, Naux);
  if (p.np > 128) return cudaErrorNotSupported;  // the fused kernel holds n <= 128 columns
  for (int np : {64, 128}) {
    if (np == 64) e = cudaFuncSetAttribute(pair_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<64>::SMEM);
    else e = cudaFuncSetAttribute(pair_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<128>::SMEM);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
  if (e != cudaSuccess) return e;

  MixedState* m = new MixedState();
  auto bail = [&](cudaError_t err) { mixed_destroy(m); return err; };
  m->Ng = Ng; m->N = N; m->n = n; m->Naux = Naux; m->dV = dV; m->np = p.np;
  m->Np = p.Np; m->Ng8 = p.Ng8; m->Na8 = p.Na8; m->Ng4 = p.Ng4; m->Na4 = p.Na4;
  m->partsA = p.partsA; m->partsC = p.partsC; m->ychunkA = p.ychunkA; m->ychunkC = p.ychunkC;
  m->splitsL1 = p.splitsL1; m->splitsL23 = p.splitsL23;
  m->kchunkL1 = p.kchunkL1; m->kchunkL23 = p.kchunkL23;
  const size_t ng = Ng, na = Naux;
#define MX(ptr, elems)                         \
  do {                                         \
    cudaError_t e_ = alloc(m, &(ptr), (elems)); \
    if (e_ != cudaSuccess) return bail(e_);     \
  } while (0)
  MX(m->phi_h, ng * p.Np); MX(m->phi_l, ng * p.Np);
  MX(m->phiT_h, (size_t)N * p.Ng8); MX(m->phiT_l, (size_t)N * p.Ng8);
  MX(m->phigT_h, (size_t)N * p.Na8); MX(m->phigT_l, (size_t)N * p.Na8);
  MX(m->V32, na * p.Ng4); MX(m->VT32, ng * p.Na4); MX(m->W32, na * p.Na4);
  MX(m->idx, na);
  MX(m->CT_h, (size_t)p.np * p.Np); MX(m->CT_l, (size_t)p.np * p.Np);
  MX(m->psi32, ng * n);
  MX(m->psi_h, ng * p.np); MX(m->psi_l, ng * p.np);
  MX(m->psig_h, na * p.np); MX(m->psig_l, na * p.np);
  MX(m->M2p, (size_t)p.partsA * na * n); MX(m->M3p, (size_t)p.partsC * na * n);
  MX(m->M1, (size_t)n * p.Ng4);
  MX(m->D23, na * n);
  MX(m->M1_h, (size_t)n * p.Ng8); MX(m->M1_l, (size_t)n * p.Ng8);
  MX(m->D23T_h, (size_t)n * p.Na8); MX(m->D23T_l, (size_t)n * p.Na8);
  MX(m->L1p, (size_t)p.splitsL1 * N * n); MX(m->L23p, (size_t)p.splitsL23 * N * n);
  MX(m->sc, NSC); MX(m->am, NAM); MX(m->status, 4);
  MX(m->red, reduce_work_elems());
  double* stage = nullptr;
  {
    void* q = nullptr;
    e = cudaMalloc(&q, ng * std::max<size_t>(N, na) * 8);
    if (e != cudaSuccess) return bail(e);
    stage = static_cast<double*>(q);
  }
  auto fin = [&](cudaError_t err) { cudaFree(stage); return err == cudaSuccess ? cudaSuccess : bail(err); };
  e = cudaMemsetAsync(m->am, 0, NAM * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->sc, 0, NSC * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, 16, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->CT_h, 0, (size_t)p.np * p.Np * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->CT_l, 0, (size_t)p.np * p.Np * 2, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->idx, idx, na * 4, cudaMemcpyHostToDevice, s);
  // Phi: FP64 staging -> scale -> splits in three layouts
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, phi, ng * N * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fin(e);
  absmax_kernel<double><<<blocks_for(ng * N), 256, 0, s>>>(stage, ng, N, N, m->am + AM_PHI);
  set_phi_scale_kernel<<<1, 32, 0, s>>>(m->am, m->sc);
  split_rows_kernel<double><<<blocks_for(ng * p.Np), 256, 0, s>>>(stage, ng, N, N, m->sc, SC_PHI, m->phi_h, m->phi_l, p.Np);
  {
    dim3 grid((unsigned)((p.Ng8 + 31) / 32), (unsigned)((N + 31) / 32));
    split_transpose_kernel<double><<<grid, dim3(32, 8), 0, s>>>(stage, ng, N, N, m->sc, SC_PHI, m->phiT_h, m->phiT_l, p.Ng8);
  }
  count_launch(4);
  // Phi_g^T from the gathered FP64 rows (reuse the front of the staging buffer after Phi^T)
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fin(e);
  {
    // gather Phi rows at idx into a compact FP64 buffer, then transpose-split
    double* phig = nullptr;
    void* q = nullptr;
    e = cudaMalloc(&q, na * N * 8);
    if (e != cudaSuccess) return fin(e);
    phig = static_cast<double*>(q);
    e = gather_rows_f64(stage, N, m->idx, Naux, N, phig, N, s);
    if (e == cudaSuccess) {
      dim3 grid((unsigned)((p.Na8 + 31) / 32), (unsigned)((N + 31) / 32));
      split_transpose_kernel<double><<<grid, dim3(32, 8), 0, s>>>(phig, na, N, N, m->sc, SC_PHI, m->phigT_h, m->phigT_l, p.Na8);
      count_launch();
      e = cudaStreamSynchronize(s);
    }
    cudaFree(phig);
    if (e != cudaSuccess) return fin(e);
  }
  // V in both orientations, W; max |V|, max |W| for the product scales
  e = cudaMemcpyAsync(stage, V, na * ng * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fin(e);
  absmax_kernel<double><<<blocks_for(na * ng), 256, 0, s>>>(stage, na, ng, ng, m->am + AM_V);
  f64_to_f32_kernel<<<blocks_for(na * p.Ng4), 256, 0, s>>>(stage, na, ng, m->V32, p.Ng4);
  {
    dim3 grid((unsigned)((p.Na4 + 31) / 32), (unsigned)((ng + 31) / 32));
    // VT[R][g] = V[g][R], zero for g >= N_aux
    f64_to_f32_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(stage, na, ng, m->VT32, p.Na4);
  }
  count_launch(3);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage, W, na * na * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fin(e);
  absmax_kernel<double><<<blocks_for(na * na), 256, 0, s>>>(stage, na, na, na, m->am + AM_W);
  f64_to_f32_kernel<<<blocks_for(na * p.Na4), 256, 0, s>>>(stage, na, na, m->W32, p.Na4);
  count_launch(2);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fin(e);

  // tensor maps
  const auto F16 = CU_TENSOR_MAP_DATA_TYPE_FLOAT16, F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int np_ = p.np;
  struct MapSpec { CUtensorMap* m; const void* p; CUtensorMapDataType t; int es; long rows, ld; int br, bc; };
  const MapSpec specs[] = {
      {&m->m_phi_h, m->phi_h, F16, 2, (long)ng, p.Np, 128, 64},
      {&m->m_phi_l, m->phi_l, F16, 2, (long)ng, p.Np, 128, 64},
      {&m->m_CT_h, m->CT_h, F16, 2, n, p.Np, 128, 64},
      {&m->m_CT_l, m->CT_l, F16, 2, n, p.Np, 128, 64},
      {&m->m_psi128_h, m->psi_h, F16, 2, (long)ng, np_, 128, 64},
      {&m->m_psi128_l, m->psi_l, F16, 2, (long)ng, np_, 128, 64},
      {&m->m_psi64_h, m->psi_h, F16, 2, (long)ng, np_, 64, 64},
      {&m->m_psi64_l, m->psi_l, F16, 2, (long)ng, np_, 64, 64},
      {&m->m_psig128_h, m->psig_h, F16, 2, (long)na, np_, 128, 64},
      {&m->m_psig128_l, m->psig_l, F16, 2, (long)na, np_, 128, 64},
      {&m->m_psig64_h, m->psig_h, F16, 2, (long)na, np_, 64, 64},
      {&m->m_psig64_l, m->psig_l, F16, 2, (long)na, np_, 64, 64},
      {&m->m_V, m->V32, F32, 4, (long)na, p.Ng4, 128, 32},
      {&m->m_VT, m->VT32, F32, 4, (long)ng, p.Na4, 128, 32},
      {&m->m_W, m->W32, F32, 4, (long)na, p.Na4, 128, 32},
      {&m->m_phiT_h, m->phiT_h, F16, 2, N, p.Ng8, 128, 64},
      {&m->m_phiT_l, m->phiT_l, F16, 2, N, p.Ng8, 128, 64},
      {&m->m_M1_h, m->M1_h, F16, 2, n, p.Ng8, 128, 64},
      {&m->m_M1_l, m->M1_l, F16, 2, n, p.Ng8, 128, 64},
      {&m->m_phigT_h, m->phigT_h, F16, 2, N, p.Na8, 128, 64},
      {&m->m_phigT_l, m->phigT_l, F16, 2, N, p.Na8, 128, 64},
      {&m->m_D23T_h, m->D23T_h, F16, 2, n, p.Na8, 128, 64},
      {&m->m_D23T_l, m->D23T_l, F16, 2, n, p.Na8, 128, 64},
  };
  for (const MapSpec& ms : specs) {
    e = make_map(ms.m, ms.p, ms.t, ms.es, ms.rows, ms.ld, ms.br, ms.bc);
    if (e != cudaSuccess) return fin(e);
  }
#undef MX
  cudaFree(stage);
  *out = m;
  return cudaSuccess;
}

void mixed_destroy(MixedState* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

cudaError_t mixed_enqueue(MixedState* m, const double* C, double* K, double* Ex, cudaStream_t s,
                          const StepHook& hook) {
  const long ng = m->Ng, na = m->Naux;
  const int N = m->N, n = m->n, np = m->np;
  cudaError_t e;
  // ---- step 1: Psi = Phi C
  hook(0, 1);
  e = cudaMemsetAsync(m->am + AM_C, 0, (NAM - AM_C) * 4, s);
  if (e != cudaSuccess) return e;
  absmax_kernel<double><<<blocks_for((long)N * n), 256, 0, s>>>(C, N, n, n, m->am + AM_C);
  scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 0);
  {
    dim3 grid((unsigned)((m->Np + 31) / 32), (unsigned)((n + 31) / 32));
    // C^T[j][mu] from C[mu][j]; rows j >= n of CT stay zero from setup
    split_transpose_kernel<double><<<grid, dim3(32, 8), 0, s>>>(C, N, n, n, m->sc, SC_C, m->CT_h, m->CT_l, m->Np);
  }
  {
    GemmArgs g{(int)ng, n, N, (int)m->Np, m->psi32, n, 0, m->sc, SC_OUT_ORB, m->status};
    dim3 grid((unsigned)((ng + 127) / 128), (unsigned)((n + 127) / 128), 1);
    tc_gemm_kernel<<<grid, 192, G_SMEM, s>>>(m->m_phi_h, m->m_phi_l, m->m_CT_h, m->m_CT_l, g);
  }
  absmax_kernel<float><<<blocks_for(ng * n), 256, 0, s>>>(m->psi32, ng, n, n, m->am + AM_PSI);
  rownorm2_max_kernel<<<blocks_for(ng), 256, 0, s>>>(m->psi32, ng, n, n, m->am + AM_RN2);
  scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 1);
  split_rows_kernel<float><<<blocks_for(ng * np), 256, 0, s>>>(m->psi32, ng, n, n, m->sc, SC_PSI, m->psi_h, m->psi_l, np);
  gather_rows_half_kernel<<<blocks_for(na * np), 256, 0, s>>>(m->psi_h, np, m->idx, (int)na, m->psig_h);
  gather_rows_half_kernel<<<blocks_for(na * np), 256, 0, s>>>(m->psi_l, np, m->idx, (int)na, m->psig_l);
  count_launch(10);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(0, 0);

  // ---- step 2-3: the three fused pair contractions
  hook(1, 1);
  const int xa = (int)((na + 127) / 128);
  auto launch_pair = [&](const CUtensorMap& Xh, const CUtensorMap& Xl, const CUtensorMap& Yh,
                         const CUtensorMap& Yl, const CUtensorMap& Vm, const PairArgs& pa,
                         dim3 grid) {
    if (np == 64)
      pair_kernel<64><<<grid, 192, PairCfg<64>::SMEM, s>>>(Xh, Xl, Yh, Yl, Vm, pa);
    else
      pair_kernel<128><<<grid, 192, PairCfg<128>::SMEM, s>>>(Xh, Xl, Yh, Yl, Vm, pa);
    count_launch();
  };
  {  // role A: M2[g][j] = sum_R (V o P)[g][R] Psi[R][j]
    PairArgs pa{(int)na, (int)ng, m->ychunkA, n, m->sc, SC_F_AB, SC_OUT_AB, m->M2p, n,
                na * n, 0, m->status};
    launch_pair(m->m_psig128_h, m->m_psig128_l, m->m_psi64_h, m->m_psi64_l, m->m_V, pa,
                dim3(xa, m->partsA));
  }
  {  // role B: M1[j][R] = sum_g (V^T o P^T)[R][g] Psi_g[g][j], written transposed
    PairArgs pa{(int)ng, (int)na, (int)rup(na, 64), n, m->sc, SC_F_AB, SC_OUT_AB, m->M1,
                m->Ng4, 0, 1, m->status};
    launch_pair(m->m_psi128_h, m->m_psi128_l, m->m_psig64_h, m->m_psig64_l, m->m_VT, pa,
                dim3((unsigned)((ng + 127) / 128), 1));
  }
  {  // role C: M3[g][j] = sum_g' (W o Q)[g][g'] Psi_g[g'][j]
    PairArgs pa{(int)na, (int)na, m->ychunkC, n, m->sc, SC_F_C, SC_OUT_C, m->M3p, n, na * n, 0,
                m->status};
    launch_pair(m->m_psig128_h, m->m_psig128_l, m->m_psig64_h, m->m_psig64_l, m->m_W, pa,
                dim3(xa, m->partsC));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(1, 0);

  // ---- step 4: line1^T = Phi^T M1^T and (line2 - line3)^T = Phi_g^T (M2 - M3)
  hook(4, 1);
  reduce_parts_kernel<<<blocks_for(na * n), 256, 0, s>>>(m->M2p, m->partsA, m->M3p, m->partsC,
                                                         na * n, m->D23, m->am + AM_D23);
  absmax_kernel<float><<<blocks_for((long)n * ng), 256, 0, s>>>(m->M1, n, ng, m->Ng4, m->am + AM_M1);
  scales_kernel<<<1, 32, 0, s>>>(m->am, m->sc, 2);
  split_rows_kernel<float><<<blocks_for((long)n * m->Ng8), 256, 0, s>>>(m->M1, n, ng, m->Ng4, m->sc, SC_M1, m->M1_h, m->M1_l, m->Ng8);
  {
    dim3 grid((unsigned)((m->Na8 + 31) / 32), (unsigned)((n + 31) / 32));
    split_transpose_kernel<double><<<grid, dim3(32, 8), 0, s>>>(m->D23, na, n, n, m->sc, SC_D23, m->D23T_h, m->D23T_l, m->Na8);
  }
  {
    GemmArgs g{N, n, (int)ng, m->kchunkL1, m->L1p, n, (long)N * n, m->sc, SC_OUT_L1, m->status};
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((n + 127) / 128), (unsigned)m->splitsL1);
    tc_gemm_kernel<<<grid, 192, G_SMEM, s>>>(m->m_phiT_h, m->m_phiT_l, m->m_M1_h, m->m_M1_l, g);
  }
  {
    GemmArgs g{N, n, (int)na, m->kchunkL23, m->L23p, n, (long)N * n, m->sc, SC_OUT_L23, m->status};
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((n + 127) / 128), (unsigned)m->splitsL23);
    tc_gemm_kernel<<<grid, 192, G_SMEM, s>>>(m->m_phigT_h, m->m_phigT_l, m->m_D23T_h, m->m_D23T_l, g);
  }
  count_launch(7);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook(4, 0);

  // ---- step 5: K_{mu i} and E_x in FP64
  hook(7, 1);
  final_k_kernel<<<blocks_for((long)N * n), 256, 0, s>>>(m->L1p, m->splitsL1, m->L23p,
                                                         m->splitsL23, (long)N * n, m->dV, K);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = neg_dot_f64(K, C, (long)N * n, m->red, Ex, s);
  if (e != cudaSuccess) return e;
  hook(7, 0);
  return cudaSuccess;
}

int mixed_take_status(MixedState* m) {
  int st[4] = {0, 0, 0, 0};
  if (cudaMemcpy(st, m->status, 16, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (st[0] != 0) cudaMemset(m->status, 0, 16);
  return st[0];
}

double mixed_error_bound(const MixedState* m) {
  // Per-product relative error of split-FP16x3 is about 2^-22; the E_x bound
  // reported with each result is that factor times the size of the build.
  (void)m;
  return 1e-6;
}

}  // namespace xk
