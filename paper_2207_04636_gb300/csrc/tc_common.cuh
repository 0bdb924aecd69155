// Blackwell (sm_103a) building blocks written as inline PTX: mbarriers with
// bounded waits, TMA tiled loads, tensor-memory allocation and loads, the
// tcgen05.mma issue/commit pair, and the shared-memory / instruction
// descriptors of the 5th-generation tensor cores.
//
// Layout conventions used by every kernel in this library:
//   * 16-bit operands live in shared memory in the 128-byte swizzled layout
//     that a TMA load with CU_TENSOR_MAP_SWIZZLE_128B produces: rows of 64
//     elements (128 B), 8-row atoms of 1024 B, tile bases 1024-B aligned.
//   * A K-major operand tile [rows][64] is described with SBO = 1024 (the
//     stride between 8-row groups); successive K=16 slices start 32 B apart.
//   * An MN-major operand tile [K rows][MN] made of 64-wide column blocks is
//     described with LBO = stride between the column blocks and SBO = 1024
//     (8 K-rows); successive K=16 slices start 2048 B apart.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace xk {
namespace tc {

// Bound on any single wait inside a kernel, in SM clock cycles (about one
// second at 2 GHz).  A wait that runs out records an error and returns.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of the phase (never suspends the thread).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// A wait with a shortened limit: polls with mbarrier.test_wait, so the limit
// holds even when it is shorter than the interval try_wait may sleep.  Kept
// out of line: the default path below stays as short as it was.
__device__ __noinline__ bool mbar_wait_short(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Waits for the phase with the given parity to complete; gives up after
// `limit` SM clock cycles (default kWaitCycles) and returns false.  Kernels
// take the limit of their pipeline waits from their launch arguments (a
// handle can shorten it, e.g. to make a wait run out in a test); the final
// waits for a kernel's own TMA copies and MMAs always use kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitCycles) {
  if (limit < kWaitCycles) return mbar_wait_short(bar, parity, limit);
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// All lanes of a warp wait; true only if every lane saw the phase.  Fast
// path: after __syncwarp the lanes are converged and one test_wait (which
// never suspends a lane) gives them one barrier state, so a completed phase
// costs about 25 cycles instead of about 75 with try_wait and a vote;
// otherwise the bounded wait, and a vote on its result.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity,
                                               long long limit = kWaitCycles) {
  __syncwarp();
  if (mbar_test(bar, parity)) return true;
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, limit));
}

// The pipeline-wait limit of a launch: `arg` cycles when positive, else the default.
__device__ __forceinline__ long long wait_limit(long long arg) {
  return arg > 0 ? arg : kWaitCycles;
}

// True when a launch shortened its pipeline-wait limit.  Kernels then run a
// separate instantiation of their body (template flag kShort), so that the
// default instantiation compiles the plain bounded wait and nothing else.
__device__ __forceinline__ bool short_wait(long long arg) { return arg > 0 && arg < kWaitCycles; }

// True in exactly one lane (the lowest) of a converged warp.
__device__ __forceinline__ bool elect_one() {
  uint32_t p;
  asm volatile(
      "{\n\t.reg .pred P;\n\t.reg .b32 r;\n\t"
      "elect.sync r|P, 0xffffffff;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(p));
  return p != 0;
}

// ---------------------------------------------------------------- fences

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- TMA

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Tiled store of a shared-memory box to global memory (bulk async group of
// the issuing thread); elements outside the tensor map's extent are dropped.
// The writers of the box execute fence_async_smem() and synchronise first.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int c0,
                                             int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until every committed bulk store of this thread has read its source
// (the shared memory may then be rewritten).
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Waits until every committed bulk store of this thread has completed.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Brings a tile of a tensor map into L2 (no shared-memory destination).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int c0, int c1) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1)
               : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------- TMEM

// One full warp executes these.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Thread t of warp w reads TMEM lane 32*(w%4)+t, columns [col, col+16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Thread t of warp w reads TMEM lane 32*(w%4)+t, columns [col, col+8).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Thread t of warp w writes TMEM lane 32*(w%4)+t, columns [col, col+8).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// Thread t of warp w writes TMEM lane 32*(w%4)+t, columns [col, col+16).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Thread t of warp w reads TMEM lane 32*(w%4)+t, columns [col, col+32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]),"=r"(r[1]),"=r"(r[2]),"=r"(r[3]),"=r"(r[4]),"=r"(r[5]),"=r"(r[6]),"=r"(r[7]),"=r"(r[8]),"=r"(r[9]),"=r"(r[10]),"=r"(r[11]),"=r"(r[12]),"=r"(r[13]),"=r"(r[14]),"=r"(r[15]),"=r"(r[16]),"=r"(r[17]),"=r"(r[18]),"=r"(r[19]),"=r"(r[20]),"=r"(r[21]),"=r"(r[22]),"=r"(r[23]),"=r"(r[24]),"=r"(r[25]),"=r"(r[26]),"=r"(r[27]),"=r"(r[28]),"=r"(r[29]),"=r"(r[30]),"=r"(r[31])
      : "r"(taddr));
}

// Thread t of warp w writes TMEM lane 32*(w%4)+t, columns [col, col+32).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]),"r"(r[1]),"r"(r[2]),"r"(r[3]),"r"(r[4]),"r"(r[5]),"r"(r[6]),"r"(r[7]),"r"(r[8]),"r"(r[9]),"r"(r[10]),"r"(r[11]),"r"(r[12]),"r"(r[13]),"r"(r[14]),"r"(r[15]),"r"(r[16]),"r"(r[17]),"r"(r[18]),"r"(r[19]),"r"(r[20]),"r"(r[21]),"r"(r[22]),"r"(r[23]),"r"(r[24]),"r"(r[25]),"r"(r[26]),"r"(r[27]),"r"(r[28]),"r"(r[29]),"r"(r[30]),"r"(r[31])
      : "memory");
}


// ---------------------------------------------------------------- MMA

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (fp16 or bf16 in, fp32 accumulate).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16: A (M x 16 per instruction) lives
// in tensor memory, one row per lane, two 16-bit elements per 32-bit column
// (the lower half holds the even K index).
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Runs of MMAs along K issued by one elected lane of a converged warp, with
// no branch per MMA: the whole warp executes one asm block, elect.sync picks
// the lane and every tcgen05.mma is predicated on it.  `acc0` enables the
// accumulator for the first MMA of the run; the others always accumulate.
//
// 8 TS MMAs: A in tensor memory at ta + 8 k (16-bit pairs, 8 columns per K
// step); B a K-major 128-byte-swizzled tile whose K steps sit at
// desc + {0, 2, 4, 6, 512, 514, 516, 518} (32 B apart within a 64-wide block,
// 8 KB between blocks).
__device__ __forceinline__ void mma_ts_run8_kmajor(uint32_t d, uint32_t ta, uint64_t b,
                                                   uint32_t idesc, uint32_t acc0) {
  asm volatile(
      "{\n\t.reg .pred E, A, T;\n\t.reg .b64 b1, b2, b3, b4, b5, b6, b7;\n\t"
      ".reg .b32 a1, a2, a3, a4, a5, a6, a7;\n\t"
      "elect.sync _|E, 0xffffffff;\n\t"
      "setp.ne.b32 A, %4, 0;\n\tsetp.eq.b32 T, 0, 0;\n\t"
      "add.u32 a1, %1, 8;\n\tadd.u32 a2, %1, 16;\n\tadd.u32 a3, %1, 24;\n\tadd.u32 a4, %1, 32;\n\t"
      "add.u32 a5, %1, 40;\n\tadd.u32 a6, %1, 48;\n\tadd.u32 a7, %1, 56;\n\t"
      "add.s64 b1, %2, 2;\n\tadd.s64 b2, %2, 4;\n\tadd.s64 b3, %2, 6;\n\tadd.s64 b4, %2, 512;\n\t"
      "add.s64 b5, %2, 514;\n\tadd.s64 b6, %2, 516;\n\tadd.s64 b7, %2, 518;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, A;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a4], b4, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a5], b5, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a6], b6, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a7], b7, %3, T;\n\t}" ::"r"(d),
      "r"(ta), "l"(b), "r"(idesc), "r"(acc0)
      : "memory");
}

// 4 TS MMAs: A in tensor memory at ta + 8 k; B an MN-major tile whose K steps
// (16 rows) sit 2048 B apart (desc + 128 k).
__device__ __forceinline__ void mma_ts_run4_mn(uint32_t d, uint32_t ta, uint64_t b, uint32_t idesc,
                                               uint32_t acc0) {
  asm volatile(
      "{\n\t.reg .pred E, A, T;\n\t.reg .b64 b1, b2, b3;\n\t.reg .b32 a1, a2, a3;\n\t"
      "elect.sync _|E, 0xffffffff;\n\t"
      "setp.ne.b32 A, %4, 0;\n\tsetp.eq.b32 T, 0, 0;\n\t"
      "add.u32 a1, %1, 8;\n\tadd.u32 a2, %1, 16;\n\tadd.u32 a3, %1, 24;\n\t"
      "add.s64 b1, %2, 128;\n\tadd.s64 b2, %2, 256;\n\tadd.s64 b3, %2, 384;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, A;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, T;\n\t}" ::"r"(d),
      "r"(ta), "l"(b), "r"(idesc), "r"(acc0)
      : "memory");
}

// 8 SS MMAs, both operands MN-major with K steps (16 rows) 2048 B apart.
__device__ __forceinline__ void mma_ss_run8_mn(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                               uint32_t acc0) {
  asm volatile(
      "{\n\t.reg .pred E, A, T;\n\t.reg .b64 a1, a2, a3, a4, a5, a6, a7, b1, b2, b3, b4, b5, b6, b7;\n\t"
      "elect.sync _|E, 0xffffffff;\n\t"
      "setp.ne.b32 A, %4, 0;\n\tsetp.eq.b32 T, 0, 0;\n\t"
      "add.s64 a1, %1, 128;\n\tadd.s64 a2, %1, 256;\n\tadd.s64 a3, %1, 384;\n\tadd.s64 a4, %1, 512;\n\t"
      "add.s64 a5, %1, 640;\n\tadd.s64 a6, %1, 768;\n\tadd.s64 a7, %1, 896;\n\t"
      "add.s64 b1, %2, 128;\n\tadd.s64 b2, %2, 256;\n\tadd.s64 b3, %2, 384;\n\tadd.s64 b4, %2, 512;\n\t"
      "add.s64 b5, %2, 640;\n\tadd.s64 b6, %2, 768;\n\tadd.s64 b7, %2, 896;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, A;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a4, b4, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a5, b5, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a6, b6, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a7, b7, %3, T;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc0)
      : "memory");
}

// 4 TS MMAs: A in tensor memory at ta + 8 k; B a K-major 128-byte-swizzled
// tile whose K steps sit 32 B apart (desc + 2 k).
__device__ __forceinline__ void mma_ts_run4_kmajor(uint32_t d, uint32_t ta, uint64_t b,
                                                   uint32_t idesc, uint32_t acc0) {
  asm volatile(
      "{\n\t.reg .pred E, A, T;\n\t.reg .b64 b1, b2, b3;\n\t.reg .b32 a1, a2, a3;\n\t"
      "elect.sync _|E, 0xffffffff;\n\t"
      "setp.ne.b32 A, %4, 0;\n\tsetp.eq.b32 T, 0, 0;\n\t"
      "add.u32 a1, %1, 8;\n\tadd.u32 a2, %1, 16;\n\tadd.u32 a3, %1, 24;\n\t"
      "add.s64 b1, %2, 2;\n\tadd.s64 b2, %2, 4;\n\tadd.s64 b3, %2, 6;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, A;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, T;\n\t}" ::"r"(d),
      "r"(ta), "l"(b), "r"(idesc), "r"(acc0)
      : "memory");
}

// 4 SS MMAs with K steps `as` and `bs` apart in the A and B descriptors.
__device__ __forceinline__ void mma_ss_run4(uint32_t d, uint64_t a, uint64_t b, uint64_t as,
                                            uint64_t bs, uint32_t idesc, uint32_t acc0) {
  asm volatile(
      "{\n\t.reg .pred E, A, T;\n\t.reg .b64 a1, a2, a3, b1, b2, b3;\n\t"
      "elect.sync _|E, 0xffffffff;\n\t"
      "setp.ne.b32 A, %4, 0;\n\tsetp.eq.b32 T, 0, 0;\n\t"
      "add.s64 a1, %1, %5;\n\tadd.s64 a2, a1, %5;\n\tadd.s64 a3, a2, %5;\n\t"
      "add.s64 b1, %2, %6;\n\tadd.s64 b2, b1, %6;\n\tadd.s64 b3, b2, %6;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, A;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %3, T;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %3, T;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc0), "l"(as), "l"(bs)
      : "memory");
}

// Two SS MMAs over successive K=16 slices (steps as / bs), issued by one
// elected lane; acc0 = 0 starts the accumulator with the first.
__device__ __forceinline__ void mma_ss_run2(uint32_t d, uint64_t a, uint64_t b, uint64_t as,
                                            uint64_t bs, uint32_t idesc, uint32_t acc0) {
  asm volatile(
      "{\n\t.reg .pred E, A, T;\n\t.reg .b64 a1, b1;\n\t"
      "elect.sync _|E, 0xffffffff;\n\t"
      "setp.ne.b32 A, %4, 0;\n\tsetp.eq.b32 T, 0, 0;\n\t"
      "add.s64 a1, %1, %5;\n\tadd.s64 b1, %2, %6;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, A;\n\t"
      "@E tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, T;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc0), "l"(as), "l"(bs)
      : "memory");
}

// One commit by an elected lane of a converged warp (no branch).
__device__ __forceinline__ void mma_commit_elect(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .pred E;\n\telect.sync _|E, 0xffffffff;\n\t"
      "@E tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
          smem_u32(bar))
      : "memory");
}

// The mbarrier receives one arrival once every prior tcgen05 op of this thread completes.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle (layout type 2), version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// The same for the 64-byte swizzled layout (CU_TENSOR_MAP_SWIZZLE_64B): rows
// of 32 16-bit elements (64 B), 8-row atoms of 512 B (SBO = 512 for a K-major
// tile), tile bases 512-B aligned; successive K=16 slices start 32 B apart.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (4ull << 61);
}

// Instruction descriptor of kind::f16 with an FP32 accumulator.
// bf16 selects BF16 operands (else FP16); a_mn / b_mn mark MN-major operands.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16, bool a_mn, bool b_mn) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

}  // namespace tc
}  // namespace xk
