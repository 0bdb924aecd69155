// Mixed-precision (split-BF16x3 on tcgen05 tensor cores) path of the
// exchange build: tables held in FP32 / BF16 pairs, FP32 accumulation in
// tensor memory, FP64 cross-tile sums, FP64 K assembly and E_x.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace xk {

struct MixedState;

// Optional callback marking the start (begin = 1) and end (begin = 0) of a
// build step (the XK_STEP_* numbering of xk.h) on the build's stream.
struct StepHook {
  void (*fn)(void* ctx, int step, int begin);
  void* ctx;
  void operator()(int step, int begin) const {
    if (fn) fn(ctx, step, begin);
  }
};

// Device bytes of the mixed-precision tables and scratch for a state that
// holds the rows of Naux of the NaT interpolation points (Naux = NaT unsharded).
size_t mixed_footprint(int64_t Ng, int N, int n, int Naux, int NaT);

// Convert and upload the per-geometry tables: FP64 phi (Ng x N), idx (all NaT
// interpolation points, host memory), and the rows [g0, g1) of V (g1 - g0 rows
// of Ng) and of W (g1 - g0 rows of NaT), in host or device memory (copies use
// cudaMemcpyDefault).  g0 = 0, g1 = NaT is the whole cell; a slice makes the
// builds return that slice's share of K and E_x (the sum over g splits).
cudaError_t mixed_create(int64_t Ng, int N, int n, int NaT, int g0, int g1, const double* phi,
                         const int32_t* idx, const double* V, const double* W, double dV,
                         cudaStream_t s, MixedState** out);
void mixed_destroy(MixedState* m);

// Enqueue one build: C_dev (N x n FP64) -> K_dev (N x n FP64), Ex_dev.
cudaError_t mixed_enqueue(MixedState* m, const double* C_dev, double* K_dev, double* Ex_dev,
                          cudaStream_t s, const StepHook& hook);

// The same build in three parts: orbitals (step 1), the pair contractions
// (steps 2-3), and the line contractions with K and E_x (steps 4-5).
cudaError_t mixed_enqueue_pre(MixedState* m, const double* C_dev, cudaStream_t s,
                              const StepHook& hook);
cudaError_t mixed_enqueue_pair(MixedState* m, cudaStream_t s, const StepHook& hook);
cudaError_t mixed_enqueue_post(MixedState* m, double* K_dev, double* Ex_dev, cudaStream_t s,
                               const StepHook& hook);

// E_x alone (no K): the orbitals, then the pair products S with the sums
// sum V' o S^2 and sum W' o S^2 only (no second product, no line
// contractions), then E_x from the closed form.  Uses the same split and
// summation order as mixed_enqueue, so for n <= 128 the two give the same E_x.
cudaError_t mixed_enqueue_energy(MixedState* m, const double* C_dev, double* Ex_dev,
                                 cudaStream_t s, const StepHook& hook);

// Full exchange matrix K_{mu nu} (N x N, FP64) of Eq. rpsEx with the three
// terms of Eq. rps: T = V o P and W o Q stored as hi/lo FP16, then
// M_A = T_A Phi, M_C = T_C Phi_g, Y = Phi_g^T M_A, Z = Phi_g^T (M_A - M_C) on
// the tensor cores and K = dV (Z + Y^T) in FP64.  mixed_full_prepare
// allocates the extra scratch (mixed_full_footprint bytes) once per state.
size_t mixed_full_footprint(int64_t Ng, int N, int n, int Naux);
cudaError_t mixed_full_prepare(MixedState* m);
cudaError_t mixed_enqueue_full(MixedState* m, const double* C_dev, double* Kfull_dev,
                               cudaStream_t s, const StepHook& hook);

// Pair contractions of several handles as one grouped launch per piece width
// (64 or 128 columns): the roles of every n <= 128 member, longest first, in
// launches of up to 16 roles; members with n > 128 run their own pair step.
struct PairGroup;
cudaError_t mixed_group_create(MixedState* const* ms, int count, PairGroup** out);
cudaError_t mixed_group_enqueue_pair(PairGroup* g, cudaStream_t s);
void mixed_group_destroy(PairGroup* g);

// Device word (4 ints) the kernels record their error codes in; the first is
// the code.  Callers snapshot and clear it on the build's stream.
int* mixed_status_ptr(MixedState* m);

// Bound, in SM clock cycles, on every pipeline wait inside the state's kernels
// (0 restores the default of about one second); waits for a kernel's own
// copies and MMAs before it exits keep the default.  Applies to launches
// enqueued afterwards.
void mixed_set_wait_limit(MixedState* m, long long cycles);

// The set-up autotuner's choices: info[0] = width of the n > 128
// back-contraction tiles (128 or 256, 0 otherwise), info[1] = the K split of
// M2 (role A for n <= 64); ms[0], ms[1] = timing of the 128- and 256-column
// shapes at set-up (0 when not timed), ms[2] = the tuned pair launch (n <= 64).
void mixed_autotune_info(const MixedState* m, int* info, double* ms);


}  // namespace xk
