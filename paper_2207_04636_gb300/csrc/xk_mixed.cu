// Mixed-precision path: not yet built in this revision; setup refuses the mode.
#include "xk_internal.h"
#include "xk_mixed.h"

namespace xk {

struct MixedState {};

size_t mixed_footprint(int64_t, int, int, int) { return 0; }

cudaError_t mixed_create(int64_t, int, int, int, const double*, const int32_t*, const double*,
                         const double*, double, cudaStream_t, MixedState**) {
  return cudaErrorNotSupported;
}

void mixed_destroy(MixedState* m) { delete m; }

cudaError_t mixed_enqueue(MixedState*, const double*, double*, double*, cudaStream_t,
                          const StepHook&) {
  return cudaErrorNotSupported;
}

double mixed_error_bound(const MixedState*) { return 0.0; }

}  // namespace xk
