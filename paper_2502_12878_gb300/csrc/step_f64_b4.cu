// Step kernels of the FP64 sweep (Eq. 6) with register budget 4 (at least
// 4 resident blocks of 256 threads per SM), all stencil sizes.
#include "step.cuh"

namespace rbffd {

StepFn pick_step_f64_b4(int n, bool persistent) {
    return pick_step_m<MODE_SWEEP64, 4>(n, persistent);
}

}  // namespace rbffd
