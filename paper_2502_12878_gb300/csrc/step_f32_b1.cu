// Step kernels of the FP32 inner sweep (Eq. 6) with register budget 1 (at least
// 1 resident block of 256 threads per SM), all stencil sizes.
#include "step.cuh"

namespace rbffd {

StepFn pick_step_f32_b1(int n, bool persistent) {
    return pick_step_m<MODE_INNER32, 1>(n, persistent);
}

}  // namespace rbffd
