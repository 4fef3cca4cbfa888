// Step kernels of the FP32 inner sweep (Eq. 6) with register budget 4 (at least
// 4 resident blocks of 256 threads per SM), all stencil sizes.
#include "step.cuh"

namespace rbffd {

StepFn pick_step_f32_b4(int n, bool persistent) {
    return pick_step_m<MODE_INNER32, 4>(n, persistent);
}

}  // namespace rbffd
