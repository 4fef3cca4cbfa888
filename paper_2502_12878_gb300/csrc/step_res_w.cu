// Resident persistent launch, 1024-thread blocks, for the stencil sizes whose
// kernel fits 64 registers a thread (n <= 31): twice the warps per SM, so a
// block sweeps its share of up to 32 slices in one round.  The tuner times
// both block sizes.
#include "step_res.cuh"

namespace rbffd {

template <int MODE, bool I16>
static StepFn pick_res_w(int n) {
#define RBFFD_WCASE(NN) \
    case NN: return resident_kernel<NN, MODE, I16, RES_THREADS_WIDE>;
    switch (n) {
        RBFFD_WCASE(12)
        RBFFD_WCASE(13)
        RBFFD_WCASE(16)
        RBFFD_WCASE(20)
        RBFFD_WCASE(24)
        RBFFD_WCASE(30)
        RBFFD_WCASE(31)
        default: return nullptr;
    }
#undef RBFFD_WCASE
}

StepFn pick_resident_wide(int mode, int n, bool i16) {
    if (mode == MODE_SWEEP64) return i16 ? pick_res_w<MODE_SWEEP64, true>(n)
                                         : pick_res_w<MODE_SWEEP64, false>(n);
    return i16 ? pick_res_w<MODE_INNER32, true>(n) : pick_res_w<MODE_INNER32, false>(n);
}

}  // namespace rbffd
