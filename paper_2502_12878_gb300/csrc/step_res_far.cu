// Resident persistent launch with far lists: every gather from shared memory
// (the kernel is resident_kernel<..., FAR = true> in step_res.cuh).  512-thread
// blocks for every compiled stencil size, 1024-thread blocks for n <= 31.
#include "step_res.cuh"

namespace rbffd {

template <int MODE>
static StepFn pick_far_512(int n) {
#define RBFFD_FCASE(NN) \
    case NN: return resident_kernel<NN, MODE, false, RES_THREADS_HOST, true>;
    switch (n) {
        RBFFD_FCASE(6)
        RBFFD_FCASE(12)
        RBFFD_FCASE(13)
        RBFFD_FCASE(16)
        RBFFD_FCASE(20)
        RBFFD_FCASE(24)
        RBFFD_FCASE(30)
        RBFFD_FCASE(31)
        RBFFD_FCASE(40)
        RBFFD_FCASE(48)
        RBFFD_FCASE(56)
        RBFFD_FCASE(57)
        RBFFD_FCASE(70)
        RBFFD_FCASE(71)
        default: return resident_kernel<0, MODE, false, RES_THREADS_HOST, true>;
    }
#undef RBFFD_FCASE
}

template <int MODE>
static StepFn pick_far_1024(int n) {
#define RBFFD_FCASE(NN) \
    case NN: return resident_kernel<NN, MODE, false, RES_THREADS_WIDE, true>;
    switch (n) {
        RBFFD_FCASE(12)
        RBFFD_FCASE(13)
        RBFFD_FCASE(16)
        RBFFD_FCASE(20)
        RBFFD_FCASE(24)
        RBFFD_FCASE(30)
        RBFFD_FCASE(31)
        default: return nullptr;
    }
#undef RBFFD_FCASE
}

StepFn pick_resident_far(int mode, int n, int threads) {
    if (threads == RES_THREADS_WIDE)
        return mode == MODE_SWEEP64 ? pick_far_1024<MODE_SWEEP64>(n)
                                    : pick_far_1024<MODE_INNER32>(n);
    return mode == MODE_SWEEP64 ? pick_far_512<MODE_SWEEP64>(n) : pick_far_512<MODE_INNER32>(n);
}

}  // namespace rbffd
