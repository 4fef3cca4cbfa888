// Split persistent launch: the kernel instantiations for every compiled
// stencil size (the kernel itself is in step_split.cuh), 512- and 1024-thread
// blocks (the generic size and n = 6: 512 only), and the shared-memory size of
// a launch.
#include "step_split.cuh"

namespace rbffd {

template <int MODE, int TH>
static StepFn pick_split_m(int n) {
#define RBFFD_SCASE(NN) \
    case NN: return split_kernel<NN, MODE, TH>;
    if constexpr (TH == RES_THREADS_WIDE) {
        switch (n) {
            RBFFD_SCASE(12)
            RBFFD_SCASE(13)
            RBFFD_SCASE(16)
            RBFFD_SCASE(20)
            RBFFD_SCASE(24)
            RBFFD_SCASE(30)
            RBFFD_SCASE(31)
            RBFFD_SCASE(40)
            RBFFD_SCASE(48)
            RBFFD_SCASE(56)
            RBFFD_SCASE(57)
            RBFFD_SCASE(70)
            RBFFD_SCASE(71)
            default: return nullptr;
        }
    } else {
    switch (n) {
        RBFFD_SCASE(6)
        RBFFD_SCASE(12)
        RBFFD_SCASE(13)
        RBFFD_SCASE(16)
        RBFFD_SCASE(20)
        RBFFD_SCASE(24)
        RBFFD_SCASE(30)
        RBFFD_SCASE(31)
        RBFFD_SCASE(40)
        RBFFD_SCASE(48)
        RBFFD_SCASE(56)
        RBFFD_SCASE(57)
        RBFFD_SCASE(70)
        RBFFD_SCASE(71)
        default: return split_kernel<0, MODE, TH>;
    }
    }
#undef RBFFD_SCASE
}

StepFn pick_split(int mode, int n, int threads) {
    if (threads == RES_THREADS_WIDE)
        return mode == MODE_SWEEP64 ? pick_split_m<MODE_SWEEP64, RES_THREADS_WIDE>(n)
                                    : pick_split_m<MODE_INNER32, RES_THREADS_WIDE>(n);
    return mode == MODE_SWEEP64 ? pick_split_m<MODE_SWEEP64, RES_THREADS_HOST>(n)
                                : pick_split_m<MODE_INNER32, RES_THREADS_HOST>(n);
}

unsigned split_smem(int64_t nslices, int mode, int grid) {
    const int64_t nsl = (nslices + grid - 1) / grid;
    return split_smem_bytes(nsl, mode == MODE_SWEEP64 ? 8 : 4);
}

}  // namespace rbffd
