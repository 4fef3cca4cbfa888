// Resident persistent launch, 512-thread blocks: the kernel instantiations
// for every compiled stencil size (the kernel itself is in step_res.cuh), and
// the shared-memory size of a launch.
#include "step_res.cuh"

namespace rbffd {

// the resident kernel for stencil size n (a specialisation for the sizes of
// the monomial orders in 2D and 3D, else the generic one)
template <int MODE, bool I16>
static StepFn pick_res_m(int n) {
#define RBFFD_RCASE(NN) \
    case NN: return resident_kernel<NN, MODE, I16, RES_THREADS_HOST>;
    switch (n) {
        RBFFD_RCASE(6)
        RBFFD_RCASE(12)
        RBFFD_RCASE(13)
        RBFFD_RCASE(16)
        RBFFD_RCASE(20)
        RBFFD_RCASE(24)
        RBFFD_RCASE(30)
        RBFFD_RCASE(31)
        RBFFD_RCASE(40)
        RBFFD_RCASE(48)
        RBFFD_RCASE(56)
        RBFFD_RCASE(57)
        RBFFD_RCASE(70)
        RBFFD_RCASE(71)
        default: return resident_kernel<0, MODE, I16, RES_THREADS_HOST>;
    }
#undef RBFFD_RCASE
}

StepFn pick_resident(int mode, int n, bool i16) {
    if (mode == MODE_SWEEP64) return i16 ? pick_res_m<MODE_SWEEP64, true>(n)
                                         : pick_res_m<MODE_SWEEP64, false>(n);
    return i16 ? pick_res_m<MODE_INNER32, true>(n) : pick_res_m<MODE_INNER32, false>(n);
}

// dynamic shared memory of a resident launch of `grid` blocks (the largest
// block's share of the slices, its halo window reaching `halo` slots beyond
// its rows; halo < 0: the planes alone)
unsigned resident_smem(int64_t nslices, int n, int mode, bool i16, int grid, int64_t halo,
                       int64_t extra) {
    const int64_t nsl = (nslices + grid - 1) / grid;
    return res_layout(nsl, n, mode == MODE_SWEEP64 ? 8 : 4, i16 ? 2 : 4, halo, extra).total;
}

}  // namespace rbffd
