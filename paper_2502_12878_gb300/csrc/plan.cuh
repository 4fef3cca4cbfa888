// Internal layout of an rbffd_plan: the node permutation and the packed
// (sliced-ELL) stencils that the explicit sweep streams, plus the device
// control block shared by the step kernels.
#pragma once

#include "common.cuh"

namespace rbffd {

static constexpr int SLICE = 32;   // rows per slice = one warp
static constexpr int GRAPH_LOG2 = 5;   // the longest captured graph: 32 step launches

// Device control block of a step loop.  Step kernels read their parameters
// here (so a captured graph can be replayed with new ones); the stop decision
// of each step is taken one step later (graph launches: at the start of the
// next step's kernels; persistent launches: after the next step's rows) and
// a run that stops records its outcome here.
struct StepCtrl {
    unsigned long long res[3];   // per-step max |r| as IEEE bits (r >= 0 orders as uint64)
    unsigned long long steps;    // graph launches: steps completed (block 0 of each adds 1)
    // persistent launches: block arrivals at step ends since the run started
    unsigned long long arrivals;
    unsigned long long pad1;
    long long k;                 // steps taken so far
    long long max_steps;
    int done;                    // 0 running, 1 converged, 2 cap, 3 non-finite, 4 diverged, 5 timeout
    int held;                    // persistent barrier: arrivals it waits for beyond the grid's
    long long spin_limit;        // persistent barrier: clock cycles a wait may last
    double dt;
    double tol;
    double res_first;            // R_0 of this run (divergence test)
    double res_last;             // R of the last step taken
};

enum : int { DONE_RUNNING = 0, DONE_CONVERGED = 1, DONE_CAP = 2, DONE_NONFINITE = 3,
             DONE_DIVERGED = 4, DONE_TIMEOUT = 5 };

struct Transpose;
void free_transpose(rbffd_plan* p);   // adjoint.cu

// stable split of ids 0..N-1 by key != 0 (key 0 first, each group ascending)
int split_by_flag(const int32_t* key, int64_t N, int32_t* out, int32_t* pos, int64_t* tmp,
                  cudaStream_t s);

}  // namespace rbffd

struct rbffd_plan {
    int d = 2;
    int64_t N = 0, NI = 0;
    int n = 0;
    int flags = 0;
    int64_t nslices = 0;
    int32_t* perm = nullptr;        // [N] slot -> original node
    int32_t* inv = nullptr;         // [N] original node -> slot
    int32_t* row_of_slot = nullptr; // [NI] slot -> row of the caller's interior list
    double* w64 = nullptr;          // [nslices][n][32]
    float* w32 = nullptr;           // [nslices][n][32]
    int32_t* col = nullptr;         // [nslices][n][32] neighbour slots
    // compact neighbour indices: per slice up to four window bases (int4,
    // x = -1 marks a slice that keeps the int32 form) and per entry a 16-bit
    // code, window k in bits 15..14 and the offset from that base in 13..0
    uint16_t* col16 = nullptr;      // [nslices][n][32] (NULL with RBFFD_PACK_IDX32)
    int4* sbase = nullptr;          // [nslices]
    int64_t rows16 = 0;             // interior rows in compact slices
    double* u[2] = {nullptr, nullptr};   // iterates in slot order [N]
    double* fs = nullptr;           // f in slot order [NI]
    float* e[2] = {nullptr, nullptr};    // DC correction [N]
    float* d32 = nullptr;           // DC defect [NI]
    double* scratch = nullptr;      // [2 * NI + 1024] reductions, power iteration
    rbffd::StepCtrl* ctrl = nullptr;
    int64_t dc_K_in = 20000;
    double dc_rho_in = 1e-3;
    // CUDA graphs of step launches, per mode (0 FP64 sweep, 1 FP32 inner
    // sweep) and length 2^b, b = 0..GRAPH_LOG2; built on first use
    void* graphs[2][6] = {};
    // persistent barrier: how long a wait may last, and (to test that path)
    // arrivals withheld from every step's barrier
    long long spin_limit = 0;
    int held_arrivals = 0;
    int grid_steps = 0;             // blocks per SM of auxiliary sweeps (defect, power)
    // tuned launch shape per mode (0 FP64 sweep, 1 FP32 inner sweep)
    bool tuned[2] = {false, false};
    bool persist[2] = {false, false};   // the step loop of each mode runs persistent
    bool resident[2] = {false, false};  // ... as the resident launch (planes in shared memory)
    bool pdl[2] = {false, false};       // graph-mode steps as programmatic dependent launches
    unsigned res_smem[2] = {0, 0};      // its dynamic shared memory per block
    int res_threads[2] = {512, 512};    // and its block size
    bool res_far[2] = {false, false};   // ... with far lists (every gather in shared memory)
    bool split[2] = {false, false};     // ... as the split launch (stencils streamed, own rows
                                        // in shared memory; res_smem / res_threads its shape)
    bool inner_first = false;           // each SM's share ordered with its inner rows first
    int32_t* inner_sl = nullptr;        // [SMs] its leading slices of inner rows only
    // far-list data per mode (built when the tuner first considers it): the
    // window reach it was built for, the most far slots of a block, the
    // entries' local indices, each block's far slots
    bool fl_built[2] = {false, false};
    bool fl_ok[2] = {false, false};
    int64_t fl_halo[2] = {0, 0};
    int64_t fl_max[2] = {0, 0};
    uint16_t* fl_idx[2] = {nullptr, nullptr};
    int32_t* fl_off[2] = {nullptr, nullptr};
    int32_t* fl_slot[2] = {nullptr, nullptr};
    int64_t res_halo[2] = {0, 0};       // and its halo reach (slots beyond a block's rows)
    int64_t res_halo_set = -2;          // a reach fixed by rbffd_plan_set_resident_halo (-2: tuned)
    int res_threads_set = 0;            // block size fixed by rbffd_plan_set_block (0: tuned)
    int minb[2] = {2, 2};
    int per_sm[2] = {2, 2};
    float tune_ms[2] = {0.f, 0.f};
    // timing of the last step loop (CUDA events on the caller's stream around
    // the step launches) and the number of kernels the last solve launched
    void* ev[2] = {nullptr, nullptr};
    double last_loop_ms = 0.0;
    long long last_loop_steps = 0;
    long long last_launches = 0;
    rbffd::Transpose* tr = nullptr;
    // Neumann boundary nodes (mixed-boundary variant): slots, supports (slots),
    // normal-derivative weights, data, scratch for the new values
    int64_t NN = 0;
    int nn = 0;
    int32_t* nslot = nullptr;
    int32_t* ncol = nullptr;
    double* nw = nullptr;
    double* ng = nullptr;
    double* ng0 = nullptr;          // zeros (homogeneous data, for the power iteration)
    double* uN = nullptr;
};
