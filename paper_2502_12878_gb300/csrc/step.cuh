// Step kernels of the explicit sweep (Eq. 6): one pass over the packed rows,
// u <- u + dt (L u - f) in FP64 (MODE_SWEEP64) or the FP32 correction sweep
// e <- e + dt32 (L e + d) of defect correction (MODE_INNER32), with the
// residual max-norm and the stop decision on the device.
//
// The kernel templates live here so that their instantiations can be spread
// over several translation units (step_f64_b*.cu, step_f32_b*.cu: one per
// arithmetic and register budget) that compile in parallel; each of those
// exports one pick function, and sweep.cu, which drives the step loop,
// dispatches through them.
#pragma once

#include "plan.cuh"

namespace rbffd {

static constexpr int STEP_THREADS = 256;
static constexpr long long SPIN_LIMIT_CYCLES = 4000000000LL;   // default: ~2 s at 2 GHz

// ------------------------------------------------------------- utilities
__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double bitsd(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// block max of a non-negative value (NaN mapped to +Inf by the caller);
// valid in thread 0
__device__ __forceinline__ double block_max(double v) {
    __shared__ double wm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wm[wid] = v;
    __syncthreads();
    double m = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wm[w]);
    __syncthreads();
    return m;
}

// ---------------------------------------------------------- row kernels
// Streaming loads of the stencil planes (read once per step: evict-first).
// Ordered asm: the compiler keeps them in program order, so the phases of
// row_dot below really put 2*CH loads in flight before the first use.
__device__ __forceinline__ double ld_stream(const double* p) {
    double v;
    asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm volatile("ld.global.cs.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.cs.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint16_t* p) {
    unsigned short v;
    asm volatile("ld.global.cs.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint32_t)v;
}
// Gather of the iterate.  Within one launch per step the iterate is
// read-only, so the non-coherent path (L1) is used; a persistent launch
// rewrites it between steps from other SMs, so it reads through L2 (.cg).
template <bool COHERENT>
__device__ __forceinline__ double ld_iter(const double* p) {
    double v;
    if (COHERENT) asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    else asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
template <bool COHERENT>
__device__ __forceinline__ float ld_iter(const float* p) {
    float v;
    if (COHERENT) asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    else asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// compact index: window k = code >> 14 selects one of the slice's four bases
// (three selects on the integer pipe), plus the 14-bit offset
__device__ __forceinline__ int32_t decode16(uint32_t v, const int4& b) {
    const uint32_t k = v >> 14;
    const int32_t base = (k & 2u) ? ((k & 1u) ? b.w : b.z) : ((k & 1u) ? b.y : b.x);
    return base + (int32_t)(v & 0x3fffu);
}

// sum_j w_j u[col_j] as an fma chain from 0, j ascending.  Loads are issued
// in phases of CH (indices, weights, then the gathers) so each thread keeps
// 2*CH streaming loads and CH gathers in flight.  I16: the indices come as
// 16-bit codes against the slice's bases `sb` (same columns, fewer bytes).
template <int NN, bool COH, bool I16, class T>
__device__ __forceinline__ T row_dot(const T* __restrict__ w, const void* __restrict__ colp,
                                     const int4& sb, const T* __restrict__ u, int n) {
    constexpr int CH = 16;
    T acc = T(0);
    const int nn = NN > 0 ? NN : n;
#pragma unroll
    for (int j0 = 0; j0 < (NN > 0 ? NN : 1 << 30); j0 += CH) {
        if (NN == 0 && j0 >= nn) break;
        int32_t c[CH];
        T wv[CH], uv[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (I16)
                    c[t] = (int32_t)ld_stream((const uint16_t*)colp + (j0 + t) * SLICE);
                else
                    c[t] = ld_stream((const int32_t*)colp + (j0 + t) * SLICE);
            }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) wv[t] = ld_stream(w + (j0 + t) * SLICE);
        if constexpr (I16) {
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < nn) c[t] = decode16((uint32_t)c[t], sb);
        }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) uv[t] = ld_iter<COH>(u + c[t]);
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (sizeof(T) == 8) acc = __fma_rn(wv[t], uv[t], acc);
                else acc = __fmaf_rn(wv[t], uv[t], acc);
            }
    }
    return acc;
}

// |x| as IEEE bits, NaN mapped to +Inf: integer ops only (keeps the FP64
// pipe for the multiply-adds)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : b;
}
__device__ __forceinline__ unsigned long long abs_bits(float x) {
    return abs_bits((double)x);
}

template <int NN, bool COH = false>
__device__ __forceinline__ double row_dot64(const double* __restrict__ w,
                                            const int32_t* __restrict__ col,
                                            const double* __restrict__ u, int n) {
    const int4 none = make_int4(0, 0, 0, 0);
    return row_dot<NN, COH, false, double>(w, col, none, u, n);
}

enum : int { MODE_SWEEP64 = 0, MODE_INNER32 = 1 };

struct StepArgs {
    const double* w64;
    const float* w32;
    const int32_t* col;
    const uint16_t* col16;   // compact codes, NULL when the plan keeps int32 only
    const int4* sbase;       // [nslices] window bases; x < 0: the slice uses col
    const double* f;      // FP64 sweep: f in slot order
    float* d32;           // FP32 inner: defect in slot order
    double* u0;
    double* u1;
    float* e0;
    float* e1;
    int64_t NI;
    int64_t nslices;
    int n;
    int spread;   // 1: consecutive slices go to different blocks (small plans)
    int64_t N;    // slots (the iterate's length)
    int64_t halo; // resident launch: slots staged beyond a block's rows on either side
    int pdl;      // graph launch with programmatic serialization: prefetch before the wait
    // resident launch with far lists: per block the sorted slots its rows
    // read outside its window (staged every step behind the window), and for
    // every stencil entry its position in the window + far values
    const uint16_t* fl_idx;   // [nslices][n][32]
    const int32_t* fl_off;    // [blocks + 1]
    const int32_t* fl_slot;
    int64_t fl_max;           // most far slots of a block
    // split launch: per block (SM) the number of leading slices of its share
    // that are inner rows only (plans ordered inner rows first)
    const int32_t* inner;
};

// The warp's first slice.  Large plans give each block runs of consecutive
// slices (their gathers share the SM's L1); plans with fewer slices than the
// blocks' warps would then leave SMs idle while others run several warps'
// FP64 chains, so there consecutive slices go to different blocks.
__device__ __forceinline__ int64_t step_warp(const StepArgs& A) {
    return A.spread ? (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x
                    : (int64_t)blockIdx.x * (STEP_THREADS / 32) + (threadIdx.x >> 5);
}

// Bulk prefetch into L2 (one lane) of the weight and index planes of slice
// sl, the warp's next one: the 16-bit code plane when the plan has one (the
// few slices that keep int32 indices then read theirs from HBM; choosing per
// slice would wait on the slice's window bases first, which measured 3 %
// slower).  Both planes start on 16-byte boundaries and their sizes (8n or 4n
// and 2n or 4n bytes per row, 32 rows) are multiples of 16.  Measured at 1M
// rows: +13 % for the FP32 sweep (HBM-latency bound); two or three slices
// ahead gain nothing.  The FP64 sweep prefetches only for n <= PF64_MAX_N:
// +3.5 % at n = 12, +1.6 % at n = 13, nothing at 16, and 3-19 % lost from
// n = 20 on, where the FP64 pipe binds.
static constexpr int PF64_MAX_N = 13;

template <int MODE>
__device__ __forceinline__ void prefetch_planes(const StepArgs& A, int64_t sl) {
    if (sl >= A.nslices) return;
    const int64_t nb = sl * (int64_t)A.n * SLICE;
    const unsigned plane = (unsigned)(A.n * SLICE);
    if (MODE == MODE_INNER32)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A.w32 + nb),
                     "r"(plane * 4u) : "memory");
    else
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A.w64 + nb),
                     "r"(plane * 8u) : "memory");
    if (A.col16)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A.col16 + nb),
                     "r"(plane * 2u) : "memory");
    else
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A.col + nb),
                     "r"(plane * 4u) : "memory");
}

// one step over the slices owned by this warp (slice0, slice0 + stride, ...);
// returns this thread's max |r| with NaN -> +Inf
template <int NN, int MODE, bool COH>
__device__ __forceinline__ unsigned long long step_rows(const StepArgs& A, int par, double dt,
                                                        float dt32, int64_t slice0,
                                                        int64_t stride) {
    const int lane = threadIdx.x & 31;
    unsigned long long m = 0;
    for (int64_t sl = slice0; sl < A.nslices; sl += stride) {
        const int64_t row = sl * SLICE + lane;
        const int64_t base = sl * (int64_t)A.n * SLICE + lane;
        const int4 sb = A.col16 ? __ldg(A.sbase + sl) : make_int4(-1, -1, -1, -1);
        if ((MODE == MODE_INNER32 || (NN > 0 && NN <= PF64_MAX_N)) && lane == 0)
            prefetch_planes<MODE>(A, sl + stride);
        if (row < A.NI) {
            if (MODE == MODE_SWEEP64) {
                const double* uin = par ? A.u1 : A.u0;
                double* uout = par ? A.u0 : A.u1;
                // the row's own f and u are issued before the dot product, so
                // their latency overlaps the stencil loads
                const double fi = ld_stream(A.f + row);
                const double ui = ld_iter<COH>(uin + row);
                double acc;
                if (sb.x >= 0)
                    acc = row_dot<NN, COH, true, double>(A.w64 + base, A.col16 + base, sb, uin,
                                                         A.n);
                else
                    acc = row_dot<NN, COH, false, double>(A.w64 + base, A.col + base, sb, uin,
                                                          A.n);
                double r = __dsub_rn(acc, fi);
                uout[row] = __fma_rn(dt, r, ui);
                m = max(m, abs_bits(r));
            } else {
                const float* ein = par ? A.e1 : A.e0;
                float* eout = par ? A.e0 : A.e1;
                const float di = ld_stream(A.d32 + row);
                const float ei = ld_iter<COH>(ein + row);
                float acc;
                if (sb.x >= 0)
                    acc = row_dot<NN, COH, true, float>(A.w32 + base, A.col16 + base, sb, ein,
                                                        A.n);
                else
                    acc = row_dot<NN, COH, false, float>(A.w32 + base, A.col + base, sb, ein,
                                                         A.n);
                float rho = __fadd_rn(acc, di);
                eout[row] = __fmaf_rn(dt32, rho, ei);
                m = max(m, abs_bits(rho));
            }
        }
    }
    return m;
}

// block max of IEEE bits; valid in thread 0
__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v) {
    __shared__ unsigned long long wm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wm[wid] = v;
    __syncthreads();
    unsigned long long m = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    return m;
}

// the stop rule after step kk with residual R (R0: step 0's), the same in
// every launch mode: non-finite, below tol, grown 1e6-fold, or the cap
__device__ __forceinline__ int stop_rule(double R, double R0, long long kk, long long kmax,
                                         double tol) {
    if (!isfinite(R)) return DONE_NONFINITE;
    if (R < tol) return DONE_CONVERGED;
    if (kk > 0 && R0 > 0.0 && R > 1e6 * R0) return DONE_DIVERGED;
    if (kk + 1 >= kmax) return DONE_CAP;
    return DONE_RUNNING;
}

// Graph launches: the state at the start of a step's kernels, read by one
// thread after the previous kernel completed.  k = steps completed; the stop
// rule is applied here to step k - 1 (whose residual slot is complete at the
// kernel boundary), so a step's kernel ends without a last-block ticket.
// `record` (one block of the step kernel, and the finish kernel): on a stop
// write the outcome, at step 0 its residual, and clear the slot step k + 1
// will use (its last reader, step k's start, has completed).  Returns true
// when the kernel should run step k.
__device__ __forceinline__ bool graph_state(StepCtrl* c, bool record, long long* k_out) {
    volatile StepCtrl* vc = c;
    const long long k = (long long)vc->steps;
    *k_out = k;
    if (vc->done != DONE_RUNNING) return false;
    const long long kmax = vc->max_steps;
    if (k > 0) {
        const long long kk = k - 1;
        const double R = bitsd(vc->res[kk % 3]);
        const double R0 = kk == 0 ? R : vc->res_first;
        const int dn = stop_rule(R, R0, kk, kmax, vc->tol);
        if (record && kk == 0) vc->res_first = R;
        if (dn != DONE_RUNNING) {
            if (record) {
                vc->res_last = R;
                vc->k = k;
                vc->done = dn;
            }
            return false;
        }
    }
    if (k >= kmax) return false;
    if (record) vc->res[(k + 1) % 3] = 0ull;
    return true;
}

// release / acquire accesses at GPU scope (PTX memory model): a release
// orders every memory access that precedes it (cumulatively, including the
// block's other threads' writes ordered by the preceding __syncthreads), an
// acquire every access that follows it.  The step ends use them instead of
// full fences around relaxed atomics: measured 4-11 % less time per step on
// 10k-90k-node plans (graph and persistent launches), 0.9 % at 1M nodes.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_max_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// graph mode: one step per launch, one slice per warp
template <int NN, int MODE, int MINB>
__global__ void __launch_bounds__(STEP_THREADS, MINB) step_kernel(StepArgs A, StepCtrl* c) {
    __shared__ long long s_k;
    __shared__ int s_skip;
    __shared__ double s_dt;
    // programmatic dependent launch: the next step's blocks may be scheduled
    // now (they take SM slots as this step's blocks leave, so its launch
    // overlaps this step's tail); every block then waits here until the
    // previous step has completed and its writes are visible.  Both are no-ops
    // for a launch without the programmatic-serialization attribute.  Before
    // waiting, such a launch has one lane of each warp prefetch its first
    // slice's planes into L2 (stencils only: nothing the previous step writes).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (A.pdl && (threadIdx.x & 31) == 0) prefetch_planes<MODE>(A, step_warp(A));
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) {
        long long k;
        s_skip = !graph_state(c, blockIdx.x == 0, &k);
        s_k = k;
        s_dt = ((volatile StepCtrl*)c)->dt;
    }
    __syncthreads();
    if (s_skip) return;
    const long long k = s_k;
    const int par = (int)(k & 1);
    const int64_t warp = step_warp(A);
    unsigned long long m = step_rows<NN, MODE, false>(A, par, s_dt, (float)s_dt, warp,
                                                      (int64_t)gridDim.x * (STEP_THREADS / 32));
    m = block_max_bits(m);
    // the block's max and (block 0) the step count: fire-and-forget; the
    // next step's kernels see both through the kernel boundary
    if (threadIdx.x == 0) {
        red_max_relaxed(&c->res[k % 3], m);
        if (blockIdx.x == 0) red_add_relaxed(&c->steps, 1ull);
    }
}

// Step ends of the persistent launches: a counter barrier, with the stop
// decision one step behind.  At the end of step k each block adds its max |r|
// to the step's residual slot and its arrival to a counter (both fire-and-
// forget reductions; the arrival releases the block's iterate writes and its
// max), and waits until the counter shows every block's arrival (bounded by
// `spin` clock cycles; `held` arrivals are added to every target - 0 in every
// solve, except a test of the timeout path, where no barrier can complete).
// Right after the barrier thread 0 starts loading the step's full residual and
// the block computes step k + 1 meanwhile; at its end every block applies the
// stop rule to step k - the same rule to the same value in every block, so all
// stop together.  A stop wastes step k + 1, which writes the other buffer: the
// result, u^{k+1}, is untouched.  The barrier's critical path is one
// reduction and one poll, against the four round trips of a barrier whose last
// arrival decides and publishes.  Block 0 clears the slot that step k + 2 will
// use (every block read its previous contents before arriving here) and, when
// the run stops, writes the outcome to the control block.
__device__ __forceinline__ void red_add_release(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct LagState {
    unsigned long long pend;   // thread 0: the last barrier's step residual (bits)
    double R0;                 // thread 0: residual of step 0
    double tol;
    long long kmax;
};

// barrier at the end of step k (m: the block's max, valid in thread 0);
// false in every thread when the wait gave up (done = DONE_TIMEOUT)
__device__ __forceinline__ bool lag_barrier(StepCtrl* c, LagState& S, long long k, long long k0,
                                            unsigned long long m, long long spin, int held) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        red_max_relaxed(&c->res[k % 3], m);
        red_add_release(&c->arrivals, 1ull);
        const unsigned long long target =
            (unsigned long long)(k - k0 + 1) * gridDim.x + (unsigned long long)held;
        const long long t0 = clock64();
        int ok = 1;
        while (ld_acquire(&c->arrivals) < target)
            if (clock64() - t0 > spin) {
                atomicExch(&c->done, DONE_TIMEOUT);
                ok = 0;
                break;
            }
        if (ok) {
            if (blockIdx.x == 0) st_relaxed(&c->res[(k + 2) % 3], 0ull);
            S.pend = ld_relaxed(&c->res[k % 3]);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// the stop rule for step kk from its residual (loaded at its barrier), in
// every thread; block 0 records the outcome of a run that stops
__device__ __forceinline__ int lag_decide(StepCtrl* c, LagState& S, long long kk) {
    __shared__ int s_dn;
    if (threadIdx.x == 0) {
        const double R = bitsd(S.pend);
        if (kk == 0) S.R0 = R;
        const int dn = stop_rule(R, S.R0, kk, S.kmax, S.tol);
        if (dn != DONE_RUNNING && blockIdx.x == 0) {
            volatile StepCtrl* vc = c;
            vc->res_first = S.R0;
            vc->res_last = R;
            vc->k = kk + 1;
            vc->done = dn;
        }
        s_dn = dn;
    }
    __syncthreads();
    return s_dn;
}

// persistent mode: all steps in one cooperative launch
template <int NN, int MODE, int MINB>
__global__ void __launch_bounds__(STEP_THREADS, MINB) persistent_kernel(StepArgs A, StepCtrl* c) {
    __shared__ long long s_k, s_max, s_spin;
    __shared__ int s_held;
    __shared__ double s_dt;
    LagState S;
    if (threadIdx.x == 0) {
        volatile StepCtrl* vc = c;
        s_k = vc->k;
        s_max = vc->max_steps;
        s_dt = vc->dt;
        constexpr long long dflt = SPIN_LIMIT_CYCLES;
        const long long lim = vc->spin_limit;
        s_spin = lim > 0 ? lim : dflt;
        s_held = vc->held;
        S.R0 = vc->res_first;
        S.tol = vc->tol;
        S.kmax = vc->max_steps;
        S.pend = 0ull;
    }
    __syncthreads();
    const double dt = s_dt;
    const long long kmax = s_max, k0 = s_k, spin = s_spin;
    const int held = s_held;
    const int64_t warp = step_warp(A);
    const int64_t nw = (int64_t)gridDim.x * (STEP_THREADS / 32);
    for (long long k = k0; k < kmax; ++k) {
        unsigned long long m = step_rows<NN, MODE, true>(A, (int)(k & 1), dt, (float)dt, warp, nw);
        // the decision of step k - 1 (its residual loaded at its barrier)
        if (k > k0 && lag_decide(c, S, k - 1) != DONE_RUNNING) return;
        m = block_max_bits(m);
        if (!lag_barrier(c, S, k, k0, m, spin, held)) return;
    }
    if (kmax > k0) lag_decide(c, S, kmax - 1);   // the last step's: it stops the run
}

// ------------------------------------------------------ dispatch by n
typedef void (*StepFn)(StepArgs, StepCtrl*);

// kernel for stencil size n: a specialisation with n fixed at compile time
// for the sizes of the monomial orders used in 2D and 3D, else the generic one
template <int MODE, int MINB>
static StepFn pick_step_m(int n, bool persistent) {
#define RBFFD_CASE(NN) \
    case NN: return persistent ? persistent_kernel<NN, MODE, MINB> : step_kernel<NN, MODE, MINB>;
    switch (n) {
        RBFFD_CASE(6)
        RBFFD_CASE(12)
        RBFFD_CASE(13)
        RBFFD_CASE(16)
        RBFFD_CASE(20)
        RBFFD_CASE(24)
        RBFFD_CASE(30)
        RBFFD_CASE(31)
        RBFFD_CASE(40)
        RBFFD_CASE(48)
        RBFFD_CASE(56)
        RBFFD_CASE(57)
        RBFFD_CASE(70)
        RBFFD_CASE(71)
        default: return persistent ? persistent_kernel<0, MODE, MINB> : step_kernel<0, MODE, MINB>;
    }
#undef RBFFD_CASE
}

// one per translation unit: FP64 sweep and FP32 inner sweep with register
// budgets 1..4 (minimum resident blocks per SM)
StepFn pick_step_f64_b1(int n, bool persistent);
StepFn pick_step_f64_b2(int n, bool persistent);
StepFn pick_step_f64_b3(int n, bool persistent);
StepFn pick_step_f64_b4(int n, bool persistent);
StepFn pick_step_f32_b1(int n, bool persistent);
StepFn pick_step_f32_b2(int n, bool persistent);
StepFn pick_step_f32_b3(int n, bool persistent);
StepFn pick_step_f32_b4(int n, bool persistent);

// the resident persistent launch (step_res.cuh): one block of RES_THREADS_HOST
// threads per SM keeps its slices' planes in shared memory; i16: the index
// planes are 16-bit codes (every slice of the plan has them).  The wide
// variant has RES_THREADS_WIDE threads a block (nullptr for stencil sizes
// without one, step_res_w.cu)
static constexpr int RES_THREADS_HOST = 512;
static constexpr int RES_THREADS_WIDE = 1024;
StepFn pick_resident(int mode, int n, bool i16);
StepFn pick_resident_wide(int mode, int n, bool i16);
// the resident launch with far lists (step_res_far.cu), `threads` a block
// (nullptr where that block size is not compiled for n)
StepFn pick_resident_far(int mode, int n, int threads);
// dynamic shared memory of a resident launch of `grid` blocks whose halo
// window reaches `halo` slots beyond each block's rows on either side, with
// room for `extra` more values behind it (the far values)
unsigned resident_smem(int64_t nslices, int n, int mode, bool i16, int grid, int64_t halo,
                       int64_t extra = 0);

}  // namespace rbffd
