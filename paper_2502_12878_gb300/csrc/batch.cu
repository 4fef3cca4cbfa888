// rbffd_batch_*: many independent domains (uneven node counts and stencil
// sizes) solved by Eq. 6 in ONE persistent launch, replayed from a CUDA graph.
//
// Each domain keeps its own plan (packed stencils, iterates, f).  A device
// table describes the domains.  Load balance (per call, on the host): a
// domain's work is its bytes per step x its step cap; with target = total
// work / blocks, a domain of at least the target gets a team of
// floor(work/target) blocks, and the smaller domains are packed first-fit-
// decreasing into the remaining blocks, each of which then runs its domains
// one after another.  A team sweeps its domain's slices, reduces the step's
// residual, and decides on its own when the domain stops (tolerance, step cap,
// non-finite, divergence).  One-block teams synchronise with __syncthreads
// and gather the iterate through L1 (their own writes are visible after the
// barrier); larger teams use a per-domain barrier whose waits give up after
// ~2 s (RBFFD_ERR_TIMEOUT) and gather through L2 (.cg), because other blocks
// of the same launch rewrite the iterate.  Slices read the plan's 16-bit
// neighbour codes where it has them, and each warp prefetches its next
// slice's planes into L2 (bulk prefetch) before it sweeps the current one.
//
// The per-call inputs (the caller's f / u pointers, dt, tol, step caps) are
// copied into a device table at a fixed address, so one captured graph -
// gather of all domains, the persistent kernel, scatter of all domains - is
// replayed for every call.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <string.h>

#include <vector>

#include "plan.cuh"

namespace rbffd {

static constexpr int BATCH_MAX_WARPS = 32;   // blocks of 256, 512, 768 or 1024 threads
static constexpr long long BATCH_SPIN_CYCLES = 4000000000LL;

struct DomDesc {           // static part (from the plan)
    const double* w64;
    const int32_t* col;
    const uint16_t* col16;     // compact neighbour codes (NULL: int32 only)
    const int4* sbase;         // per slice window bases; x < 0: the slice uses col
    double* fs;            // plan's f in slot order
    double* u0;            // plan's iterates in slot order
    double* u1;
    const int32_t* perm;
    const int32_t* row_of_slot;
    int64_t N, NI, nslices;
    int n, pad;
};

struct DomCall {           // per-call part
    const double* f;       // caller's f [NI] (interior-list order)
    double* u;             // caller's u [N] in/out
    double dt, tol;
    long long max_steps;
};

struct DomState {          // per-domain control, written by the kernel
    unsigned long long res[3];
    unsigned long long arrivals;   // team barrier: block arrivals since the solve started
    long long k;
    int done, pad;
    double res_first, res_last;
    unsigned long long t_start, t_end;   // %globaltimer (ns) at the domain's first / last step
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct TeamDesc {
    int dom, rank, size, pad;
};

}  // namespace rbffd

struct rbffd_batch {
    int ndom = 0;
    int grid = 0;
    int minb = 2;
    int per_sm = 2;
    int threads = 256;                    // block size
    rbffd::DomDesc* d_desc = nullptr;
    rbffd::DomCall* d_call = nullptr;
    rbffd::DomState* d_state = nullptr;
    rbffd::TeamDesc* d_team = nullptr;    // assignments (CSR by block)
    int* d_first = nullptr;
    rbffd::TeamDesc* h_team = nullptr;    // pinned staging
    int* h_first = nullptr;
    rbffd::DomCall* h_call = nullptr;     // pinned staging
    rbffd::DomState* h_state = nullptr;   // pinned read-back
    std::vector<rbffd::DomDesc> desc;
    std::vector<double> work;
    void* graph = nullptr;
    int coop = 0;                         // graph holds a cooperative kernel node
    void* ev[2] = {nullptr, nullptr};
    double last_ms = 0.0;
};

namespace rbffd {

__device__ __forceinline__ double bld_cg(const double* p) {
    double v;
    asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double bld_ca(const double* p) {
    double v;
    asm volatile("ld.global.ca.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double bld_cs(const double* p) {
    double v;
    asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t bld_cs(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.cs.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t bld_cs(const uint16_t* p) {
    unsigned short v;
    asm volatile("ld.global.cs.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint32_t)v;
}

// window k = code >> 14 of the slice's four bases, plus the 14-bit offset
__device__ __forceinline__ int32_t bdecode16(uint32_t v, const int4& b) {
    const uint32_t k = v >> 14;
    const int32_t base = (k & 2u) ? ((k & 1u) ? b.w : b.z) : ((k & 1u) ? b.y : b.x);
    return base + (int32_t)(v & 0x3fffu);
}

// sum_j w_j u[col_j], an fma chain from 0 in j order; loads in phases of CH
// (indices, weights, then the gathers).  I16: 16-bit codes against the
// slice's window bases `sb` (the same columns, fewer bytes).
template <int NN, bool COH, int CH, bool I16>
__device__ __forceinline__ double brow(const double* __restrict__ w, const void* __restrict__ colp,
                                       const int4& sb, const double* __restrict__ u, int n) {
    double acc = 0.0;
    const int nn = NN > 0 ? NN : n;
#pragma unroll
    for (int j0 = 0; j0 < (NN > 0 ? NN : 1 << 30); j0 += CH) {
        if (NN == 0 && j0 >= nn) break;
        int32_t c[CH];
        double wv[CH], uv[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (I16)
                    c[t] = (int32_t)bld_cs((const uint16_t*)colp + (j0 + t) * SLICE);
                else
                    c[t] = bld_cs((const int32_t*)colp + (j0 + t) * SLICE);
            }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) wv[t] = bld_cs(w + (j0 + t) * SLICE);
        if constexpr (I16) {
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < nn) c[t] = bdecode16((uint32_t)c[t], sb);
        }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) uv[t] = COH ? bld_cg(u + c[t]) : bld_ca(u + c[t]);
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) acc = __fma_rn(wv[t], uv[t], acc);
    }
    return acc;
}

__device__ __forceinline__ unsigned long long babs_bits(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : b;
}

// bulk prefetch into L2 (one lane) of the weight and index planes of slice
// sl, the warp's next one: the 16-bit code plane when the plan has one.  Both
// planes start on 16-byte boundaries and their sizes (8n and 2n or 4n bytes
// per row, 32 rows) are multiples of 16.
__device__ __forceinline__ void bprefetch(const DomDesc& D, int64_t sl) {
    if (sl >= D.nslices) return;
    const int64_t nb = sl * (int64_t)D.n * SLICE;
    const unsigned plane = (unsigned)(D.n * SLICE);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(D.w64 + nb), "r"(plane * 8u)
                 : "memory");
    if (D.col16)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(D.col16 + nb),
                     "r"(plane * 2u) : "memory");
    else
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(D.col + nb),
                     "r"(plane * 4u) : "memory");
}

// one step of domain D over the slices of this team member; returns max |r| bits
template <int NN, bool COH, int CH>
__device__ __noinline__ unsigned long long bstep(const DomDesc& D, int par, double dt, int64_t s0,
                                                 int64_t stride) {
    const int lane = threadIdx.x & 31;
    const double* uin = par ? D.u1 : D.u0;
    double* uout = par ? D.u0 : D.u1;
    unsigned long long m = 0;
    for (int64_t sl = s0; sl < D.nslices; sl += stride) {
        const int64_t row = sl * SLICE + lane;
        const int64_t base = sl * (int64_t)D.n * SLICE + lane;
        const int4 sb = D.col16 ? __ldg(D.sbase + sl) : make_int4(-1, -1, -1, -1);
        if (lane == 0) bprefetch(D, sl + stride);
        if (row < D.NI) {
            const double fi = bld_cs(D.fs + row);
            const double ui = COH ? bld_cg(uin + row) : bld_ca(uin + row);
            double acc = sb.x >= 0
                             ? brow<NN, COH, CH, true>(D.w64 + base, D.col16 + base, sb, uin, D.n)
                             : brow<NN, COH, CH, false>(D.w64 + base, D.col + base, sb, uin, D.n);
            double r = __dsub_rn(acc, fi);
            uout[row] = __fma_rn(dt, r, ui);
            m = max(m, babs_bits(r));
        }
    }
    return m;
}

template <bool COH, int CH>
__device__ unsigned long long bstep_any(const DomDesc& D, int par, double dt, int64_t s0,
                                        int64_t stride) {
    switch (D.n) {
        case 12: return bstep<12, COH, CH>(D, par, dt, s0, stride);
        case 30: return bstep<30, COH, CH>(D, par, dt, s0, stride);
        case 56: return bstep<56, COH, CH>(D, par, dt, s0, stride);
        default: return bstep<0, COH, CH>(D, par, dt, s0, stride);
    }
}

// release / acquire accesses at GPU scope for the team barrier
__device__ __forceinline__ void bred_max(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void bred_add_release(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long bld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long bld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// the stop rule for step kk with residual R (R0: step 0's), in thread 0;
// rank 0 of the team records a stop in the domain's state
__device__ __forceinline__ int bdecide(DomState* st, const DomCall& C, int rank, long long kk,
                                       double R, double* R0) {
    if (kk == 0) *R0 = R;
    int dn;
    if (!isfinite(R)) dn = DONE_NONFINITE;
    else if (R < C.tol) dn = DONE_CONVERGED;
    else if (kk > 0 && *R0 > 0.0 && R > 1e6 * *R0) dn = DONE_DIVERGED;
    else if (kk + 1 >= C.max_steps) dn = DONE_CAP;
    else dn = DONE_RUNNING;
    if (rank == 0 && dn != DONE_RUNNING) {
        st->k = kk + 1;
        st->res_first = *R0;
        st->res_last = R;
        st->done = dn;
        st->t_end = gtimer();
    }
    return dn;
}

// one domain's solve by one team member (rank of size blocks); returns false
// when a team wait gave up.  CH: neighbours per load phase (8 where the
// register budget is below 80 per thread).  A one-block team decides right
// after each step (its residual is the block's).  Larger teams end a step
// with a counter barrier (each block adds its max |r| to the step's residual
// slot and its arrival to the domain's counter - both fire-and-forget, the
// arrival a release - and polls the counter, bounded), load the step's full
// residual right after it and apply the stop rule to it after their next
// step: the same rule to the same value in every member, so the team stops
// together.  A stop wastes that next step, which writes the other buffer; the
// result u^{k+1} is untouched.  Rank 0 clears the slot step k + 2 will use.
template <int CH>
__device__ bool run_domain(const TeamDesc T, const DomDesc* __restrict__ desc,
                           const DomCall* __restrict__ call, DomState* state,
                           unsigned long long* wmax, int* s_stop) {
    const DomDesc D = desc[T.dom];
    const DomCall C = call[T.dom];
    DomState* st = state + T.dom;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5);
    const int64_t s0 = (int64_t)T.rank * nw + wid;
    const int64_t stride = (int64_t)T.size * nw;
    double R0 = 0.0;
    unsigned long long pend = 0ull;   // thread 0: the last barrier's step residual
    bool decided = false;
    if (threadIdx.x == 0 && T.rank == 0) st->t_start = gtimer();
    for (long long k = 0; k < C.max_steps; ++k) {
        unsigned long long m = T.size == 1
                                   ? bstep_any<false, CH>(D, (int)(k & 1), C.dt, s0, stride)
                                   : bstep_any<true, CH>(D, (int)(k & 1), C.dt, s0, stride);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) wmax[wid] = m;
        __syncthreads();
        if (wid == 0) {
            m = lane < nw ? wmax[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
        if (threadIdx.x == 0) {
            int dn = DONE_RUNNING;
            if (T.size == 1) {
                dn = bdecide(st, C, T.rank, k, __longlong_as_double((long long)m), &R0);
            } else {
                if (k > 0) dn = bdecide(st, C, T.rank, k - 1, __longlong_as_double((long long)pend),
                                        &R0);
                if (dn == DONE_RUNNING) {
                    bred_max(&st->res[k % 3], m);
                    bred_add_release(&st->arrivals, 1ull);
                    const unsigned long long target = (unsigned long long)(k + 1) * T.size;
                    const long long t0 = clock64();
                    while (bld_acquire(&st->arrivals) < target)
                        if (clock64() - t0 > BATCH_SPIN_CYCLES) {
                            atomicExch(&st->done, DONE_TIMEOUT);
                            dn = -1;
                            break;
                        }
                    if (dn == DONE_RUNNING) {
                        if (T.rank == 0) atomicExch(&st->res[(k + 2) % 3], 0ull);
                        pend = bld_relaxed(&st->res[k % 3]);
                    }
                }
            }
            *s_stop = dn;
        }
        __syncthreads();
        const int dn = *s_stop;
        __syncthreads();   // every thread has read it before thread 0 writes the next
        if (dn == -1) return false;
        if (dn != DONE_RUNNING) {
            decided = true;
            break;
        }
    }
    // a larger team's last step (the cap): its rule, from the residual of its barrier
    if (!decided && T.size > 1 && C.max_steps > 0 && threadIdx.x == 0)
        bdecide(st, C, T.rank, C.max_steps - 1, __longlong_as_double((long long)pend), &R0);
    __syncthreads();
    return true;
}

template <int MINB, int TH>
__global__ void __launch_bounds__(TH, MINB)
    batch_kernel(const DomDesc* __restrict__ desc, const DomCall* __restrict__ call,
                 DomState* state, const TeamDesc* __restrict__ assign,
                 const int* __restrict__ first) {
    constexpr int CH = 65536 / (TH * MINB) >= 80 ? 16 : 8;
    __shared__ unsigned long long wmax[BATCH_MAX_WARPS];
    __shared__ int s_stop;
    for (int a = first[blockIdx.x]; a < first[blockIdx.x + 1]; ++a)
        if (!run_domain<CH>(assign[a], desc, call, state, wmax, &s_stop)) return;
}

// gather f and u of every domain into its plan (one launch for all domains)
__global__ void batch_gather(const DomDesc* desc, const DomCall* call, DomState* state,
                             int ndom) {
    for (int dI = blockIdx.y; dI < ndom; dI += gridDim.y) {
        const DomDesc D = desc[dI];
        const DomCall C = call[dI];
        for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < D.N;
             p += (int64_t)gridDim.x * blockDim.x) {
            double v = C.u[D.perm[p]];
            D.u0[p] = v;
            D.u1[p] = v;
            if (p < D.NI) D.fs[p] = C.f[D.row_of_slot[p]];
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            DomState& s = state[dI];
            s.res[0] = s.res[1] = s.res[2] = 0ull;
            s.arrivals = 0ull;
            s.k = 0;
            s.done = C.max_steps <= 0 ? DONE_CAP : DONE_RUNNING;
            s.res_first = s.res_last = 0.0;
            s.t_start = s.t_end = 0ull;
        }
    }
}

__global__ void batch_scatter(const DomDesc* desc, const DomCall* call, const DomState* state,
                              int ndom) {
    for (int dI = blockIdx.y; dI < ndom; dI += gridDim.y) {
        const DomDesc D = desc[dI];
        const DomCall C = call[dI];
        const double* us = (state[dI].k & 1) ? D.u1 : D.u0;
        for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < D.NI;
             p += (int64_t)gridDim.x * blockDim.x)
            C.u[D.perm[p]] = us[p];
    }
}

typedef void (*BatchFn)(const DomDesc*, const DomCall*, DomState*, const TeamDesc*, const int*);

// launch shapes: (register budget, block size) with TH x MINB <= 1024 threads
static bool batch_shape_ok(int minb, int threads) {
    return (threads == 256 && minb >= 1 && minb <= 3) || (threads == 512 && minb >= 1 && minb <= 2) ||
           ((threads == 768 || threads == 1024) && minb == 1);
}

static BatchFn batch_fn(int minb, int threads) {
    if (threads == 1024) return batch_kernel<1, 1024>;
    if (threads == 768) return batch_kernel<1, 768>;
    if (threads == 512) return minb == 2 ? batch_kernel<2, 512> : batch_kernel<1, 512>;
    switch (minb) {
        case 1: return batch_kernel<1, 256>;
        case 3: return batch_kernel<3, 256>;
        default: return batch_kernel<2, 256>;
    }
}

// Assignment of domains to the blocks of the persistent grid, minimising the
// largest block load.  work[i] = cost of domain i (cost per step x step cap).
// For a candidate load T: a domain with work > T gets a team of ceil(work/T)
// blocks (each member carries work/size); the others are placed longest first
// on the least-loaded block (LPT), after any team domain of that block.  T is the smallest value (binary
// search) for which every block stays within T.  Returns per-block
// assignment lists in CSR form.
static bool try_assign(const std::vector<double>& work, int grid, double T,
                       std::vector<std::vector<TeamDesc>>* out) {
    const int nd = (int)work.size();
    std::vector<int> team(nd, 0);
    long long used = 0;
    for (int i = 0; i < nd; ++i)
        if (work[i] > T) {
            team[i] = (int)ceil(work[i] / T);
            used += team[i];
        }
    if (used > grid) return false;
    std::vector<int> order;
    for (int i = 0; i < nd; ++i)
        if (team[i] == 0) order.push_back(i);
    std::sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
    std::vector<double> load(grid, 0.0);
    std::vector<std::vector<TeamDesc>> per(grid);
    int b = 0;
    for (int i = 0; i < nd; ++i)
        for (int r = 0; r < team[i]; ++r) {
            per[b].push_back({i, r, team[i], 0});
            load[b] = work[i] / team[i];
            ++b;
        }
    // LPT over all blocks (a heap would do; domain counts are small).  A team
    // member runs its team's domain first - all members start it together -
    // and then any small domains placed on its block.
    for (int i : order) {
        int best = 0;
        for (int q = 1; q < grid; ++q)
            if (load[q] < load[best]) best = q;
        if (load[best] + work[i] > T * (1.0 + 1e-9)) return false;
        per[best].push_back({i, 0, 1, 0});
        load[best] += work[i];
    }
    if (out) out->swap(per);
    return true;
}

static void make_assignment(const std::vector<double>& work, int grid, std::vector<TeamDesc>& asg,
                            std::vector<int>& first) {
    double tot = std::accumulate(work.begin(), work.end(), 0.0);
    double mx = *std::max_element(work.begin(), work.end());
    double lo = tot / std::max(grid, 1), hi = std::max(mx, lo) * 2.0 + 1e-300;
    // hi is always feasible when grid >= number of domains or small domains pack;
    // grow it until feasible
    for (int g = 0; g < 64 && !try_assign(work, grid, hi, nullptr); ++g) hi *= 2.0;
    for (int it = 0; it < 40; ++it) {
        double mid = 0.5 * (lo + hi);
        if (try_assign(work, grid, mid, nullptr)) hi = mid;
        else lo = mid;
    }
    std::vector<std::vector<TeamDesc>> per;
    try_assign(work, grid, hi, &per);
    per.resize(grid);
    asg.clear();
    first.assign(grid + 1, 0);
    for (int q = 0; q < grid; ++q) {
        first[q] = (int)asg.size();
        for (auto& t : per[q]) asg.push_back(t);
    }
    first[grid] = (int)asg.size();
}

// captures on a private stream (capture records, it runs nothing)
static int batch_capture(rbffd_batch* B) {
    if (B->graph) {
        cudaGraphExecDestroy((cudaGraphExec_t)B->graph);
        B->graph = nullptr;
    }
    BatchFn fn = batch_fn(B->minb, B->threads);
    cudaStream_t cs;
    RBFFD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaErrorUnknown;
    // first try a cooperative kernel node; if capture refuses it, a plain node
    // (the grid was checked to fit on the device at once; waits are bounded)
    for (int coop = 1; coop >= 0 && e != cudaSuccess; --coop) {
        cudaGraph_t g;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            dim3 gg(64, (unsigned)std::min(B->ndom, 65535));
            batch_gather<<<gg, 256, 0, cs>>>(B->d_desc, B->d_call, B->d_state, B->ndom);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(B->grid);
            cfg.blockDim = dim3(B->threads);
            cfg.stream = cs;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = coop;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, fn, (const DomDesc*)B->d_desc, (const DomCall*)B->d_call,
                                   B->d_state, (const TeamDesc*)B->d_team, (const int*)B->d_first);
            if (e == cudaSuccess) {
                batch_scatter<<<gg, 256, 0, cs>>>(B->d_desc, B->d_call, B->d_state, B->ndom);
                e = cudaStreamEndCapture(cs, &g);
            } else {
                cudaGraph_t dummy;
                cudaStreamEndCapture(cs, &dummy);
            }
        }
        if (e == cudaSuccess) {
            cudaGraphExec_t ex;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e == cudaSuccess) {
                B->graph = (void*)ex;
                B->coop = coop;
            }
        }
        if (e != cudaSuccess) cudaGetLastError();
    }
    cudaStreamDestroy(cs);
    RBFFD_CHECK_CUDA(e);
    return RBFFD_OK;
}

static void batch_free(rbffd_batch* B) {
    if (!B) return;
    void* dv[] = {B->d_desc, B->d_call, B->d_state, B->d_team, B->d_first};
    for (void* p : dv)
        if (p) cudaFree(p);
    if (B->h_team) cudaFreeHost(B->h_team);
    if (B->h_first) cudaFreeHost(B->h_first);
    if (B->h_call) cudaFreeHost(B->h_call);
    if (B->h_state) cudaFreeHost(B->h_state);
    if (B->graph) cudaGraphExecDestroy((cudaGraphExec_t)B->graph);
    for (void* e : B->ev)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    delete B;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_batch_create(rbffd_plan* const* plans, int ndom, int blocks_per_sm,
                                  rbffd_batch** out, void* stream) {
    clear_error();
    RBFFD_ARG(plans && out && ndom >= 1, "rbffd_batch_create: bad argument");
    RBFFD_ARG(blocks_per_sm >= 0 && blocks_per_sm <= 8, "rbffd_batch_create: blocks_per_sm in [0, 8]");
    for (int i = 0; i < ndom; ++i) RBFFD_ARG(plans[i] != nullptr, "rbffd_batch_create: NULL plan %d", i);
    *out = nullptr;
    cudaStream_t s = as_stream(stream);
    rbffd_batch* B = new rbffd_batch();
    B->ndom = ndom;
    for (int i = 0; i < ndom; ++i) {
        const rbffd_plan* p = plans[i];
        DomDesc d;
        d.w64 = p->w64;
        d.col = p->col;
        d.col16 = p->col16;
        d.sbase = p->sbase;
        d.fs = p->fs;
        d.u0 = p->u[0];
        d.u1 = p->u[1];
        d.perm = p->perm;
        d.row_of_slot = p->row_of_slot;
        d.N = p->N;
        d.NI = p->NI;
        d.nslices = p->nslices;
        d.n = p->n;
        d.pad = 0;
        B->desc.push_back(d);
        // default cost of one step: memory rounds of its slices (one per chunk of
        // 16 neighbours plus one), which is what latency-bound blocks pay
        B->work.push_back((double)p->nslices * (double)((p->n + 15) / 16 + 1));
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_desc, sizeof(DomDesc) * ndom);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_call, sizeof(DomCall) * ndom);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_state, sizeof(DomState) * ndom);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_call, sizeof(DomCall) * ndom);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_state, sizeof(DomState) * ndom);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreate(&ev);
        if (e == cudaSuccess) B->ev[i] = (void*)ev;
    }
    int sms = device_sm_count();
    const size_t max_asg = (size_t)sms * 8 + ndom;
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_team, sizeof(TeamDesc) * max_asg);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_team, sizeof(TeamDesc) * max_asg);
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_first, sizeof(int) * ((size_t)sms * 8 + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_first, sizeof(int) * ((size_t)sms * 8 + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_desc, B->desc.data(), sizeof(DomDesc) * ndom, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_state, 0, sizeof(DomState) * ndom, s);
    if (e != cudaSuccess) {
        set_error("rbffd_batch_create: %s", cudaGetErrorString(e));
        batch_free(B);
        return RBFFD_ERR_CUDA;
    }
    // launch shape: register budget minb and blocks per SM; blocks_per_sm = 0 -> tune
    // (the tuner times one short solve per candidate in rbffd_batch_tune)
    int per_sm_max = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_max, (const void*)batch_fn(2, 256), 256,
                                                  0);
    B->minb = 2;
    B->threads = 256;
    B->per_sm = blocks_per_sm > 0 ? std::min(blocks_per_sm, std::max(per_sm_max, 1))
                                  : std::min(2, std::max(per_sm_max, 1));
    B->grid = sms * B->per_sm;
    int maxres = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxres, (const void*)batch_fn(B->minb, 256), 256,
                                                  0);
    if (B->grid > maxres * sms) {
        set_error("rbffd_batch_create: %d domains need %d co-resident blocks, the device holds %d",
                  ndom, B->grid, maxres * sms);
        batch_free(B);
        return RBFFD_ERR_CAPACITY;
    }
    int st = batch_capture(B);
    if (st) {
        batch_free(B);
        return st;
    }
    *out = B;
    return RBFFD_OK;
}

extern "C" int rbffd_batch_destroy(rbffd_batch* B) {
    clear_error();
    if (!B) return RBFFD_OK;
    cudaDeviceSynchronize();
    batch_free(B);
    return RBFFD_OK;
}

extern "C" int rbffd_solve_batch(rbffd_batch* B, const double* const* f, double* const* u,
                                 const double* dt, const int64_t* max_steps, const double* tol,
                                 int64_t* h_steps, double* h_res, int* h_status, void* stream) {
    clear_error();
    RBFFD_ARG(B && f && u && dt && max_steps && tol, "rbffd_solve_batch: NULL argument");
    cudaStream_t s = as_stream(stream);
    for (int i = 0; i < B->ndom; ++i) {
        RBFFD_ARG(f[i] && u[i], "rbffd_solve_batch: NULL f/u of domain %d", i);
        RBFFD_ARG(dt[i] > 0.0 && isfinite(dt[i]) && tol[i] >= 0.0 && max_steps[i] >= 0,
                  "rbffd_solve_batch: bad dt / tol / max_steps of domain %d", i);
        B->h_call[i].f = f[i];
        B->h_call[i].u = u[i];
        B->h_call[i].dt = dt[i];
        B->h_call[i].tol = tol[i];
        B->h_call[i].max_steps = max_steps[i];
    }
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(B->d_call, B->h_call, sizeof(DomCall) * B->ndom,
                                     cudaMemcpyHostToDevice, s));
    {
        std::vector<double> work(B->ndom);
        for (int i = 0; i < B->ndom; ++i) work[i] = B->work[i] * (double)std::max<int64_t>(max_steps[i], 1);
        std::vector<TeamDesc> asg;
        std::vector<int> first;
        make_assignment(work, B->grid, asg, first);
        // the pinned staging may still be read by a previous call's copy
        RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
        memcpy(B->h_team, asg.data(), sizeof(TeamDesc) * asg.size());
        memcpy(B->h_first, first.data(), sizeof(int) * first.size());
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(B->d_team, B->h_team, sizeof(TeamDesc) * asg.size(),
                                         cudaMemcpyHostToDevice, s));
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(B->d_first, B->h_first, sizeof(int) * first.size(),
                                         cudaMemcpyHostToDevice, s));
    }
    RBFFD_CHECK_CUDA(cudaEventRecord((cudaEvent_t)B->ev[0], s));
    RBFFD_CHECK_CUDA(cudaGraphLaunch((cudaGraphExec_t)B->graph, s));
    RBFFD_CHECK_CUDA(cudaEventRecord((cudaEvent_t)B->ev[1], s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(B->h_state, B->d_state, sizeof(DomState) * B->ndom,
                                     cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, (cudaEvent_t)B->ev[0], (cudaEvent_t)B->ev[1]);
    B->last_ms = ms;
    int worst = RBFFD_OK;
    for (int i = 0; i < B->ndom; ++i) {
        const DomState& st = B->h_state[i];
        int code;
        switch (st.done) {
            case DONE_CONVERGED: code = RBFFD_OK; break;
            case DONE_CAP: code = RBFFD_NOT_CONVERGED; break;
            case DONE_NONFINITE: code = RBFFD_ERR_NONFINITE; break;
            case DONE_DIVERGED: code = RBFFD_ERR_DIVERGED; break;
            case DONE_TIMEOUT: code = RBFFD_ERR_TIMEOUT; break;
            default: code = RBFFD_ERR_CUDA; break;
        }
        if (h_steps) h_steps[i] = st.k;
        if (h_res) h_res[i] = st.res_last;
        if (h_status) h_status[i] = code;
        if (code < 0 && (worst >= 0 || code < worst)) worst = code;
        if (worst >= 0 && code == RBFFD_NOT_CONVERGED) worst = RBFFD_NOT_CONVERGED;
    }
    if (worst < 0) set_error("rbffd_solve_batch: a domain ended with status %d", worst);
    return worst;
}

extern "C" int rbffd_batch_set_shape(rbffd_batch* B, int minb, int blocks_per_sm, int threads,
                                     void* stream) {
    clear_error();
    RBFFD_ARG(B && blocks_per_sm >= 1 && blocks_per_sm <= 8 && batch_shape_ok(minb, threads),
              "rbffd_batch_set_shape: bad argument");
    int sms = device_sm_count();
    int maxres = 0;
    RBFFD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &maxres, (const void*)batch_fn(minb, threads), threads, 0));
    int grid = sms * blocks_per_sm;
    if (grid > maxres * sms) {
        set_error("rbffd_batch_set_shape: %d blocks cannot be co-resident (max %d)", grid,
                  maxres * sms);
        return RBFFD_ERR_CAPACITY;
    }
    B->minb = minb;
    B->per_sm = blocks_per_sm;
    B->threads = threads;
    B->grid = grid;
    (void)stream;
    return batch_capture(B);
}

extern "C" int rbffd_batch_stats(const rbffd_batch* B, double* h_ms, int* h_shape) {
    clear_error();
    RBFFD_ARG(B, "rbffd_batch_stats: NULL batch");
    if (h_ms) *h_ms = B->last_ms;
    if (h_shape) {
        h_shape[0] = B->minb;
        h_shape[1] = B->per_sm;
        h_shape[2] = B->grid;
        h_shape[3] = B->coop;
        h_shape[4] = B->threads;
    }
    return RBFFD_OK;
}

extern "C" int rbffd_batch_domain_times(const rbffd_batch* B, double* h_start_ms, double* h_end_ms,
                                        int* h_block, int* h_team) {
    clear_error();
    RBFFD_ARG(B && B->h_state, "rbffd_batch_domain_times: NULL batch");
    unsigned long long t0 = ~0ull;
    for (int i = 0; i < B->ndom; ++i)
        if (B->h_state[i].t_start) t0 = std::min(t0, B->h_state[i].t_start);
    for (int i = 0; i < B->ndom; ++i) {
        const DomState& st = B->h_state[i];
        if (h_start_ms) h_start_ms[i] = st.t_start ? (st.t_start - t0) * 1e-6 : -1.0;
        if (h_end_ms) h_end_ms[i] = st.t_end ? (st.t_end - t0) * 1e-6 : -1.0;
        if (h_block) h_block[i] = -1;
        if (h_team) h_team[i] = 0;
    }
    for (int q = 0; q < B->grid; ++q)
        for (int a = B->h_first[q]; a < B->h_first[q + 1]; ++a) {
            const TeamDesc& t = B->h_team[a];
            if (t.rank == 0) {
                if (h_block) h_block[t.dom] = q;
                if (h_team) h_team[t.dom] = t.size;
            }
        }
    return RBFFD_OK;
}

extern "C" int rbffd_batch_set_costs(rbffd_batch* B, const double* h_cost_per_step) {
    clear_error();
    RBFFD_ARG(B && h_cost_per_step, "rbffd_batch_set_costs: NULL argument");
    for (int i = 0; i < B->ndom; ++i)
        RBFFD_ARG(h_cost_per_step[i] > 0.0 && isfinite(h_cost_per_step[i]),
                  "rbffd_batch_set_costs: cost of domain %d must be positive", i);
    for (int i = 0; i < B->ndom; ++i) B->work[i] = h_cost_per_step[i];
    return RBFFD_OK;
}

