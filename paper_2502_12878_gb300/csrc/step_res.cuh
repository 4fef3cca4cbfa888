// Resident persistent launch of the explicit sweep (Eq. 6): for plans whose
// packed stencils fit in the shared memory of one block per SM, every block
// keeps its slices' weight and index planes (and their rows' f or d32) in
// shared memory for the whole run, and at the start of every step stages the
// halo of its rows - a window of the iterate around its own slots, which in
// Morton order holds nearly all of its rows' neighbours - into shared memory
// too, so the gathers read shared memory and only the neighbours outside the
// window go to L2.  Both are TMA bulk copies (cp.async.bulk, global ->
// shared, completion on an mbarrier: the planes once per launch on its first
// phase, the halo every step on the next); every wait is bounded.  The arithmetic is that of the other step kernels - the same fused
// multiply-add chain per row in support order - so the results are the same
// bit for bit.
#pragma once

#include <type_traits>

#include "step.cuh"

namespace rbffd {
static constexpr unsigned RES_COPY_CHUNK = 32768;   // bytes per bulk copy

// shared-memory layout of one block (byte offsets; every region 128-aligned):
// the mbarrier, the weight and index planes, the rows' f (or d32), two
// buffers of the block's own rows' iterate, the slice order, and the halo
// window of the iterate (plus `extra` far values behind it)
struct ResLayout {
    unsigned w, idx, f, o, ord, h, total;
};

__host__ __device__ __forceinline__ unsigned res_align(unsigned x) { return (x + 127u) & ~127u; }

// the layout for at most `nsl` slices of n entries: weights of `wbytes`,
// indices of `ibytes` (2: 16-bit codes, 4: int32 slots); the halo window
// holds the block's rows and `halo` slots on either side (halo < 0: no window)
__host__ __device__ __forceinline__ unsigned res_window(int64_t nsl, int64_t halo) {
    return halo < 0 ? 0u : (unsigned)(nsl * SLICE + 2 * halo + 8);
}
__host__ __device__ __forceinline__ ResLayout res_layout(int64_t nsl, int n, int wbytes,
                                                         int ibytes, int64_t halo,
                                                         int64_t extra = 0) {
    ResLayout L;
    const unsigned ent = (unsigned)(nsl * n * SLICE);
    const unsigned rows = (unsigned)(nsl * SLICE);
    L.w = 128;   // the mbarrier lives at offset 0
    L.idx = L.w + res_align(ent * (unsigned)wbytes);
    L.f = L.idx + res_align(ent * (unsigned)ibytes);
    L.o = L.f + res_align(rows * (unsigned)wbytes);
    L.ord = L.o + res_align(2u * rows * (unsigned)wbytes);
    L.h = L.ord + res_align((unsigned)nsl * 2u);
    L.total = L.h + res_align((res_window(nsl, halo) + (unsigned)extra) * (unsigned)wbytes);
    return L;
}

// slices of block b of G: a contiguous range, sizes differing by at most one
__device__ __forceinline__ void res_range(int64_t nslices, int64_t* s0, int64_t* s1) {
    *s0 = nslices * blockIdx.x / gridDim.x;
    *s1 = nslices * (blockIdx.x + 1) / gridDim.x;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// bounded wait on phase `parity` of the mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long spin) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > spin) return false;
    }
}

// the iterate at slot c: from the block's halo window [lo, lo + W) in shared
// memory, else through L2 (.cg: other blocks rewrite the iterate between steps)
template <class T>
__device__ __forceinline__ T res_u(const T* hs, int32_t lo, uint32_t W, const T* __restrict__ u,
                                   int32_t c) {
    const uint32_t o = (uint32_t)(c - lo);
    return o < W ? hs[o] : ld_iter<true>(u + c);
}

// sum_j w_j u[col_j] with the planes in shared memory (entries at stride 32),
// an fma chain from 0 in j order; the iterate from the halo window where it
// covers the neighbour, CH gathers in flight at a time
template <int NN, bool I16, class T>
__device__ __forceinline__ T row_dot_res(const T* w, const void* colp, const int4& sb,
                                         const T* hs, int32_t lo, uint32_t W,
                                         const T* __restrict__ u, int n) {
    constexpr int CH = 16;
    T acc = T(0);
    const int nn = NN > 0 ? NN : n;
#pragma unroll
    for (int j0 = 0; j0 < (NN > 0 ? NN : 1 << 30); j0 += CH) {
        if (NN == 0 && j0 >= nn) break;
        int32_t c[CH];
        T uv[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (I16)
                    c[t] = decode16((uint32_t)((const uint16_t*)colp)[(j0 + t) * SLICE], sb);
                else
                    c[t] = ((const int32_t*)colp)[(j0 + t) * SLICE];
            }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) uv[t] = res_u<T>(hs, lo, W, u, c[t]);
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (sizeof(T) == 8) acc = __fma_rn(w[(j0 + t) * SLICE], uv[t], acc);
                else acc = __fmaf_rn(w[(j0 + t) * SLICE], uv[t], acc);
            }
    }
    return acc;
}

// FAR: sum_j w_j v_j with every v_j in shared memory at the entry's local
// index (window position, or the window's length plus its far position)
template <int NN, class T>
__device__ __forceinline__ T row_dot_far(const T* w, const uint16_t* li, const T* hs, int n) {
    constexpr int CH = 16;
    T acc = T(0);
    const int nn = NN > 0 ? NN : n;
#pragma unroll
    for (int j0 = 0; j0 < (NN > 0 ? NN : 1 << 30); j0 += CH) {
        if (NN == 0 && j0 >= nn) break;
        T uv[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) uv[t] = hs[li[(j0 + t) * SLICE]];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (sizeof(T) == 8) acc = __fma_rn(w[(j0 + t) * SLICE], uv[t], acc);
                else acc = __fmaf_rn(w[(j0 + t) * SLICE], uv[t], acc);
            }
    }
    return acc;
}

// the slot of entry e of the block's index planes (FAR: its local index)
template <bool I16, bool FAR>
__device__ __forceinline__ int32_t res_col(const unsigned char* idx_s, int32_t e, const int4& sb) {
    if constexpr (FAR) return (int32_t)((const uint16_t*)idx_s)[e];
    else if constexpr (I16) return decode16((uint32_t)((const uint16_t*)idx_s)[e], sb);
    else return ((const int32_t*)idx_s)[e];
}

// sum_j w_j u[col_j] for a row whose neighbours are all rows of the block
// itself: the iterate from the block's own-row buffer o (at slot - base), the
// same fma chain from 0 in j order as the other row sums
template <int NN, bool I16, bool FAR, class T>
__device__ __forceinline__ T row_dot_own(const T* w, const unsigned char* idx_s, int32_t eo,
                                         const int4& sb, const T* o, int32_t base, int n) {
    constexpr int CH = 16;
    T acc = T(0);
    const int nn = NN > 0 ? NN : n;
#pragma unroll
    for (int j0 = 0; j0 < (NN > 0 ? NN : 1 << 30); j0 += CH) {
        if (NN == 0 && j0 >= nn) break;
        T uv[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) uv[t] = o[res_col<I16, FAR>(idx_s, eo + (j0 + t) * SLICE, sb) - base];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (sizeof(T) == 8) acc = __fma_rn(w[(j0 + t) * SLICE], uv[t], acc);
                else acc = __fmaf_rn(w[(j0 + t) * SLICE], uv[t], acc);
            }
    }
    return acc;
}

// The step barrier of the resident launch, split in its two halves so that a
// block can compute between them: at the end of step k every block adds its
// max |r| to the step's residual slot and its arrival to the counter (both
// fire-and-forget; the arrival releases the block's iterate writes), and at
// the start of step k + 1 one thread waits for every block's arrival (bounded
// by `spin` clock cycles; `held`: arrivals added to every target, 0 but in a
// test of the timeout path), then loads step k's full residual, to which the
// stop rule is applied once the block has staged step k + 1's window (every
// block the same rule to the same value, so all stop together, before step
// k + 1 writes more than the other buffer), and block 0 clears the slot step
// k + 2 will use.  Thread 0 only.
__device__ __forceinline__ void res_arrive(StepCtrl* c, long long k, unsigned long long m) {
    red_max_relaxed(&c->res[k % 3], m);
    red_add_release(&c->arrivals, 1ull);
}
__device__ __forceinline__ bool res_wait(StepCtrl* c, LagState& S, long long k, long long k0,
                                         long long spin, int held) {
    const unsigned long long target =
        (unsigned long long)(k - k0 + 1) * gridDim.x + (unsigned long long)held;
    const long long t0 = clock64();
    while (ld_acquire(&c->arrivals) < target)
        if (clock64() - t0 > spin) {
            atomicExch(&c->done, DONE_TIMEOUT);
            return false;
        }
    if (blockIdx.x == 0) st_relaxed(&c->res[(k + 2) % 3], 0ull);
    S.pend = ld_relaxed(&c->res[k % 3]);
    return true;
}

// the stop rule for step kk from its residual (loaded at its barrier); block 0
// records the outcome of a run that stops.  Thread 0 only.
__device__ __forceinline__ int res_decide(StepCtrl* c, LagState& S, long long kk) {
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
    return dn;
}

// block max of IEEE bits over TH threads, valid in thread 0: one shared-memory
// round and a warp-wide reduction in warp 0
template <int TH>
__device__ __forceinline__ unsigned long long res_block_max(unsigned long long v) {
    __shared__ unsigned long long wm[TH / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < TH / 32 ? wm[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// All steps of a run in one cooperative launch of one block per SM.  The
// index planes are the 16-bit codes when every slice of the plan has them
// (I16), else the int32 slots.
// TH: threads per block (one block per SM): 512, or 1024 where the kernel
// fits 64 registers - one round of slices per step for more blocks' shares.
// FAR: the index planes are the entries' local indices (A.fl_idx) and every
// step the block's far values (the slots outside its window that its rows
// read: A.fl_slot) are loaded behind the window, so every gather reads
// shared memory (no L2 round trip in the rows' chains).
//
// Overlap of the step barrier: the block's slices are ordered once, inner
// slices first - those whose rows read only the block's own rows.  Step k + 1
// of an inner slice needs nothing but the block's own u^{k+1}, which it keeps
// in shared memory, so while warp 0 waits for the other blocks' arrivals of
// step k and then stages the halo window, the other warps compute the inner
// slices into the second own-row buffer; their results go to the iterate
// only after the barrier (slower blocks may still read the buffer they
// overwrite).  Then all warps compute the remaining slices from the window.
// Each row's arithmetic is the same whichever phase computes it.  Shares are
// ordered with their inner rows first at plan creation, so whole slices of
// them lead.
template <int NN, int MODE, bool I16, int TH, bool FAR = false>
__global__ void __launch_bounds__(TH, 1) resident_kernel(StepArgs A, StepCtrl* c) {
    typedef typename std::conditional<MODE == MODE_SWEEP64, double, float>::type T;
    extern __shared__ __align__(128) unsigned char rsm[];
    __shared__ long long s_k, s_max, s_spin;
    __shared__ int s_held, s_fail, s_nin, s_dn;
    __shared__ double s_dt;
    LagState S;
    int64_t s0, s1;
    res_range(A.nslices, &s0, &s1);
    const int64_t nsl = s1 - s0;
    const int n = NN > 0 ? NN : A.n;
    constexpr bool IDX2 = I16 || FAR;   // 2-byte index planes
    const ResLayout L = res_layout(nsl, n, (int)sizeof(T), IDX2 ? 2 : 4, A.halo,
                                   FAR ? A.fl_max : 0);
    const int32_t f0 = FAR ? A.fl_off[blockIdx.x] : 0;
    const int32_t nfar = FAR ? A.fl_off[blockIdx.x + 1] - f0 : 0;
    T* w_s = reinterpret_cast<T*>(rsm + L.w);
    unsigned char* idx_s = rsm + L.idx;
    T* f_s = reinterpret_cast<T*>(rsm + L.f);
    T* o_s = reinterpret_cast<T*>(rsm + L.o);
    uint16_t* ord = reinterpret_cast<uint16_t*>(rsm + L.ord);
    T* h_s = reinterpret_cast<T*>(rsm + L.h);
    // the halo window: the block's rows and A.halo slots on either side, its
    // start rounded down and its length down to 16-byte multiples (a TMA bulk
    // copy's rule), within [0, N)
    // (A.halo < 0: no window, every gather through L2)
    const int64_t lo64 = max((int64_t)0, s0 * SLICE - A.halo) & ~(int64_t)3;
    const int64_t hi64 = min(A.N, s1 * SLICE + A.halo);
    const uint32_t W =
        A.halo >= 0 && hi64 > lo64 ? (uint32_t)((hi64 - lo64) & ~(int64_t)3) : 0u;
    const int32_t lo = (int32_t)lo64;
    // the block's own rows: slots [r0, r0 + nown); in the index planes they
    // are the values [obase, obase + nown) (FAR: window positions)
    const int64_t r0 = s0 * SLICE;
    const int32_t nown = (int32_t)max((int64_t)0, min(s1 * SLICE, A.NI) - r0);
    const int32_t obase = FAR ? (int32_t)(r0 - lo64) : (int32_t)r0;
    const uint32_t mbar = smem_addr(rsm);
    if (threadIdx.x == 0) {
        volatile StepCtrl* vc = c;
        s_k = vc->k;
        s_max = vc->max_steps;
        s_dt = vc->dt;
        constexpr long long dflt = SPIN_LIMIT_CYCLES;
        const long long lim = vc->spin_limit;
        s_spin = lim > 0 ? lim : dflt;
        s_held = vc->held;
        s_fail = 0;
        S.R0 = vc->res_first;
        S.tol = vc->tol;
        S.kmax = vc->max_steps;
        S.pend = 0ull;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // stage the block's planes: one thread announces the bytes and issues the
    // bulk copies in chunks; sources and destinations are 16-byte aligned and
    // every size a multiple of 16 (planes of 32 rows of 2-, 4- or 8-byte entries)
    const unsigned ent = (unsigned)(nsl * n * SLICE);
    const unsigned wb = ent * (unsigned)sizeof(T), ib = ent * (IDX2 ? 2u : 4u);
    const unsigned fb = (unsigned)(nsl * SLICE) * (unsigned)sizeof(T);
    if (threadIdx.x == 0 && nsl > 0) {
        const T* wg = (MODE == MODE_SWEEP64 ? (const T*)(const void*)A.w64
                                            : (const T*)(const void*)A.w32) +
                      s0 * (int64_t)n * SLICE;
        const unsigned char* ig =
            FAR   ? (const unsigned char*)(A.fl_idx + s0 * (int64_t)n * SLICE)
            : I16 ? (const unsigned char*)(A.col16 + s0 * (int64_t)n * SLICE)
                  : (const unsigned char*)(A.col + s0 * (int64_t)n * SLICE);
        const T* fg = (MODE == MODE_SWEEP64 ? (const T*)(const void*)A.f
                                            : (const T*)(const void*)A.d32) +
                      s0 * SLICE;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                     "r"(wb + ib + fb) : "memory");
        const void* src[3] = {wg, ig, fg};
        const uint32_t dst[3] = {smem_addr(w_s), smem_addr(idx_s), smem_addr(f_s)};
        const unsigned bytes[3] = {wb, ib, fb};
        for (int q = 0; q < 3; ++q)
            for (unsigned o = 0; o < bytes[q]; o += RES_COPY_CHUNK) {
                const unsigned sz = min(RES_COPY_CHUNK, bytes[q] - o);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                    "[%0], [%1], %2, [%3];" ::"r"(dst[q] + o),
                    "l"((const unsigned char*)src[q] + o), "r"(sz), "r"(mbar)
                    : "memory");
            }
    } else if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
    }
    // the rows' f (or the inner sweep's d32) beyond NI in the last slice are
    // padding of the plan's arrays; the planes stay valid for every row < NI
    if (!mbar_wait(mbar, 0, s_spin)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
        // give the copies a second bounded wait before the block leaves
        if (threadIdx.x == 0) {
            atomicExch(&c->done, DONE_TIMEOUT);
            mbar_wait(mbar, 0, s_spin);
        }
        __syncthreads();
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = TH / 32;
    // order the slices, inner first (flags in the own-row buffer, which the
    // first step's rows overwrite)
    {
        unsigned char* inner = reinterpret_cast<unsigned char*>(o_s);
        for (int64_t ls = warp; ls < nsl; ls += NW) {
            const int64_t row = (s0 + ls) * SLICE + lane;
            bool in = true;
            if (row < A.NI) {
                const int64_t eo = ls * (int64_t)n * SLICE + lane;
                const int4 sb = (I16 && !FAR) ? __ldg(A.sbase + s0 + ls) : make_int4(0, 0, 0, 0);
                for (int j = 0; j < n; ++j)
                    in = in && (uint32_t)(res_col<I16, FAR>(idx_s, eo + j * SLICE, sb) - obase) <
                                   (uint32_t)nown;
            }
            in = __all_sync(0xffffffffu, in);
            if (lane == 0) inner[ls] = in ? 1 : 0;
        }
        __syncthreads();
        if (warp == 0) {
            const unsigned below = (1u << lane) - 1u;
            int nin = 0;
            for (int64_t b = 0; b < nsl; b += 32)
                nin += __popc(__ballot_sync(0xffffffffu, b + lane < nsl && inner[b + lane]));
            int pi = 0, ph = nin;
            for (int64_t b = 0; b < nsl; b += 32) {
                const bool valid = b + lane < nsl;
                const bool f = valid && inner[b + lane];
                const unsigned bi = __ballot_sync(0xffffffffu, f);
                const unsigned bh = __ballot_sync(0xffffffffu, valid && !f);
                if (f) ord[pi + __popc(bi & below)] = (uint16_t)(b + lane);
                else if (valid) ord[ph + __popc(bh & below)] = (uint16_t)(b + lane);
                pi += __popc(bi);
                ph += __popc(bh);
            }
            if (lane == 0) s_nin = nin;
        }
        __syncthreads();
    }
    const int npre_max = s_nin;
    // a resident plan's slots fit 32 bits (its share of every SM's shared memory)
    const int32_t r0i = (int32_t)r0, NI32 = (int32_t)A.NI;
    const double dt = s_dt;
    const float dt32 = (float)dt;
    const long long kmax = s_max, k0 = s_k, spin = s_spin;
    const int held = s_held;
    for (long long k = k0; k < kmax; ++k) {
        const int par = (int)(k & 1);
        const T* ucur = MODE == MODE_SWEEP64 ? (const T*)(const void*)(par ? A.u1 : A.u0)
                                             : (const T*)(const void*)(par ? A.e1 : A.e0);
        T* unext = MODE == MODE_SWEEP64 ? (T*)(void*)(par ? A.u0 : A.u1)
                                        : (T*)(void*)(par ? A.e0 : A.e1);
        // the own-row buffers: u^k (read by phase 1) and u^{k+1} (written)
        const T* o_cur = o_s + (k & 1) * (int64_t)(nsl * SLICE);
        T* o_next = o_s + ((k + 1) & 1) * (int64_t)(nsl * SLICE);
        // phase 1 (from the second step on): inner slices
        const int npre = k > k0 ? npre_max : 0;
        unsigned long long m = 0;
        if (warp == 0) {
            if (lane == 0) {
                // the barrier of step k - 1 and its stop decision, then this
                // step's halo window of the iterate (one bulk copy on the
                // mbarrier's next phase).  The other blocks' writes of the
                // previous step were acquired at the barrier; the proxy fence
                // orders them before the copy, which reads through the async proxy.
                const bool ok = k == k0 || res_wait(c, S, k - 1, k0, spin, held);
                s_fail = ok ? 0 : 1;
                if (ok && A.halo >= 0) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    if (W > 0) {
                        const unsigned hb = W * (unsigned)sizeof(T);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                         mbar),
                                     "r"(hb) : "memory");
                        for (unsigned o = 0; o < hb; o += RES_COPY_CHUNK)
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                                "[%0], [%1], %2, [%3];" ::"r"(smem_addr(h_s) + o),
                                "l"((const unsigned char*)(ucur + lo) + o),
                                "r"(min(RES_COPY_CHUNK, hb - o)), "r"(mbar)
                                : "memory");
                    } else {
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar)
                                     : "memory");
                    }
                }
            }
        } else {
            for (int i = warp - 1; i < npre; i += NW - 1) {
                const int ls = ord[i];
                const int32_t row = r0i + ls * SLICE + lane;
                if (row < NI32) {
                    const int32_t eo = ls * n * SLICE + lane;
                    const int4 sb = (I16 && !FAR) ? __ldg(A.sbase + s0 + ls) : make_int4(0, 0, 0, 0);
                    const T acc = row_dot_own<NN, I16, FAR, T>(w_s + eo, idx_s, eo, sb, o_cur, obase, n);
                    const T ui = o_cur[row - r0i];
                    if constexpr (MODE == MODE_SWEEP64) {
                        const double r = __dsub_rn(acc, f_s[ls * SLICE + lane]);
                        o_next[row - r0i] = __fma_rn(dt, r, ui);
                        m = max(m, abs_bits(r));
                    } else {
                        const float rho = __fadd_rn(acc, f_s[ls * SLICE + lane]);
                        o_next[row - r0i] = __fmaf_rn(dt32, rho, ui);
                        m = max(m, abs_bits(rho));
                    }
                }
            }
        }
        __syncthreads();
        if (s_fail) return;   // the barrier gave up (done = DONE_TIMEOUT); no copy issued
        // phase 1's rows: to the iterate, now that no block reads its old
        // values (each thread its own rows: no barrier between)
        if (warp > 0)
            for (int i = warp - 1; i < npre; i += NW - 1) {
                const int32_t row = r0i + ord[i] * SLICE + lane;
                if (row < NI32) unext[row] = o_next[row - r0i];
            }
        // far values: plain loads through L2 (acquired at the barrier like the
        // window's source), stored behind the window - other addresses than
        // the bulk copy's, ordered for the readers by the barrier below
        if constexpr (FAR)
            for (int32_t i = threadIdx.x; i < nfar; i += TH)
                h_s[W + i] = ld_iter<true>(ucur + __ldg(A.fl_slot + f0 + i));
        // the stop decision for step k - 1 (its residual was loaded at the
        // barrier, off the path of this step's copy)
        if (threadIdx.x == 0) s_dn = k > k0 ? res_decide(c, S, k - 1) : DONE_RUNNING;
        const uint32_t phase = (uint32_t)((k - k0 + 1) & 1);
        if (A.halo >= 0 && !mbar_wait(mbar, phase, spin)) s_fail = 1;
        __syncthreads();
        // the run stopped after step k - 1: its result u^k is complete (phase
        // 1 wrote only the other buffer) and this step's copy has landed
        if (s_dn != DONE_RUNNING && !s_fail) return;
        if (s_fail) {
            if (threadIdx.x == 0) {
                atomicExch(&c->done, DONE_TIMEOUT);
                mbar_wait(mbar, phase, spin);
            }
            __syncthreads();
            return;
        }
        // phase 2: the other slices, from the window (and L2); every row's
        // u^{k+1} also goes to the own-row buffer for the next step's phase 1
        for (int i = npre + warp; i < nsl; i += NW) {
            const int ls = ord[i];
            const int32_t row = r0i + ls * SLICE + lane;
            if (row >= NI32) continue;
            const int32_t eo = ls * n * SLICE + lane;
            const int4 sb = (I16 && !FAR) ? __ldg(A.sbase + s0 + ls) : make_int4(0, 0, 0, 0);
            const void* cp = IDX2 ? (const void*)((const uint16_t*)idx_s + eo)
                                  : (const void*)((const int32_t*)idx_s + eo);
            if constexpr (MODE == MODE_SWEEP64) {
                const double* uin = (const double*)(const void*)ucur;
                const double ui = FAR ? ((const double*)h_s)[row - lo]
                                      : res_u<double>((const double*)h_s, lo, W, uin,
                                                      row);
                const double acc =
                    FAR ? row_dot_far<NN, double>(w_s + eo, (const uint16_t*)cp,
                                                  (const double*)h_s, n)
                        : row_dot_res<NN, I16, double>(w_s + eo, cp, sb, (const double*)h_s, lo,
                                                       W, uin, n);
                const double r = __dsub_rn(acc, f_s[ls * SLICE + lane]);
                const double v = __fma_rn(dt, r, ui);
                unext[row] = v;
                o_next[row - r0i] = v;
                m = max(m, abs_bits(r));
            } else {
                const float* ein = (const float*)(const void*)ucur;
                const float ei = FAR ? ((const float*)h_s)[row - lo]
                                     : res_u<float>((const float*)h_s, lo, W, ein, row);
                const float acc =
                    FAR ? row_dot_far<NN, float>(w_s + eo, (const uint16_t*)cp,
                                                 (const float*)h_s, n)
                        : row_dot_res<NN, I16, float>(w_s + eo, cp, sb, (const float*)h_s, lo, W,
                                                      ein, n);
                const float rho = __fadd_rn(acc, f_s[ls * SLICE + lane]);
                const float v = __fmaf_rn(dt32, rho, ei);
                unext[row] = v;
                o_next[row - r0i] = v;
                m = max(m, abs_bits(rho));
            }
        }
        m = res_block_max<TH>(m);
        if (threadIdx.x == 0) res_arrive(c, k, m);
    }
    // the last step's barrier and decision: it stops the run
    if (kmax > k0 && threadIdx.x == 0 && res_wait(c, S, kmax - 1, k0, spin, held))
        res_decide(c, S, kmax - 1);
}

}  // namespace rbffd
