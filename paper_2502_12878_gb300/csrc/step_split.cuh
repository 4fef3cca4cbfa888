// Split persistent launch of the explicit sweep (Eq. 6) for plans whose
// stencils stream from HBM every step: one block per SM owns a contiguous
// share of the slices (the resident launch's partition), keeps the iterate of
// its own rows in shared memory (two buffers: u^k and u^{k+1}) and splits
// every step in two.  The inner slices - rows whose supports lie inside the
// share, which plan creation puts first in each share - need only the
// block's own u^k, so they are computed while warp 0 waits at the barrier of
// the previous step; their results go to the iterate once that barrier has
// passed (a slower block may still be reading the buffer they overwrite).
// Then all warps compute the remaining slices, gathering the other shares'
// rows through L2.  The stencil planes are streamed as in the one-launch-
// per-step kernel, and each row's arithmetic is the same fused multiply-add
// chain, so the results are the same bit for bit.
#pragma once

#include "step_res.cuh"

namespace rbffd {

// shared memory of one block: the two own-row buffers
__host__ __device__ __forceinline__ unsigned split_smem_bytes(int64_t nsl, int wbytes) {
    return res_align((unsigned)(2 * nsl * SLICE) * (unsigned)wbytes);
}

// sum_j w_j u[col_j], the planes streamed (indices, weights, then the
// gathers, CH at a time, as row_dot); the iterate from the own-row buffer o
// (at c - r0) where the column is a row of the block, else through L2.  OWN:
// every column is.
template <int NN, bool OWN, bool I16, int CH, class T>
__device__ __forceinline__ T row_dot_split(const T* __restrict__ w, const void* __restrict__ colp,
                                           const int4& sb, const T* o, int32_t r0, uint32_t nown,
                                           const T* __restrict__ u, int n) {
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
            if (j0 + t < nn) {
                const uint32_t q = (uint32_t)(c[t] - r0);
                if constexpr (OWN) uv[t] = o[q];
                else uv[t] = q < nown ? o[q] : ld_iter<true>(u + c[t]);
            }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < nn) {
                if constexpr (sizeof(T) == 8) acc = __fma_rn(wv[t], uv[t], acc);
                else acc = __fmaf_rn(wv[t], uv[t], acc);
            }
    }
    return acc;
}

// |x| of a float as IEEE bits, NaN mapped to +Inf: orders like |x| (widened to
// double once per step, it gives the residual slot's bits without an FP64
// conversion per row)
__device__ __forceinline__ unsigned abs_bits32(float x) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    return b > 0x7f800000u ? 0x7f800000u : b;
}

// one row of the split launch: its stencil from the packed planes (16-bit
// codes where the slice has them), u_i from the own-row buffer; returns the
// new value and folds |r| into m (FP64: as double bits; FP32 inner sweep: as
// float bits, widened at the step's end)
template <int NN, int MODE, bool OWN, int TH, class T>
__device__ __forceinline__ T split_row(const StepArgs& A, int64_t sl, int32_t row, int lane,
                                       const T* o, int32_t r0, uint32_t nown, const T* u,
                                       double dt, float dt32, unsigned long long& m) {
    const int64_t base = sl * (int64_t)A.n * SLICE + lane;
    const int4 sb = A.col16 ? __ldg(A.sbase + sl) : make_int4(-1, -1, -1, -1);
    // loads in flight per thread: fewer for the generic size and in the FP64
    // 1024-thread blocks (64 registers), so nothing spills (12 fit from n = 30
    // on, 8 for the smaller sizes: by the compiler's register report)
    constexpr int CH = NN == 0                                    ? 8
                       : !(MODE == MODE_SWEEP64 && TH >= 1024)    ? 16
                       : NN >= 30                                 ? 12
                                                                  : 8;
    if constexpr (MODE == MODE_SWEEP64) {
        const double fi = ld_stream(A.f + row);
        const double ui = o[row - r0];
        const double acc =
            sb.x >= 0 ? row_dot_split<NN, OWN, true, CH, double>(A.w64 + base, A.col16 + base, sb, o,
                                                             r0, nown, u, A.n)
                      : row_dot_split<NN, OWN, false, CH, double>(A.w64 + base, A.col + base, sb, o,
                                                              r0, nown, u, A.n);
        const double r = __dsub_rn(acc, fi);
        m = max(m, abs_bits(r));
        return __fma_rn(dt, r, ui);
    } else {
        const float di = ld_stream(A.d32 + row);
        const float ei = o[row - r0];
        const float acc =
            sb.x >= 0 ? row_dot_split<NN, OWN, true, CH, float>(A.w32 + base, A.col16 + base, sb, o,
                                                            r0, nown, u, A.n)
                      : row_dot_split<NN, OWN, false, CH, float>(A.w32 + base, A.col + base, sb, o,
                                                             r0, nown, u, A.n);
        const float rho = __fadd_rn(acc, di);
        m = max(m, (unsigned long long)abs_bits32(rho));
        return __fmaf_rn(dt32, rho, ei);
    }
}

// release / acquire of a flag in shared memory at block scope: what warp 0
// acquired at the step barrier (the other blocks' iterate writes) is ordered
// before what the warps that read the flag do next
__device__ __forceinline__ void st_release_cta(unsigned* p, unsigned v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v)
                 : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cta(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p))
                 : "memory");
    return v;
}

// All steps of a run in one cooperative launch of one block of TH threads
// per SM (the grid is the SM count; block b owns slices [nslices b / G,
// nslices (b+1) / G)).  Within a step no block-wide barrier separates the two
// halves: each warp computes its share of the inner slices, waits for warp
// 0's flag that the step barrier has passed, stores its inner rows, and then
// takes the remaining slices one at a time from a shared counter, so their
// L2-bound gathers overlap the other warps' inner slices.
template <int NN, int MODE, int TH>
__global__ void __launch_bounds__(TH, 1) split_kernel(StepArgs A, StepCtrl* c) {
    typedef typename std::conditional<MODE == MODE_SWEEP64, double, float>::type T;
    extern __shared__ __align__(128) unsigned char ssm[];
    __shared__ long long s_k, s_max, s_spin;
    __shared__ int s_held, s_fail, s_dn, s_next;
    __shared__ unsigned s_go;   // steps whose barrier warp 0 has passed (k - k0 + 1)
    __shared__ double s_dt;
    __shared__ float s_dt32;
    // the stop decision's state lives in shared memory: only thread 0 uses it,
    // and registers are the 1024-thread blocks' tight budget
    __shared__ LagState S;
    int64_t s0w, s1w;
    res_range(A.nslices, &s0w, &s1w);
    // a share's slots fit 32 bits (its own rows sit in shared memory)
    const int32_t s0 = (int32_t)s0w, nsl = (int32_t)(s1w - s0w);
    const int32_t r0 = s0 * SLICE;
    const int32_t NI32 = (int32_t)A.NI;
    const int32_t nown = max(0, min((int32_t)(s1w * SLICE), NI32) - r0);
    T* o_s = reinterpret_cast<T*>(ssm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = TH / 32;
    if (threadIdx.x == 0) {
        volatile StepCtrl* vc = c;
        s_k = vc->k;
        s_max = vc->max_steps;
        s_dt = vc->dt;
        s_dt32 = (float)vc->dt;
        constexpr long long dflt = SPIN_LIMIT_CYCLES;
        const long long lim = vc->spin_limit;
        s_spin = lim > 0 ? lim : dflt;
        s_held = vc->held;
        s_fail = 0;
        s_dn = DONE_RUNNING;
        S.R0 = vc->res_first;
        S.tol = vc->tol;
        S.kmax = vc->max_steps;
        S.pend = 0ull;
    }
    __syncthreads();
    const long long kmax = s_max, k0 = s_k, spin = s_spin;
    const int held = s_held;
    const int32_t rows = nsl * SLICE;
    // the own rows of u^{k0} into the buffer of step k0
    {
        const int par = (int)(k0 & 1);
        const T* u0 = MODE == MODE_SWEEP64 ? (const T*)(const void*)(par ? A.u1 : A.u0)
                                           : (const T*)(const void*)(par ? A.e1 : A.e0);
        T* o0 = o_s + (k0 & 1) * rows;
        for (int32_t i = threadIdx.x; i < nown; i += TH) o0[i] = ld_iter<true>(u0 + r0 + i);
    }
    // the share's leading slices of inner rows (plan creation ordered them first)
    const int npre = min(A.inner[blockIdx.x], nsl);
    if (threadIdx.x == 0) {
        s_next = npre;
        s_go = 0u;
    }
    __syncthreads();
    for (long long k = k0; k < kmax; ++k) {
        const int par = (int)(k & 1);
        const T* ucur = MODE == MODE_SWEEP64 ? (const T*)(const void*)(par ? A.u1 : A.u0)
                                             : (const T*)(const void*)(par ? A.e1 : A.e0);
        T* unext = MODE == MODE_SWEEP64 ? (T*)(void*)(par ? A.u0 : A.u1)
                                        : (T*)(void*)(par ? A.e0 : A.e1);
        const T* o_cur = o_s + (k & 1) * rows;
        T* o_next = o_s + ((k + 1) & 1) * rows;
        const unsigned go = (unsigned)(k - k0 + 1);
        unsigned long long m = 0;
        if (warp == 0) {
            // the barrier of step k - 1 and its stop decision, then the flag
            if (lane == 0) {
                bool ok = true;
                int dn = DONE_RUNNING;
                if (k > k0) {
                    ok = res_wait(c, S, k - 1, k0, spin, held);
                    dn = ok ? res_decide(c, S, k - 1) : DONE_RUNNING;
                }
                s_fail = ok ? 0 : 1;
                s_dn = dn;
                st_release_cta(&s_go, go);
            }
            __syncwarp();
        } else {
            // inner slices, from the block's own u^k only; one lane prefetches
            // the warp's next slice's planes into L2 where that pays (as in the
            // one-launch-per-step kernel)
            for (int i = warp - 1; i < npre; i += NW - 1) {
                if ((MODE == MODE_INNER32 || (NN > 0 && NN <= PF64_MAX_N)) && lane == 0 &&
                    i + NW - 1 < npre)
                    prefetch_planes<MODE>(A, s0 + i + NW - 1);
                const int32_t row = r0 + i * SLICE + lane;
                if (row < NI32)
                    o_next[row - r0] =
                        split_row<NN, MODE, true, TH, T>(A, s0 + i, row, lane, o_cur, r0,
                                                         (uint32_t)nown, ucur, s_dt, s_dt32, m);
            }
            // warp 0's flag (its own wait is bounded by `spin`)
            if (lane == 0) {
                const long long t0 = clock64();
                while (ld_acquire_cta(&s_go) != go)
                    if (clock64() - t0 > 4 * spin) {
                        atomicExch(&c->done, DONE_TIMEOUT);
                        break;
                    }
            }
            __syncwarp();
        }
        // the barrier gave up (done = DONE_TIMEOUT), or the run stopped after
        // step k - 1 (its result u^k complete; nothing of step k stored)
        if (s_fail || s_dn != DONE_RUNNING || ld_acquire_cta(&s_go) != go) return;
        // the inner rows to the iterate, now that no block reads its old values
        // (each thread its own rows)
        if (warp > 0)
            for (int i = warp - 1; i < npre; i += NW - 1) {
                const int32_t row = r0 + i * SLICE + lane;
                if (row < NI32) unext[row] = o_next[row - r0];
            }
        // the other slices, one at a time from the shared counter: the other
        // shares' rows of u^k through L2
        for (;;) {
            int i = 0;
            if (lane == 0) i = atomicAdd(&s_next, 1);
            i = __shfl_sync(0xffffffffu, i, 0);
            if (i >= nsl) break;
            const int32_t row = r0 + i * SLICE + lane;
            if (row < NI32) {
                const T v = split_row<NN, MODE, false, TH, T>(A, s0 + i, row, lane, o_cur, r0,
                                                              (uint32_t)nown, ucur, s_dt, s_dt32, m);
                unext[row] = v;
                o_next[row - r0] = v;
            }
        }
        if constexpr (MODE == MODE_INNER32) m = abs_bits((double)__uint_as_float((unsigned)m));
        m = res_block_max<TH>(m);
        if (threadIdx.x == 0) {
            res_arrive(c, k, m);
            s_next = npre;   // every warp is past this step's counter
        }
    }
    // the last step's barrier and decision: it stops the run
    if (kmax > k0 && threadIdx.x == 0 && res_wait(c, S, kmax - 1, k0, spin, held))
        res_decide(c, S, kmax - 1);
}

// kernel of the split launch for stencil size n, mode and block size (512, or
// 1024 for the compiled sizes from 12 on; nullptr otherwise), and its dynamic
// shared memory with `grid` blocks
StepFn pick_split(int mode, int n, int threads);
unsigned split_smem(int64_t nslices, int mode, int grid);

}  // namespace rbffd
