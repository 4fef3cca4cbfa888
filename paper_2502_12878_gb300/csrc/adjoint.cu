// rbffd_adjoint: reverse sweep of K explicit steps of Eq. 6 (the adjoint is
// an addition of this library; the paper only runs the forward iteration).
//
// The forward step is u^{k+1}_I = u^k_I + dt (W_II u^k_I + W_IB g - f).  Its
// transpose needs W^T: built once per plan as a column-major copy of the
// packed stencils (count per column, scan, scatter, then each column's
// entries sorted by the caller's interior row so every column sums in the
// same order as a row-ascending scatter would).  The columns are stored as
// 32-column slices [slice][j][lane] padded to the slice's longest column with
// zero weights, so the reverse step is the same coalesced thread-per-column
// gather as the forward sweep - no atomics, deterministic.  As in the forward
// layout, an interior slice whose rows fit in four windows of 2^14 placed
// positions also stores each row as a 16-bit code (window in bits 15..14,
// offset from the window's base in 13..0), which the reverse step reads
// instead of the int32 row: 10 bytes per entry instead of 12.
#include <math.h>

#include <algorithm>

#include "plan.cuh"

namespace rbffd {

// Interior columns are placed within windows of TR_WINDOW consecutive slots by
// decreasing length (ties by slot), so a slice holds columns of nearly equal
// length and little padding; a window of consecutive Morton slots is a small
// patch of the domain, so the gathers stay local.  Everything indexed by an
// interior column or row (lambda, S, the rows of the entries) is held in that
// placed order; boundary columns keep their slots.
static constexpr int TR_WINDOW = 256;

typedef void (*AdjStepFn)(const struct Transpose, const int64_t, const double, const double*,
                          double*, double*);

struct Transpose {
    int64_t nslices = 0;      // over all N columns (placed order)
    AdjStepFn step = nullptr; // the reverse-step shape the tuner picked (on first use)
    unsigned step_grid = 0;   // and its grid
    bool step_pdl = false;    // and whether consecutive steps are programmatic dependent launches
    int64_t* off = nullptr;   // [nslices + 1] element offset of each slice
    int32_t* len = nullptr;   // [nslices] padded length of each slice
    int32_t* row = nullptr;   // placed position of each entry's row
    double* w = nullptr;      // weight of each entry (0 for padding)
    // 16-bit row codes (NULL when the plan keeps int32 indices) and per
    // interior slice its four window bases (x = -1: the slice reads row)
    uint16_t* row16 = nullptr;
    int4* tbase = nullptr;
    int64_t entries = 0;      // stored entries of the interior slices
    int64_t cols16 = 0;       // interior columns in slices with codes
    int64_t entries16 = 0;    // and those slices' stored entries
    int32_t* colof = nullptr; // [N] slot of the column at each placed position
    int32_t* posof = nullptr; // [N] placed position of each slot
    double* lam[2] = {nullptr, nullptr};   // [NI] placed order
    double* S = nullptr;      // [NI] sum of lambda^k, placed order
};

void free_transpose(rbffd_plan* p) {
    if (!p || !p->tr) return;
    Transpose* t = p->tr;
    void* b[] = {t->off,   t->len,   t->row,    t->w,      t->colof, t->posof,
                 t->lam[0], t->lam[1], t->S,      t->row16,  t->tbase};
    for (void* x : b)
        if (x) cudaFree(x);
    delete t;
    p->tr = nullptr;
}

__global__ void tr_count(const int32_t* col, int64_t NI, int n, int32_t* cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t base = (p / SLICE) * (int64_t)n * SLICE + (p % SLICE);
        for (int j = 0; j < n; ++j) atomicAdd(&cnt[col[base + j * SLICE]], 1);
    }
}

__global__ void tr_scatter(const int32_t* col, const double* w64, const int32_t* row_of_slot,
                           int64_t NI, int n, int32_t* cursor, int32_t* erow, int32_t* ekey,
                           double* ew) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t base = (p / SLICE) * (int64_t)n * SLICE + (p % SLICE);
        for (int j = 0; j < n; ++j) {
            int c = col[base + j * SLICE];
            int pos = atomicAdd(&cursor[c], 1);
            erow[pos] = (int32_t)p;
            ekey[pos] = row_of_slot[p];
            ew[pos] = w64[base + j * SLICE];
        }
    }
}

// each column's entries into ascending caller row order
__global__ void tr_sort(const int32_t* start, int64_t N, int32_t* erow, int32_t* ekey, double* ew) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        int b = start[c], e = start[c + 1];
        for (int i = b + 1; i < e; ++i) {
            int32_t k = ekey[i], r = erow[i];
            double wv = ew[i];
            int j = i - 1;
            while (j >= b && ekey[j] > k) {
                ekey[j + 1] = ekey[j];
                erow[j + 1] = erow[j];
                ew[j + 1] = ew[j];
                --j;
            }
            ekey[j + 1] = k;
            erow[j + 1] = r;
            ew[j + 1] = wv;
        }
    }
}

// placement of the interior columns: one warp per window ranks each column
// by (length descending, slot ascending); boundary columns stay in place
__global__ void tr_place(const int32_t* start, int64_t NI, int64_t N, int32_t* colof,
                         int32_t* posof) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nwin = (NI + TR_WINDOW - 1) / TR_WINDOW;
    for (int64_t win = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); win < nwin;
         win += nw) {
        const int64_t c0 = win * TR_WINDOW, c1 = min(NI, c0 + TR_WINDOW);
        for (int64_t c = c0 + lane; c < c1; c += 32) {
            const int lc = start[c + 1] - start[c];
            int rank = 0;
            for (int64_t q = c0; q < c1; ++q) {
                const int lq = start[q + 1] - start[q];
                rank += (lq > lc) || (lq == lc && q < c);
            }
            colof[c0 + rank] = (int32_t)c;
            posof[c] = (int32_t)(c0 + rank);
        }
    }
    for (int64_t c = NI + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        colof[c] = (int32_t)c;
        posof[c] = (int32_t)c;
    }
}

__global__ void tr_slice_len(const int32_t* start, const int32_t* colof, int64_t N, int64_t nsl,
                             int32_t* len, int64_t* size) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsl;
         s += (int64_t)gridDim.x * blockDim.x) {
        int L = 0;
        for (int l = 0; l < SLICE; ++l) {
            int64_t q = s * SLICE + l;
            if (q < N) {
                const int32_t c = colof[q];
                L = max(L, start[c + 1] - start[c]);
            }
        }
        len[s] = L;
        size[s] = (int64_t)L * SLICE;
    }
}

__global__ void tr_fill(const int32_t* start, const int32_t* erow, const double* ew,
                        const int32_t* colof, const int32_t* posof, int64_t N, int64_t nsl,
                        const int64_t* off, const int32_t* len, int32_t* trow, double* tw) {
    const int64_t total = nsl * SLICE;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = q / SLICE, l = q % SLICE;
        int L = len[s];
        const int32_t c = q < N ? colof[q] : 0;
        int b = q < N ? start[c] : 0, e = q < N ? start[c + 1] : 0;
        for (int j = 0; j < L; ++j) {
            int64_t o = off[s] + (int64_t)j * SLICE + l;
            if (b + j < e) {
                trow[o] = posof[erow[b + j]];
                tw[o] = ew[b + j];
            } else {
                trow[o] = 0;
                tw[o] = 0.0;
            }
        }
    }
}

// 16-bit row codes of the interior slices (one warp per slice): the fewest
// windows of 2^14 placed positions, greedy from the left, that cover every
// stored row of the slice's interior columns.  Padding entries (and the lanes
// of boundary columns, which the reverse step skips) get code 0, i.e. the
// first window's base: a row of this slice, read with weight 0 as the int32
// padding reads row 0.  A slice that needs more than four windows (tbase x =
// -1) stores as each entry's code its own position in the slice, through
// which the reverse step reads the int32 row: one code form for every slice,
// so the reverse step has one loop.
static constexpr int32_t TR_WINDOW16 = 1 << 14;

__global__ void tr_pack16(const int32_t* __restrict__ start, const int32_t* __restrict__ colof,
                          int64_t NI, int64_t nsl_int, const int64_t* __restrict__ off,
                          const int32_t* __restrict__ len, const int32_t* __restrict__ trow,
                          uint16_t* __restrict__ row16, int4* __restrict__ tbase,
                          unsigned long long* cnt, int* err) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < nsl_int;
         sl += nw) {
        const int64_t q = sl * SLICE + lane;
        const bool valid = q < NI;
        int Lc = 0;   // this column's stored (unpadded) entries
        if (valid) {
            const int32_t c = colof[q];
            Lc = start[c + 1] - start[c];
        }
        const int L = len[sl];
        const int64_t base = off[sl] + lane;
        int32_t b[4];
        int64_t thr = INT64_MIN;   // rows >= thr are not yet covered
        int used = 0;
        for (int k = 0; k < 4; ++k) {
            int32_t mn = INT32_MAX;
            for (int j = 0; j < Lc; ++j) {
                const int32_t v = trow[base + (int64_t)j * SLICE];
                if ((int64_t)v >= thr) mn = min(mn, v);
            }
            mn = __reduce_min_sync(0xffffffffu, mn);
            if (mn == INT32_MAX) break;   // warp-uniform
            b[k] = mn;
            used = k + 1;
            thr = (int64_t)mn + TR_WINDOW16;
        }
        for (int k = used; k < 4; ++k) b[k] = used ? b[used - 1] : 0;
        bool left = false;
        for (int j = 0; j < Lc; ++j) left |= (int64_t)trow[base + (int64_t)j * SLICE] >= thr;
        const bool wide = __any_sync(0xffffffffu, left) && used == 4;
        if (lane == 0)
            tbase[sl] = wide ? make_int4(-1, -1, -1, -1) : make_int4(b[0], b[1], b[2], b[3]);
        if (wide) {   // each entry's code is its own position j * 32 + lane (< 2^16)
            for (int j = 0; j < L; ++j)
                row16[base + (int64_t)j * SLICE] = (uint16_t)(j * SLICE + lane);
            continue;
        }
        const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, valid));
        if (lane == 0) {
            atomicAdd(&cnt[0], (unsigned long long)nvalid);
            atomicAdd(&cnt[1], (unsigned long long)L * SLICE);
        }
        for (int j = 0; j < L; ++j) {
            uint16_t code = 0;
            if (j < Lc) {
                const int32_t v = trow[base + (int64_t)j * SLICE];
                const int k = (v >= b[1]) + (v >= b[2]) + (v >= b[3]);
                const int32_t o = v - (k == 0 ? b[0] : k == 1 ? b[1] : k == 2 ? b[2] : b[3]);
                if (o < 0 || o >= TR_WINDOW16) atomicExch(err, 1);   // cannot happen
                code = (uint16_t)(((uint32_t)k << 14) | ((uint32_t)o & 0x3fffu));
            }
            row16[base + (int64_t)j * SLICE] = code;
        }
    }
}

// exclusive scan of int64 slice sizes (single block; slice counts are modest)
__global__ void scan64_single(const int64_t* in, int64_t n, int64_t* out) {
    __shared__ int64_t carry;
    __shared__ int64_t buf[256];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += 256) {
        int64_t i = b + threadIdx.x;
        buf[threadIdx.x] = i < n ? in[i] : 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t run = carry;
            for (int k = 0; k < 256 && b + k < n; ++k) {
                int64_t v = buf[k];
                out[b + k] = run;
                run += v;
            }
            carry = run;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// Ordered streaming loads: asm volatile keeps the loads of one phase ahead of
// the first use, so each thread has 2*CH loads and then CH gathers in flight
// (plain loads were issued one dependent pair at a time).  CH = 8 with four
// 256-thread blocks per SM fits 64 registers without spills.
__device__ __forceinline__ double adj_ld_cs(const double* p) {
    double v;
    asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t adj_ld_cs(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.cs.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t adj_ld_cs(const uint16_t* p) {
    unsigned short v;
    asm volatile("ld.global.cs.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return (uint32_t)v;
}
__device__ __forceinline__ double adj_ld_nc(const double* p) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

// 16-bit row code -> placed row: window k = code >> 14 selects one of the
// slice's four bases, plus the 14-bit offset
__device__ __forceinline__ int32_t adj_decode16(uint32_t v, const int4& b) {
    const uint32_t k = v >> 14;
    const int32_t base = (k & 2u) ? ((k & 1u) ? b.w : b.z) : ((k & 1u) ? b.y : b.x);
    return base + (int32_t)(v & 0x3fffu);
}

// sum over a column's L stored entries (stride SLICE) of w * lam[row], an fma
// chain from 0 in entry order; loads in phases of CH (rows, weights, then
// the gathers).  I16: rows as 16-bit codes against the slice's bases.
// sum over a column's L stored entries (stride SLICE) of w * lam[row], an fma
// chain from 0 in entry order; loads in phases of CH (rows, weights, then
// the gathers).  I16: each entry's 16-bit code is decoded against the
// slice's window bases, or, in a slice the windows cannot cover (sb.x < 0),
// is the entry's own position in the slice, which reads its int32 row.
template <int CH, bool I16>
__device__ __forceinline__ double adj_col_sum(const double* wp, const void* rp,
                                              const int32_t* rows, const int4& sb,
                                              const double* __restrict__ lam, int L) {
    double acc = 0.0;
    for (int j0 = 0; j0 < L; j0 += CH) {
        int32_t r[CH];
        double wv[CH], lv[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < L) {
                if constexpr (I16)
                    r[t] = (int32_t)adj_ld_cs((const uint16_t*)rp + (int64_t)(j0 + t) * SLICE);
                else
                    r[t] = adj_ld_cs((const int32_t*)rp + (int64_t)(j0 + t) * SLICE);
            }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < L) wv[t] = adj_ld_cs(wp + (int64_t)(j0 + t) * SLICE);
        if constexpr (I16) {
            if (sb.x >= 0) {
#pragma unroll
                for (int t = 0; t < CH; ++t)
                    if (j0 + t < L) r[t] = adj_decode16((uint32_t)r[t], sb);
            } else {
#pragma unroll
                for (int t = 0; t < CH; ++t)
                    if (j0 + t < L) r[t] = adj_ld_cs(rows + r[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < L) lv[t] = adj_ld_nc(lam + r[t]);
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (j0 + t < L) acc = __fma_rn(wv[t], lv[t], acc);
    }
    return acc;
}

// one reverse step over interior columns c < NI:
//   S_c += lam_c;  lam'_c = fma(dt, sum_rows w_rc lam_r, lam_c)
// the column sum is an fma chain from 0 over the column's entries in order
// (padding entries carry weight 0, so they add exact zeros).  Shapes: CH
// entries per load phase (rows, weights, then gathers) and a register budget
// for MINB resident blocks of 256 threads; every shape, and either row form,
// gives the same bits.  One lane prefetches the warp's next slice (weight
// plane and row codes, or rows when the plan keeps int32 indices) into L2:
// both planes start on 16-byte boundaries (slice offsets are multiples of 32
// entries) and span a multiple of 16 bytes.
template <int CH, bool I16>
__device__ __forceinline__ void adj_slices(const Transpose& T, const int64_t NI, const double dt,
                                           const double* __restrict__ lam,
                                           double* __restrict__ lam_out,
                                           double* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int64_t nsl_int = (NI + SLICE - 1) / SLICE;
    const int64_t stride = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); s < nsl_int;
         s += stride) {
        if (lane == 0 && s + stride < nsl_int) {
            const int64_t o = __ldg(T.off + s + stride);
            const unsigned Ln = (unsigned)__ldg(T.len + s + stride) * SLICE;
            if (Ln) {
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(T.w + o),
                             "r"(Ln * 8u) : "memory");
                if (I16)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(T.row16 + o),
                                 "r"(Ln * 2u) : "memory");
                else
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(T.row + o),
                                 "r"(Ln * 4u) : "memory");
            }
        }
        const int64_t c = s * SLICE + lane;
        if (c >= NI) continue;
        const int L = __ldg(T.len + s);
        const int64_t off = __ldg(T.off + s);
        double acc, lc, Sc;
        if constexpr (I16) {
            const int4 sb = __ldg(T.tbase + s);
            // (the window bases take the registers that would hold the
            // column's own lambda and S through the sum)
            acc = adj_col_sum<CH, true>(T.w + off + lane, T.row16 + off + lane, T.row + off, sb,
                                        lam, L);
            lc = lam[c];
            Sc = S[c];
        } else {
            // the column's own lambda and S are issued before the sum, so
            // their latency overlaps the entry loads
            lc = lam[c];
            Sc = S[c];
            acc = adj_col_sum<CH, false>(T.w + off + lane, T.row + off + lane, nullptr,
                                         make_int4(-1, -1, -1, -1), lam, L);
        }
        S[c] = __dadd_rn(Sc, lc);
        lam_out[c] = __fma_rn(dt, acc, lc);
    }
}

// As a programmatic dependent launch (the tuner's choice in rbffd_adjoint's
// step loop) a step waits for the previous step before its first read of
// lambda, and lets the next step's blocks be scheduled as its own blocks
// finish their slices; both are no-ops in a plain launch.
template <int CH, int MINB>
__global__ void __launch_bounds__(256, MINB)
adjoint_step(const Transpose T, const int64_t NI, const double dt,
             const double* __restrict__ lam, double* __restrict__ lam_out,
             double* __restrict__ S) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (T.row16) adj_slices<CH, true>(T, NI, dt, lam, lam_out, S);
    else adj_slices<CH, false>(T, NI, dt, lam, lam_out, S);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// boundary columns: grad_g[node] = dt * sum_rows w_rc S_r + dLdu[node] (the
// loss's direct dependence on u^K at a boundary node, where u^K = g)
__global__ void adjoint_grad_g(const Transpose T, const int64_t NI, const int64_t N,
                               const double dt, const double* __restrict__ S,
                               const int32_t* perm, const double* __restrict__ dLdu,
                               double* grad_g) {
    for (int64_t c = NI + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = c / SLICE, lane = c % SLICE;
        const int L = T.len[s];
        const int64_t o = T.off[s] + lane;
        double acc = 0.0;
        for (int j = 0; j < L; ++j)
            acc = __fma_rn(T.w[o + (int64_t)j * SLICE], S[T.row[o + (int64_t)j * SLICE]], acc);
        const int32_t node = perm[c];
        grad_g[node] = __dadd_rn(__dmul_rn(dt, acc), dLdu[node]);
    }
}

__global__ void adj_gather(const double* src, const int32_t* row_of_slot, int64_t NI,
                           double* dst) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = src[row_of_slot[p]];
}

// lambda^K = the interior entries of dL/du^K (caller's node order) into the
// placed order
__global__ void adj_gather_placed(const double* dLdu, const int32_t* perm, const int32_t* colof,
                                  int64_t NI, double* dst) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < NI;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = dLdu[perm[colof[q]]];
}

// S and lambda^0 (placed order) out to the caller's order
__global__ void adj_outputs(const double* S, const double* lam, const int32_t* row_of_slot,
                            const int32_t* colof, const int32_t* perm, int64_t NI, double dt,
                            double* grad_f, double* grad_g, double* lam0) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < NI;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = colof[q];
        const int32_t r = row_of_slot[c];
        grad_f[r] = __dmul_rn(-dt, S[q]);
        grad_g[perm[c]] = 0.0;
        if (lam0) lam0[r] = lam[q];
    }
}

// replay of one forward step (Eq. 6) from uin to uout, both in slot order:
// interior rows updated, boundary slots copied (the same arithmetic as the
// forward sweep, so the replayed iterates are the forward's bit for bit)
__global__ void __launch_bounds__(256, 4)
replay_step(const double* __restrict__ w64, const int32_t* __restrict__ col,
            const double* __restrict__ fs, const double* __restrict__ uin,
            double* __restrict__ uout, int64_t NI, int64_t N, int n, double dt) {
    constexpr int CH = 8;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (p >= NI) {
            uout[p] = uin[p];
            continue;
        }
        const int64_t base = (p / SLICE) * (int64_t)n * SLICE + (p % SLICE);
        double acc = 0.0;
        for (int j0 = 0; j0 < n; j0 += CH) {
            int32_t c[CH];
            double wv[CH], uv[CH];
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) c[t] = adj_ld_cs(col + base + (int64_t)(j0 + t) * SLICE);
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) wv[t] = adj_ld_cs(w64 + base + (int64_t)(j0 + t) * SLICE);
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) uv[t] = adj_ld_nc(uin + c[t]);
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) acc = __fma_rn(wv[t], uv[t], acc);
        }
        double r = __dsub_rn(acc, fs[p]);
        uout[p] = __fma_rn(dt, r, uin[p]);
    }
}

// weight-gradient accumulation with lambda^{k+1} and u^k in the slice layout:
// G[s][j][lane] = fma(lambda_p, u^k[col], G[s][j][lane])
__global__ void __launch_bounds__(256, 4)
wgrad_accum(const int32_t* __restrict__ col, const double* __restrict__ lam,
            const int32_t* __restrict__ posof, const double* __restrict__ uk,
            double* __restrict__ G, int64_t NI, int n) {
    constexpr int CH = 8;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = (p / SLICE) * (int64_t)n * SLICE + (p % SLICE);
        const double lp = lam[posof[p]];   // lambda is held in the placed order
        for (int j0 = 0; j0 < n; j0 += CH) {
            int32_t c[CH];
            double gv[CH], uv[CH];
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) c[t] = adj_ld_cs(col + base + (int64_t)(j0 + t) * SLICE);
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) gv[t] = G[base + (int64_t)(j0 + t) * SLICE];
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) uv[t] = adj_ld_nc(uk + c[t]);
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (j0 + t < n) G[base + (int64_t)(j0 + t) * SLICE] = __fma_rn(lp, uv[t], gv[t]);
        }
    }
}

// grad_w in the caller's layout [NI][n] = dt * G
__global__ void wgrad_unpack(const double* __restrict__ G, const int32_t* row_of_slot, int64_t NI,
                             int n, double dt, double* grad_w) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = (p / SLICE) * (int64_t)n * SLICE + (p % SLICE);
        const int64_t r = row_of_slot[p];
        for (int j = 0; j < n; ++j) grad_w[r * n + j] = __dmul_rn(dt, G[base + j * SLICE]);
    }
}

__global__ void ckpt_gather(const double* u, const int32_t* perm, int64_t N, double* out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = u[perm[p]];
}

// reverse-step shapes the tuner times: (phase width, register budget), each
// with one warp per slice (the full grid) or a grid-stride loop over slices
// on the resident blocks
// (with 16-bit row codes the window bases need registers: at four blocks
// per SM phases of 8 spill and phases of 6 or 7 fit)
static const AdjStepFn adj_shapes[] = {adjoint_step<8, 4>,  adjoint_step<7, 4>,
                                       adjoint_step<6, 4>,  adjoint_step<12, 3>,
                                       adjoint_step<16, 2>, adjoint_step<8, 3>};
static constexpr int N_ADJ_SHAPES = 6;

// one reverse step; `pdl`: as a programmatic dependent launch
static cudaError_t adj_launch(AdjStepFn fn, unsigned grid, bool pdl, cudaStream_t s,
                              const Transpose& T, int64_t NI, double dt, const double* lam,
                              double* lam_out, double* S) {
    if (!pdl) {
        fn<<<grid, 256, 0, s>>>(T, NI, dt, lam, lam_out, S);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, T, NI, dt, lam, lam_out, S);
}

static unsigned adj_grid(const rbffd_plan* p) {
    const int64_t nsl_int = (p->NI + SLICE - 1) / SLICE;
    return (unsigned)std::max<int64_t>(1, (nsl_int + 7) / 8);
}

// Time every reverse-step shape and grid on this plan's transpose (a few
// steps each on scratch vectors, dt = 0; an untimed round first, then the
// best of three interleaved rounds) and keep the fastest.  Once per plan.
static int tune_adjoint(rbffd_plan* p, cudaStream_t s) {
    Transpose& T = *p->tr;
    if (T.step) return RBFFD_OK;
    const int64_t NI = p->NI;
    const int sms = device_sm_count();
    // shapes x (the full grid, the resident grid) x (plain, programmatic
    // dependent launches; RBFFD_LAUNCH_PDL / _NO_PDL fix that choice)
    AdjStepFn cf[4 * N_ADJ_SHAPES];
    unsigned cg[4 * N_ADJ_SHAPES];
    bool cp[4 * N_ADJ_SHAPES];
    int nc = 0;
    const int pdl_lo = (p->flags & RBFFD_LAUNCH_PDL) ? 1 : 0;
    const int pdl_hi = (p->flags & RBFFD_LAUNCH_NO_PDL) ? 1 : 2;
    for (int c = 0; c < N_ADJ_SHAPES; ++c) {
        int per_sm = 0;
        RBFFD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, (const void*)adj_shapes[c], 256, 0));
        const unsigned res = (unsigned)(sms * std::max(1, per_sm));
        for (int pdl = pdl_lo; pdl < pdl_hi; ++pdl) {
            cf[nc] = adj_shapes[c];
            cg[nc] = adj_grid(p);
            cp[nc++] = pdl != 0;
            if (res < adj_grid(p)) {
                cf[nc] = adj_shapes[c];
                cg[nc] = res;
                cp[nc++] = pdl != 0;
            }
        }
    }
    RBFFD_CHECK_CUDA(cudaMemsetAsync(T.lam[0], 0, sizeof(double) * NI, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(T.lam[1], 0, sizeof(double) * NI, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(T.S, 0, sizeof(double) * NI, s));
    const int reps = (int)std::max<int64_t>(4, std::min<int64_t>(64, 200000000 / (NI * p->n + 1)));
    cudaEvent_t e0, e1;
    RBFFD_CHECK_CUDA(cudaEventCreate(&e0));
    RBFFD_CHECK_CUDA(cudaEventCreate(&e1));
    float best[4 * N_ADJ_SHAPES];
    for (float& b : best) b = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int round = 0; round < 4 && e == cudaSuccess; ++round)
        for (int c = 0; c < nc && e == cudaSuccess; ++c) {
            cudaEventRecord(e0, s);
            for (int k = 0; k < reps && e == cudaSuccess; ++k)
                e = adj_launch(cf[c], cg[c], cp[c], s, T, NI, 0.0, T.lam[k & 1],
                               T.lam[(k + 1) & 1], T.S);
            cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            float ms = 0.f;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            if (round) best[c] = std::min(best[c], ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RBFFD_CHECK_CUDA(e);
    int bi = 0;
    for (int c = 1; c < nc; ++c)
        if (best[c] < best[bi]) bi = c;
    T.step = cf[bi];
    T.step_grid = cg[bi];
    T.step_pdl = cp[bi];
    return RBFFD_OK;
}

static int build_transpose(rbffd_plan* p, cudaStream_t s) {
    if (p->tr) return RBFFD_OK;
    const int64_t N = p->N, NI = p->NI;
    const int n = p->n;
    const int64_t nnz = NI * n;
    const int sms = device_sm_count();
    Transpose* t = new Transpose();
    t->nslices = (N + SLICE - 1) / SLICE;
    Scratch start, cursor, erow, ekey, ew, tmp, size;
    cudaError_t e = cudaSuccess;
    int64_t total = 0;
    do {
        if ((e = start.alloc(sizeof(int32_t) * (N + 1), s))) break;
        if ((e = cursor.alloc(sizeof(int32_t) * (N + 1), s))) break;
        if ((e = erow.alloc(sizeof(int32_t) * nnz, s))) break;
        if ((e = ekey.alloc(sizeof(int32_t) * nnz, s))) break;
        if ((e = ew.alloc(sizeof(double) * nnz, s))) break;
        if ((e = tmp.alloc(sizeof(int64_t) * scan_tmp_elems(N), s))) break;
        if ((e = size.alloc(sizeof(int64_t) * t->nslices, s))) break;
        if ((e = cudaMalloc((void**)&t->off, sizeof(int64_t) * (t->nslices + 1)))) break;
        if ((e = cudaMalloc((void**)&t->len, sizeof(int32_t) * t->nslices))) break;
        if ((e = cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * (N + 1), s))) break;
        tr_count<<<sms * 8, 256, 0, s>>>(p->col, NI, n, cursor.as<int32_t>());
        if ((e = exclusive_scan_i32(cursor.as<int32_t>(), start.as<int32_t>(), N,
                                    tmp.as<int64_t>(), s)))
            break;
        if ((e = cudaMemcpyAsync(cursor.p, start.p, sizeof(int32_t) * N,
                                 cudaMemcpyDeviceToDevice, s)))
            break;
        tr_scatter<<<sms * 8, 256, 0, s>>>(p->col, p->w64, p->row_of_slot, NI, n,
                                           cursor.as<int32_t>(), erow.as<int32_t>(),
                                           ekey.as<int32_t>(), ew.as<double>());
        tr_sort<<<sms * 8, 256, 0, s>>>(start.as<int32_t>(), N, erow.as<int32_t>(),
                                        ekey.as<int32_t>(), ew.as<double>());
        if ((e = cudaMalloc((void**)&t->colof, sizeof(int32_t) * N))) break;
        if ((e = cudaMalloc((void**)&t->posof, sizeof(int32_t) * N))) break;
        tr_place<<<sms * 8, 256, 0, s>>>(start.as<int32_t>(), NI, N, t->colof, t->posof);
        tr_slice_len<<<sms * 4, 256, 0, s>>>(start.as<int32_t>(), t->colof, N, t->nslices,
                                             t->len, size.as<int64_t>());
        scan64_single<<<1, 256, 0, s>>>(size.as<int64_t>(), t->nslices, t->off);
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(&total, t->off + t->nslices, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s)))
            break;
        if ((e = cudaStreamSynchronize(s))) break;
        if ((e = cudaMalloc((void**)&t->row, sizeof(int32_t) * std::max<int64_t>(total, 1)))) break;
        if ((e = cudaMalloc((void**)&t->w, sizeof(double) * std::max<int64_t>(total, 1)))) break;
        if ((e = cudaMalloc((void**)&t->lam[0], sizeof(double) * NI))) break;
        if ((e = cudaMalloc((void**)&t->lam[1], sizeof(double) * NI))) break;
        if ((e = cudaMalloc((void**)&t->S, sizeof(double) * NI))) break;
        tr_fill<<<sms * 8, 256, 0, s>>>(start.as<int32_t>(), erow.as<int32_t>(), ew.as<double>(),
                                        t->colof, t->posof, N, t->nslices, t->off, t->len, t->row,
                                        t->w);
        if ((e = cudaGetLastError())) break;
        const int64_t nsl_int = (NI + SLICE - 1) / SLICE;
        if ((e = cudaMemcpyAsync(&t->entries, t->off + nsl_int, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s)))
            break;
        if (p->col16 && nsl_int > 0) {   // the plan's index form: codes unless RBFFD_PACK_IDX32
            Scratch cnt;
            // columns and stored entries of the compact slices, then an error flag
            if ((e = cnt.alloc(3 * sizeof(unsigned long long), s))) break;
            if ((e = cudaMemsetAsync(cnt.p, 0, 3 * sizeof(unsigned long long), s))) break;
            if ((e = cudaMalloc((void**)&t->row16, sizeof(uint16_t) * std::max<int64_t>(total, 1))))
                break;
            if ((e = cudaMalloc((void**)&t->tbase, sizeof(int4) * nsl_int))) break;
            unsigned long long* dc = cnt.as<unsigned long long>();
            tr_pack16<<<sms * 8, 256, 0, s>>>(start.as<int32_t>(), t->colof, NI, nsl_int, t->off,
                                              t->len, t->row, t->row16, t->tbase, dc,
                                              reinterpret_cast<int*>(dc + 2));
            if ((e = cudaGetLastError())) break;
            unsigned long long hc[2];
            int herr = 0;
            if ((e = cudaMemcpyAsync(hc, dc, sizeof(hc), cudaMemcpyDeviceToHost, s))) break;
            if ((e = cudaMemcpyAsync(&herr, dc + 2, sizeof(int), cudaMemcpyDeviceToHost, s)))
                break;
            if ((e = cudaStreamSynchronize(s))) break;
            if (herr) {
                e = cudaErrorUnknown;
                break;
            }
            t->cols16 = (int64_t)hc[0];
            t->entries16 = (int64_t)hc[1];
        } else {
            e = cudaStreamSynchronize(s);
        }
    } while (0);
    p->tr = t;
    if (e != cudaSuccess) {
        set_error("rbffd_adjoint: building the transpose: %s", cudaGetErrorString(e));
        free_transpose(p);
        return RBFFD_ERR_CUDA;
    }
    return RBFFD_OK;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_transpose(rbffd_plan* p, void* stream) {
    clear_error();
    RBFFD_ARG(p, "rbffd_transpose: NULL plan");
    return build_transpose(p, as_stream(stream));
}

extern "C" int rbffd_transpose_layout(const rbffd_plan* p, int64_t* h_slices, int64_t* h_cols16,
                                      int64_t* h_entries, double* h_bytes) {
    clear_error();
    RBFFD_ARG(p, "rbffd_transpose_layout: NULL plan");
    RBFFD_ARG(p->tr, "rbffd_transpose_layout: the transpose is not built (rbffd_transpose)");
    const Transpose& T = *p->tr;
    const int64_t nsl_int = (p->NI + SLICE - 1) / SLICE;
    // with codes: entries of compact slices are 2 + 8 bytes, those of the
    // other slices 2 + 4 + 8 (code, int32 row, weight); without: 4 + 8.  Per
    // slice its offset and length (and window bases); per column lambda and
    // S read, both written
    const double e16 = (double)T.entries16, ew = (double)(T.entries - T.entries16);
    const double bytes = (T.row16 ? 10.0 * e16 + 14.0 * ew + 28.0 * nsl_int
                                  : 12.0 * (double)T.entries + 12.0 * nsl_int) +
                         32.0 * (double)p->NI;
    if (h_slices) *h_slices = nsl_int;
    if (h_cols16) *h_cols16 = T.cols16;
    if (h_entries) *h_entries = T.entries;
    if (h_bytes) *h_bytes = bytes;
    return RBFFD_OK;
}

extern "C" int rbffd_adjoint(rbffd_plan* p, const double* dLdu, int64_t K, double dt,
                             double* grad_f, double* grad_g, double* lam0, void* stream) {
    clear_error();
    RBFFD_ARG(p && dLdu && grad_f && grad_g, "rbffd_adjoint: NULL argument");
    RBFFD_ARG(K >= 0 && isfinite(dt), "rbffd_adjoint: bad K / dt");
    cudaStream_t s = as_stream(stream);
    int st = build_transpose(p, s);
    if (st) return st;
    if ((st = tune_adjoint(p, s))) return st;
    Transpose& T = *p->tr;
    const int sms = device_sm_count();
    const unsigned G = (unsigned)sms * 8;
    adj_gather_placed<<<G, 256, 0, s>>>(dLdu, p->perm, T.colof, p->NI, T.lam[0]);
    RBFFD_CHECK_CUDA(cudaMemsetAsync(T.S, 0, sizeof(double) * p->NI, s));
    for (int64_t k = 0; k < K; ++k)
        RBFFD_CHECK_CUDA(adj_launch(T.step, T.step_grid, T.step_pdl && k > 0, s, T, p->NI, dt,
                                    T.lam[k & 1], T.lam[(k + 1) & 1], T.S));
    adjoint_grad_g<<<G, 256, 0, s>>>(T, p->NI, p->N, dt, T.S, p->perm, dLdu, grad_g);
    adj_outputs<<<G, 256, 0, s>>>(T.S, T.lam[K & 1], p->row_of_slot, T.colof, p->perm, p->NI,
                                  dt, grad_f,
                                  grad_g, lam0);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}

extern "C" int rbffd_adjoint_w(rbffd_plan* p, const double* f, const double* ckpt, int64_t every,
                               const double* dLdu, int64_t K, double dt, double* grad_w,
                               double* grad_f, double* grad_g, double* lam0, void* stream) {
    clear_error();
    RBFFD_ARG(p && f && ckpt && dLdu && grad_w && grad_f && grad_g,
              "rbffd_adjoint_w: NULL argument");
    RBFFD_ARG(K >= 0 && every >= 1 && isfinite(dt), "rbffd_adjoint_w: bad K / every / dt");
    cudaStream_t s = as_stream(stream);
    int st = build_transpose(p, s);
    if (st) return st;
    if ((st = tune_adjoint(p, s))) return st;
    Transpose& T = *p->tr;
    const int sms = device_sm_count();
    const unsigned G = (unsigned)sms * 8;
    const int64_t N = p->N, NI = p->NI;
    const int n = p->n;
    const int64_t seg = std::min<int64_t>(every, std::max<int64_t>(K, 1));
    Scratch segbuf, gacc;
    RBFFD_CHECK_CUDA(segbuf.alloc(sizeof(double) * (size_t)seg * N, s));
    RBFFD_CHECK_CUDA(gacc.alloc(sizeof(double) * (size_t)p->nslices * n * SLICE, s));
    double* U = segbuf.as<double>();
    double* Gw = gacc.as<double>();
    RBFFD_CHECK_CUDA(cudaMemsetAsync(Gw, 0, sizeof(double) * (size_t)p->nslices * n * SLICE, s));
    // f in slot order for the replays; lambda^K in slot order
    adj_gather<<<G, 256, 0, s>>>(f, p->row_of_slot, NI, p->fs);
    adj_gather_placed<<<G, 256, 0, s>>>(dLdu, p->perm, T.colof, NI, T.lam[0]);
    RBFFD_CHECK_CUDA(cudaMemsetAsync(T.S, 0, sizeof(double) * NI, s));
    const int64_t nseg = (K + every - 1) / every;
    const unsigned agrid = T.step_grid;
    int cur = 0;   // lambda^{k+1} lives in T.lam[cur]
    for (int64_t sidx = nseg - 1; sidx >= 0; --sidx) {
        const int64_t k0 = sidx * every, k1 = std::min(K, k0 + every);
        // u^{k0} from its checkpoint, then replay u^{k0+1} .. u^{k1-1}
        ckpt_gather<<<G, 256, 0, s>>>(ckpt + sidx * N, p->perm, N, U);
        for (int64_t k = k0; k + 1 < k1; ++k)
            replay_step<<<G, 256, 0, s>>>(p->w64, p->col, p->fs, U + (k - k0) * N,
                                          U + (k - k0 + 1) * N, NI, N, n, dt);
        for (int64_t k = k1 - 1; k >= k0; --k) {
            wgrad_accum<<<G, 256, 0, s>>>(p->col, T.lam[cur], T.posof, U + (k - k0) * N, Gw, NI,
                                          n);
            T.step<<<agrid, 256, 0, s>>>(T, NI, dt, T.lam[cur], T.lam[cur ^ 1], T.S);
            cur ^= 1;
        }
        RBFFD_CHECK_CUDA(cudaGetLastError());
    }
    adjoint_grad_g<<<G, 256, 0, s>>>(T, NI, N, dt, T.S, p->perm, dLdu, grad_g);
    adj_outputs<<<G, 256, 0, s>>>(T.S, T.lam[cur], p->row_of_slot, T.colof, p->perm, NI, dt,
                                  grad_f,
                                  grad_g, lam0);
    wgrad_unpack<<<G, 256, 0, s>>>(Gw, p->row_of_slot, NI, n, dt, grad_w);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}

