// The explicit solver of Eq. 6 (jacobi_step) on one GPU:
//   rbffd_apply           Eq. 1 on the caller's row-major layout
//   rbffd_plan_create     node reordering + packed stencil layout
//   rbffd_solve_explicit  FP64 sweep (or FP32 defect correction)
//   rbffd_solve_dc        FP64 defect correction around an FP32 inner sweep
//   rbffd_stable_dt       power-iteration bound for dt (Eq. 7 is a guideline)
//
// Layout.  Nodes are renumbered into "slots": interior nodes first, then
// boundary nodes, each group in Morton order of a uniform cell grid (the
// paper's subdomain idea of Sec. II-A reused as on-chip locality blocking).
// Interior rows are grouped into slices of 32 rows; a slice stores its
// weights and neighbour slots as [slice][j][lane], so one warp reads each
// j-plane as a contiguous 256-byte (FP64) or 128-byte (FP32/int32) line.
// Thread = row, so each row's sum is the same fused multiply-add chain in
// support order as the definition.  Weights and indices are streamed with
// evict-first loads; the iterate (8 bytes per node) stays in L2.
//
// Step loop.  One step = one pass over all rows.  Launch modes:
//  graph       one launch per step, a chunk of launches captured once into a
//              CUDA graph and replayed; the next step's kernels apply the
//              stop rule to the completed step (its residual slot in a device
//              control block) at their start, one small kernel after the
//              replays to the last step.
//  persistent  one cooperative launch runs the steps, separated by a counter
//              barrier whose waits are bounded in time (RBFFD_ERR_TIMEOUT);
//              the stop rule for a step is applied after the next one.
//  resident    the persistent launch with each block's stencil planes held
//              in shared memory (step_res.cuh).
// The residual max-norm is reduced warp -> block -> a max reduction on its
// IEEE bits (non-negative doubles order like unsigned integers).
#include <math.h>

#include <algorithm>
#include <vector>

#include "step.cuh"
#include "step_split.cuh"

namespace rbffd {

// ------------------------------------------------------ dispatch
// launch shape of a step kernel: the register budget (min resident blocks per
// SM the compiler must allow: more blocks = fewer registers = fewer loads in
// flight per thread) and the grid (blocks per SM of the grid-stride sweep).
// Budgets 1..4 (255, 128, 80 and 64 registers per thread); the fourth suits
// the FP32 inner sweep and the FP64 sweep at small stencils.
static constexpr int N_MINB = 4;

static StepFn pick(int mode, int n, bool persistent, int minb) {
    if (mode == MODE_SWEEP64) {
        switch (minb) {
            case 1: return pick_step_f64_b1(n, persistent);
            case 2: return pick_step_f64_b2(n, persistent);
            case 3: return pick_step_f64_b3(n, persistent);
            default: return pick_step_f64_b4(n, persistent);
        }
    }
    switch (minb) {
        case 1: return pick_step_f32_b1(n, persistent);
        case 2: return pick_step_f32_b2(n, persistent);
        case 3: return pick_step_f32_b3(n, persistent);
        default: return pick_step_f32_b4(n, persistent);
    }
}

// ------------------------------------------------------- plan building
__device__ __forceinline__ uint32_t spread2(uint32_t x) {
    x &= 0x0000ffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x000003ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// key = (boundary ? cells : 0) + Morton index of the node's cell
__global__ void morton_keys(const double* xyz, const uint8_t* is_bnd, int64_t N, GridGeom g,
                            int64_t cells, int32_t* key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[3] = {0, 0, 0};
        for (int a = 0; a < g.d; ++a)
            c[a] = (uint32_t)cell_coord(xyz[(int64_t)a * N + i], g.org[a], g.cs, g.G[a]);
        uint32_t mk;
        if (g.d == 1) mk = c[0];
        else if (g.d == 2) mk = spread2(c[0]) | (spread2(c[1]) << 1);
        else mk = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
        key[i] = (int32_t)((is_bnd[i] ? cells : 0) + (int64_t)mk);
    }
}

__global__ void bnd_keys(const uint8_t* is_bnd, int64_t N, int32_t* key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        key[i] = is_bnd[i] ? 1 : 0;
}

__global__ void invert_perm(const int32_t* perm, int64_t N, int32_t* inv) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x)
        inv[perm[p]] = (int32_t)p;
}

// random bijection of [0, NI) by a 4-round Feistel network on 2^(2b) with
// cycle walking; keys from SplitMix64
__device__ uint32_t feistel(uint32_t x, int hb, uint64_t seed) {
    uint32_t mask = (1u << hb) - 1u;
    uint32_t L = x >> hb, R = x & mask;
    for (int r = 0; r < 4; ++r) {
        uint64_t z = seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull + R;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        uint32_t t = L ^ ((uint32_t)z & mask);
        L = R;
        R = t;
    }
    return (L << hb) | R;
}

__global__ void random_interior_perm(const int32_t* ordered, int64_t NI, int hb, uint64_t seed,
                                     int32_t* perm) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)p;
        do {
            x = feistel(x, hb, seed);
        } while ((int64_t)x >= NI);
        perm[p] = ordered[x];
    }
}

__global__ void check_interior(const uint8_t* is_bnd, const int32_t* interior, const int32_t* inv,
                               int64_t N, int64_t NI, int32_t* row_of_slot, int* err) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < NI;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t node = interior[r];
        if (node < 0 || node >= N || is_bnd[node]) {
            atomicExch(err, 1);
            continue;
        }
        int32_t p = inv[node];
        if (p >= NI) {
            atomicExch(err, 1);
            continue;
        }
        if (atomicExch(&row_of_slot[p], (int32_t)r) != -1) atomicExch(err, 2);
    }
}

__global__ void count_interior(const uint8_t* is_bnd, int64_t N, unsigned long long* cnt) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        c += is_bnd[i] ? 0 : 1;
    atomicAdd(cnt, c);
}

__global__ void pack_stencils(const int32_t* row_of_slot, const int32_t* inv, const int32_t* idx,
                              const double* w, int64_t NI, int64_t nslices, int n, int64_t N,
                              double* w64, float* w32, int32_t* col, int* err) {
    const int64_t total = nslices * SLICE;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t sl = p / SLICE, lane = p % SLICE;
        int64_t base = sl * (int64_t)n * SLICE + lane;
        int32_t r = p < NI ? row_of_slot[p] : -1;
        if (p < NI && (r < 0 || r >= NI)) {
            atomicExch(err, 2);   // slot not covered by the interior list
            r = -1;
        }
        if (r >= 0) {
            for (int j = 0; j < n; ++j) {
                int32_t nb = idx[(int64_t)r * n + j];
                if (nb < 0 || nb >= N) {
                    atomicExch(err, 3);
                    nb = 0;
                }
                double wv = w[(int64_t)r * n + j];
                w64[base + j * SLICE] = wv;
                w32[base + j * SLICE] = (float)wv;
                col[base + j * SLICE] = inv[nb];
            }
        } else {
            for (int j = 0; j < n; ++j) {
                w64[base + j * SLICE] = 0.0;
                w32[base + j * SLICE] = 0.0f;
                col[base + j * SLICE] = 0;
            }
        }
    }
}

// Compact form of one slice's neighbour slots (one warp per slice).  The
// windows are chosen greedily from the left: base b0 = the smallest slot the
// slice's rows use, b1 = the smallest slot >= b0 + 2^14, and so on; a slice
// whose slots need more than four windows keeps the int32 form (x = -1).
// Greedy from the left covers with the fewest windows, and every slot v of a
// compact slice lies in window k = #{bases <= v} - 1 at offset v - b_k < 2^14.
static constexpr int32_t IDX16_WINDOW = 1 << 14;

__global__ void pack_idx16(const int32_t* __restrict__ col, int64_t NI, int64_t nslices, int n,
                           uint16_t* __restrict__ col16, int4* __restrict__ sbase,
                           unsigned long long* rows16, int* err) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sl = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < nslices;
         sl += nw) {
        const bool valid = sl * SLICE + lane < NI;
        const int64_t base = sl * (int64_t)n * SLICE + lane;
        int32_t b[4];
        int64_t thr = INT64_MIN;   // slots >= thr are not yet covered
        int used = 0;
        for (int k = 0; k < 4; ++k) {
            int32_t mn = INT32_MAX;
            if (valid)
                for (int j = 0; j < n; ++j) {
                    const int32_t v = col[base + (int64_t)j * SLICE];
                    if ((int64_t)v >= thr) mn = min(mn, v);
                }
            mn = __reduce_min_sync(0xffffffffu, mn);
            if (mn == INT32_MAX) break;   // warp-uniform
            b[k] = mn;
            used = k + 1;
            thr = (int64_t)mn + IDX16_WINDOW;
        }
        for (int k = used; k < 4; ++k) b[k] = used ? b[used - 1] : 0;
        bool left = false;
        if (valid)
            for (int j = 0; j < n; ++j) left |= (int64_t)col[base + (int64_t)j * SLICE] >= thr;
        const bool wide = __any_sync(0xffffffffu, left) && used == 4;
        if (lane == 0)
            sbase[sl] = wide ? make_int4(-1, -1, -1, -1) : make_int4(b[0], b[1], b[2], b[3]);
        if (wide) continue;
        const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, valid));
        if (lane == 0) atomicAdd(rows16, (unsigned long long)nvalid);
        for (int j = 0; j < n; ++j) {
            uint16_t code = 0;
            if (valid) {
                const int32_t v = col[base + (int64_t)j * SLICE];
                const int k = (v >= b[1]) + (v >= b[2]) + (v >= b[3]);
                const int32_t off = v - (k == 0 ? b[0] : k == 1 ? b[1] : k == 2 ? b[2] : b[3]);
                if (off < 0 || off >= IDX16_WINDOW) atomicExch(err, 4);   // cannot happen
                code = (uint16_t)(((uint32_t)k << 14) | ((uint32_t)off & 0x3fffu));
            }
            col16[base + (int64_t)j * SLICE] = code;
        }
    }
}

__global__ void gather_f(const double* f, const int32_t* row_of_slot, int64_t NI, double* fs) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x)
        fs[p] = f[row_of_slot[p]];
}

__global__ void gather_u(const double* u, const int32_t* perm, int64_t N, double* a, double* b) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double v = u[perm[p]];
        a[p] = v;
        b[p] = v;
    }
}

__global__ void scatter_u(const double* us, const int32_t* perm, int64_t NI, double* u) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x)
        u[perm[p]] = us[p];
}

// ---------------------------------------------------- Neumann boundary nodes
// Before each step, every Neumann node b takes the value that meets its
// normal-derivative condition with the previous iterate of its other support
// nodes: acc = fma-chain_{j>=1} nw_bj u_j, u_b = (g_b - acc) / nw_b0.  Two
// kernels (new values into uN, then into both iterate buffers), so supports
// that contain other Neumann nodes read their previous values.
__global__ void neumann_update(const int32_t* __restrict__ ncol, const double* __restrict__ nw,
                               const double* __restrict__ ng, int64_t NN, int nn,
                               const double* u0, const double* u1, double* uN, StepCtrl* c) {
    __shared__ int s_skip, s_par;
    if (threadIdx.x == 0) {
        long long k = 0;
        s_skip = c ? !graph_state(c, false, &k) : 0;
        s_par = (int)(k & 1);
    }
    __syncthreads();
    if (s_skip) return;
    const double* uin = s_par ? u1 : u0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < NN;
         b += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 1; j < nn; ++j) acc = __fma_rn(nw[b * nn + j], uin[ncol[b * nn + j]], acc);
        uN[b] = __ddiv_rn(__dsub_rn(ng[b], acc), nw[b * nn]);
    }
}

__global__ void neumann_scatter(const int32_t* __restrict__ nslot, const double* __restrict__ uN,
                                int64_t NN, double* u0, double* u1, StepCtrl* c) {
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        long long k = 0;
        s_skip = c ? !graph_state(c, false, &k) : 0;
    }
    __syncthreads();
    if (s_skip) return;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < NN;
         b += (int64_t)gridDim.x * blockDim.x) {
        u0[nslot[b]] = uN[b];
        if (u1) u1[nslot[b]] = uN[b];
    }
}

__global__ void neumann_out(const int32_t* nslot, const double* us, const int32_t* perm,
                            int64_t NN, double* u) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < NN;
         b += (int64_t)gridDim.x * blockDim.x)
        u[perm[nslot[b]]] = us[nslot[b]];
}

// graph launches: after the last replayed step, the stop rule for it (the
// next step's kernels would apply it at their start); records the outcome
__global__ void graph_finish(StepCtrl* c) {
    long long k;
    graph_state(c, true, &k);
}

// --------------------------------------------------------- DC kernels
// d = W u - f (FP64 chain), d32 = (float) d; max |d| into *dmax (bits); the
// register budget and index codes as power_apply below
template <int NN>
__global__ void __launch_bounds__(STEP_THREADS, NN > 0 ? 4 : 1) defect_kernel(StepArgs A, const double* u,
                                                                 unsigned long long* dmax) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (STEP_THREADS / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (STEP_THREADS / 32);
    double m = 0.0;
    for (int64_t sl = warp; sl < A.nslices; sl += nw) {
        const int64_t row = sl * SLICE + lane;
        const int64_t base = sl * (int64_t)A.n * SLICE + lane;
        if (row < A.NI) {
            const int4 sb = A.col16 ? __ldg(A.sbase + sl) : make_int4(-1, -1, -1, -1);
            const double acc =
                sb.x >= 0 ? row_dot<NN, false, true, double>(A.w64 + base, A.col16 + base, sb, u,
                                                             A.n)
                          : row_dot64<NN>(A.w64 + base, A.col + base, u, A.n);
            double dr = __dsub_rn(acc, A.f[row]);
            A.d32[row] = (float)dr;
            double a = fabs(dr);
            m = (a != a || isinf(a)) ? INFINITY : fmax(m, a);
        }
    }
    m = block_max(m);
    if (threadIdx.x == 0) atomicMax(dmax, dbits(m));
}

__global__ void dc_update(double* u, const float* e, int64_t NI) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x)
        u[p] = __dadd_rn(u[p], (double)e[p]);
}

// ----------------------------------------------- power iteration kernels
// y = W_II v (v in slot order, boundary slots 0); partial sums of y^2 per
// block.  Four blocks of 256 per SM (the register budget of 64; no budget for
// the generic stencil size, which needs more) and the plan's 16-bit neighbour
// codes where a slice has them, as the step kernels: the same columns, so the
// same sums.
template <int NN>
__global__ void __launch_bounds__(STEP_THREADS, NN > 0 ? 4 : 1) power_apply(StepArgs A, const double* v,
                                                               double* y, double* part) {
    __shared__ double ws[STEP_THREADS / 32];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (STEP_THREADS / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (STEP_THREADS / 32);
    double s = 0.0;
    for (int64_t sl = warp; sl < A.nslices; sl += nw) {
        const int64_t row = sl * SLICE + lane;
        const int64_t base = sl * (int64_t)A.n * SLICE + lane;
        if (row < A.NI) {
            const int4 sb = A.col16 ? __ldg(A.sbase + sl) : make_int4(-1, -1, -1, -1);
            const double acc =
                sb.x >= 0 ? row_dot<NN, false, true, double>(A.w64 + base, A.col16 + base, sb, v,
                                                             A.n)
                          : row_dot64<NN>(A.w64 + base, A.col + base, v, A.n);
            y[row] = acc;
            s = __fma_rn(acc, acc, s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < STEP_THREADS / 32; ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// single block: norm = sqrt(sum part) in a fixed order; v = y / norm
__global__ void power_normalize(const double* part, int nparts, const double* y, double* v,
                                int64_t NI, double* norm_out) {
    __shared__ double sh[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += part[i];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    double nrm = sqrt(sh[0]);
    if (threadIdx.x == 0) *norm_out = nrm;
    for (int64_t p = threadIdx.x; p < NI; p += blockDim.x) v[p] = y[p] / nrm;
}

__global__ void power_scale(const double* norm, const double* y, double* v, int64_t NI) {
    double nrm = *norm;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x)
        v[p] = y[p] / nrm;
}

__global__ void norm_partials(const double* v, int64_t NI, double* part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NI;
         p += (int64_t)gridDim.x * blockDim.x)
        s = __fma_rn(v[p], v[p], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_to_norm(const double* part, int nparts, double* norm_out) {
    __shared__ double sh[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += part[i];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *norm_out = sqrt(sh[0]);
}

// ------------------------------------------------------------ apply (Eq. 1)
__global__ void apply_rowmajor(const double* w, const int32_t* idx, int64_t nc, int n,
                               const double* u, double* Lu) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nc;
         r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j)
            acc = __fma_rn(w[r * n + j], __ldg(u + idx[r * n + j]), acc);
        Lu[r] = acc;
    }
}

// ------------------------------------------------------------ host side
// One graph-mode step launch.  With programmatic stream serialization (pdl)
// the next launch of a captured chunk can start while this one drains.  The
// autotuner times every graph shape with and without it (measured: on plans
// of 10k-90k nodes the FP32 inner sweep gained 6-13 % per step and the FP64
// sweep up to 9 %; at 1M nodes, without the prefetch before the wait, the
// FP64 sweep lost 1 %).
static cudaError_t launch_step(StepFn fn, int grid, cudaStream_t s, const StepArgs& A,
                               StepCtrl* ctrl, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(STEP_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    StepArgs a = A;
    a.pdl = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fn, a, ctrl);
}

// fewer slices than one block of warps per SM: spread them over all SMs
static bool spread_slices(const rbffd_plan* p) {
    return (p->nslices + STEP_THREADS / 32 - 1) / (STEP_THREADS / 32) < device_sm_count();
}

static StepArgs make_args(const rbffd_plan* p) {
    StepArgs A;
    A.w64 = p->w64;
    A.w32 = p->w32;
    A.col = p->col;
    A.col16 = p->col16;
    A.sbase = p->sbase;
    A.f = p->fs;
    A.d32 = p->d32;
    A.u0 = p->u[0];
    A.u1 = p->u[1];
    A.e0 = p->e[0];
    A.e1 = p->e[1];
    A.NI = p->NI;
    A.nslices = p->nslices;
    A.n = p->n;
    A.spread = spread_slices(p) ? 1 : 0;
    A.N = p->N;
    A.halo = 0;
    A.pdl = 0;
    A.fl_idx = nullptr;
    A.fl_off = nullptr;
    A.fl_slot = nullptr;
    A.fl_max = 0;
    A.inner = p->inner_sl;
    return A;
}

// the far-list fields of the resident launch of mode mi
static void far_args(const rbffd_plan* p, int mi, StepArgs* A) {
    A->fl_idx = p->fl_idx[mi];
    A->fl_off = p->fl_off[mi];
    A->fl_slot = p->fl_slot[mi];
    A->fl_max = p->fl_max[mi];
}

static void drop_graphs(rbffd_plan* p) {
    for (auto& per_mode : p->graphs)
        for (void*& g : per_mode)
            if (g) {
                cudaGraphExecDestroy((cudaGraphExec_t)g);
                g = nullptr;
            }
}

static void free_plan(rbffd_plan* p) {
    if (!p) return;
    void* bufs[] = {p->perm, p->inv, p->row_of_slot, p->w64, p->w32, p->col, p->u[0], p->u[1],
                    p->fs, p->e[0], p->e[1], p->d32, p->scratch, p->ctrl, p->nslot, p->ncol,
                    p->nw, p->ng, p->ng0, p->uN, p->col16, p->sbase,
                    p->fl_idx[0], p->fl_idx[1], p->fl_off[0], p->fl_off[1],
                    p->fl_slot[0], p->fl_slot[1], p->inner_sl};
    for (void* b : bufs)
        if (b) cudaFree(b);
    drop_graphs(p);
    for (void* e : p->ev)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    free_transpose(p);
    delete p;
}

// blocks of a grid-stride launch with `per_sm` blocks per SM (fewer,
// longer-lived blocks avoid the tail of many short ones)
static int grid_for(const rbffd_plan* p, int per_sm) {
    int64_t warps = p->nslices;
    // spread plans: one slice per block at most, so every SM takes a share
    int64_t blocks = spread_slices(p) ? warps : (warps + STEP_THREADS / 32 - 1) / (STEP_THREADS / 32);
    int64_t cap = (int64_t)device_sm_count() * std::max(1, per_sm);
    return (int)std::max<int64_t>(1, std::min(blocks, cap));
}
static int step_grid(const rbffd_plan* p) { return grid_for(p, p->grid_steps); }

// resident blocks of a persistent launch, no more than the slices need
// (spread plans: one block per SM at most)
static int persistent_grid(StepFn fn, const rbffd_plan* p) {
    const int64_t nslices = p->nslices;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, STEP_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int sms = device_sm_count();
    int64_t need = (nslices + STEP_THREADS / 32 - 1) / (STEP_THREADS / 32);
    if (spread_slices(p)) need = std::min<int64_t>(nslices, sms);
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, need));
}

// reset the control block for a run of at most max_steps steps; `held`:
// arrivals the persistent barrier waits for beyond the grid's (0 but in a
// test of the timeout path, rbffd_plan_set_wait)
static int ctrl_reset(rbffd_plan* p, double dt, double tol, long long max_steps, cudaStream_t s,
                      int held = 0) {
    StepCtrl h;
    memset(&h, 0, sizeof(h));
    h.max_steps = max_steps;
    h.dt = dt;
    h.tol = tol;
    h.done = max_steps <= 0 ? DONE_CAP : DONE_RUNNING;
    h.held = held;
    h.spin_limit = p->spin_limit;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(p->ctrl, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    return RBFFD_OK;
}

// launch modes the autotuner may choose from: persistent only when asked for
// (or left to it) and the plan has no Neumann phase, which only graphs replay
static bool may_persist(const rbffd_plan* p) {
    return (p->flags & (RBFFD_LAUNCH_PERSISTENT | RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_RESIDENT |
                        RBFFD_LAUNCH_FAR | RBFFD_LAUNCH_SPLIT)) != 0 &&
           p->NN == 0;
}
static bool may_graph(const rbffd_plan* p) {
    return !(p->flags & (RBFFD_LAUNCH_PERSISTENT | RBFFD_LAUNCH_RESIDENT | RBFFD_LAUNCH_FAR |
                         RBFFD_LAUNCH_SPLIT)) ||
           p->NN > 0;
}

// The resident persistent launch (step_res.cu): one block per SM keeping its
// slices' planes in shared memory.  Its index planes are the 16-bit codes when
// every slice has them.  Returns its kernel and dynamic shared memory, or
// nullptr when the plan's share per SM does not fit.
static bool res_i16(const rbffd_plan* p) { return p->col16 && p->rows16 == p->NI; }
// The halo window (the slots staged in shared memory each step) reaches
// `*halo` slots beyond the block's rows on either side: at most as far as the
// shared memory left beside the planes allows (returned in *halo; the tuner
// tries shorter reaches, and none), up to the whole iterate.
static StepFn resident_fn(rbffd_plan* p, int mode, int threads, unsigned* smem, int64_t* halo) {
    const int grid = device_sm_count();
    const bool i16 = res_i16(p);
    int dev = 0, optin = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const unsigned room = (unsigned)optin - 1024u;   // static shared memory and slack
    const unsigned planes = resident_smem(p->nslices, p->n, mode, i16, grid, -1);
    if (planes > room) return nullptr;
    const int64_t rows = (p->nslices + grid - 1) / grid * SLICE;
    const int64_t elem = mode == MODE_SWEEP64 ? 8 : 4;
    const int64_t fit = (int64_t)(room - planes) / elem - 8;   // alignment slack
    int64_t h = fit > rows ? (fit - rows) / 2 : 0;
    h = std::min<int64_t>(h, p->N);
    const unsigned bytes = resident_smem(p->nslices, p->n, mode, i16, grid, h);
    if (bytes > room) return nullptr;
    StepFn fn = threads == RES_THREADS_WIDE ? pick_resident_wide(mode, p->n, i16)
                                            : pick_resident(mode, p->n, i16);
    if (!fn) return nullptr;
    if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, threads,
                                                      bytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return nullptr;
    }
    *smem = bytes;
    *halo = h;
    return fn;
}

// Far lists of the resident launch (mode mi, grid = SMs; block b owns slices
// [nslices b / G, nslices (b+1) / G)): with the window reach h, block b stages
// slots [lo, lo + W) (lo = (b's first slot - h) rounded down to 4, W its span
// to b's last slot + h, rounded down to 4, both within [0, N)) - the kernel's
// own formula - and every other slot its rows read is a far slot, kept in a
// sorted per-block list and staged behind the window each step.  Each stencil
// entry gets its local index: c - lo in the window, W + its position in the
// list otherwise.  h starts at the largest window that fits beside the planes
// and shrinks until the window and the largest far list fit; the build fails
// (fl_ok false) when own rows fall outside the window or indices exceed 16 bits.
static int build_far(rbffd_plan* p, int mode, cudaStream_t s) {
    const int mi = mode == MODE_SWEEP64 ? 0 : 1;
    if (p->fl_built[mi]) return RBFFD_OK;
    p->fl_built[mi] = true;
    p->fl_ok[mi] = false;
    const int G = device_sm_count();
    const int64_t NI = p->NI, N = p->N, nsl = p->nslices;
    const int n = p->n;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        cudaGetLastError();
        return RBFFD_OK;
    }
    const int64_t room = (int64_t)optin - 1024;
    const int64_t elem = mode == MODE_SWEEP64 ? 8 : 4;
    const int64_t planes = resident_smem(nsl, n, mode, true, G, -1);
    const int64_t rows = (nsl + G - 1) / G * SLICE;
    if (planes + (rows + 8) * elem > room || NI > 4000000) return RBFFD_OK;
    const int64_t ent = nsl * n * SLICE;
    std::vector<int32_t> col(ent);
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(col.data(), p->col, sizeof(int32_t) * ent,
                                     cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    std::vector<uint16_t> lidx(ent, 0);
    std::vector<int32_t> off(G + 1, 0);
    std::vector<int32_t> slots;
    int64_t h = std::max<int64_t>(0, (room - planes) / elem - 8 - rows) / 2;
    for (int attempt = 0; attempt < 12; ++attempt) {
        slots.clear();
        int64_t fmax = 0;
        bool bad = false;
        for (int b = 0; b < G && !bad; ++b) {
            const int64_t s0 = nsl * b / G, s1 = nsl * (b + 1) / G;
            const int64_t lo = std::max<int64_t>(0, s0 * SLICE - h) & ~(int64_t)3;
            const int64_t hi = std::min<int64_t>(N, s1 * SLICE + h);
            const int64_t W = hi > lo ? (hi - lo) & ~(int64_t)3 : 0;
            const int64_t r1 = std::min<int64_t>(s1 * SLICE, NI);
            if (r1 > s0 * SLICE && r1 - lo > W) {
                bad = true;
                break;
            }
            std::vector<int32_t> far;
            for (int64_t sl = s0; sl < s1; ++sl)
                for (int j = 0; j < n; ++j)
                    for (int l = 0; l < SLICE; ++l) {
                        if (sl * SLICE + l >= NI) continue;
                        const int32_t c = col[(sl * n + j) * SLICE + l];
                        if (c < lo || c >= lo + W) far.push_back(c);
                    }
            std::sort(far.begin(), far.end());
            far.erase(std::unique(far.begin(), far.end()), far.end());
            if (W + (int64_t)far.size() > 65535) {
                bad = true;
                break;
            }
            fmax = std::max<int64_t>(fmax, (int64_t)far.size());
            for (int64_t sl = s0; sl < s1; ++sl)
                for (int j = 0; j < n; ++j)
                    for (int l = 0; l < SLICE; ++l) {
                        const int64_t e = (sl * n + j) * SLICE + l;
                        if (sl * SLICE + l >= NI) continue;
                        const int32_t c = col[e];
                        lidx[e] = (uint16_t)(c >= lo && c < lo + W
                                                 ? c - lo
                                                 : W + (std::lower_bound(far.begin(), far.end(),
                                                                         c) -
                                                        far.begin()));
                    }
            off[b] = (int32_t)slots.size();
            slots.insert(slots.end(), far.begin(), far.end());
        }
        off[G] = (int32_t)slots.size();
        if (bad) return RBFFD_OK;
        const int64_t need = resident_smem(nsl, n, mode, true, G, h, fmax);
        if (need <= room) {
            cudaError_t e = cudaSuccess;
            auto up = [&](void** dst, const void* src, size_t bytes) {
                if (e == cudaSuccess) e = cudaMalloc(dst, bytes);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
            };
            if (slots.empty()) slots.push_back(0);
            up((void**)&p->fl_idx[mi], lidx.data(), sizeof(uint16_t) * lidx.size());
            up((void**)&p->fl_off[mi], off.data(), sizeof(int32_t) * off.size());
            up((void**)&p->fl_slot[mi], slots.data(), sizeof(int32_t) * slots.size());
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            RBFFD_CHECK_CUDA(e);
            p->fl_halo[mi] = h;
            p->fl_max[mi] = fmax;
            p->fl_ok[mi] = true;
            return RBFFD_OK;
        }
        if (h == 0) return RBFFD_OK;
        h = std::max<int64_t>(0, h - ((need - room) / elem + 127) / 2 - 64);
    }
    return RBFFD_OK;
}

// Autotuner: time every launch shape of `mode` for a few steps on this plan's
// own stencils (u / e buffers zeroed; dt = 0 so nothing moves) and keep the
// fastest.  Candidates: register budget minb in {1, 2, 3, 4} x blocks per SM
// in {1, 2, 3, 4} x plain or programmatic dependent launches (graph mode,
// timed as a captured chunk of launches: what solves replay), and minb alone
// (persistent mode,
// whose grid is the resident maximum); RBFFD_LAUNCH_AUTO times both modes and
// keeps the faster.  The candidates are timed in interleaved rounds, one
// untimed warm-up round first, each keeping its best round: timing them one
// after another let drift (clocks, caches) favour whichever came last.  Runs
// once per plan and mode, on `s`.
struct TuneCand {
    int minb, per_sm;
    bool pdl;        // graph shapes: steps as programmatic dependent launches
    bool persistent;
    bool resident;   // the resident persistent launch (smem bytes, halo, threads below)
    bool far;        // ... with far lists
    bool split;      // the split persistent launch (smem bytes, threads below)
    int threads;
    unsigned smem;
    int64_t halo;
    StepFn fn;
    int grid;
    cudaGraphExec_t gx;
    float ms;
};

static int tune_shape(rbffd_plan* p, int mode, cudaStream_t s) {
    const int mi = mode == MODE_SWEEP64 ? 0 : 1;
    if (p->tuned[mi]) return RBFFD_OK;
    RBFFD_CHECK_CUDA(cudaMemsetAsync(p->u[0], 0, sizeof(double) * p->N, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(p->u[1], 0, sizeof(double) * p->N, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(p->e[0], 0, sizeof(float) * p->N, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(p->e[1], 0, sizeof(float) * p->N, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(p->d32, 0, sizeof(float) * p->NI, s));
    StepArgs A = make_args(p);
    // enough steps to time reliably on small plans (a step there costs a few
    // microseconds of mostly latency, so a short trial is noise), few on large ones
    const long long reps =
        std::max<long long>(10, std::min<long long>(600, 400000000 / (p->NI * p->n + 1)));
    const int n_minb = N_MINB;
    // candidate c: graph shapes per_sm = c (1..4), then the persistent launch (c = 5)
    const bool only_far = (p->flags & RBFFD_LAUNCH_FAR) != 0;
    const bool only_split = (p->flags & RBFFD_LAUNCH_SPLIT) != 0;
    const bool only_res = (p->flags & RBFFD_LAUNCH_RESIDENT) != 0 || only_far || only_split;
    const int c_lo = may_graph(p) ? 1 : 5, c_hi = may_persist(p) ? 5 : 4;
    std::vector<TuneCand> cands;
    const int pdl_lo = (p->flags & RBFFD_LAUNCH_PDL) ? 1 : 0;
    const int pdl_hi = (p->flags & RBFFD_LAUNCH_NO_PDL) ? 1 : 2;
    for (int minb = 1; minb <= n_minb && !only_res; ++minb)
        for (int c = c_lo; c <= c_hi; ++c)
            for (int pdl = c == 5 ? 0 : pdl_lo; pdl < (c == 5 ? 1 : pdl_hi); ++pdl) {
                TuneCand t;
                t.minb = minb;
                t.pdl = pdl != 0;
                t.persistent = c == 5;
                t.resident = false;
                t.far = false;
                t.split = false;
                t.threads = STEP_THREADS;
                t.smem = 0;
                t.halo = 0;
                t.per_sm = t.persistent ? 1 : c;
                t.fn = pick(mode, p->n, t.persistent, minb);
                t.grid = t.persistent ? persistent_grid(t.fn, p) : grid_for(p, t.per_sm);
                t.gx = nullptr;
                t.ms = 1e30f;
                cands.push_back(t);
            }
    // the resident persistent launch, when asked for (or left to the tuner)
    // and the plan's planes fit one block per SM; its halo reach is tuned: no
    // window, the block's own rows, 256, 1024, 4096 slots, the most that fits;
    // and its block size: 512 threads, and 1024 where the stencil size has it
    bool res_any = false;
    for (int wide = 0; wide < 2 && may_persist(p) && !only_far && !only_split &&
                       (p->flags & (RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_RESIDENT));
         ++wide) {
        TuneCand t;
        int64_t hmax = 0;
        t.threads = wide ? RES_THREADS_WIDE : RES_THREADS_HOST;
        if (p->res_threads_set && t.threads != p->res_threads_set) continue;
        t.far = false;
        t.split = false;
        t.fn = resident_fn(p, mode, t.threads, &t.smem, &hmax);
        if (t.fn) {
            res_any = true;
            t.minb = 1;
            t.pdl = false;
            t.per_sm = 1;
            t.persistent = true;
            t.resident = true;
            t.grid = device_sm_count();
            t.gx = nullptr;
            t.ms = 1e30f;
            const unsigned smax = t.smem;
            const int64_t reach[] = {-1, 0, 256, 1024, 4096, hmax};
            for (int q = 0; q < 6; ++q) {
                // a reach set by rbffd_plan_set_resident_halo replaces the list
                if (p->res_halo_set >= -1 && q > 0) break;
                if (p->res_halo_set < -1 && (reach[q] > hmax || (q == 5 && hmax <= 4096)))
                    continue;
                t.halo = p->res_halo_set >= -1 ? std::min(p->res_halo_set, hmax) : reach[q];
                t.smem = std::min(smax, resident_smem(p->nslices, p->n, mode, res_i16(p),
                                                      t.grid, t.halo));
                cands.push_back(t);
            }
        }
    }
    // the resident launch with far lists (its reach fixed by the build; not
    // when rbffd_plan_set_resident_halo fixed one)
    if (may_persist(p) && !only_split &&
        (p->flags & (RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_RESIDENT | RBFFD_LAUNCH_FAR)) &&
        p->res_halo_set < -1) {
        int st0 = build_far(p, mode, s);
        if (st0) return st0;
        for (int wide = 0; wide < 2 && p->fl_ok[mi]; ++wide) {
            TuneCand t;
            t.threads = wide ? RES_THREADS_WIDE : RES_THREADS_HOST;
            if (p->res_threads_set && t.threads != p->res_threads_set) continue;
            t.fn = pick_resident_far(mode, p->n, t.threads);
            if (!t.fn) continue;
            t.smem = resident_smem(p->nslices, p->n, mode, true, device_sm_count(),
                                   p->fl_halo[mi], p->fl_max[mi]);
            int per_sm = 0;
            if (cudaFuncSetAttribute((const void*)t.fn,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)t.smem) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)t.fn,
                                                              t.threads, t.smem) !=
                    cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                continue;
            }
            t.minb = 1;
            t.pdl = false;
            t.per_sm = 1;
            t.persistent = true;
            t.resident = true;
            t.far = true;
            t.split = false;
            t.halo = p->fl_halo[mi];
            t.grid = device_sm_count();
            t.gx = nullptr;
            t.ms = 1e30f;
            res_any = true;
            cands.push_back(t);
        }
    }
    // the split launch: Morton plans ordered with each share's inner rows first
    // (plan creation), when its own-row buffers fit one block per SM
    bool split_any = false;
    for (int wide = 0; wide < 2 && may_persist(p) && p->inner_first &&
                       (p->flags & (RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_PERSISTENT | RBFFD_LAUNCH_SPLIT));
         ++wide) {
        TuneCand t;
        t.threads = wide ? RES_THREADS_WIDE : RES_THREADS_HOST;
        if (p->res_threads_set && t.threads != p->res_threads_set) continue;
        t.fn = pick_split(mode, p->n, t.threads);
        if (!t.fn) continue;
        t.grid = device_sm_count();
        t.smem = split_smem(p->nslices, mode, t.grid);
        int dev = 0, optin = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
                cudaSuccess ||
            t.smem + 1024u > (unsigned)optin ||
            cudaFuncSetAttribute((const void*)t.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t.smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)t.fn, t.threads,
                                                          t.smem) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            continue;
        }
        t.minb = 1;
        t.pdl = false;
        t.per_sm = 1;
        t.persistent = true;
        t.resident = false;
        t.far = false;
        t.split = true;
        t.halo = 0;
        t.gx = nullptr;
        t.ms = 1e30f;
        split_any = true;
        cands.push_back(t);
    }
    if (only_split && !split_any) {
        set_error("split launch: not available for this plan (a Morton plan created with "
                  "RBFFD_LAUNCH_SPLIT whose share of rows per SM fits shared memory)");
        return RBFFD_ERR_CAPACITY;
    }
    if (only_res && !only_split && !res_any) {
        set_error("resident launch: the plan's stencils do not fit in shared memory "
                  "(%lld slices of %d entries)", (long long)p->nslices, p->n);
        return RBFFD_ERR_CAPACITY;
    }
    int st = RBFFD_OK;
    // capture one chunk of `reps` launches per graph candidate
    for (TuneCand& t : cands) {
        if (t.persistent) continue;
        cudaStream_t cs;
        cudaGraph_t gg;
        cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (ce == cudaSuccess) {
            ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                cudaError_t le = cudaSuccess;
                for (long long i = 0; i < reps && le == cudaSuccess; ++i)
                    le = launch_step(t.fn, t.grid, cs, A, p->ctrl, t.pdl);
                ce = cudaStreamEndCapture(cs, &gg);
                if (ce == cudaSuccess && le != cudaSuccess) {
                    cudaGraphDestroy(gg);
                    ce = le;
                } else if (ce == cudaSuccess) {
                    ce = cudaGraphInstantiate(&t.gx, gg, 0);
                    cudaGraphDestroy(gg);
                }
            }
            cudaStreamDestroy(cs);
        }
        if (ce != cudaSuccess) {
            set_error("autotune: capture: %s", cudaGetErrorString(ce));
            st = RBFFD_ERR_CUDA;
            break;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == RBFFD_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        set_error("autotune: event creation failed");
        st = RBFFD_ERR_CUDA;
    }
    // round 0 warms up; rounds 1..3 are timed
    for (int round = 0; round < 4 && st == RBFFD_OK; ++round) {
        for (TuneCand& t : cands) {
            if ((st = ctrl_reset(p, 0.0, 0.0, reps, s))) break;
            cudaEventRecord(e0, s);
            if (t.persistent) {
                StepCtrl* c = p->ctrl;
                A.halo = t.halo;
                far_args(p, mi, &A);
                void* args[] = {(void*)&A, (void*)&c};
                cudaLaunchCooperativeKernel((const void*)t.fn, dim3(t.grid),
                                            dim3(t.resident || t.split ? t.threads : STEP_THREADS),
                                            args, t.smem, s);
            } else {
                cudaGraphLaunch(t.gx, s);
            }
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                set_error("autotune: %s", cudaGetErrorString(e));
                st = RBFFD_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (round) t.ms = std::min(t.ms, ms);
        }
    }
    for (TuneCand& t : cands)
        if (t.gx) cudaGraphExecDestroy(t.gx);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) return st;
    const TuneCand* best = &cands[0];
    for (const TuneCand& t : cands)
        if (t.ms < best->ms) best = &t;
    p->minb[mi] = best->minb;
    p->per_sm[mi] = best->per_sm;
    p->pdl[mi] = best->pdl;
    p->persist[mi] = best->persistent;
    p->resident[mi] = best->resident;
    p->res_smem[mi] = best->smem;
    p->res_threads[mi] = best->resident || best->split ? best->threads : RES_THREADS_HOST;
    p->res_far[mi] = best->resident && best->far;
    p->split[mi] = best->split;
    p->res_halo[mi] = best->halo;
    p->tune_ms[mi] = best->ms / (float)reps;
    p->tuned[mi] = true;
    return RBFFD_OK;
}

// build (once) a graph of 2^b step launches of the given mode
static int ensure_graph(rbffd_plan* p, int mode, int b, cudaStream_t s) {
    const int mi = mode == MODE_SWEEP64 ? 0 : 1;
    void** slot = &p->graphs[mi][b];
    if (*slot) return RBFFD_OK;
    int st = tune_shape(p, mode, s);
    if (st) return st;
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    StepFn fn = pick(mode, p->n, false, p->minb[mi]);
    cudaStream_t cs;
    RBFFD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    StepArgs A = make_args(p);
    int grid = grid_for(p, p->per_sm[mi]);
    cudaGraph_t g;
    cudaError_t le = cudaSuccess;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const unsigned ng = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->NN + 255) / 256, 1024));
        for (int i = 0; i < (1 << b); ++i) {
            if (mode == MODE_SWEEP64 && p->NN > 0) {
                neumann_update<<<ng, 256, 0, cs>>>(p->ncol, p->nw, p->ng, p->NN, p->nn, p->u[0],
                                                   p->u[1], p->uN, p->ctrl);
                neumann_scatter<<<ng, 256, 0, cs>>>(p->nslot, p->uN, p->NN, p->u[0], p->u[1],
                                                    p->ctrl);
            }
            if (le == cudaSuccess) le = launch_step(fn, grid, cs, A, p->ctrl, p->pdl[mi]);
        }
        e = cudaStreamEndCapture(cs, &g);
        // a launch refused during capture would leave a graph short of steps
        if (e == cudaSuccess && le != cudaSuccess) {
            cudaGraphDestroy(g);
            e = le;
        }
    }
    if (e == cudaSuccess) {
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e == cudaSuccess) *slot = (void*)ex;
    }
    cudaStreamDestroy(cs);
    RBFFD_CHECK_CUDA(e);
    return RBFFD_OK;
}

// Tune the launch shape of `mode` and build its graph if the chosen mode
// replays one; both clobber the iterate buffers, which are saved and restored.
// Leaves the control block reset for the run.
static int prepare_mode(rbffd_plan* p, int mode, double dt, double tol, long long max_steps,
                        cudaStream_t s) {
    const int mi = mode == MODE_SWEEP64 ? 0 : 1;
    const bool graph_missing = !p->graphs[mi][GRAPH_LOG2];
    if (p->tuned[mi] && (p->persist[mi] || !graph_missing)) return RBFFD_OK;
    Scratch save;
    RBFFD_CHECK_CUDA(save.alloc(sizeof(double) * 2 * p->N + sizeof(float) * 2 * p->N, s));
    double* sv = save.as<double>();
    float* se = reinterpret_cast<float*>(sv + 2 * p->N);
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(sv, p->u[0], sizeof(double) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(sv + p->N, p->u[1], sizeof(double) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(se, p->e[0], sizeof(float) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(se + p->N, p->e[1], sizeof(float) * p->N, cudaMemcpyDeviceToDevice, s));
    Scratch saved32;
    RBFFD_CHECK_CUDA(saved32.alloc(sizeof(float) * p->NI, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(saved32.p, p->d32, sizeof(float) * p->NI, cudaMemcpyDeviceToDevice, s));
    int st = tune_shape(p, mode, s);
    if (st) return st;
    if (!p->persist[mi]) {
        st = ensure_graph(p, mode, GRAPH_LOG2, s);
        if (st) return st;
    }
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(p->u[0], sv, sizeof(double) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(p->u[1], sv + p->N, sizeof(double) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(p->e[0], se, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(p->e[1], se + p->N, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(p->d32, saved32.p, sizeof(float) * p->NI, cudaMemcpyDeviceToDevice, s));
    return ctrl_reset(p, dt, tol, max_steps, s, p->held_arrivals);
}

// run the step loop of `mode` until the control block says done.
// Reads back done / k / res_last.
static int run_steps(rbffd_plan* p, int mode, double dt, double tol, long long max_steps,
                     cudaStream_t s, long long* steps, double* res, int* done) {
    int st = ctrl_reset(p, dt, tol, max_steps, s, p->held_arrivals);
    if (st) return st;
    StepCtrl h;
    if (max_steps > 0) {
        const int mi = mode == MODE_SWEEP64 ? 0 : 1;
        st = prepare_mode(p, mode, dt, tol, max_steps, s);
        if (st) return st;
        if (p->persist[mi]) {
            // resident and split launches: one block of res_threads per SM
            const bool res = p->resident[mi] || p->split[mi];
            StepFn fn = p->split[mi] ? pick_split(mode, p->n, p->res_threads[mi])
                        : p->resident[mi]
                            ? (p->res_far[mi] ? pick_resident_far(mode, p->n, p->res_threads[mi])
                               : p->res_threads[mi] == RES_THREADS_WIDE
                                   ? pick_resident_wide(mode, p->n, res_i16(p))
                                   : pick_resident(mode, p->n, res_i16(p)))
                            : pick(mode, p->n, true, p->minb[mi]);
            int grid = res ? device_sm_count() : persistent_grid(fn, p);
            StepArgs A = make_args(p);
            A.halo = p->resident[mi] ? p->res_halo[mi] : 0;
            far_args(p, mi, &A);
            StepCtrl* c = p->ctrl;
            void* args[] = {(void*)&A, (void*)&c};
            RBFFD_CHECK_CUDA(cudaEventRecord((cudaEvent_t)p->ev[0], s));
            RBFFD_CHECK_CUDA(cudaLaunchCooperativeKernel(
                (const void*)fn, dim3(grid), dim3(res ? p->res_threads[mi] : STEP_THREADS), args,
                res ? p->res_smem[mi] : 0, s));
            RBFFD_CHECK_CUDA(cudaEventRecord((cudaEvent_t)p->ev[1], s));
            p->last_launches += 1;
        } else {
            // max_steps launches exactly: chunks of 2^GRAPH_LOG2 launches, then one
            // graph per set bit of the remainder, longest first
            const long long chunk = 1LL << GRAPH_LOG2;
            const long long full = max_steps >> GRAPH_LOG2;
            const long long rem = max_steps & (chunk - 1);
            for (int b = 0; b < GRAPH_LOG2; ++b)
                if ((rem >> b) & 1) {
                    st = ensure_graph(p, mode, b, s);
                    if (st) return st;
                }
            std::vector<int> tail;
            for (int b = GRAPH_LOG2 - 1; b >= 0; --b)
                if ((rem >> b) & 1) tail.push_back(b);
            const long long ngraphs = full + (long long)tail.size();
            long long launched = 0, g = 0;
            // check the device decision every `per_check` graphs
            const long long per_check = std::max<long long>(1, std::min<long long>(64, full));
            RBFFD_CHECK_CUDA(cudaEventRecord((cudaEvent_t)p->ev[0], s));
            for (;;) {
                for (long long i = 0; i < per_check && g < ngraphs; ++i, ++g) {
                    const int b = g < full ? GRAPH_LOG2 : tail[(size_t)(g - full)];
                    RBFFD_CHECK_CUDA(cudaGraphLaunch((cudaGraphExec_t)p->graphs[mi][b], s));
                    launched += 1LL << b;
                }
                RBFFD_CHECK_CUDA(cudaEventRecord((cudaEvent_t)p->ev[1], s));
                RBFFD_CHECK_CUDA(cudaMemcpyAsync(&h, p->ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
                RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
                if (h.done != DONE_RUNNING || g >= ngraphs) break;
            }
            // the last step's stop rule (a stop found earlier by a step's
            // kernels only makes the rest of the replayed kernels skip)
            graph_finish<<<1, 1, 0, s>>>(p->ctrl);
            RBFFD_CHECK_CUDA(cudaGetLastError());
            p->last_launches += launched + 1;
        }
    }
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&h, p->ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    *steps = h.k;
    *res = h.res_last;
    *done = h.done;
    if (max_steps > 0) {
        float ms = 0.f;
        RBFFD_CHECK_CUDA(cudaEventElapsedTime(&ms, (cudaEvent_t)p->ev[0], (cudaEvent_t)p->ev[1]));
        p->last_loop_ms += ms;
        p->last_loop_steps += h.k;
    }
    return RBFFD_OK;
}

static int done_status(int done) {
    switch (done) {
        case DONE_CONVERGED: return RBFFD_OK;
        case DONE_CAP: return RBFFD_NOT_CONVERGED;
        case DONE_NONFINITE: set_error("residual became non-finite"); return RBFFD_ERR_NONFINITE;
        case DONE_DIVERGED: set_error("residual grew 1e6-fold: dt above the stability bound?");
            return RBFFD_ERR_DIVERGED;
        case DONE_TIMEOUT: set_error("grid barrier wait timed out"); return RBFFD_ERR_TIMEOUT;
        default: set_error("step loop ended in an unknown state"); return RBFFD_ERR_CUDA;
    }
}

// stable split by a 0/1 flag: ids with flag 0 first, each group ascending
__global__ void flag_invert(const int32_t* key, int64_t N, int32_t* f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] = key[i] ? 0 : 1;
}
__global__ void split_write(const int32_t* pos0, int64_t N, int32_t* out) {
    int64_t n0 = pos0[N];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool zero = pos0[i + 1] != pos0[i];
        int64_t o = zero ? pos0[i] : n0 + (i - pos0[i]);
        out[o] = (int32_t)i;
    }
}
int split_by_flag(const int32_t* key, int64_t N, int32_t* out, int32_t* pos, int64_t* tmp,
                  cudaStream_t s) {
    int sms = device_sm_count();
    flag_invert<<<sms * 8, 256, 0, s>>>(key, N, pos);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(exclusive_scan_i32(pos, pos, N, tmp, s));
    split_write<<<sms * 8, 256, 0, s>>>(pos, N, out);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}
}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_apply(const double* w, const int32_t* idx, int64_t nc, int n, const double* u,
                           double* Lu, void* stream) {
    clear_error();
    RBFFD_ARG(nc >= 0 && n >= 1, "rbffd_apply: bad sizes");
    if (nc == 0) return RBFFD_OK;
    RBFFD_ARG(w && idx && u && Lu, "rbffd_apply: NULL argument");
    int sms = device_sm_count();
    int64_t blocks = std::min<int64_t>((nc + 255) / 256, (int64_t)sms * 16);
    apply_rowmajor<<<(unsigned)blocks, 256, 0, as_stream(stream)>>>(w, idx, nc, n, u, Lu);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}

// Shares of the resident and split launches: block b of their grid (one
// block per SM) owns slices [nslices b / G, nslices (b+1) / G).  For a Morton
// plan that asks for one of them (or leaves the choice to the autotuner) and
// that one could fit, the rows of each share are reordered once at creation:
// the rows whose stencils read only rows of the same share ("inner" rows)
// first, then the others, each group in its Morton order.  The share's rows
// stay the same set, so the same rows are inner; now the leading slices of a
// share are whole slices of inner rows, which those kernels compute while
// they wait for the other blocks at the step barrier.
static bool inner_first_applies(const rbffd_plan* p, int flags) {
    if ((flags & 15) != RBFFD_ORDER_MORTON ||
        !(flags & (RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_RESIDENT | RBFFD_LAUNCH_FAR |
                   RBFFD_LAUNCH_PERSISTENT | RBFFD_LAUNCH_SPLIT)))
        return false;
    const int G = device_sm_count();
    if (p->nslices < 2 * (int64_t)G) return false;   // a share of less than two slices
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // the smaller (FP32) planes with 16-bit indices: the resident launch of at
    // least one arithmetic may fit; else the split launch's own-row buffers
    if (flags & (RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_RESIDENT | RBFFD_LAUNCH_FAR))
        if (resident_smem(p->nslices, p->n, MODE_INNER32, true, G, -1) + 1024u <= (unsigned)optin)
            return true;
    return (flags & (RBFFD_LAUNCH_AUTO | RBFFD_LAUNCH_PERSISTENT | RBFFD_LAUNCH_SPLIT)) &&
           split_smem(p->nslices, MODE_INNER32, G) + 1024u <= (unsigned)optin;
}

// the share (block of G) that owns slice sl: nsl b / G <= sl < nsl (b+1) / G
__device__ __forceinline__ int share_of(int64_t sl, int64_t nsl, int G) {
    int64_t b = sl * G / nsl;
    while (b > 0 && nsl * b / G > sl) --b;
    while (b + 1 < G && nsl * (b + 1) / G <= sl) ++b;
    return (int)b;
}

// per interior slot: 1 when every neighbour slot of its row lies in its share
__global__ void share_inner_flags(const int32_t* __restrict__ col, int64_t NI, int64_t nsl, int n,
                                  int G, uint8_t* __restrict__ flag) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < NI;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = r / SLICE;
        const int b = share_of(sl, nsl, G);
        const int64_t c0 = nsl * b / G * SLICE;
        const int64_t c1e = nsl * (b + 1) / G * SLICE;
        const int64_t c1 = c1e < NI ? c1e : NI;
        const int64_t base = sl * n * SLICE + r % SLICE;
        bool in = true;
        for (int j = 0; j < n && in; ++j) {
            const int32_t c = col[base + (int64_t)j * SLICE];
            in = c >= c0 && c < c1;
        }
        flag[r] = in ? 1 : 0;
    }
}

// One block per share: the share's slots of perm_in in a stable partition,
// inner rows first, written to perm_out; inner_sl[b] = its leading slices of
// inner rows only.  Block size 1024 (32 warps).
__global__ void __launch_bounds__(1024) share_partition(const uint8_t* __restrict__ flag,
                                                         const int32_t* __restrict__ perm_in,
                                                         int32_t* __restrict__ perm_out,
                                                         int64_t NI, int64_t nsl, int G,
                                                         int32_t* __restrict__ inner_sl) {
    __shared__ int s_wi[32], s_wo[32];
    __shared__ int s_total;
    const int b = blockIdx.x;
    const int64_t r0 = nsl * b / G * SLICE;
    const int64_t r1e = nsl * (b + 1) / G * SLICE;
    const int64_t r1 = r1e < NI ? r1e : NI;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // the share's inner rows
    int cnt = 0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) cnt += flag[r];
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) s_wi[wid] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_wi[w];
        s_total = t;
    }
    __syncthreads();
    const int64_t ninner = s_total;
    // each chunk of blockDim slots in order: ranks among the chunk's inner and
    // other rows by warp ballots, then the warps' offsets
    int64_t run_i = 0, run_o = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int64_t c = r0; c < r1; c += blockDim.x) {
        const int64_t r = c + threadIdx.x;
        const bool valid = r < r1;
        const bool f = valid && flag[r];
        const unsigned bi = __ballot_sync(0xffffffffu, f);
        const unsigned bo = __ballot_sync(0xffffffffu, valid && !f);
        __syncthreads();   // the previous chunk's offsets are read
        if (lane == 0) {
            s_wi[wid] = __popc(bi);
            s_wo[wid] = __popc(bo);
        }
        __syncthreads();
        int oi = 0, oo = 0, ti = 0, to = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < wid) {
                oi += s_wi[w];
                oo += s_wo[w];
            }
            ti += s_wi[w];
            to += s_wo[w];
        }
        if (f) perm_out[r0 + run_i + oi + __popc(bi & below)] = perm_in[r];
        else if (valid) perm_out[r0 + ninner + run_o + oo + __popc(bo & below)] = perm_in[r];
        run_i += ti;
        run_o += to;
    }
    if (threadIdx.x == 0) inner_sl[b] = (int32_t)(ninner / SLICE);
}

extern "C" int rbffd_plan_create(const double* xyz, const uint8_t* is_bnd, int64_t N, int d,
                                 const int32_t* interior, const int32_t* idx, const double* w,
                                 int64_t NI, int n, int flags, uint64_t seed, rbffd_plan** out,
                                 void* stream) {
    clear_error();
    RBFFD_ARG(xyz && is_bnd && interior && idx && w && out, "rbffd_plan_create: NULL argument");
    RBFFD_ARG(d >= 1 && d <= 3, "rbffd_plan_create: d must be 1, 2 or 3");
    RBFFD_ARG(N >= 1 && N < (int64_t(1) << 31) && NI >= 1 && NI <= N,
              "rbffd_plan_create: bad N / NI");
    RBFFD_ARG(n >= 1 && n <= 128, "rbffd_plan_create: n must be in [1, 128]");
    int order = flags & 15;
    RBFFD_ARG(order <= RBFFD_ORDER_RANDOM, "rbffd_plan_create: unknown order flag");
    RBFFD_ARG((flags & (RBFFD_LAUNCH_PDL | RBFFD_LAUNCH_NO_PDL)) !=
                  (RBFFD_LAUNCH_PDL | RBFFD_LAUNCH_NO_PDL),
              "rbffd_plan_create: RBFFD_LAUNCH_PDL and RBFFD_LAUNCH_NO_PDL together");
    *out = nullptr;
    cudaStream_t s = as_stream(stream);
    rbffd_plan* p = new rbffd_plan();
    p->d = d;
    p->N = N;
    p->NI = NI;
    p->n = n;
    p->flags = flags;
    p->nslices = (NI + SLICE - 1) / SLICE;
    p->grid_steps = 2;
    const size_t ell = (size_t)p->nslices * n * SLICE;
    cudaError_t e = cudaSuccess;
#define RBFFD_ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes));
    RBFFD_ALLOC(p->perm, sizeof(int32_t) * N);
    RBFFD_ALLOC(p->inv, sizeof(int32_t) * N);
    RBFFD_ALLOC(p->row_of_slot, sizeof(int32_t) * NI);
    RBFFD_ALLOC(p->w64, sizeof(double) * ell);
    RBFFD_ALLOC(p->w32, sizeof(float) * ell);
    RBFFD_ALLOC(p->col, sizeof(int32_t) * ell);
    RBFFD_ALLOC(p->u[0], sizeof(double) * N);
    RBFFD_ALLOC(p->u[1], sizeof(double) * N);
    // f and d32 padded to whole slices (the resident launch copies whole slices)
    RBFFD_ALLOC(p->fs, sizeof(double) * p->nslices * SLICE);
    RBFFD_ALLOC(p->e[0], sizeof(float) * N);
    RBFFD_ALLOC(p->e[1], sizeof(float) * N);
    RBFFD_ALLOC(p->d32, sizeof(float) * p->nslices * SLICE);
    RBFFD_ALLOC(p->scratch, sizeof(double) * (2 * NI + 4096));
    RBFFD_ALLOC(p->ctrl, sizeof(StepCtrl));
#undef RBFFD_ALLOC
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreate(&ev);
        if (e == cudaSuccess) p->ev[i] = (void*)ev;
    }
    if (e != cudaSuccess) {
        set_error("rbffd_plan_create: cudaMalloc: %s", cudaGetErrorString(e));
        free_plan(p);
        return RBFFD_ERR_CUDA;
    }
    int st = RBFFD_OK;
    int sms = device_sm_count();
    const unsigned G = (unsigned)sms * 8;
    do {
        Scratch key, start, err;
        if ((e = key.alloc(sizeof(int32_t) * N, s)) != cudaSuccess) break;
        if ((e = err.alloc(4 * sizeof(unsigned long long), s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(err.p, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess)
            break;
        count_interior<<<G, 256, 0, s>>>(is_bnd, N, err.as<unsigned long long>() + 1);
        if (order == RBFFD_ORDER_MORTON) {
            double lo[3], hi[3];
            st = bounding_box(xyz, N, d, lo, hi, s);
            if (st) break;
            GridGeom g = make_grid(d, lo, hi, N, 1.0);
            int bits = d == 1 ? 26 : (d == 2 ? 12 : 8);
            for (int a = 0; a < d; ++a) {
                while (g.G[a] > (1 << bits)) {   // coarsen until the Morton key fits
                    g.cs *= 1.25;
                    for (int b = 0; b < d; ++b) g.G[b] = (int)floor((hi[b] - lo[b]) / g.cs) + 1;
                }
            }
            int maxG = 1;
            for (int a = 0; a < d; ++a) maxG = std::max(maxG, g.G[a]);
            int64_t P2 = 1;
            while (P2 < maxG) P2 <<= 1;
            int64_t cells = 1;
            for (int a = 0; a < d; ++a) cells *= P2;
            if ((e = start.alloc(sizeof(int32_t) * (2 * cells + 1), s)) != cudaSuccess) break;
            morton_keys<<<G, 256, 0, s>>>(xyz, is_bnd, N, g, cells, key.as<int32_t>());
            st = counting_sort_by_key(key.as<int32_t>(), N, 2 * cells, start.as<int32_t>(),
                                      p->perm, s);
            if (st) break;
        } else {
            if ((e = start.alloc(sizeof(int32_t) * 3, s)) != cudaSuccess) break;
            bnd_keys<<<G, 256, 0, s>>>(is_bnd, N, key.as<int32_t>());
            // two keys: a stable split by an ordered compaction (scan per key)
            Scratch flag, tmp;
            if ((e = flag.alloc(sizeof(int32_t) * (N + 1), s)) != cudaSuccess) break;
            if ((e = tmp.alloc(sizeof(int64_t) * scan_tmp_elems(N), s)) != cudaSuccess) break;
            st = split_by_flag(key.as<int32_t>(), N, p->perm, flag.as<int32_t>(),
                               tmp.as<int64_t>(), s);
            if (st) break;
            if (order == RBFFD_ORDER_RANDOM) {
                int hb = 1;
                while ((int64_t(1) << (2 * hb)) < NI) ++hb;
                if ((e = cudaMemcpyAsync(key.p, p->perm, sizeof(int32_t) * NI,
                                         cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                    break;
                random_interior_perm<<<G, 256, 0, s>>>(key.as<int32_t>(), NI, hb, seed, p->perm);
            }
        }
        invert_perm<<<G, 256, 0, s>>>(p->perm, N, p->inv);
        if ((e = cudaMemsetAsync(p->row_of_slot, 0xff, sizeof(int32_t) * NI, s)) != cudaSuccess)
            break;
        check_interior<<<G, 256, 0, s>>>(is_bnd, interior, p->inv, N, NI, p->row_of_slot,
                                         err.as<int>());
        pack_stencils<<<G, 256, 0, s>>>(p->row_of_slot, p->inv, idx, w, NI, p->nslices, n, N,
                                        p->w64, p->w32, p->col, err.as<int>());
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        unsigned long long hv[2] = {0, 0};
        if ((e = cudaMemcpyAsync(hv, err.p, sizeof(hv), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        int herr = (int)(hv[0] & 0xffffffffull);
        if (!herr && (int64_t)hv[1] != NI) herr = 1;
        if (herr) {
            set_error(herr == 3 ? "rbffd_plan_create: support index out of range"
                                : "rbffd_plan_create: `interior` must list each non-boundary node "
                                  "exactly once (NI = number of interior nodes)");
            st = RBFFD_ERR_ARG;
            break;
        }
        if (inner_first_applies(p, flags)) {
            // on the device: each row's flag, then per share a stable partition
            // of its slots (perm copied to `key` first)
            Scratch fl;
            if ((e = fl.alloc(NI, s)) != cudaSuccess) break;
            if ((e = cudaMalloc((void**)&p->inner_sl, sizeof(int32_t) * sms)) != cudaSuccess) break;
            share_inner_flags<<<G, 256, 0, s>>>(p->col, NI, p->nslices, n, sms, fl.as<uint8_t>());
            if ((e = cudaMemcpyAsync(key.p, p->perm, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess)
                break;
            share_partition<<<sms, 1024, 0, s>>>(fl.as<uint8_t>(), key.as<int32_t>(), p->perm, NI,
                                                 p->nslices, sms, p->inner_sl);
            p->inner_first = true;
            invert_perm<<<G, 256, 0, s>>>(p->perm, N, p->inv);
            if ((e = cudaMemsetAsync(p->row_of_slot, 0xff, sizeof(int32_t) * NI, s)) !=
                cudaSuccess)
                break;
            check_interior<<<G, 256, 0, s>>>(is_bnd, interior, p->inv, N, NI, p->row_of_slot,
                                             err.as<int>());
            pack_stencils<<<G, 256, 0, s>>>(p->row_of_slot, p->inv, idx, w, NI, p->nslices, n, N,
                                            p->w64, p->w32, p->col, err.as<int>());
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(hv, err.p, sizeof(hv), cudaMemcpyDeviceToHost, s)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                break;
            if (hv[0] & 0xffffffffull) {
                set_error("rbffd_plan_create: repacking the resident shares failed");
                st = RBFFD_ERR_CUDA;
                break;
            }
        }
        if (!(flags & RBFFD_PACK_IDX32)) {
            if ((e = cudaMalloc((void**)&p->col16, sizeof(uint16_t) * ell)) != cudaSuccess) break;
            if ((e = cudaMalloc((void**)&p->sbase, sizeof(int4) * p->nslices)) != cudaSuccess)
                break;
            if ((e = cudaMemsetAsync(err.p, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess)
                break;
            pack_idx16<<<G, 256, 0, s>>>(p->col, NI, p->nslices, n, p->col16, p->sbase,
                                         err.as<unsigned long long>() + 1, err.as<int>());
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(hv, err.p, sizeof(hv), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
                break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            if (hv[0] & 0xffffffffull) {
                set_error("rbffd_plan_create: compact index packing failed");
                st = RBFFD_ERR_CUDA;
                break;
            }
            p->rows16 = (int64_t)hv[1];
        }
    } while (0);
    if (e != cudaSuccess && st == RBFFD_OK) {
        set_error("rbffd_plan_create: %s", cudaGetErrorString(e));
        st = RBFFD_ERR_CUDA;
    }
    if (st) {
        free_plan(p);
        return st;
    }
    *out = p;
    return RBFFD_OK;
}


extern "C" int rbffd_plan_destroy(rbffd_plan* plan) {
    clear_error();
    if (!plan) return RBFFD_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return RBFFD_OK;
}

extern "C" int rbffd_plan_perm(const rbffd_plan* p, int32_t* perm, void* stream) {
    clear_error();
    RBFFD_ARG(p && perm, "rbffd_plan_perm: NULL argument");
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(perm, p->perm, sizeof(int32_t) * p->N,
                                     cudaMemcpyDeviceToDevice, as_stream(stream)));
    return RBFFD_OK;
}

extern "C" int rbffd_plan_set_dc(rbffd_plan* p, int64_t K_in, double rho_in) {
    clear_error();
    RBFFD_ARG(p && K_in >= 1 && rho_in >= 0.0, "rbffd_plan_set_dc: bad argument");
    p->dc_K_in = K_in;
    p->dc_rho_in = rho_in;
    return RBFFD_OK;
}

// the launch shapes are tuned again on the next solve
static void retune(rbffd_plan* p) {
    for (int mi = 0; mi < 2; ++mi) {
        p->tuned[mi] = false;
        p->persist[mi] = p->resident[mi] = p->split[mi] = false;
    }
    drop_graphs(p);
}

extern "C" int rbffd_plan_set_resident_halo(rbffd_plan* p, int64_t halo) {
    clear_error();
    RBFFD_ARG(p && halo >= -2, "rbffd_plan_set_resident_halo: bad argument");
    p->res_halo_set = halo;
    retune(p);
    return RBFFD_OK;
}

extern "C" int rbffd_plan_set_block(rbffd_plan* p, int threads) {
    clear_error();
    RBFFD_ARG(p && (threads == 0 || threads == RES_THREADS_HOST || threads == RES_THREADS_WIDE),
              "rbffd_plan_set_block: threads must be 0, 512 or 1024");
    p->res_threads_set = threads;
    retune(p);
    return RBFFD_OK;
}

extern "C" int rbffd_plan_set_wait(rbffd_plan* p, double timeout_ms, int held_arrivals) {
    clear_error();
    RBFFD_ARG(p && isfinite(timeout_ms) && timeout_ms <= 60000.0 && held_arrivals >= 0 &&
                  held_arrivals <= 1024,
              "rbffd_plan_set_wait: bad argument");
    long long cycles = 0;
    if (timeout_ms > 0.0) {
        int dev = 0, khz = 0;
        RBFFD_CHECK_CUDA(cudaGetDevice(&dev));
        RBFFD_CHECK_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
        cycles = std::max<long long>(1, (long long)(timeout_ms * (double)khz));
    }
    p->spin_limit = cycles;
    p->held_arrivals = held_arrivals;
    return RBFFD_OK;
}

static int load_problem(rbffd_plan* p, const double* f, const double* u, cudaStream_t s) {
    int sms = device_sm_count();
    p->last_loop_ms = 0.0;
    p->last_loop_steps = 0;
    p->last_launches = 2;   // gather_f, gather_u (+ the step kernels, + scatter_u)
    gather_f<<<sms * 8, 256, 0, s>>>(f, p->row_of_slot, p->NI, p->fs);
    gather_u<<<sms * 8, 256, 0, s>>>(u, p->perm, p->N, p->u[0], p->u[1]);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}

extern "C" int rbffd_solve_dc(rbffd_plan* p, const double* f, double* u, double dt, double tol,
                              int64_t max_outer, int64_t K_in, double rho_in, int64_t* h_outer_out,
                              int64_t* h_inner_out, double* h_res_out, void* stream) {
    clear_error();
    RBFFD_ARG(p && f && u, "rbffd_solve_dc: NULL argument");
    RBFFD_ARG(dt > 0.0 && isfinite(dt) && tol >= 0.0, "rbffd_solve_dc: bad dt / tol");
    RBFFD_ARG(max_outer >= 0 && K_in >= 1 && rho_in >= 0.0, "rbffd_solve_dc: bad loop limits");
    RBFFD_ARG(p->NN == 0, "rbffd_solve_dc: plans with Neumann nodes use FP64 sweeps only");
    cudaStream_t s = as_stream(stream);
    int st = load_problem(p, f, u, s);
    if (st) return st;
    StepArgs A = make_args(p);
    const int sms = device_sm_count();
    const int grid = grid_for(p, 4);
    unsigned long long* dmax = reinterpret_cast<unsigned long long*>(p->scratch);
    typedef void (*DefFn)(StepArgs, const double*, unsigned long long*);
    DefFn def;
    switch (p->n) {
        case 12: def = defect_kernel<12>; break;
        case 30: def = defect_kernel<30>; break;
        case 56: def = defect_kernel<56>; break;
        case 70: def = defect_kernel<70>; break;
        default: def = defect_kernel<0>; break;
    }
    int64_t outer = 0, inner_total = 0;
    double D = 0.0;
    int status = RBFFD_NOT_CONVERGED;
    // the FP64 iterate lives in u[0]; the inner loop ping-pongs e[0]/e[1]
    for (outer = 0; outer <= max_outer; ++outer) {
        RBFFD_CHECK_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s));
        def<<<grid, STEP_THREADS, 0, s>>>(A, p->u[0], dmax);
        RBFFD_CHECK_CUDA(cudaGetLastError());
        p->last_launches += 1;
        unsigned long long hb = 0;
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(&hb, dmax, sizeof(hb), cudaMemcpyDeviceToHost, s));
        RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
        memcpy(&D, &hb, sizeof(D));
        if (!isfinite(D)) {
            status = RBFFD_ERR_NONFINITE;
            set_error("defect became non-finite");
            break;
        }
        if (D < tol) {
            status = RBFFD_OK;
            break;
        }
        if (outer == max_outer) break;
        RBFFD_CHECK_CUDA(cudaMemsetAsync(p->e[0], 0, sizeof(float) * p->N, s));
        RBFFD_CHECK_CUDA(cudaMemsetAsync(p->e[1], 0, sizeof(float) * p->N, s));
        long long steps = 0;
        double R = 0.0;
        int done = 0;
        st = run_steps(p, MODE_INNER32, dt, rho_in * D, K_in, s, &steps, &R, &done);
        if (st) return st;
        inner_total += steps;
        if (done == DONE_NONFINITE) {
            status = RBFFD_ERR_NONFINITE;
            set_error("inner residual became non-finite");
            D = INFINITY;
            break;
        }
        if (done == DONE_TIMEOUT) return done_status(done);
        const float* ef = p->e[steps & 1];
        dc_update<<<sms * 8, 256, 0, s>>>(p->u[0], ef, p->NI);
        RBFFD_CHECK_CUDA(cudaGetLastError());
        p->last_launches += 1;
    }
    scatter_u<<<sms * 8, 256, 0, s>>>(p->u[0], p->perm, p->NI, u);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    p->last_launches += 1;
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h_outer_out) *h_outer_out = outer;
    if (h_inner_out) *h_inner_out = inner_total;
    if (h_res_out) *h_res_out = D;
    return status;
}

extern "C" int rbffd_solve_explicit(rbffd_plan* p, const double* f, double* u, double dt,
                                    int64_t max_steps, double tol, int precision,
                                    int64_t* h_steps_out, double* h_res_out, void* stream) {
    clear_error();
    RBFFD_ARG(p && f && u, "rbffd_solve_explicit: NULL argument");
    RBFFD_ARG(dt > 0.0 && isfinite(dt), "rbffd_solve_explicit: dt must be positive and finite");
    RBFFD_ARG(max_steps >= 0 && tol >= 0.0, "rbffd_solve_explicit: bad max_steps / tol");
    RBFFD_ARG(precision == 0 || precision == 1, "rbffd_solve_explicit: precision must be 0 or 1");
    if (precision == 1) {
        int64_t outer_cap = std::max<int64_t>(1, max_steps / p->dc_K_in);
        int64_t outer = 0, inner = 0;
        int st = rbffd_solve_dc(p, f, u, dt, tol, outer_cap, p->dc_K_in, p->dc_rho_in, &outer,
                                &inner, h_res_out, stream);
        if (h_steps_out) *h_steps_out = inner;
        return st;
    }
    cudaStream_t s = as_stream(stream);
    int st = load_problem(p, f, u, s);
    if (st) return st;
    long long steps = 0;
    double R = 0.0;
    int done = 0;
    st = run_steps(p, MODE_SWEEP64, dt, tol, max_steps, s, &steps, &R, &done);
    if (st) return st;
    int sms = device_sm_count();
    scatter_u<<<sms * 8, 256, 0, s>>>(p->u[steps & 1], p->perm, p->NI, u);
    p->last_launches += 1;
    if (p->NN > 0) {
        neumann_out<<<sms * 2, 256, 0, s>>>(p->nslot, p->u[steps & 1], p->perm, p->NN, u);
        p->last_launches += 1;
    }
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h_steps_out) *h_steps_out = steps;
    if (h_res_out) *h_res_out = R;
    if (max_steps == 0) return RBFFD_NOT_CONVERGED;
    return done_status(done);
}

extern "C" int rbffd_stable_dt(rbffd_plan* p, const double* v0, int iters, double safety,
                               double* h_dt_out, double* h_rho_out, void* stream) {
    clear_error();
    RBFFD_ARG(p && v0 && iters >= 1 && safety > 0.0, "rbffd_stable_dt: bad argument");
    cudaStream_t s = as_stream(stream);
    const int sms = device_sm_count();
    // v lives in u[0] (slot order; boundary slots 0), y in scratch[1024 ..]
    double* v = p->u[0];
    double* y = p->scratch + 4096;
    double* part = p->scratch + 8;
    double* nrm = p->scratch;
    const int nparts = 1024;
    RBFFD_CHECK_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * p->N, s));
    gather_f<<<sms * 8, 256, 0, s>>>(v0, p->row_of_slot, p->NI, y);
    norm_partials<<<nparts, 256, 0, s>>>(y, p->NI, part);
    sum_to_norm<<<1, 256, 0, s>>>(part, nparts, nrm);
    power_scale<<<sms * 8, 256, 0, s>>>(nrm, y, v, p->NI);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    StepArgs A = make_args(p);
    typedef void (*PowFn)(StepArgs, const double*, double*, double*);
    PowFn pf;
    switch (p->n) {
        case 12: pf = power_apply<12>; break;
        case 30: pf = power_apply<30>; break;
        case 56: pf = power_apply<56>; break;
        case 70: pf = power_apply<70>; break;
        default: pf = power_apply<0>; break;
    }
    const int grid = std::min(grid_for(p, 4), nparts);
    for (int it = 0; it < iters; ++it) {
        if (p->NN > 0) {   // Neumann values of v from its interior values (data 0)
            const unsigned ngr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->NN + 255) / 256, 1024));
            neumann_update<<<ngr, 256, 0, s>>>(p->ncol, p->nw, p->ng0, p->NN, p->nn, v, v, p->uN,
                                               nullptr);
            neumann_scatter<<<ngr, 256, 0, s>>>(p->nslot, p->uN, p->NN, v, nullptr, nullptr);
        }
        pf<<<grid, STEP_THREADS, 0, s>>>(A, v, y, part);
        sum_to_norm<<<1, 256, 0, s>>>(part, grid, nrm);
        power_scale<<<sms * 8, 256, 0, s>>>(nrm, y, v, p->NI);
    }
    RBFFD_CHECK_CUDA(cudaGetLastError());
    double rho = 0.0;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&rho, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (!(rho > 0.0) || !isfinite(rho)) {
        set_error("rbffd_stable_dt: spectral radius estimate is %g", rho);
        return RBFFD_ERR_NONFINITE;
    }
    if (h_rho_out) *h_rho_out = rho;
    if (h_dt_out) *h_dt_out = 2.0 / (safety * rho);
    return RBFFD_OK;
}

extern "C" int rbffd_plan_stats(const rbffd_plan* p, double* h_loop_ms, int64_t* h_loop_steps,
                                int64_t* h_launches, int* h_shape) {
    clear_error();
    RBFFD_ARG(p, "rbffd_plan_stats: NULL plan");
    if (h_loop_ms) *h_loop_ms = p->last_loop_ms;
    if (h_loop_steps) *h_loop_steps = p->last_loop_steps;
    if (h_launches) *h_launches = p->last_launches;
    if (h_shape) {
        for (int mi = 0; mi < 2; ++mi) {
            h_shape[2 * mi] = p->resident[mi] ? p->res_threads[mi] / 512 + (p->res_far[mi] ? 4 : 0)
                              : p->split[mi] ? p->res_threads[mi] / 512
                                             : p->minb[mi];
            h_shape[2 * mi + 1] = p->persist[mi]
                                      ? (p->resident[mi] ? -1 : p->split[mi] ? -2 : 0)
                                      : p->per_sm[mi] + (p->pdl[mi] ? 16 : 0);
        }
    }
    return RBFFD_OK;
}

extern "C" int rbffd_plan_layout(const rbffd_plan* p, int64_t* h_nslices, int64_t* h_rows16,
                                 double* h_bytes64, double* h_bytes32) {
    clear_error();
    RBFFD_ARG(p, "rbffd_plan_layout: NULL plan");
    const double NI = (double)p->NI, n = (double)p->n, r16 = (double)p->rows16;
    // index bytes streamed per step: 2 per entry of a compact row, 4 otherwise,
    // plus the slices' window bases
    const double idx = 2.0 * n * r16 + 4.0 * n * (NI - r16) + (p->col16 ? 16.0 * p->nslices : 0.0);
    if (h_nslices) *h_nslices = p->nslices;
    if (h_rows16) *h_rows16 = p->rows16;
    if (h_bytes64) *h_bytes64 = NI * (8.0 * n + 24.0) + idx;
    if (h_bytes32) *h_bytes32 = NI * (4.0 * n + 12.0) + idx;
    return RBFFD_OK;
}

namespace rbffd {
__global__ void neumann_map(const int32_t* nodes, const int32_t* idx, const double* w,
                            const double* g, int64_t NN, int nn, int64_t NI, int64_t N,
                            const int32_t* inv, int32_t* nslot, int32_t* ncol, double* nw,
                            double* ng, double* ng0, int* err) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < NN;
         b += (int64_t)gridDim.x * blockDim.x) {
        int32_t node = nodes[b];
        if (node < 0 || node >= N || idx[b * nn] != node || inv[node] < NI) {
            atomicExch(err, 1);   // not a boundary node, or not first in its support
            continue;
        }
        nslot[b] = inv[node];
        for (int j = 0; j < nn; ++j) {
            int32_t q = idx[b * nn + j];
            if (q < 0 || q >= N) {
                atomicExch(err, 2);
                q = node;
            }
            ncol[b * nn + j] = inv[q];
            nw[b * nn + j] = w[b * nn + j];
        }
        ng[b] = g ? g[b] : 0.0;
        ng0[b] = 0.0;
    }
}
}  // namespace rbffd

extern "C" int rbffd_plan_set_neumann(rbffd_plan* p, int64_t NN, const int32_t* nodes,
                                      const int32_t* idx, const double* w, int nn, const double* g,
                                      void* stream) {
    clear_error();
    RBFFD_ARG(p && NN >= 0 && (NN == 0 || (nodes && idx && w && nn >= 2)),
              "rbffd_plan_set_neumann: bad argument");
    cudaStream_t s = as_stream(stream);
    void* old[] = {p->nslot, p->ncol, p->nw, p->ng, p->ng0, p->uN};
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (void* o : old)
        if (o) cudaFree(o);
    p->nslot = p->ncol = nullptr;
    p->nw = p->ng = p->ng0 = p->uN = nullptr;
    p->NN = 0;
    p->nn = 0;
    // captured graphs include (or not) the Neumann phase: capture again; the
    // launch modes may change with it (plans with Neumann nodes replay
    // graphs), so the shapes are tuned again too
    drop_graphs(p);
    for (int mi = 0; mi < 2; ++mi) {
        p->tuned[mi] = false;
        p->persist[mi] = false;
    }
    if (NN == 0) return RBFFD_OK;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->nslot, sizeof(int32_t) * NN);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->ncol, sizeof(int32_t) * NN * nn);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->nw, sizeof(double) * NN * nn);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->ng, sizeof(double) * NN);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->ng0, sizeof(double) * NN);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->uN, sizeof(double) * NN);
    RBFFD_CHECK_CUDA(e);
    Scratch err;
    RBFFD_CHECK_CUDA(err.alloc(sizeof(int), s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    int sms = device_sm_count();
    neumann_map<<<sms * 2, 256, 0, s>>>(nodes, idx, w, g, NN, nn, p->NI, p->N, p->inv, p->nslot,
                                        p->ncol, p->nw, p->ng, p->ng0, err.as<int>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    int herr = 0;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    p->NN = NN;
    p->nn = nn;
    if (herr) {
        set_error(herr == 1 ? "rbffd_plan_set_neumann: each Neumann node must be a boundary node "
                              "and the first entry of its own support"
                            : "rbffd_plan_set_neumann: support index out of range");
        rbffd_plan_set_neumann(p, 0, nullptr, nullptr, nullptr, 0, nullptr, stream);
        return RBFFD_ERR_ARG;
    }
    return RBFFD_OK;
}

