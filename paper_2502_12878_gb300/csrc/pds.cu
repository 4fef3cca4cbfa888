// rbffd_nodes_pds: Poisson-disc node placement in 2D (Sec. II-C, last
// paragraph, after the method of Slak and Kosec that the paper cites).
//
// The method walks a node list first in, first out: the list starts with the
// boundary nodes (seeds); node p proposes K candidates at distance h, a fixed
// set of K directions rotated by an angle drawn for p; a candidate inside the
// domain is appended when no node in the list is closer than zeta h.
//
// Walking the list in order is a breadth-first walk by generation: the
// children of generation g are appended while generation g is walked, and
// none of them is walked before all of generation g.  So one generation can
// be processed in parallel with the same result:
//   * every candidate of the generation is tested against the nodes of all
//     earlier generations (a uniform grid with at most one node per cell);
//   * among the candidates that pass, the walk accepts, in key order
//     (parent's position, direction j), each candidate that no accepted
//     candidate of lower key is closer to than zeta h.  That is the
//     lexicographically first maximal independent set of the conflict graph;
//     a candidate is decided IN once all its lower-key neighbours are OUT,
//     and OUT once one of them is IN.  Repeated passes reach the same set the
//     sequential walk does (each pass decides at least the lowest undecided
//     candidate, so the passes end).  The conflict graph (each candidate's
//     lower-key neighbours, CSR) is built by the whole grid; the passes run
//     in one block on states held in shared memory, each thread walking a
//     contiguous range of about 32 keys in ascending order, so a chain of
//     conflicts inside a range resolves in one pass.
//   * the accepted candidates are appended in key order: they are the next
//     generation, and their positions in the list are those of the walk.
// Arithmetic (angles, rotations, squared distances) is a fixed sequence of
// separately rounded IEEE operations, so the node list is reproducible bit
// for bit by a sequential implementation of the same definition.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "nodegen.cuh"

namespace rbffd {

static constexpr int PDS_KMAX = 64;
static constexpr int PDS_BLOCK = 1024;

enum : int { PDS_UND = 0, PDS_IN = 1, PDS_OUT = 2 };

struct PdsCtrl {
    long long lo, hi;   // the generation being walked: nodes [lo, hi)
    long long N;        // nodes in the list
    long long rounds;   // generations walked
    long long nv;       // candidates of the generation that passed the first tests
    long long passes;   // conflict-resolution passes over all generations
    int err;            // 1 two nodes in one grid cell, 2 generation too large, 3 list
                        // full, 4 conflict graph too large
    int pad;
};

struct PdsArgs {
    double* X;
    double* Y;
    uint8_t* B;
    double* rc;          // [maxn] cos of each node's rotation angle (set when it is added)
    double* rs;          // [maxn] sin
    int32_t* cell;       // [G*G] node id per cell, -1 empty
    int32_t* chead;      // [G*G] candidate list heads, -1 empty
    int32_t* cnext;      // [capC]
    double* cx;          // [capC] candidates of the generation, index a*K + j
    double* cy;
    int32_t* ccell;      // [capC] grid cell of each candidate inside the domain
    uint8_t* cflag;      // [capC] passed the domain and earlier-generation tests
    int32_t* V;          // [capC] keys of the passing candidates, ascending
    int32_t* state;      // [capC] by position in V (when shared memory is too small)
    int32_t* deg;        // [capC] lower-key conflicts of each passing candidate; after the
                         // passes, the rank of an accepted candidate (-1 otherwise)
    int32_t* off;        // [capC + 1] their CSR offsets
    int32_t* adj;        // [capA] the conflicting lower-key positions
    const double* ex;    // [K] fixed candidate directions
    const double* ey;
    PdsCtrl* ctrl;
    int shape, K;
    double h, cs, r2;
    float inv_cs;        // 1 / cs in FP32, for grid cells
    int64_t G, maxn, capF, capA;
    uint64_t seed;
};

__device__ __forceinline__ bool pds_inside(int shape, double x, double y) {
    if (shape == 0) return x > 0.0 && x < 1.0 && y > 0.0 && y < 1.0;
    double dx = __dsub_rn(x, 0.5), dy = __dsub_rn(y, 0.5);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < 0.25;
}

__device__ __forceinline__ double pds_d2(double ax, double ay, double bx, double by) {
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Grid cell of a point in [0, 1]^2, in FP32.  The grid only accelerates the
// proximity tests (every decision compares exact FP64 squared distances), so
// any cell map keeping two properties gives the same node list: at most one
// node per cell and every node within zeta h of a point inside the 5 x 5
// cells around the point's cell.  With cells of side 0.99 zeta h / sqrt 2,
// FP32 rounding (below 1e-7 in the unit square, h >= 5e-5) moves a point by
// far less than the 1 % margin on both.  One FP64 division per axis would
// cost more than the rest of a candidate's work on this GPU's FP64 pipe.
__device__ __forceinline__ void pds_cell_xy(const PdsArgs& A, double x, double y, int64_t* gx,
                                            int64_t* gy) {
    int64_t a = (int64_t)__fmul_rn(__double2float_rn(x), A.inv_cs);
    int64_t b = (int64_t)__fmul_rn(__double2float_rn(y), A.inv_cs);
    *gx = a < 0 ? 0 : (a >= A.G ? A.G - 1 : a);
    *gy = b < 0 ? 0 : (b >= A.G ? A.G - 1 : b);
}

__device__ __forceinline__ int64_t pds_cell_of(const PdsArgs& A, double x, double y) {
    int64_t gx, gy;
    pds_cell_xy(A, x, y, &gx, &gy);
    return gx * A.G + gy;
}

// seeds: the boundary grid points of the square in row-major order, or the
// disk's boundary nodes at angles 2 pi k / Nb
__global__ void pds_seeds(PdsArgs A, int Kg, int64_t nb) {
    const double two_pi = 6.283185307179586;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nb;
         s += (int64_t)gridDim.x * blockDim.x) {
        double x, y;
        if (A.shape == 0) {
            int64_t i, j;
            const int64_t first = (int64_t)Kg + 1, mid = 2 * ((int64_t)Kg - 1);
            if (s < first) {
                i = 0;
                j = s;
            } else if (s < first + mid) {
                int64_t r = s - first;
                i = 1 + r / 2;
                j = (r & 1) ? Kg : 0;
            } else {
                i = Kg;
                j = s - first - mid;
            }
            x = __dmul_rn((double)i, A.h);
            y = __dmul_rn((double)j, A.h);
        } else {
            double a = __ddiv_rn(__dmul_rn(two_pi, (double)s), (double)nb);
            double ux, uy;
            unit_dir(a, &ux, &uy);
            x = __dadd_rn(0.5, __dmul_rn(0.5, ux));
            y = __dadd_rn(0.5, __dmul_rn(0.5, uy));
        }
        A.X[s] = x;
        A.Y[s] = y;
        A.B[s] = 1;
        if (atomicCAS(&A.cell[pds_cell_of(A, x, y)], -1, (int32_t)s) != -1)
            atomicExch(&A.ctrl->err, 1);
        unit_dir(__dmul_rn(two_pi, unit_draw(A.seed, (uint64_t)s)), &A.rc[s], &A.rs[s]);
    }
}

// the fixed directions e_j at angles 2 pi j / K
__global__ void pds_dirs(int K, double* ex, double* ey) {
    const double two_pi = 6.283185307179586;
    int j = threadIdx.x;
    if (j < K) unit_dir(__ddiv_rn(__dmul_rn(two_pi, (double)j), (double)K), &ex[j], &ey[j]);
}

// candidates of the generation, tested against the domain and the nodes of
// earlier generations (5 x 5 cells: 2 cs > zeta h); one thread per candidate
// (a warp-wide FP64 instruction costs the FP64 pipe the same whatever the
// number of active lanes, so the lanes each take a candidate)
__global__ void pds_gen(PdsArgs A) {
    const long long lo = A.ctrl->lo, hi = A.ctrl->hi;
    if (A.ctrl->err || hi <= lo) return;
    if (hi - lo > A.capF) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&A.ctrl->err, 2);
        return;
    }
    const long long total = (hi - lo) * A.K;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long p = lo + e / A.K;
        const int j = (int)(e % A.K);
        const double c = A.rc[p], s = A.rs[p];
        const double ux = __dsub_rn(__dmul_rn(c, A.ex[j]), __dmul_rn(s, A.ey[j]));
        const double uy = __dadd_rn(__dmul_rn(s, A.ex[j]), __dmul_rn(c, A.ey[j]));
        const double x = __dadd_rn(A.X[p], __dmul_rn(A.h, ux));
        const double y = __dadd_rn(A.Y[p], __dmul_rn(A.h, uy));
        A.cx[e] = x;
        A.cy[e] = y;
        bool ok = pds_inside(A.shape, x, y);
        if (ok) {
            int64_t gx, gy;
            pds_cell_xy(A, x, y, &gx, &gy);
            A.ccell[e] = (int32_t)(gx * A.G + gy);
            for (int64_t a = gx - 2; a <= gx + 2 && ok; ++a) {
                if (a < 0 || a >= A.G) continue;
                for (int64_t b = gy - 2; b <= gy + 2 && ok; ++b) {
                    if (b < 0 || b >= A.G) continue;
                    const int32_t q = A.cell[a * A.G + b];
                    if (q >= 0 && pds_d2(x, y, A.X[q], A.Y[q]) < A.r2) ok = false;
                }
            }
        }
        A.cflag[e] = ok ? 1 : 0;
    }
}

// exclusive scan of one value per thread over a PDS_BLOCK-thread block;
// returns the thread's offset and sets *total
__device__ long long block_excl_scan(long long v, long long* total) {
    __shared__ long long ws[PDS_BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = lane < PDS_BLOCK / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < PDS_BLOCK / 32) ws[lane] = t;
    }
    __syncthreads();
    const long long before = (wid ? ws[wid - 1] : 0) + x - v;
    *total = ws[PDS_BLOCK / 32 - 1];
    __syncthreads();
    return before;
}

// one generation, step 1 (one block): the passing candidates in key order
// (flags read four at a time, tiles of 4 x PDS_BLOCK keys), and per grid cell
// the list of them
__global__ void __launch_bounds__(PDS_BLOCK, 1) pds_compact(PdsArgs A) {
    __shared__ long long s_total;
    __shared__ int s_skip;
    const int t = threadIdx.x;
    if (t == 0) {
        volatile PdsCtrl* c = A.ctrl;
        s_skip = c->err != 0 || c->hi <= c->lo;
        s_total = (c->hi - c->lo) * A.K;
        if (s_skip) c->nv = 0;
    }
    __syncthreads();
    if (s_skip) return;
    const long long total = s_total;
    long long nv = 0;
    for (long long base = 0; base < total; base += 4 * PDS_BLOCK) {
        const long long e = base + 4 * (long long)t;
        unsigned f = 0;
        if (e + 3 < total) {
            const uchar4 q = *reinterpret_cast<const uchar4*>(A.cflag + e);
            f = (q.x ? 1u : 0u) | (q.y ? 2u : 0u) | (q.z ? 4u : 0u) | (q.w ? 8u : 0u);
        } else {
            for (int i = 0; i < 4; ++i)
                if (e + i < total && A.cflag[e + i]) f |= 1u << i;
        }
        long long tile_n;
        long long pos = nv + block_excl_scan(__popc(f), &tile_n);
        for (int i = 0; i < 4; ++i)
            if (f & (1u << i)) A.V[pos++] = (int32_t)(e + i);
        nv += tile_n;
    }
    __syncthreads();
    for (long long v = t; v < nv; v += PDS_BLOCK) {
        const int32_t e = A.V[v];
        A.cnext[v] = atomicExch(&A.chead[A.ccell[e]], (int32_t)v);
    }
    if (t == 0) A.ctrl->nv = nv;
}

// step 2 (whole grid): the lower-key conflicts of each passing candidate;
// FILL = false counts them, FILL = true writes them at the CSR offsets.  One
// thread per candidate: the 25 list heads are loaded first (independent
// loads), then the few non-empty lists are walked.
template <bool FILL>
__global__ void pds_conflicts(PdsArgs A) {
    const long long nv = ((volatile PdsCtrl*)A.ctrl)->nv;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x) {
        const int32_t ev = A.V[v];
        const double x = A.cx[ev], y = A.cy[ev];
        const int32_t cv = A.ccell[ev];
        const long long gx = cv / A.G, gy = cv % A.G;
        int32_t head[25];
#pragma unroll
        for (int l = 0; l < 25; ++l) {
            const long long a = gx - 2 + l / 5, b = gy - 2 + l % 5;
            head[l] = (a >= 0 && a < A.G && b >= 0 && b < A.G) ? A.chead[a * A.G + b] : -1;
        }
        int32_t k = FILL ? A.off[v] : 0;
#pragma unroll
        for (int l = 0; l < 25; ++l) {
            for (int32_t w = head[l]; w >= 0; w = A.cnext[w]) {
                if (w >= v) continue;
                const int32_t ew = A.V[w];
                if (!(pds_d2(x, y, A.cx[ew], A.cy[ew]) < A.r2)) continue;
                if (FILL) A.adj[k] = w;
                ++k;
            }
        }
        if (!FILL) A.deg[v] = k;
    }
}

// step 3 (one block): CSR offsets of the conflict lists
__global__ void __launch_bounds__(PDS_BLOCK, 1) pds_offsets(PdsArgs A) {
    const long long nv = ((volatile PdsCtrl*)A.ctrl)->nv;
    if (nv == 0) return;
    const int t = threadIdx.x;
    const long long per = (nv + PDS_BLOCK - 1) / PDS_BLOCK;
    const long long v0 = min(nv, (long long)t * per), v1 = min(nv, v0 + per);
    long long cnt = 0;
    for (long long v = v0; v < v1; ++v) cnt += A.deg[v];
    long long nnz;
    long long pos = block_excl_scan(cnt, &nnz);
    for (long long v = v0; v < v1; ++v) {
        A.off[v] = (int32_t)pos;
        pos += A.deg[v];
    }
    if (t == 0) {
        A.off[nv] = (int32_t)nnz;
        if (nnz > A.capA) {
            atomicExch(&A.ctrl->err, 4);
            ((volatile PdsCtrl*)A.ctrl)->nv = 0;
        }
    }
}

// The passes of the walk's choice over states st, CSR lists off/adj; thread t
// walks keys [t*per, (t+1)*per) in ascending order.  Returns the number of
// passes.  Each candidate is a chain of dependent loads (its state, its list
// bounds, a neighbour, the neighbour's state), so the loads' latency is the
// cost: the range length is odd, so the 32 lanes of a warp read 32 different
// shared-memory banks, and states are whole words.  A thread need not see the
// other threads' updates within a pass (only its own, in program order, and
// all of them after the barrier), so the states are plain memory.
__device__ __forceinline__ int resolve_passes(int32_t* st, const int32_t* off,
                                              const int32_t* adj, int nv, int t) {
    // ranges of about 32 keys: long enough that most conflict chains stay
    // inside one range, short enough that the passes are short
    int per = (nv + PDS_BLOCK - 1) / PDS_BLOCK;
    per = per < 31 ? 31 : per;
    per |= 1;
    const int v0 = min(nv, t * per), v1 = min(nv, v0 + per);
    int pass = 0;
    for (; pass <= nv; ++pass) {
        int open = 0;
        for (int v = v0; v < v1; ++v) {
            if (st[v] != PDS_UND) continue;
            bool in_lower = false, und_lower = false;
            const int k1 = off[v + 1];
            for (int k = off[v]; k < k1; ++k) {
                const int sw = st[adj[k]];
                if (sw == PDS_IN) {
                    in_lower = true;
                    break;
                }
                if (sw == PDS_UND) und_lower = true;
            }
            if (in_lower) st[v] = PDS_OUT;
            else if (!und_lower) st[v] = PDS_IN;
            else open = 1;
        }
        if (!__syncthreads_or(open)) break;
    }
    return pass + 1;
}

// step 4 (one block): the walk's choice, then the accepted candidates
// appended in key order.  Dynamic shared memory holds the states and, when
// it fits, a copy of the conflict lists (the passes then read shared memory
// only); otherwise both stay in global memory.
__global__ void __launch_bounds__(PDS_BLOCK, 1) pds_resolve(PdsArgs A, int smem_bytes) {
    extern __shared__ int4 s_dyn[];
    __shared__ long long s_N, s_nv;
    __shared__ int s_skip;
    const int t = threadIdx.x;
    if (t == 0) {
        volatile PdsCtrl* c = A.ctrl;
        s_N = c->N;
        s_nv = c->nv;
        s_skip = c->err != 0 || c->hi <= c->lo;
    }
    __syncthreads();
    if (s_skip) return;
    const long long nv = s_nv;
    const long long nnz = nv ? A.off[nv] : 0;   // no offsets are written for nv = 0
    const long long st_bytes = (4 * nv + 15) / 16 * 16;
    const long long off4 = (nv + 1 + 3) / 4, adj4 = (nnz + 3) / 4;   // int4 units
    const bool fit = st_bytes + 16 * (off4 + adj4) <= (long long)smem_bytes;
    int32_t* st;
    int passes;
    if (fit) {
        signed char* base = reinterpret_cast<signed char*>(s_dyn);
        int32_t* sst = reinterpret_cast<int32_t*>(base);
        int4* so = reinterpret_cast<int4*>(base + st_bytes);
        // the conflict lists into shared memory, four independent 16-byte loads
        // per thread in flight (the buffers are padded to whole int4s)
        const int4* go = reinterpret_cast<const int4*>(A.off);
        const int4* ga = reinterpret_cast<const int4*>(A.adj);
        for (long long i = t; i < off4 + adj4; i += 4 * PDS_BLOCK) {
            int4 r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long k = i + (long long)u * PDS_BLOCK;
                if (k < off4 + adj4) r[u] = __ldcg(k < off4 ? go + k : ga + (k - off4));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long k = i + (long long)u * PDS_BLOCK;
                if (k < off4 + adj4) so[k] = r[u];
            }
        }
        for (long long v = t; v < nv; v += PDS_BLOCK) sst[v] = PDS_UND;
        __syncthreads();
        passes = resolve_passes(sst, reinterpret_cast<const int32_t*>(so),
                                reinterpret_cast<const int32_t*>(so + off4), (int)nv, t);
        st = sst;
    } else {
        for (long long v = t; v < nv; v += PDS_BLOCK) A.state[v] = PDS_UND;
        __syncthreads();
        passes = resolve_passes(A.state, A.off, A.adj, (int)nv, t);
        st = A.state;
    }
    // rank of each accepted candidate in key order (its place in the list);
    // the appending is left to pds_commit (many blocks)
    const long long per = (nv + PDS_BLOCK - 1) / PDS_BLOCK;
    const long long v0 = min(nv, (long long)t * per), v1 = min(nv, v0 + per);
    long long cnt = 0;
    for (long long v = v0; v < v1; ++v) cnt += st[v] == PDS_IN;
    long long nacc;
    long long pos = block_excl_scan(cnt, &nacc);
    for (long long v = v0; v < v1; ++v) A.deg[v] = st[v] == PDS_IN ? (int32_t)pos++ : -1;
    if (t == 0) {
        A.ctrl->lo = s_N;
        A.ctrl->hi = s_N + nacc;
        A.ctrl->N = s_N + nacc;
        A.ctrl->rounds += 1;
        A.ctrl->passes += passes;
    }
}

// step 5 (whole grid): append the accepted candidates at their ranks (the
// new generation [lo, hi)), with their rotation angles 2 pi U_id; empty the
// candidate lists
__global__ void pds_commit(PdsArgs A) {
    const double two_pi = 6.283185307179586;
    volatile PdsCtrl* c = A.ctrl;
    if (c->err) return;
    const long long nv = c->nv, lo = c->lo;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (long long)gridDim.x * blockDim.x) {
        const int32_t e = A.V[v];
        const int32_t cell = A.ccell[e];
        A.chead[cell] = -1;
        const int32_t r = A.deg[v];
        if (r < 0) continue;
        const long long id = lo + r;
        if (id >= A.maxn) {
            atomicExch(&A.ctrl->err, 3);
            continue;
        }
        A.X[id] = A.cx[e];
        A.Y[id] = A.cy[e];
        A.B[id] = 0;
        if (atomicCAS(&A.cell[cell], -1, (int32_t)id) != -1) atomicExch(&A.ctrl->err, 1);
        unit_dir(__dmul_rn(two_pi, unit_draw(A.seed, (uint64_t)id)), &A.rc[id], &A.rs[id]);
    }
}

__global__ void pds_copy_out(const PdsArgs A, int64_t N, double* xyz, uint8_t* is_bnd,
                             int64_t cap) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        xyz[i] = A.X[i];
        xyz[cap + i] = A.Y[i];
        is_bnd[i] = A.B[i];
    }
}

static double pds_cell_side(double zeta, double h) {
    return (0.99 * (zeta * h)) / 1.4142135623730951;
}

// cells per axis over [0, 1] (one spare column for FP32 rounding at x = 1)
static int64_t pds_cells_per_axis(int Kg, double zeta) {
    return (int64_t)(1.0 / pds_cell_side(zeta, 1.0 / (double)Kg)) + 2;
}

// one attempt with room for generations of at most capF nodes; returns
// RBFFD_OK, or RBFFD_ERR_CAPACITY with *grow set when a generation was larger
static int pds_run(int shape, int Kg, int K, double zeta, uint64_t seed, int64_t capF,
                   int64_t capA, double* xyz, uint8_t* is_bnd, int64_t cap, int64_t* h_n,
                   int64_t* h_rounds, int* grow, cudaStream_t s) {
    *grow = 0;
    const double h = 1.0 / (double)Kg;
    const int64_t G = pds_cells_per_axis(Kg, zeta);
    const int64_t maxn = G * G;
    const int64_t capC = capF * K;
    const double t = zeta * h;
    PdsArgs A;
    A.shape = shape;
    A.K = K;
    A.h = h;
    A.cs = pds_cell_side(zeta, h);
    A.inv_cs = (float)(1.0 / A.cs);
    A.r2 = t * t;
    A.G = G;
    A.maxn = maxn;
    A.capF = capF;
    A.capA = capA;
    A.seed = seed;
    Scratch bX, bY, bB, brc, brs, bcell, bhead, bnext, bcx, bcy, bflag, bV, bst, bdir, bctl;
    Scratch bdeg, boff, badj, bccell;
    RBFFD_CHECK_CUDA(bccell.alloc(sizeof(int32_t) * capC, s));
    RBFFD_CHECK_CUDA(bdeg.alloc(sizeof(int32_t) * capC, s));
    RBFFD_CHECK_CUDA(boff.alloc(sizeof(int32_t) * (capC + 8), s));   // padded to whole int4s
    RBFFD_CHECK_CUDA(badj.alloc(sizeof(int32_t) * (capA + 8), s));
    RBFFD_CHECK_CUDA(bX.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(bY.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(bB.alloc(maxn, s));
    RBFFD_CHECK_CUDA(brc.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(brs.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(bcell.alloc(sizeof(int32_t) * maxn, s));
    RBFFD_CHECK_CUDA(bhead.alloc(sizeof(int32_t) * maxn, s));
    RBFFD_CHECK_CUDA(bnext.alloc(sizeof(int32_t) * capC, s));
    RBFFD_CHECK_CUDA(bcx.alloc(sizeof(double) * capC, s));
    RBFFD_CHECK_CUDA(bcy.alloc(sizeof(double) * capC, s));
    RBFFD_CHECK_CUDA(bflag.alloc(capC, s));
    RBFFD_CHECK_CUDA(bV.alloc(sizeof(int32_t) * capC, s));
    RBFFD_CHECK_CUDA(bst.alloc(sizeof(int32_t) * capC, s));
    RBFFD_CHECK_CUDA(bdir.alloc(sizeof(double) * 2 * PDS_KMAX, s));
    RBFFD_CHECK_CUDA(bctl.alloc(sizeof(PdsCtrl), s));
    A.X = bX.as<double>();
    A.Y = bY.as<double>();
    A.B = bB.as<uint8_t>();
    A.rc = brc.as<double>();
    A.rs = brs.as<double>();
    A.cell = bcell.as<int32_t>();
    A.chead = bhead.as<int32_t>();
    A.cnext = bnext.as<int32_t>();
    A.cx = bcx.as<double>();
    A.cy = bcy.as<double>();
    A.cflag = bflag.as<uint8_t>();
    A.V = bV.as<int32_t>();
    A.state = bst.as<int32_t>();
    A.ex = bdir.as<double>();
    A.ey = bdir.as<double>() + PDS_KMAX;
    A.ctrl = bctl.as<PdsCtrl>();
    A.ccell = bccell.as<int32_t>();
    A.deg = bdeg.as<int32_t>();
    A.off = boff.as<int32_t>();
    A.adj = badj.as<int32_t>();
    RBFFD_CHECK_CUDA(cudaMemsetAsync(A.cell, 0xff, sizeof(int32_t) * maxn, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(A.chead, 0xff, sizeof(int32_t) * maxn, s));
    const int64_t nb = shape == 0 ? 4 * (int64_t)Kg
                                  : (int64_t)floor((6.283185307179586 * 0.5) / h + 0.5);
    PdsCtrl c0 = {0, nb, nb, 0, 0, 0, 0, 0};
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(A.ctrl, &c0, sizeof(c0), cudaMemcpyHostToDevice, s));
    pds_dirs<<<1, PDS_KMAX, 0, s>>>(K, bdir.as<double>(), bdir.as<double>() + PDS_KMAX);
    pds_seeds<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(A, Kg, nb);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    const unsigned grid = (unsigned)device_sm_count() * 4;
    // shared memory of the resolving block: states and conflict lists
    const int smem_bytes = 200 * 1024;
    RBFFD_CHECK_CUDA(cudaFuncSetAttribute(pds_resolve,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes));
    PdsCtrl hc = c0;
    // each generation appends at least one node until the walk ends, so the
    // walk takes at most maxn generations
    for (int64_t r = 0; r < maxn; r += 16) {
        for (int b = 0; b < 16; ++b) {
            pds_gen<<<grid, 256, 0, s>>>(A);
            pds_compact<<<1, PDS_BLOCK, 0, s>>>(A);
            pds_conflicts<false><<<grid, 256, 0, s>>>(A);
            pds_offsets<<<1, PDS_BLOCK, 0, s>>>(A);
            pds_conflicts<true><<<grid, 256, 0, s>>>(A);
            pds_resolve<<<1, PDS_BLOCK, smem_bytes, s>>>(A, smem_bytes);
            pds_commit<<<grid, 256, 0, s>>>(A);
        }
        RBFFD_CHECK_CUDA(cudaGetLastError());
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(&hc, A.ctrl, sizeof(hc), cudaMemcpyDeviceToHost, s));
        RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
        if (hc.err || hc.hi <= hc.lo) break;
    }
    if (hc.err == 2 || hc.err == 4) {
        *grow = hc.err;
        return RBFFD_ERR_CAPACITY;
    }
    if (hc.err) {
        set_error("rbffd_nodes_pds: internal error %d (grid cell collision or list full)",
                  hc.err);
        return RBFFD_ERR_CUDA;
    }
    if (hc.hi > hc.lo) {
        set_error("rbffd_nodes_pds: the walk did not end");
        return RBFFD_ERR_CUDA;
    }
    *h_n = hc.N;
    if (h_rounds) {
        h_rounds[0] = hc.rounds;
        h_rounds[1] = hc.passes;
    }
    if (hc.N > cap) {
        set_error("rbffd_nodes_pds: %lld nodes, capacity %lld", (long long)hc.N,
                  (long long)cap);
        return RBFFD_ERR_CAPACITY;
    }
    pds_copy_out<<<grid, 256, 0, s>>>(A, hc.N, xyz, is_bnd, cap);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    return RBFFD_OK;
}

// the 3D walk (pds3.cu)
int pds3_run(int Kg, int K, double zeta, uint64_t seed, double* xyz, uint8_t* is_bnd,
             int64_t cap, int64_t* h_n, int64_t* h_rounds, cudaStream_t s);
int64_t pds3_node_bound(int Kg, double zeta);

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_nodes_pds_cap(int d, int Kg, double zeta, int64_t* h_cap) {
    clear_error();
    RBFFD_ARG(h_cap, "rbffd_nodes_pds_cap: NULL argument");
    RBFFD_ARG(d == 2 || d == 3, "rbffd_nodes_pds_cap: d must be 2 or 3");
    RBFFD_ARG(Kg >= 2 && Kg <= (d == 2 ? 20000 : 1000) && zeta > 0.0 && zeta <= 1.0,
              "rbffd_nodes_pds_cap: bad Kg / zeta");
    if (d == 3) {
        *h_cap = pds3_node_bound(Kg, zeta);
        return RBFFD_OK;
    }
    const int64_t G = pds_cells_per_axis(Kg, zeta);
    *h_cap = G * G;
    return RBFFD_OK;
}

extern "C" int rbffd_nodes_pds(int d, int shape, int Kg, int K, double zeta, uint64_t seed,
                               double* xyz, uint8_t* is_bnd, int64_t cap, int64_t* h_n_out,
                               int64_t* h_rounds, void* stream) {
    clear_error();
    RBFFD_ARG(d == 2 || d == 3, "rbffd_nodes_pds: d must be 2 or 3");
    RBFFD_ARG(shape == 0 || (shape == 1 && d == 2),
              "rbffd_nodes_pds: shape must be 0 (square / cube) or 1 (disk, d = 2)");
    RBFFD_ARG(Kg >= 2 && Kg <= (d == 2 ? 20000 : 1000),
              "rbffd_nodes_pds: Kg must be in [2, 20000] (d = 2) or [2, 1000] (d = 3)");
    RBFFD_ARG(K >= 1 && K <= (d == 2 ? PDS_KMAX : 256),
              "rbffd_nodes_pds: K must be in [1, 64] (d = 2) or [1, 256] (d = 3)");
    RBFFD_ARG(zeta > 0.0 && zeta <= 1.0, "rbffd_nodes_pds: zeta must be in (0, 1]");
    RBFFD_ARG(h_n_out && (cap == 0 || (xyz && is_bnd)), "rbffd_nodes_pds: NULL argument");
    cudaStream_t s = as_stream(stream);
    if (d == 3) return pds3_run(Kg, K, zeta, seed, xyz, is_bnd, cap, h_n_out, h_rounds, s);
    const int64_t G = pds_cells_per_axis(Kg, zeta);
    int64_t capF = std::min<int64_t>(G * G, 64 * G + 4096);
    int64_t capA = 8 * capF * K;
    for (int attempt = 0; attempt < 8; ++attempt) {
        int grow = 0;
        int st = pds_run(shape, Kg, K, zeta, seed, capF, capA, xyz, is_bnd, cap, h_n_out,
                         h_rounds, &grow, s);
        if (!grow) return st;
        if (grow == 2) capF = std::min<int64_t>(G * G, capF * 4);
        capA *= 4;
        if (capA > (int64_t(1) << 31) - 1) break;
    }
    set_error("rbffd_nodes_pds: a generation outgrew the scratch buffers");
    return RBFFD_ERR_CUDA;
}
