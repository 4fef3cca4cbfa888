// rbffd_knn: support selection (Sec. II, text after Eq. 1) - for each centre
// the n nearest nodes, centre included, ordered by the key (d2, node index).
//
// Design: nodes are binned into a uniform cell grid (about one node per
// cell; counting sort, ids ascending inside a cell).  One warp serves one
// centre.  It scans the cells of a box of Chebyshev radius r around the
// centre's cell, streaming candidates through a warp-local top-n (candidates
// that cannot beat the current n-th key are dropped by a ballot; survivors are
// merged by exact rank), then grows the box until every node outside it is
// provably farther than the current n-th key.  Growing only scans the new
// shell.  Squared distances are formed exactly like the definition
// (fl(fl(dx*dx) + fl(dy*dy) ...), no contraction), so ties resolve by index
// and the result is bit-identical to any exact implementation.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace rbffd {

static constexpr int KNN_NMAX = 128;
static constexpr int KNN_BUF = 64;
static constexpr int KNN_WARPS = 4;

// distances are kept as the IEEE bits of d2: for non-negative doubles the
// unsigned integer order is the numeric order, so the (d2, index) key
// comparisons of the merges run on the integer pipes, not the FP64 pipe
struct KnnSmem {
    unsigned long long bd[2][KNN_NMAX];
    int32_t bj[2][KNN_NMAX];
    unsigned long long cd[KNN_BUF];
    int32_t cj[KNN_BUF];
    int32_t rb[32], rpre[32];   // range begin, inclusive prefix of lengths
};

struct KnnArgs {
    const double* xyz;
    int64_t N;
    int d;
    const int32_t* centres;
    int64_t nc;
    int n;
    int32_t* idx;
    GridGeom g;
    const int32_t* cell_start;
    const int32_t* sorted;
    const uint8_t* cand;   // NULL, or only nodes with cand != 0 (and the centre) qualify
    int r0;
    int* err;
};

__device__ __forceinline__ bool kless(unsigned long long da, int32_t ja, unsigned long long db,
                                      int32_t jb) {
    return da < db || (da == db && ja < jb);
}

__device__ __forceinline__ double sqdist(const double* xyz, int64_t N, int d, int32_t j,
                                         const double* q) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        double t = __dsub_rn(xyz[(int64_t)a * N + j], q[a]);
        double sq = __dmul_rn(t, t);
        s = (a == 0) ? sq : __dadd_rn(s, sq);
    }
    return s;
}

// merge best[cur] (nb entries) with the buffer (nbuf) into best[cur^1]; keep n
__device__ void knn_merge(KnnSmem& sm, int& cur, int& nb, int nbuf, int n, int lane) {
    __syncwarp();
    int L = nb + nbuf;
    for (int e = lane; e < L; e += 32) {
        unsigned long long de = e < nb ? sm.bd[cur][e] : sm.cd[e - nb];
        int32_t je = e < nb ? sm.bj[cur][e] : sm.cj[e - nb];
        int rank = 0;
        for (int f = 0; f < nb; ++f) rank += kless(sm.bd[cur][f], sm.bj[cur][f], de, je);
        for (int f = 0; f < nbuf; ++f) rank += kless(sm.cd[f], sm.cj[f], de, je);
        if (rank < n) {
            sm.bd[cur ^ 1][rank] = de;
            sm.bj[cur ^ 1][rank] = je;
        }
    }
    __syncwarp();
    cur ^= 1;
    nb = L < n ? L : n;
}

__global__ void __launch_bounds__(32 * KNN_WARPS) knn_kernel(KnnArgs A) {
    __shared__ KnnSmem smem[KNN_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    KnnSmem& sm = smem[wib];
    const GridGeom& g = A.g;
    const int d = A.d, n = A.n;
    const int last = d - 1;   // contiguous axis of the row-major cell grid
    const int64_t warps = (int64_t)gridDim.x * KNN_WARPS;

    for (int64_t qi = (int64_t)blockIdx.x * KNN_WARPS + wib; qi < A.nc; qi += warps) {
        const int32_t c = A.centres[qi];
        double q[3] = {0, 0, 0};
        int cc[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            q[a] = A.xyz[(int64_t)a * A.N + c];
            cc[a] = cell_coord(q[a], g.org[a], g.cs, g.G[a]);
        }
        int cur = 0, nb = 0, nbuf = 0;
        int r = A.r0, prev = -1;
        bool done = false;
        for (int guard = 0; guard < 1 << 20 && !done; ++guard) {
            // rows of the box: all axes but the last; each row gives two slots
            // (left and right of the previous box, or the whole row)
            int side = 2 * r + 1;
            int64_t nrows = 1;
            for (int a = 0; a < last; ++a) nrows *= side;
            int64_t nslots = 2 * nrows;
            for (int64_t s0 = 0; s0 < nslots; s0 += 32) {
                // lane k describes slot s0 + k as a range of `sorted`
                int64_t s = s0 + lane;
                int32_t beg = 0, len = 0;
                if (s < nslots) {
                    int64_t row = s >> 1;
                    int half = (int)(s & 1);
                    bool ok = true, inside_prev = (prev >= 0);
                    int64_t cell_row = 0;
                    int64_t rem = row;
                    int crow[3] = {0, 0, 0};
                    for (int a = last - 1; a >= 0; --a) {
                        crow[a] = cc[a] - r + (int)(rem % side);
                        rem /= side;
                    }
                    for (int a = 0; a < last; ++a) {
                        if (crow[a] < 0 || crow[a] >= g.G[a]) ok = false;
                        int dd = crow[a] - cc[a];
                        if (dd < -prev || dd > prev) inside_prev = false;
                        cell_row = cell_row * g.G[a] + crow[a];
                    }
                    int lo = cc[last] - r, hi = cc[last] + r;
                    if (inside_prev) {
                        if (half == 0) hi = cc[last] - prev - 1;
                        else lo = cc[last] + prev + 1;
                    } else if (half == 1) {
                        ok = false;
                    }
                    if (lo < 0) lo = 0;
                    if (hi > g.G[last] - 1) hi = g.G[last] - 1;
                    if (ok && lo <= hi) {
                        int64_t base = cell_row * g.G[last];
                        beg = A.cell_start[base + lo];
                        len = A.cell_start[base + hi + 1] - beg;
                    }
                }
                int32_t pre = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int32_t t = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += t;
                }
                sm.rb[lane] = beg;
                sm.rpre[lane] = pre;
                int32_t total = __shfl_sync(0xffffffffu, pre, 31);
                __syncwarp();
                for (int32_t v0 = 0; v0 < total; v0 += 32) {
                    if (nbuf + 32 > KNN_BUF) {
                        knn_merge(sm, cur, nb, nbuf, n, lane);
                        nbuf = 0;
                    }
                    int32_t v = v0 + lane;
                    bool acc = false;
                    unsigned long long dv = 0;
                    int32_t jv = 0;
                    if (v < total) {
                        int k = 0;   // first slot with inclusive prefix > v
                        for (int step = 16; step > 0; step >>= 1)
                            if (sm.rpre[k + step - 1] <= v) k += step;
                        int32_t off = v - (k ? sm.rpre[k - 1] : 0);
                        jv = A.sorted[sm.rb[k] + off];
                        dv = (unsigned long long)__double_as_longlong(sqdist(A.xyz, A.N, d, jv, q));
                        acc = (nb < n) || kless(dv, jv, sm.bd[cur][n - 1], sm.bj[cur][n - 1]);
                        if (A.cand && !A.cand[jv] && jv != c) acc = false;
                    }
                    unsigned m = __ballot_sync(0xffffffffu, acc);
                    if (acc) {
                        int p = nbuf + __popc(m & ((1u << lane) - 1u));
                        sm.cd[p] = dv;
                        sm.cj[p] = jv;
                    }
                    nbuf += __popc(m);
                }
                __syncwarp();
            }
            if (nbuf > 0) {
                knn_merge(sm, cur, nb, nbuf, n, lane);
                nbuf = 0;
            }
            // termination: every node outside the box is farther than the n-th key
            double bound = INFINITY;
            bool whole = true;
            for (int a = 0; a < d; ++a) {
                int lo = cc[a] - r, hi = cc[a] + r;
                if (lo > 0) {
                    whole = false;
                    bound = fmin(bound, q[a] - (g.org[a] + (double)lo * g.cs));
                }
                if (hi < g.G[a] - 1) {
                    whole = false;
                    bound = fmin(bound, (g.org[a] + (double)(hi + 1) * g.cs) - q[a]);
                }
            }
            if (whole) {
                done = true;
            } else if (nb == n) {
                double be = bound - 1e-6 * g.cs;
                double worst = __longlong_as_double((long long)sm.bd[cur][n - 1]);
                if (be > 0.0 && worst < be * be * (1.0 - 1e-12)) {
                    done = true;
                } else {
                    int need = (int)ceil(sqrt(worst) / g.cs) + 1;
                    prev = r;
                    r = need > r + 1 ? need : r + 1;
                }
            } else {
                prev = r;
                r = r + 1;
            }
        }
        if (!done && lane == 0) atomicExch(A.err, 1);
        if (done && nb < n && lane == 0) atomicExch(A.err, 2);   // too few candidates
        __syncwarp();
        for (int k = lane; k < n; k += 32)
            A.idx[qi * n + k] = k < nb ? sm.bj[cur][k] : -1;
        __syncwarp();
    }
}

}  // namespace rbffd

using namespace rbffd;

static int knn_impl(const double* xyz, int64_t N, int d, const uint8_t* cand,
                    const int32_t* centres, int64_t nc, int n, int32_t* idx, void* stream) {
    RBFFD_ARG(nc >= 0, "rbffd_knn: negative centre count");
    if (nc == 0) return RBFFD_OK;
    RBFFD_ARG(xyz && centres && idx, "rbffd_knn: NULL argument");
    RBFFD_ARG(d >= 1 && d <= 3, "rbffd_knn: d must be 1, 2 or 3");
    RBFFD_ARG(N >= 1 && N < (int64_t(1) << 31), "rbffd_knn: bad N");
    RBFFD_ARG(n >= 1 && n <= KNN_NMAX && n <= N, "rbffd_knn: need 1 <= n <= min(N, %d)",
              KNN_NMAX);
    cudaStream_t s = as_stream(stream);
    double lo[3], hi[3];
    int st = bounding_box(xyz, N, d, lo, hi, s);
    if (st) return st;
    GridGeom g = make_grid(d, lo, hi, N, 1.0);
    int64_t ncell = g.ncell();
    Scratch start, sorted, err;
    RBFFD_CHECK_CUDA(start.alloc(sizeof(int32_t) * (size_t)(ncell + 1), s));
    RBFFD_CHECK_CUDA(sorted.alloc(sizeof(int32_t) * (size_t)N, s));
    RBFFD_CHECK_CUDA(err.alloc(sizeof(int), s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    st = build_cell_lists(xyz, N, g, start.as<int32_t>(), sorted.as<int32_t>(), s);
    if (st) return st;
    // initial box radius: cells holding about n nodes in a ball at mean density
    double per_cell = (double)N / (double)ncell;
    const double ball[4] = {0, 2.0, M_PI, 4.0 * M_PI / 3.0};
    double rad = pow((double)n / (ball[d] * per_cell), 1.0 / d);
    KnnArgs A;
    A.xyz = xyz;
    A.N = N;
    A.d = d;
    A.centres = centres;
    A.nc = nc;
    A.n = n;
    A.idx = idx;
    A.g = g;
    A.cell_start = start.as<int32_t>();
    A.sorted = sorted.as<int32_t>();
    A.cand = cand;
    A.r0 = (int)ceil(rad) > 1 ? (int)ceil(rad) : 1;
    A.err = err.as<int>();
    int sms = device_sm_count();
    int64_t blocks = (nc + KNN_WARPS - 1) / KNN_WARPS;
    int64_t cap = (int64_t)sms * 64;
    knn_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 32 * KNN_WARPS, 0, s>>>(A);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    int herr = 0;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (herr == 2) {
        set_error("rbffd_knn: fewer than n candidate nodes");
        return RBFFD_ERR_ARG;
    }
    if (herr) {
        set_error("rbffd_knn: ring search did not terminate");
        return RBFFD_ERR_CAPACITY;
    }
    return RBFFD_OK;
}

extern "C" int rbffd_knn(const double* xyz, int64_t N, int d, const int32_t* centres, int64_t nc,
                         int n, int32_t* idx, void* stream) {
    clear_error();
    return knn_impl(xyz, N, d, nullptr, centres, nc, n, idx, stream);
}

extern "C" int rbffd_knn_masked(const double* xyz, int64_t N, int d, const uint8_t* cand,
                                const int32_t* centres, int64_t nc, int n, int32_t* idx,
                                void* stream) {
    clear_error();
    RBFFD_ARG(cand != nullptr || nc == 0, "rbffd_knn_masked: NULL candidate mask");
    return knn_impl(xyz, N, d, cand, centres, nc, n, idx, stream);
}



// ---------------------------------------------------------------------------
// rbffd_knn_noalloc: the same support selection for callers that cannot
// allocate device memory while they run.  Its working memory is one
// file-scope __device__ array of fixed size (every GPU that loads the library
// holds it until the process exits), reached from host code through the
// address that cudaGetSymbolAddress returns for the current device.
// ---------------------------------------------------------------------------
namespace rbffd {

static constexpr int64_t NA_MAX_NODES = RBFFD_KNN_NOALLOC_MAX_NODES;
static constexpr int64_t NA_MAX_CELLS = 2 * NA_MAX_NODES;
static constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
static constexpr int NA_BBOX_BLOCKS = 256;
// byte offsets of the regions inside the scratch array (each 256-aligned)
static constexpr size_t NA_OFF_PART = 0;                                       // bbox partials
static constexpr size_t NA_OFF_ERR = NA_OFF_PART + na_round(sizeof(double) * 6 * NA_BBOX_BLOCKS);
static constexpr size_t NA_OFF_START = NA_OFF_ERR + 256;                         // cell starts
static constexpr size_t NA_OFF_COUNT = NA_OFF_START + na_round(4 * (NA_MAX_CELLS + 1));
static constexpr size_t NA_OFF_TMP = NA_OFF_COUNT + na_round(4 * (NA_MAX_CELLS + 1));
static constexpr int64_t NA_TMP_ELEMS = (NA_MAX_CELLS + 2047) / 2048 + 1;      // scan tiles
static constexpr size_t NA_OFF_KEY = NA_OFF_TMP + na_round(8 * NA_TMP_ELEMS);
static constexpr size_t NA_OFF_SORTED = NA_OFF_KEY + na_round(4 * NA_MAX_NODES);
static constexpr size_t NA_BYTES = NA_OFF_SORTED + na_round(4 * NA_MAX_NODES);

static __device__ __align__(256) unsigned char g_knn_noalloc_scratch[NA_BYTES];

// device address of the scratch array for the current device, looked up once
// per device (host code may not use the array's name as a device pointer)
static int noalloc_scratch(unsigned char** out) {
    static std::mutex mu;
    static void* addr[128] = {};
    int dev = 0;
    RBFFD_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) {
        set_error("rbffd_knn_noalloc: device ordinal %d out of range", dev);
        return RBFFD_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_knn_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("rbffd_knn_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return RBFFD_ERR_CUDA;
        }
        addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(addr[dev]);
    return RBFFD_OK;
}

}  // namespace rbffd

extern "C" int rbffd_knn_noalloc(const double* xyz, int64_t N, int d, const int32_t* centres,
                                 int64_t nc, int n, int32_t* idx, void* stream) {
    clear_error();
    RBFFD_ARG(nc >= 0, "rbffd_knn_noalloc: negative centre count");
    RBFFD_ARG(d >= 1 && d <= 3, "rbffd_knn_noalloc: d must be 1, 2 or 3");
    RBFFD_ARG(N >= 1, "rbffd_knn_noalloc: bad N");
    if (N > NA_MAX_NODES) {
        set_error("rbffd_knn_noalloc: %lld nodes exceed the fixed scratch limit of %lld "
                  "(use rbffd_knn)", (long long)N, (long long)NA_MAX_NODES);
        return RBFFD_ERR_CAPACITY;
    }
    RBFFD_ARG(n >= 1 && n <= KNN_NMAX && n <= N, "rbffd_knn_noalloc: need 1 <= n <= min(N, %d)",
              KNN_NMAX);
    if (nc == 0) return RBFFD_OK;
    RBFFD_ARG(xyz && centres && idx, "rbffd_knn_noalloc: NULL argument");
    cudaStream_t s = as_stream(stream);
    unsigned char* base = nullptr;
    int st = noalloc_scratch(&base);
    if (st) return st;
    double* part = reinterpret_cast<double*>(base + NA_OFF_PART);
    int* err = reinterpret_cast<int*>(base + NA_OFF_ERR);
    int32_t* start = reinterpret_cast<int32_t*>(base + NA_OFF_START);
    int32_t* count = reinterpret_cast<int32_t*>(base + NA_OFF_COUNT);
    int64_t* tmp = reinterpret_cast<int64_t*>(base + NA_OFF_TMP);
    int32_t* key = reinterpret_cast<int32_t*>(base + NA_OFF_KEY);
    int32_t* sorted = reinterpret_cast<int32_t*>(base + NA_OFF_SORTED);

    // bounding box (partials in the scratch array, final reduction on the host)
    double hpart[NA_BBOX_BLOCKS * 6];
    bbox_partial<<<NA_BBOX_BLOCKS, 256, 0, s>>>(xyz, N, d, part);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(hpart, part, sizeof(hpart), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
        for (int b = 0; b < NA_BBOX_BLOCKS; ++b) {
            lo[a] = fmin(lo[a], hpart[b * 6 + a]);
            hi[a] = fmax(hi[a], hpart[b * 6 + 3 + a]);
        }
        if (a >= d) lo[a] = hi[a] = 0.0;
    }
    for (int a = 0; a < d; ++a)
        RBFFD_ARG(isfinite(lo[a]) && isfinite(hi[a]), "rbffd_knn_noalloc: coordinates not finite");
    // cell grid of about one node per cell, coarsened to fit the fixed cell arrays
    GridGeom g = make_grid(d, lo, hi, N, 1.0);
    while (g.ncell() > NA_MAX_CELLS) {
        g.cs *= 1.25;
        for (int a = 0; a < d; ++a) g.G[a] = (int)floor((hi[a] - lo[a]) / g.cs) + 1;
    }
    const int64_t ncell = g.ncell();
    const int sms = device_sm_count();
    // the scratch keeps the previous call's contents: clear what must start at 0
    RBFFD_CHECK_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * (ncell + 1), s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    cells_key<<<sms * 8, 256, 0, s>>>(xyz, N, g, key);
    keys_count<<<sms * 8, 256, 0, s>>>(key, N, count);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(exclusive_scan_i32(count, start, ncell, tmp, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(count, start, sizeof(int32_t) * ncell,
                                     cudaMemcpyDeviceToDevice, s));
    cells_scatter<<<sms * 8, 256, 0, s>>>(N, key, count, sorted);
    cells_sort<<<sms * 8, 256, 0, s>>>(ncell, start, sorted);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    double per_cell = (double)N / (double)ncell;
    const double ball[4] = {0, 2.0, M_PI, 4.0 * M_PI / 3.0};
    double rad = pow((double)n / (ball[d] * per_cell), 1.0 / d);
    KnnArgs A;
    A.xyz = xyz;
    A.N = N;
    A.d = d;
    A.centres = centres;
    A.nc = nc;
    A.n = n;
    A.idx = idx;
    A.g = g;
    A.cell_start = start;
    A.sorted = sorted;
    A.cand = nullptr;
    A.r0 = (int)ceil(rad) > 1 ? (int)ceil(rad) : 1;
    A.err = err;
    int64_t blocks = (nc + KNN_WARPS - 1) / KNN_WARPS;
    int64_t cap = (int64_t)sms * 64;
    knn_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 32 * KNN_WARPS, 0, s>>>(A);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    int herr = 0;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("rbffd_knn_noalloc: ring search did not terminate");
        return RBFFD_ERR_CAPACITY;
    }
    return RBFFD_OK;
}

