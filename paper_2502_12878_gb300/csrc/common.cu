// Internal helpers: error strings, scans, bounding box and cell lists.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace rbffd {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

// ------------------------------------------------------------------- scans
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_PER_THREAD = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// block-wide exclusive scan of one value per thread; returns the block total
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* excl) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int64_t base = 0, total = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        if (w < wid) base += warp_tot[w];
        total += warp_tot[w];
    }
    *excl = base + inc - v;
    __syncthreads();
    return total;
}

__global__ void scan_tile_sums(const int32_t* in, int64_t n, int64_t* tmp) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int64_t s = 0;
    for (int k = 0; k < SCAN_PER_THREAD; ++k)
        if (base + k < n) s += in[base + k];
    int64_t ex;
    int64_t tot = block_exclusive_scan(s, &ex);
    if (threadIdx.x == 0) tmp[blockIdx.x] = tot;
}

__global__ void scan_tile_offsets(int64_t* tmp, int64_t ntiles) {
    // single block: exclusive scan of tmp[0..ntiles) in place, total in tmp[ntiles]
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += SCAN_THREADS) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < ntiles ? tmp[i] : 0;
        int64_t ex;
        int64_t tot = block_exclusive_scan(v, &ex);
        if (i < ntiles) tmp[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) tmp[ntiles] = carry;
}

__global__ void scan_tile_apply(const int32_t* in, int32_t* out, int64_t n, const int64_t* tmp,
                                int64_t ntiles) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int32_t v[SCAN_PER_THREAD];
    int64_t s = 0;
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t ex;
    block_exclusive_scan(s, &ex);
    int64_t run = tmp[blockIdx.x] + ex;
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (base + k < n) out[base + k] = (int32_t)run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)tmp[ntiles];
}

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* tmp,
                               cudaStream_t s) {
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    }
    scan_tile_sums<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, n, tmp);
    scan_tile_offsets<<<1, SCAN_THREADS, 0, s>>>(tmp, ntiles);
    // in-place is safe: each tile reads all of its inputs before writing
    scan_tile_apply<<<(unsigned)ntiles, SCAN_THREADS, 0, s>>>(in, out, n, tmp, ntiles);
    return cudaGetLastError();
}

// ----------------------------------------------------------- bounding box
__global__ void bbox_partial(const double* xyz, int64_t N, int d, double* part) {
    __shared__ double smin[3][256], smax[3][256];
    for (int a = 0; a < 3; ++a) {
        double lo = INFINITY, hi = -INFINITY;
        if (a < d)
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
                 i += (int64_t)gridDim.x * blockDim.x) {
                double x = xyz[(int64_t)a * N + i];
                lo = fmin(lo, x);
                hi = fmax(hi, x);
            }
        smin[a][threadIdx.x] = lo;
        smax[a][threadIdx.x] = hi;
    }
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int a = 0; a < 3; ++a) {
                smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + o]);
                smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            part[blockIdx.x * 6 + a] = smin[a][0];
            part[blockIdx.x * 6 + 3 + a] = smax[a][0];
        }
}

int bounding_box(const double* xyz, int64_t N, int d, double* lo, double* hi, cudaStream_t s) {
    const int B = 256;
    double hpart[B * 6];
    Scratch part;
    RBFFD_CHECK_CUDA(part.alloc(sizeof(double) * B * 6, s));
    bbox_partial<<<B, 256, 0, s>>>(xyz, N, d, part.as<double>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(hpart, part.p, sizeof(hpart), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
        for (int b = 0; b < B; ++b) {
            lo[a] = fmin(lo[a], hpart[b * 6 + a]);
            hi[a] = fmax(hi[a], hpart[b * 6 + 3 + a]);
        }
        if (a >= d) lo[a] = hi[a] = 0.0;
    }
    for (int a = 0; a < d; ++a)
        if (!isfinite(lo[a]) || !isfinite(hi[a])) {
            set_error("node coordinates are not finite");
            return RBFFD_ERR_ARG;
        }
    return RBFFD_OK;
}

GridGeom make_grid(int d, const double* lo, const double* hi, int64_t N, double per_cell) {
    GridGeom g;
    g.d = d;
    double vol = 1.0, maxext = 0.0;
    for (int a = 0; a < d; ++a) {
        double e = hi[a] - lo[a];
        maxext = std::max(maxext, e);
    }
    if (!(maxext > 0)) maxext = 1.0;
    for (int a = 0; a < d; ++a) vol *= std::max(hi[a] - lo[a], maxext * 1e-6);
    double cs = pow(vol * per_cell / (double)std::max<int64_t>(N, 1), 1.0 / d);
    // keep the cell count below 2^26 and no cell thinner than the extent allows
    for (;;) {
        int64_t tot = 1;
        for (int a = 0; a < d; ++a) {
            double e = hi[a] - lo[a];
            int64_t Ga = (int64_t)floor(e / cs) + 1;
            tot *= Ga;
        }
        if (tot <= (int64_t(1) << 26)) break;
        cs *= 1.25;
    }
    g.cs = cs;
    for (int a = 0; a < 3; ++a) {
        if (a < d) {
            g.org[a] = lo[a];
            g.G[a] = (int)floor((hi[a] - lo[a]) / cs) + 1;
        } else {
            g.org[a] = 0.0;
            g.G[a] = 1;
        }
    }
    return g;
}

__device__ inline int64_t cell_of(const double* xyz, int64_t N, int64_t i, const GridGeom& g) {
    int64_t c = 0;
    for (int a = 0; a < g.d; ++a) {
        int ca = cell_coord(xyz[(int64_t)a * N + i], g.org[a], g.cs, g.G[a]);
        c = c * g.G[a] + ca;
    }
    return c;
}

__global__ void cells_key(const double* xyz, int64_t N, GridGeom g, int32_t* key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        key[i] = (int32_t)cell_of(xyz, N, i, g);
}

__global__ void keys_count(const int32_t* key, int64_t N, int32_t* count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&count[key[i]], 1);
}

__global__ void cells_scatter(int64_t N, const int32_t* cellof, int32_t* cursor, int32_t* sorted) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int pos = atomicAdd(&cursor[cellof[i]], 1);
        sorted[pos] = (int32_t)i;
    }
}

// ids inside each cell into ascending order (cells hold a handful of nodes)
__global__ void cells_sort(int64_t ncell, const int32_t* start, int32_t* sorted) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        int b = start[c], e = start[c + 1];
        for (int i = b + 1; i < e; ++i) {
            int v = sorted[i];
            int j = i - 1;
            while (j >= b && sorted[j] > v) {
                sorted[j + 1] = sorted[j];
                --j;
            }
            sorted[j + 1] = v;
        }
    }
}

int counting_sort_by_key(const int32_t* key, int64_t N, int64_t nkeys, int32_t* start,
                         int32_t* sorted, cudaStream_t s) {
    Scratch count, tmp;
    RBFFD_CHECK_CUDA(count.alloc(sizeof(int32_t) * (size_t)(nkeys + 1), s));
    RBFFD_CHECK_CUDA(tmp.alloc(sizeof(int64_t) * (size_t)scan_tmp_elems(nkeys), s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(count.p, 0, sizeof(int32_t) * (size_t)(nkeys + 1), s));
    int sms = device_sm_count();
    keys_count<<<sms * 8, 256, 0, s>>>(key, N, count.as<int32_t>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(exclusive_scan_i32(count.as<int32_t>(), start, nkeys, tmp.as<int64_t>(), s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(count.p, start, sizeof(int32_t) * (size_t)nkeys,
                                     cudaMemcpyDeviceToDevice, s));
    cells_scatter<<<sms * 8, 256, 0, s>>>(N, key, count.as<int32_t>(), sorted);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    cells_sort<<<sms * 8, 256, 0, s>>>(nkeys, start, sorted);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}

int build_cell_lists(const double* xyz, int64_t N, const GridGeom& g, int32_t* cell_start,
                     int32_t* sorted, cudaStream_t s) {
    Scratch key;
    RBFFD_CHECK_CUDA(key.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(N, 1), s));
    int sms = device_sm_count();
    cells_key<<<sms * 8, 256, 0, s>>>(xyz, N, g, key.as<int32_t>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return counting_sort_by_key(key.as<int32_t>(), N, g.ncell(), cell_start, sorted, s);
}

}  // namespace rbffd

extern "C" const char* rbffd_last_error(void) { return rbffd::g_err; }
extern "C" int rbffd_version(void) { return 100; }
