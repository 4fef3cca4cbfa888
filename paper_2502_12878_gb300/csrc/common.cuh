// Internal helpers shared by the librbffd translation units: status/error
// reporting, stream-ordered scratch, exclusive scans, and the uniform cell
// grid (counting sort of nodes into cells) used by support selection and by
// the plan's node reordering.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "../../include/rbffd.h"

namespace rbffd {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();

#define RBFFD_CHECK_CUDA(expr)                                                        \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess) {                                                      \
            ::rbffd::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,            \
                               cudaGetErrorString(_e));                               \
            return RBFFD_ERR_CUDA;                                                    \
        }                                                                             \
    } while (0)

#define RBFFD_ARG(cond, ...)                                                          \
    do {                                                                              \
        if (!(cond)) {                                                                \
            ::rbffd::set_error(__VA_ARGS__);                                          \
            return RBFFD_ERR_ARG;                                                     \
        }                                                                             \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int device_sm_count();

// --------------------------------------------------- stream-ordered scratch
// RAII holder for cudaMallocAsync memory; freed on the same stream.
struct Scratch {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    Scratch() = default;
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return cudaMallocAsync(&p, bytes < 256 ? 256 : bytes, st);
    }
    template <class T>
    T* as() const { return reinterpret_cast<T*>(p); }
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

// ------------------------------------------------------------------- scans
// Exclusive prefix sum of n int32 counts into out[0..n] (out[n] = total).
// out may alias in only if out has n+1 slots and in == out.
// tmp must hold scan_tmp_elems(n) int64 values.
int64_t scan_tmp_elems(int64_t n);
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* tmp,
                               cudaStream_t s);

// ------------------------------------------------------------- cell grid
struct GridGeom {
    int d = 2;
    int G[3] = {1, 1, 1};     // cells per axis
    double org[3] = {0, 0, 0};
    double cs = 1.0;          // cell edge
    int64_t ncell() const { return (int64_t)G[0] * G[1] * G[2]; }
};

// Bounding box of the node set on the device, copied to the host (syncs).
int bounding_box(const double* xyz, int64_t N, int d, double* lo, double* hi, cudaStream_t s);

// Geometry with about `per_cell` nodes per cell over the bounding box.
GridGeom make_grid(int d, const double* lo, const double* hi, int64_t N, double per_cell);

__host__ __device__ inline int cell_coord(double x, double org, double cs, int G) {
    double t = (x - org) / cs;
    int c = (int)floor(t);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

// Counting sort of node ids by cell (row-major cells, last axis fastest):
// cell_start [ncell+1], sorted [N]; inside a cell ids ascend.
int build_cell_lists(const double* xyz, int64_t N, const GridGeom& g, int32_t* cell_start,
                     int32_t* sorted, cudaStream_t s);

// Counting sort of ids 0..N-1 by key[i] in [0, nkeys): start [nkeys+1],
// sorted [N]; ids ascend inside a key (insertion sort per key: meant for keys
// that hold a handful of ids each).
int counting_sort_by_key(const int32_t* key, int64_t N, int64_t nkeys, int32_t* start,
                         int32_t* sorted, cudaStream_t s);

// kernels of common.cu that other translation units launch directly
__global__ void bbox_partial(const double* xyz, int64_t N, int d, double* part);
__global__ void cells_key(const double* xyz, int64_t N, GridGeom g, int32_t* key);
__global__ void keys_count(const int32_t* key, int64_t N, int32_t* count);
__global__ void cells_scatter(int64_t N, const int32_t* cellof, int32_t* cursor, int32_t* sorted);
__global__ void cells_sort(int64_t ncell, const int32_t* start, int32_t* sorted);

}  // namespace rbffd
