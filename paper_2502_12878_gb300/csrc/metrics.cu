// rbffd_error: error of an iterate against a reference field (Eq. 8 of the
// paper: e = (1/N) sum |u_i - u^a_i| over the nodes of the domain), plus the
// max-norm.  Two-pass deterministic reduction: per-block partials in a fixed
// grid, then one block sums them in a fixed order.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace rbffd {

static constexpr int ERR_BLOCKS = 512;

__global__ void error_partials(const double* u, const double* ua, int64_t N, double* part) {
    __shared__ double ss[256];
    __shared__ unsigned long long sm[256];
    double s = 0.0;
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double e = fabs(__dsub_rn(u[i], ua[i]));
        s = __dadd_rn(s, e);
        unsigned long long b = (unsigned long long)__double_as_longlong(e);
        if (e != e) b = 0x7ff8000000000000ull;   // NaN dominates the max
        m = max(m, b);
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] = __dadd_rn(ss[threadIdx.x], ss[threadIdx.x + o]);
            sm[threadIdx.x] = max(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = __longlong_as_double((long long)sm[0]);
    }
}

__global__ void error_final(const double* part, int nparts, int64_t N, double* out) {
    __shared__ double ss[256];
    __shared__ unsigned long long sm[256];
    double s = 0.0;
    unsigned long long m = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s = __dadd_rn(s, part[2 * i]);
        m = max(m, (unsigned long long)__double_as_longlong(part[2 * i + 1]));
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] = __dadd_rn(ss[threadIdx.x], ss[threadIdx.x + o]);
            sm[threadIdx.x] = max(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = __longlong_as_double((long long)sm[0]);
        out[1] = __ddiv_rn(ss[0], (double)N);
    }
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_error(const double* u, const double* ua, int64_t N, double* h_max,
                           double* h_mean, void* stream) {
    clear_error();
    RBFFD_ARG(N >= 1, "rbffd_error: N must be positive");
    RBFFD_ARG(u && ua, "rbffd_error: NULL argument");
    cudaStream_t s = as_stream(stream);
    Scratch part;
    RBFFD_CHECK_CUDA(part.alloc(sizeof(double) * (2 * ERR_BLOCKS + 2), s));
    double* p = part.as<double>();
    error_partials<<<ERR_BLOCKS, 256, 0, s>>>(u, ua, N, p);
    error_final<<<1, 256, 0, s>>>(p, ERR_BLOCKS, N, p + 2 * ERR_BLOCKS);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    double out[2];
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(out, p + 2 * ERR_BLOCKS, sizeof(out), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h_max) *h_max = out[0];
    if (h_mean) *h_mean = out[1];
    return RBFFD_OK;
}

// ---------------------------------------------------------------------------
// rbffd_fp64_fma_rate: the device's FP64 fused multiply-add rate, measured -
// the roofline of the kernels the FP64 pipe binds (the explicit sweep at
// larger stencils, the weight build).  Not part of the paper's method.
// Every thread runs CH independent chains acc <- fma(w, v, acc), four fmas per
// chain per loop iteration, with v read from shared memory - as the sweeps'
// operands arrive from loads.  (Chains whose operands all stay in registers
// saturate near 1.6-1.7 fma/clk/SM on this GPU, below the rate that the
// sweeps themselves reach; with one operand from a load they reach the pipe's
// 2 fma/clk/SM.)  The result is kept alive by a store that never happens.
// Shapes with 4 and 8 chains per thread at the largest resident grid of
// 256-thread blocks are timed and the fastest kept.
// ---------------------------------------------------------------------------
namespace rbffd {

static __device__ double g_fma_sink;

template <int CH>
__global__ void __launch_bounds__(256) fp64_fma_chains(long long iters) {
    __shared__ double sv[256];
    sv[threadIdx.x] = 0.5 + 1e-6 * (double)threadIdx.x;
    __syncthreads();
    double acc[CH], w[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        acc[c] = 0.0;
        w[c] = 1e-3 * (double)(threadIdx.x + 3 * c + 1);
    }
    const int t = (int)threadIdx.x;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c)
                acc[c] = __fma_rn(w[c], sv[(t + 4 * c + u) & 255], acc[c]);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s = __dadd_rn(s, acc[c]);
    if (s == -1.0) g_fma_sink = s;
}
template <int CH>
static cudaError_t time_fma_shape(long long fmas_per_thread, cudaStream_t s, double* rate,
                                  float* ms_out) {
    int per_sm = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_chains<CH>, 256, 0);
    if (e != cudaSuccess) return e;
    const int grid = device_sm_count() * std::max(1, per_sm);
    const long long iters = std::max<long long>(1, fmas_per_thread / (4 * CH));
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    fp64_fma_chains<CH><<<grid, 256, 0, s>>>(std::max<long long>(1, iters / 16));   // warm-up
    cudaEventRecord(e0, s);
    fp64_fma_chains<CH><<<grid, 256, 0, s>>>(iters);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) {
        *rate = (double)grid * 256.0 * 4.0 * CH * (double)iters / (ms * 1e-3);
        *ms_out = ms;
    }
    return e;
}

}  // namespace rbffd

extern "C" int rbffd_fp64_fma_rate(int64_t iters, double* h_fma_per_s, double* h_ms,
                                   void* stream) {
    using namespace rbffd;
    clear_error();
    RBFFD_ARG(iters >= 1 && iters <= (int64_t(1) << 32) && h_fma_per_s,
              "rbffd_fp64_fma_rate: bad argument");
    cudaStream_t s = as_stream(stream);
    // `iters` fmas per thread in each timed launch
    double best = 0.0, r = 0.0;
    float best_ms = 0.f, ms = 0.f;
    RBFFD_CHECK_CUDA(time_fma_shape<4>(iters, s, &r, &ms));
    if (r > best) { best = r; best_ms = ms; }
    RBFFD_CHECK_CUDA(time_fma_shape<8>(iters, s, &r, &ms));
    if (r > best) { best = r; best_ms = ms; }
    *h_fma_per_s = best;
    if (h_ms) *h_ms = best_ms;
    return RBFFD_OK;
}
