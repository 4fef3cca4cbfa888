// rbffd_error: error of an iterate against a reference field (Eq. 8 of the
// paper: e = (1/N) sum |u_i - u^a_i| over the nodes of the domain), plus the
// max-norm.  Two-pass deterministic reduction: per-block partials in a fixed
// grid, then one block sums them in a fixed order.
#include <math.h>

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
