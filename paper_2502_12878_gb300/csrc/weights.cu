// rbffd_weights: batched RBF-FD Laplacian weights (Eq. 2-3), phi(r) = r^3
// augmented with every monomial of degree <= m, solved in FP64.
//
// One warp owns one local system at a time.  The (n+M) x (n+M+1) augmented
// matrix lives in shared memory (odd row pitch, so column walks are
// bank-conflict free); the warp assembles it, eliminates with partial
// pivoting (lanes across columns for the trailing update, the pivot row kept
// in registers), and back-substitutes by columns.  Every element sees the
// same sequence of IEEE operations as the textbook algorithm (multiplier by
// division, update by fused multiply-add, first row of largest |pivot|), so
// the result does not depend on how lanes split the work.
//
// The work is FP64-ALU bound: (2/3) s^3 multiply-adds per stencil.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace rbffd {

static constexpr int W_SMAX = 128;

struct WeightArgs {
    const double* xyz;
    int64_t N;
    int d;
    const int32_t* idx;
    int64_t nc;
    int n, M, s, pitch;
    double* w;
    int8_t* status;
    unsigned char ex[W_SMAX][3];   // monomial exponents, graded order
    double lap_phi;                // 3 (d + 1): Laplacian of r^3 is 3(d+1) r
};

__device__ __forceinline__ double powi(double x, int e) {
    double p = 1.0;
    for (int k = 0; k < e; ++k) p = __dmul_rn(p, x);
    return p;
}

__global__ void weights_kernel(WeightArgs A, int warps_per_block) {
    extern __shared__ double wsm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int n = A.n, M = A.M, s = A.s, P = A.pitch, d = A.d;
    double* G = wsm + (size_t)wib * ((size_t)s * P + 3 * n);
    double* xi = G + (size_t)s * P;
    const int64_t warps = (int64_t)gridDim.x * warps_per_block;

    for (int64_t r = (int64_t)blockIdx.x * warps_per_block + wib; r < A.nc; r += warps) {
        const int32_t* sup = A.idx + r * n;
        const int32_t c = sup[0];
        // scale sigma = max_j |x_j - x_c|
        double sig = 0.0;
        for (int j = lane; j < n; j += 32) {
            int32_t id = sup[j];
            double s2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double t = __dsub_rn(A.xyz[(int64_t)a * A.N + id], A.xyz[(int64_t)a * A.N + c]);
                double sq = __dmul_rn(t, t);
                s2 = a == 0 ? sq : __dadd_rn(s2, sq);
            }
            sig = fmax(sig, __dsqrt_rn(s2));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sig = fmax(sig, __shfl_xor_sync(0xffffffffu, sig, o));
        if (!(sig > 0.0)) {
            for (int j = lane; j < n; j += 32) A.w[r * n + j] = 0.0;
            if (lane == 0) A.status[r] = 1;
            continue;
        }
        for (int j = lane; j < n; j += 32) {
            int32_t id = sup[j];
            for (int a = 0; a < d; ++a) {
                double t = __dsub_rn(A.xyz[(int64_t)a * A.N + id], A.xyz[(int64_t)a * A.N + c]);
                xi[3 * j + a] = __ddiv_rn(t, sig);
            }
        }
        __syncwarp();
        // assemble [[A P] [P^T 0]] | rhs
        for (int e = lane; e < n * n; e += 32) {
            int j = e / n, k = e - j * n;
            double r2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double t = __dsub_rn(xi[3 * j + a], xi[3 * k + a]);
                double sq = __dmul_rn(t, t);
                r2 = a == 0 ? sq : __dadd_rn(r2, sq);
            }
            double rr = __dsqrt_rn(r2);
            G[j * P + k] = __dmul_rn(__dmul_rn(rr, rr), rr);
        }
        for (int e = lane; e < n * M; e += 32) {
            int j = e / M, al = e - j * M;
            double p = powi(xi[3 * j + 0], A.ex[al][0]);
            if (d >= 2) p = __dmul_rn(p, powi(xi[3 * j + 1], A.ex[al][1]));
            if (d >= 3) p = __dmul_rn(p, powi(xi[3 * j + 2], A.ex[al][2]));
            G[j * P + n + al] = p;
            G[(n + al) * P + j] = p;
        }
        for (int e = lane; e < M * M; e += 32) {
            int a1 = e / M, a2 = e - a1 * M;
            G[(n + a1) * P + n + a2] = 0.0;
        }
        for (int j = lane; j < n; j += 32) {
            double rc2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double sq = __dmul_rn(xi[3 * j + a], xi[3 * j + a]);
                rc2 = a == 0 ? sq : __dadd_rn(rc2, sq);
            }
            G[j * P + s] = __dmul_rn(A.lap_phi, __dsqrt_rn(rc2));
        }
        for (int al = lane; al < M; al += 32) {
            int e0 = A.ex[al][0], e1 = A.ex[al][1], e2 = A.ex[al][2];
            bool pure2 = (e0 + e1 + e2 == 2) && (e0 == 2 || e1 == 2 || e2 == 2);
            G[(n + al) * P + s] = pure2 ? 2.0 : 0.0;
        }
        __syncwarp();

        // elimination with partial pivoting
        int bad = 0;
        for (int k = 0; k < s; ++k) {
            // pivot: the first row of largest |a_ik| (NaN entries below the
            // diagonal never win; a NaN on the diagonal makes the row singular)
            const bool diag_nan = isnan(G[k * P + k]);
            double bv = -1.0;
            int bi = s;
            for (int i = k + lane; i < s; i += 32) {
                double v = fabs(G[i * P + k]);
                if (v != v) v = -1.0;
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (diag_nan || !(bv > 1e-300) || isinf(bv)) {
                bad = 1;
                break;
            }
            if (bi != k)
                for (int j = k + lane; j <= s; j += 32) {
                    double t = G[k * P + j];
                    G[k * P + j] = G[bi * P + j];
                    G[bi * P + j] = t;
                }
            __syncwarp();
            const double piv = G[k * P + k];
            for (int i = k + 1 + lane; i < s; i += 32) G[i * P + k] = __ddiv_rn(G[i * P + k], piv);
            __syncwarp();
            // trailing update, pivot row in registers
            double pr[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int j = k + 1 + lane + 32 * q;
                pr[q] = j <= s ? G[k * P + j] : 0.0;
            }
            for (int i = k + 1; i < s; ++i) {
                const double l = G[i * P + k];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int j = k + 1 + lane + 32 * q;
                    if (j <= s) G[i * P + j] = __fma_rn(-l, pr[q], G[i * P + j]);
                }
            }
            __syncwarp();
        }
        if (!bad) {
            // back substitution by columns; x_j overwrites the rhs entry of row j
            for (int j = s - 1; j >= 0; --j) {
                double xj = __ddiv_rn(G[j * P + s], G[j * P + j]);
                if (!isfinite(xj)) {
                    bad = 1;
                    break;
                }
                __syncwarp();
                for (int i = lane; i < j; i += 32)
                    G[i * P + s] = __fma_rn(-G[i * P + j], xj, G[i * P + s]);
                if (lane == 0) G[j * P + s] = xj;
                __syncwarp();
            }
        }
        const double sig2 = __dmul_rn(sig, sig);
        for (int j = lane; j < n; j += 32) A.w[r * n + j] = bad ? 0.0 : __ddiv_rn(G[j * P + s], sig2);
        if (lane == 0) A.status[r] = (int8_t)bad;
        __syncwarp();
    }
}

__global__ void count_bad(const int8_t* st, int64_t nc, unsigned long long* cnt,
                          unsigned long long* first) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nc;
         r += (int64_t)gridDim.x * blockDim.x)
        if (st[r]) {
            atomicAdd(cnt, 1ull);
            atomicMin(first, (unsigned long long)r);
        }
}

// monomial exponents of degree <= m in graded order: degree ascending, then
// the x exponent descending, then the y exponent descending
static int graded_monomials(int d, int m, unsigned char ex[][3], int cap) {
    int M = 0;
    for (int deg = 0; deg <= m; ++deg)
        for (int a = deg; a >= 0; --a)
            for (int b = (d >= 2 ? deg - a : 0); b >= 0; --b) {
                int c = deg - a - b;
                if ((d == 1 && a != deg) || (d == 2 && c != 0)) continue;
                if (M < cap) {
                    ex[M][0] = (unsigned char)a;
                    ex[M][1] = (unsigned char)b;
                    ex[M][2] = (unsigned char)c;
                }
                ++M;
            }
    return M;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_weights(const double* xyz, int64_t N, int d, const int32_t* idx, int64_t nc,
                             int n, int m, double* w, int8_t* status, int64_t* h_n_bad,
                             int64_t* h_first_bad, void* stream) {
    clear_error();
    if (nc == 0 && n >= 1) {
        if (h_n_bad) *h_n_bad = 0;
        if (h_first_bad) *h_first_bad = -1;
        return RBFFD_OK;
    }
    RBFFD_ARG(xyz && idx && w && status, "rbffd_weights: NULL argument");
    RBFFD_ARG(d >= 1 && d <= 3, "rbffd_weights: d must be 1, 2 or 3");
    RBFFD_ARG(m >= 0 && m <= 12, "rbffd_weights: m must be in [0, 12]");
    RBFFD_ARG(n >= 1 && nc >= 0 && N >= 1, "rbffd_weights: bad sizes");
    WeightArgs A;
    int M = graded_monomials(d, m, A.ex, W_SMAX);
    RBFFD_ARG(n + M <= W_SMAX, "rbffd_weights: n + M = %d exceeds %d", n + M, W_SMAX);
    if (h_n_bad) *h_n_bad = 0;
    if (h_first_bad) *h_first_bad = -1;
    if (nc == 0) return RBFFD_OK;
    cudaStream_t s = as_stream(stream);
    A.xyz = xyz;
    A.N = N;
    A.d = d;
    A.idx = idx;
    A.nc = nc;
    A.n = n;
    A.M = M;
    A.s = n + M;
    A.pitch = (A.s + 1) | 1;   // odd pitch: column walks hit distinct banks
    A.w = w;
    A.status = status;
    A.lap_phi = (double)(3 * (d + 1));
    size_t per_warp = sizeof(double) * ((size_t)A.s * A.pitch + 3 * (size_t)n);
    const size_t smem_cap = 200 * 1024;
    int wpb = (int)std::min<size_t>(8, smem_cap / per_warp);
    if (wpb < 1) wpb = 1;
    size_t smem = per_warp * wpb;
    RBFFD_CHECK_CUDA(cudaFuncSetAttribute(weights_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)std::max<size_t>(smem, 48 * 1024)));
    int sms = device_sm_count();
    int per_sm = std::max(1, (int)(220 * 1024 / smem));
    int64_t want = (nc + wpb - 1) / wpb;
    int64_t grid = std::min<int64_t>(want, (int64_t)sms * per_sm * 4);
    weights_kernel<<<(unsigned)grid, 32 * wpb, smem, s>>>(A, wpb);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    Scratch cnt;
    RBFFD_CHECK_CUDA(cnt.alloc(2 * sizeof(unsigned long long), s));
    unsigned long long init[2] = {0ull, ~0ull};
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(cnt.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
    count_bad<<<sms * 4, 256, 0, s>>>(status, nc, cnt.as<unsigned long long>(),
                                      cnt.as<unsigned long long>() + 1);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    unsigned long long out[2];
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(out, cnt.p, sizeof(out), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h_n_bad) *h_n_bad = (int64_t)out[0];
    if (h_first_bad) *h_first_bad = out[0] ? (int64_t)out[1] : -1;
    if (out[0]) {
        set_error("rbffd_weights: %llu singular stencils, first row %llu", out[0], out[1]);
        return RBFFD_ERR_SINGULAR;
    }
    return RBFFD_OK;
}
