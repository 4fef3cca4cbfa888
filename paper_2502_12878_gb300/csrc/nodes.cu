// rbffd_nodes / rbffd_interior: seeded jittered-grid node sets (stand-in for
// the Poisson-disc sampler of Sec. II-C) and the interior-node list.
//
// Every coordinate is a fixed sequence of separately rounded IEEE operations
// (explicit __d*_rn intrinsics), so a CPU implementation of the same
// definition reproduces the node set bit for bit.
#include <math.h>

#include "common.cuh"
#include "nodegen.cuh"

namespace rbffd {

struct NodeGen {
    int d, shape, Kg;
    double h, amp;
    uint64_t seed;
    int64_t side;
};

// position of generator point `lin`; returns the boundary code: 0 interior,
// 1 Dirichlet (any index 0, or any index Kg in the unit cube), 2 Neumann
// (half cube: an index Kg and no index 0; those coordinates are exactly 1/2)
__device__ int grid_point(const NodeGen& g, int64_t lin, double* p) {
    int64_t gi[3] = {0, 0, 0};
    int64_t rem = lin;
    for (int a = g.d - 1; a >= 0; --a) {
        gi[a] = rem % g.side;
        rem /= g.side;
    }
    int bnd = 0, lo = 0;
    for (int a = 0; a < g.d; ++a) {
        if (gi[a] == 0 || gi[a] == g.Kg) bnd = 1;
        if (gi[a] == 0) lo = 1;
    }
    if (g.shape == 2 && bnd) bnd = lo ? 1 : 2;
    for (int a = 0; a < g.d; ++a) {
        double base = __dmul_rn((double)gi[a], g.h);
        if (g.shape == 0 && bnd) {
            p[a] = base;
        } else if (g.shape == 2 && bnd) {
            p[a] = gi[a] == g.Kg ? 0.5 : base;
        } else {
            double U = unit_draw(g.seed, (uint64_t)lin * (uint64_t)g.d + (uint64_t)a);
            double t = __dsub_rn(__dmul_rn(2.0, U), 1.0);
            p[a] = __dadd_rn(base, __dmul_rn(t, g.amp));
        }
    }
    return bnd;
}

__device__ bool disk_keep(const NodeGen& g, const double* p) {
    double dx = __dsub_rn(p[0], 0.5), dy = __dsub_rn(p[1], 0.5);
    double lim = __dsub_rn(0.5, __dmul_rn(0.5, g.h));
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(lim, lim);
}

__global__ void nodes_cube(NodeGen g, int64_t total, double* xyz, uint8_t* is_bnd, int64_t cap) {
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < total;
         lin += (int64_t)gridDim.x * blockDim.x) {
        double p[3];
        int bnd = grid_point(g, lin, p);
        for (int a = 0; a < g.d; ++a) xyz[(int64_t)a * cap + lin] = p[a];
        is_bnd[lin] = (uint8_t)bnd;
    }
}

__global__ void nodes_disk_flags(NodeGen g, int64_t total, int32_t* keep) {
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < total;
         lin += (int64_t)gridDim.x * blockDim.x) {
        double p[3];
        grid_point(g, lin, p);
        keep[lin] = disk_keep(g, p) ? 1 : 0;
    }
}

__global__ void nodes_disk_write(NodeGen g, int64_t total, const int32_t* pos, double* xyz,
                                 uint8_t* is_bnd, int64_t cap) {
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < total;
         lin += (int64_t)gridDim.x * blockDim.x) {
        if (pos[lin + 1] == pos[lin]) continue;   // not kept
        double p[3];
        grid_point(g, lin, p);
        int64_t o = pos[lin];
        xyz[o] = p[0];
        xyz[cap + o] = p[1];
        is_bnd[o] = 0;
    }
}

__global__ void nodes_disk_boundary(int64_t Nb, int64_t first, double* xyz, uint8_t* is_bnd,
                                    int64_t cap) {
    const double two_pi = 6.283185307179586;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < Nb;
         k += (int64_t)gridDim.x * blockDim.x) {
        double a = __ddiv_rn(__dmul_rn(two_pi, (double)k), (double)Nb);
        double cx, cy;
        unit_dir(a, &cx, &cy);
        int64_t o = first + k;
        xyz[o] = __dadd_rn(0.5, __dmul_rn(0.5, cx));
        xyz[cap + o] = __dadd_rn(0.5, __dmul_rn(0.5, cy));
        is_bnd[o] = 1;
    }
}

__global__ void interior_flags(const uint8_t* is_bnd, int64_t N, int32_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = is_bnd[i] ? 0 : 1;
}

__global__ void interior_write(int64_t N, const int32_t* pos, int32_t* interior) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        if (pos[i + 1] != pos[i]) interior[pos[i]] = (int32_t)i;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_nodes(int d, int shape, int Kg, double jitter_frac, uint64_t seed,
                           double* xyz, uint8_t* is_bnd, int64_t cap, int64_t* h_n_out,
                           void* stream) {
    clear_error();
    RBFFD_ARG(h_n_out != nullptr, "rbffd_nodes: h_n_out is NULL");
    RBFFD_ARG(shape >= 0 && shape <= 2,
              "rbffd_nodes: shape must be 0 (cube), 1 (disk) or 2 (half cube)");
    RBFFD_ARG(shape != 1 ? (d >= 1 && d <= 3) : d == 2, "rbffd_nodes: bad dimension %d", d);
    RBFFD_ARG(Kg >= 2 && Kg <= (1 << 20), "rbffd_nodes: Kg must be in [2, 2^20]");
    RBFFD_ARG(jitter_frac >= 0.0 && jitter_frac < 0.5, "rbffd_nodes: jitter_frac in [0, 0.5)");
    RBFFD_ARG(cap >= 0, "rbffd_nodes: negative capacity");
    cudaStream_t s = as_stream(stream);
    NodeGen g;
    g.d = d;
    g.shape = shape;
    g.Kg = Kg;
    g.h = (shape == 2 ? 0.5 : 1.0) / (double)Kg;
    g.amp = jitter_frac * g.h;
    g.seed = seed;
    g.side = (int64_t)Kg + 1;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= g.side;
    RBFFD_ARG(total < (int64_t(1) << 31), "rbffd_nodes: more than 2^31 grid points");
    int sms = device_sm_count();
    if (shape != 1) {
        *h_n_out = total;
        if (cap == 0) return RBFFD_OK;
        if (total > cap) {
            set_error("rbffd_nodes: %lld nodes exceed capacity %lld", (long long)total,
                      (long long)cap);
            return RBFFD_ERR_CAPACITY;
        }
        RBFFD_ARG(xyz && is_bnd, "rbffd_nodes: NULL output");
        nodes_cube<<<sms * 8, 256, 0, s>>>(g, total, xyz, is_bnd, cap);
        RBFFD_CHECK_CUDA(cudaGetLastError());
        return RBFFD_OK;
    }
    // disk: keep flags, ordered compaction, then the boundary ring
    const double two_pi = 6.283185307179586;
    int64_t Nb = (int64_t)floor((two_pi * 0.5) / g.h + 0.5);
    Scratch pos, tmp;
    RBFFD_CHECK_CUDA(pos.alloc(sizeof(int32_t) * (size_t)(total + 1), s));
    RBFFD_CHECK_CUDA(tmp.alloc(sizeof(int64_t) * (size_t)scan_tmp_elems(total), s));
    nodes_disk_flags<<<sms * 8, 256, 0, s>>>(g, total, pos.as<int32_t>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(exclusive_scan_i32(pos.as<int32_t>(), pos.as<int32_t>(), total,
                                        tmp.as<int64_t>(), s));
    int32_t ni = 0;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&ni, pos.as<int32_t>() + total, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    int64_t N = (int64_t)ni + Nb;
    *h_n_out = N;
    if (cap == 0) return RBFFD_OK;
    if (N > cap) {
        set_error("rbffd_nodes: %lld nodes exceed capacity %lld", (long long)N, (long long)cap);
        return RBFFD_ERR_CAPACITY;
    }
    RBFFD_ARG(xyz && is_bnd, "rbffd_nodes: NULL output");
    nodes_disk_write<<<sms * 8, 256, 0, s>>>(g, total, pos.as<int32_t>(), xyz, is_bnd, cap);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    nodes_disk_boundary<<<(unsigned)((Nb + 255) / 256), 256, 0, s>>>(Nb, ni, xyz, is_bnd, cap);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    return RBFFD_OK;
}

extern "C" int rbffd_interior(const uint8_t* is_bnd, int64_t N, int32_t* interior,
                              int64_t* h_ni_out, void* stream) {
    clear_error();
    RBFFD_ARG(is_bnd && interior && h_ni_out, "rbffd_interior: NULL argument");
    RBFFD_ARG(N >= 1 && N < (int64_t(1) << 31), "rbffd_interior: bad N");
    cudaStream_t s = as_stream(stream);
    Scratch pos, tmp;
    RBFFD_CHECK_CUDA(pos.alloc(sizeof(int32_t) * (size_t)(N + 1), s));
    RBFFD_CHECK_CUDA(tmp.alloc(sizeof(int64_t) * (size_t)scan_tmp_elems(N), s));
    int sms = device_sm_count();
    interior_flags<<<sms * 8, 256, 0, s>>>(is_bnd, N, pos.as<int32_t>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(exclusive_scan_i32(pos.as<int32_t>(), pos.as<int32_t>(), N,
                                        tmp.as<int64_t>(), s));
    interior_write<<<sms * 8, 256, 0, s>>>(N, pos.as<int32_t>(), interior);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    int32_t ni = 0;
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(&ni, pos.as<int32_t>() + N, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    *h_ni_out = ni;
    return RBFFD_OK;
}
