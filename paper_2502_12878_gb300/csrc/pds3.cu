// Poisson-disc node placement in the unit cube (the 3D case of
// rbffd_nodes_pds; Sec. II-C, last paragraph).
//
// The same first-in first-out walk as in 2D, with candidates on a sphere:
// node p proposes c_j = p + h R_p e_j, e_j the j-th of K Fibonacci-sphere
// points, R_p the uniform random rotation of Shoemake's quaternion from the
// (3p..3p+2)-th SplitMix64 draws.  One generation at a time, as in 2D (the
// lexicographically first maximal independent set of a generation's passing
// candidates is the sequential walk's choice), but a 3D front is large
// (~10^5 - 10^6 passing candidates per generation), so every step runs on
// the whole grid and the host drives the generation: candidates, scans of
// the passing flags, the conflict graph, passes until no candidate is
// undecided, ranks, append.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "nodegen.cuh"

namespace rbffd {

static constexpr int PDS3_KMAX = 256;
enum : int { P3_UND = 0, P3_IN = 1, P3_OUT = 2 };

struct Pds3Args {
    double* X;
    double* Y;
    double* Z;
    uint8_t* B;
    double* R;           // [maxn][9] rotation of each node (set when it is added)
    int32_t* cell;       // [G^3] node per cell, -1 empty
    int32_t* chead;      // [Gc^3] candidate lists on the coarse grid, -1 empty
    const double* E;     // [K][3] Fibonacci-sphere directions
    // per generation (capacity capC candidates)
    double* cx;
    double* cy;
    double* cz;
    int32_t* cflag;      // passed (domain and earlier generations); then reused
    int32_t* ccell;      // fine (node) cell of each candidate inside the cube
    int32_t* ccoarse;    // coarse (candidate) cell
    int32_t* pos;        // [capC + 1] scan of cflag
    int32_t* V;          // passing keys, ascending
    int32_t* cnext;
    int32_t* deg;        // [capC + 1]
    int32_t* off;        // [capC + 1]
    int32_t* adj;        // [capA]
    int32_t* st;         // states
    int32_t* rank;       // [capC + 1]
    int* flags;          // [0] undecided after a pass, [1] cell collision, [2] list full
    int K;
    double h, cs, r2;
    float inv_cs;
    float inv_csc;       // coarse cells: side 1.01 zeta h, so candidates closer than
                         // zeta h lie in adjacent coarse cells (3 x 3 x 3 searched)
    int64_t G, Gc, maxn;
    uint64_t seed;
};

__device__ __forceinline__ int64_t p3_cell(const Pds3Args& A, double x, double y, double z) {
    int64_t a = (int64_t)__fmul_rn(__double2float_rn(x), A.inv_cs);
    int64_t b = (int64_t)__fmul_rn(__double2float_rn(y), A.inv_cs);
    int64_t c = (int64_t)__fmul_rn(__double2float_rn(z), A.inv_cs);
    a = a < 0 ? 0 : (a >= A.G ? A.G - 1 : a);
    b = b < 0 ? 0 : (b >= A.G ? A.G - 1 : b);
    c = c < 0 ? 0 : (c >= A.G ? A.G - 1 : c);
    return (a * A.G + b) * A.G + c;
}

__device__ __forceinline__ int64_t p3_coarse(const Pds3Args& A, double x, double y, double z) {
    int64_t a = (int64_t)__fmul_rn(__double2float_rn(x), A.inv_csc);
    int64_t b = (int64_t)__fmul_rn(__double2float_rn(y), A.inv_csc);
    int64_t c = (int64_t)__fmul_rn(__double2float_rn(z), A.inv_csc);
    a = a < 0 ? 0 : (a >= A.Gc ? A.Gc - 1 : a);
    b = b < 0 ? 0 : (b >= A.Gc ? A.Gc - 1 : b);
    c = c < 0 ? 0 : (c >= A.Gc ? A.Gc - 1 : c);
    return (a * A.Gc + b) * A.Gc + c;
}

__device__ __forceinline__ double p3_d2(double ax, double ay, double az, double bx, double by,
                                        double bz) {
    const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Shoemake's uniform rotation of node p, as a row-major matrix
__device__ void p3_rotation(uint64_t seed, uint64_t p, double* R) {
    const double two_pi = 6.283185307179586;
    const double u1 = unit_draw(seed, 3 * p), u2 = unit_draw(seed, 3 * p + 1),
                 u3 = unit_draw(seed, 3 * p + 2);
    const double s1 = __dsqrt_rn(__dsub_rn(1.0, u1)), s2 = __dsqrt_rn(u1);
    double c2, n2, c3, n3;
    unit_dir(__dmul_rn(two_pi, u2), &c2, &n2);
    unit_dir(__dmul_rn(two_pi, u3), &c3, &n3);
    const double x = __dmul_rn(s1, n2), y = __dmul_rn(s1, c2), z = __dmul_rn(s2, n3),
                 w = __dmul_rn(s2, c3);
    const double xx = __dmul_rn(x, x), yy = __dmul_rn(y, y), zz = __dmul_rn(z, z);
    const double xy = __dmul_rn(x, y), xz = __dmul_rn(x, z), yz = __dmul_rn(y, z);
    const double xw = __dmul_rn(x, w), yw = __dmul_rn(y, w), zw = __dmul_rn(z, w);
    R[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(yy, zz)));
    R[1] = __dmul_rn(2.0, __dsub_rn(xy, zw));
    R[2] = __dmul_rn(2.0, __dadd_rn(xz, yw));
    R[3] = __dmul_rn(2.0, __dadd_rn(xy, zw));
    R[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, zz)));
    R[5] = __dmul_rn(2.0, __dsub_rn(yz, xw));
    R[6] = __dmul_rn(2.0, __dsub_rn(xz, yw));
    R[7] = __dmul_rn(2.0, __dadd_rn(yz, xw));
    R[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, yy)));
}

// the j-th Fibonacci-sphere point: z = 1 - (2j+1)/K, rho = sqrt(1 - z^2),
// angle j GA reduced to [0, 2 pi), GA = pi (3 - sqrt 5)
__global__ void p3_dirs(int K, double* E) {
    const double two_pi = 6.283185307179586;
    const double ga = 2.399963229728653;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const double z = __dsub_rn(1.0, __ddiv_rn((double)(2 * j + 1), (double)K));
        const double rho = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(z, z)));
        const double t = __dmul_rn((double)j, ga);
        const double phi = __dsub_rn(t, __dmul_rn(floor(__ddiv_rn(t, two_pi)), two_pi));
        double c, s;
        unit_dir(phi, &c, &s);
        E[3 * j] = __dmul_rn(rho, c);
        E[3 * j + 1] = __dmul_rn(rho, s);
        E[3 * j + 2] = z;
    }
}

// seeds: the cube's surface grid points in row-major order (k fastest):
// slabs i = 0 and i = Kg whole, the slabs between them as rings
__global__ void p3_seeds(Pds3Args A, int Kg, int64_t nb) {
    const int64_t side = (int64_t)Kg + 1, full = side * side, ring = 4 * (int64_t)Kg;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nb;
         s += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        if (s < full) {
            i = 0;
            j = s / side;
            k = s % side;
        } else if (s < full + (Kg - 1) * ring) {
            const int64_t r = s - full;
            i = 1 + r / ring;
            const int64_t q = r % ring;    // the ring of a (j, k) square, row-major
            if (q < side) {
                j = 0;
                k = q;
            } else if (q < side + 2 * ((int64_t)Kg - 1)) {
                const int64_t t = q - side;
                j = 1 + t / 2;
                k = (t & 1) ? Kg : 0;
            } else {
                j = Kg;
                k = q - side - 2 * ((int64_t)Kg - 1);
            }
        } else {
            const int64_t r = s - full - (Kg - 1) * ring;
            i = Kg;
            j = r / side;
            k = r % side;
        }
        const double x = __dmul_rn((double)i, A.h), y = __dmul_rn((double)j, A.h),
                     z = __dmul_rn((double)k, A.h);
        A.X[s] = x;
        A.Y[s] = y;
        A.Z[s] = z;
        A.B[s] = 1;
        if (atomicCAS(&A.cell[p3_cell(A, x, y, z)], -1, (int32_t)s) != -1) atomicExch(&A.flags[1], 1);
        p3_rotation(A.seed, (uint64_t)s, A.R + 9 * s);
    }
}

// candidates of the generation [lo, hi), tested against the domain and the
// nodes of earlier generations (5 x 5 x 5 cells: 2 cs > zeta h)
__global__ void p3_gen(Pds3Args A, int64_t lo, int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = lo + e / A.K;
        const int j = (int)(e % A.K);
        const double* R = A.R + 9 * p;
        const double* E = A.E + 3 * j;
        const double P[3] = {A.X[p], A.Y[p], A.Z[p]};
        double c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double u = __dadd_rn(__dadd_rn(__dmul_rn(R[3 * a], E[0]), __dmul_rn(R[3 * a + 1], E[1])),
                                       __dmul_rn(R[3 * a + 2], E[2]));
            c[a] = __dadd_rn(P[a], __dmul_rn(A.h, u));
        }
        A.cx[e] = c[0];
        A.cy[e] = c[1];
        A.cz[e] = c[2];
        bool ok = c[0] > 0.0 && c[0] < 1.0 && c[1] > 0.0 && c[1] < 1.0 && c[2] > 0.0 && c[2] < 1.0;
        if (ok) {
            const int64_t g = p3_cell(A, c[0], c[1], c[2]);
            A.ccell[e] = (int32_t)g;
            A.ccoarse[e] = (int32_t)p3_coarse(A, c[0], c[1], c[2]);
            const int64_t g0 = g / (A.G * A.G), g1 = (g / A.G) % A.G, g2 = g % A.G;
            // the 27 nearest cells first (most blocking nodes are there), then
            // the rest of the 5 x 5 x 5 block; the first conflict ends the test
            for (int shell = 0; shell < 2 && ok; ++shell) {
                for (int64_t a = g0 - 2; a <= g0 + 2 && ok; ++a) {
                    if (a < 0 || a >= A.G) continue;
                    for (int64_t b = g1 - 2; b <= g1 + 2 && ok; ++b) {
                        if (b < 0 || b >= A.G) continue;
                        for (int64_t d = g2 - 2; d <= g2 + 2 && ok; ++d) {
                            if (d < 0 || d >= A.G) continue;
                            const bool inner = a >= g0 - 1 && a <= g0 + 1 && b >= g1 - 1 &&
                                               b <= g1 + 1 && d >= g2 - 1 && d <= g2 + 1;
                            if (inner != (shell == 0)) continue;
                            const int32_t q = A.cell[(a * A.G + b) * A.G + d];
                            if (q >= 0 &&
                                p3_d2(c[0], c[1], c[2], A.X[q], A.Y[q], A.Z[q]) < A.r2)
                                ok = false;
                        }
                    }
                }
            }
        }
        A.cflag[e] = ok ? 1 : 0;
    }
}

// keys of the passing candidates in order, and the per-cell lists of them
__global__ void p3_compact(Pds3Args A, int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!A.cflag[e]) continue;
        const int32_t v = A.pos[e];
        A.V[v] = (int32_t)e;
        A.cnext[v] = atomicExch(&A.chead[A.ccoarse[e]], v);
        A.st[v] = P3_UND;
    }
}

// lower-key conflicts of each passing candidate (FILL = false counts them),
// from the 3 x 3 x 3 coarse cells around it
template <bool FILL>
__global__ void p3_conflicts(Pds3Args A, int64_t nv) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t ev = A.V[v];
        const double x = A.cx[ev], y = A.cy[ev], z = A.cz[ev];
        const int64_t g = A.ccoarse[ev];
        const int64_t Gc = A.Gc;
        const int64_t g0 = g / (Gc * Gc), g1 = (g / Gc) % Gc, g2 = g % Gc;
        int32_t k = FILL ? A.off[v] : 0;
        for (int64_t a = g0 - 1; a <= g0 + 1; ++a) {
            if (a < 0 || a >= Gc) continue;
            for (int64_t b = g1 - 1; b <= g1 + 1; ++b) {
                if (b < 0 || b >= Gc) continue;
                for (int64_t d = g2 - 1; d <= g2 + 1; ++d) {
                    if (d < 0 || d >= Gc) continue;
                    for (int32_t w = A.chead[(a * Gc + b) * Gc + d]; w >= 0; w = A.cnext[w]) {
                        if (w >= v) continue;
                        const int32_t ew = A.V[w];
                        if (!(p3_d2(x, y, z, A.cx[ew], A.cy[ew], A.cz[ew]) < A.r2)) continue;
                        if (FILL) A.adj[k] = w;
                        ++k;
                    }
                }
            }
        }
        if (!FILL) A.deg[v] = k;
    }
}

// one pass of the walk's choice: thread t walks keys [t per, (t+1) per) in
// ascending order (odd per); flags[0] counts the candidates left undecided
__global__ void p3_pass(Pds3Args A, int64_t nv, int per) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t v0 = t * per;
    if (v0 >= nv) return;
    const int64_t v1 = min(nv, v0 + per);
    int open = 0;
    for (int64_t v = v0; v < v1; ++v) {
        if (A.st[v] != P3_UND) continue;
        bool in_lower = false, und_lower = false;
        const int32_t k1 = A.off[v + 1];
        for (int32_t k = A.off[v]; k < k1; ++k) {
            const int sw = ((volatile int32_t*)A.st)[A.adj[k]];
            if (sw == P3_IN) {
                in_lower = true;
                break;
            }
            if (sw == P3_UND) und_lower = true;
        }
        if (in_lower) A.st[v] = P3_OUT;
        else if (!und_lower) A.st[v] = P3_IN;
        else ++open;
    }
    if (open) atomicAdd(&A.flags[0], open);
}

__global__ void p3_in_flags(Pds3Args A, int64_t nv) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        A.deg[v] = A.st[v] == P3_IN ? 1 : 0;
}

// append the accepted at their ranks, with their rotations; empty the lists
__global__ void p3_commit(Pds3Args A, int64_t nv, int64_t N) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = A.V[v];
        const int32_t cell = A.ccell[e];
        A.chead[A.ccoarse[e]] = -1;
        if (A.st[v] != P3_IN) continue;
        const int64_t id = N + A.rank[v];
        if (id >= A.maxn) {
            atomicExch(&A.flags[2], 1);
            continue;
        }
        A.X[id] = A.cx[e];
        A.Y[id] = A.cy[e];
        A.Z[id] = A.cz[e];
        A.B[id] = 0;
        if (atomicCAS(&A.cell[cell], -1, (int32_t)id) != -1) atomicExch(&A.flags[1], 1);
        p3_rotation(A.seed, (uint64_t)id, A.R + 9 * id);
    }
}

__global__ void p3_copy_out(const Pds3Args A, int64_t N, double* xyz, uint8_t* is_bnd,
                            int64_t cap) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        xyz[i] = A.X[i];
        xyz[cap + i] = A.Y[i];
        xyz[2 * cap + i] = A.Z[i];
        is_bnd[i] = A.B[i];
    }
}

static double p3_cell_side(double zeta, double h) {
    return (0.99 * (zeta * h)) / 1.7320508075688772;
}

// node-count bound: points at mutual distance >= t in the unit cube; the
// periodic extension with period 1 + t is a packing of balls of diameter t,
// so N (pi/6) t^3 <= (pi/sqrt 18)(1 + t)^3 (Hales), N <= sqrt 2 (1 + t)^3 / t^3
int64_t pds3_node_bound(int Kg, double zeta) {
    const double t = zeta / (double)Kg;
    const double b = 1.4142135623730951 * (1.0 + t) * (1.0 + t) * (1.0 + t) / (t * t * t);
    return (int64_t)(1.01 * b) + 64;
}

// scratch that grows to the largest generation seen (stream-ordered: a
// buffer is released on the stream before its replacement is allocated)
struct Grow {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    Grow() = default;
    Grow(const Grow&) = delete;
    Grow& operator=(const Grow&) = delete;
    ~Grow() {
        if (p) cudaFreeAsync(p, st);
    }
    template <class T>
    cudaError_t need(size_t n, cudaStream_t s, T** out) {
        const size_t want = sizeof(T) * std::max<size_t>(n, 1);
        if (want > bytes) {
            if (p) cudaFreeAsync(p, st);
            p = nullptr;
            bytes = 0;
            st = s;
            cudaError_t e = cudaMallocAsync(&p, want + want / 4, s);
            if (e != cudaSuccess) {
                p = nullptr;
                return e;
            }
            bytes = want + want / 4;
        }
        *out = reinterpret_cast<T*>(p);
        return cudaSuccess;
    }
};

int pds3_run(int Kg, int K, double zeta, uint64_t seed, double* xyz, uint8_t* is_bnd,
             int64_t cap, int64_t* h_n, int64_t* h_rounds, cudaStream_t s) {
    const double h = 1.0 / (double)Kg;
    const double cs = p3_cell_side(zeta, h);
    const int64_t G = (int64_t)(1.0 / cs) + 2;
    const int64_t ncell = G * G * G;
    const int64_t maxn = std::min<int64_t>(ncell, pds3_node_bound(Kg, zeta));
    const double t = zeta * h;
    const double csc = 1.01 * t;
    const int64_t Gc = (int64_t)(1.0 / csc) + 2;
    const int64_t ncoarse = Gc * Gc * Gc;
    Pds3Args A = {};
    A.K = K;
    A.h = h;
    A.cs = cs;
    A.inv_cs = (float)(1.0 / cs);
    A.inv_csc = (float)(1.0 / csc);
    A.Gc = Gc;
    A.r2 = t * t;
    A.G = G;
    A.maxn = maxn;
    A.seed = seed;
    Scratch bX, bY, bZ, bB, bR, bcell, bhead, bE, bflags;
    RBFFD_CHECK_CUDA(bX.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(bY.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(bZ.alloc(sizeof(double) * maxn, s));
    RBFFD_CHECK_CUDA(bB.alloc(maxn, s));
    RBFFD_CHECK_CUDA(bR.alloc(sizeof(double) * 9 * maxn, s));
    RBFFD_CHECK_CUDA(bcell.alloc(sizeof(int32_t) * ncell, s));
    RBFFD_CHECK_CUDA(bhead.alloc(sizeof(int32_t) * ncoarse, s));
    RBFFD_CHECK_CUDA(bE.alloc(sizeof(double) * 3 * PDS3_KMAX, s));
    RBFFD_CHECK_CUDA(bflags.alloc(sizeof(int) * 4, s));
    A.X = bX.as<double>();
    A.Y = bY.as<double>();
    A.Z = bZ.as<double>();
    A.B = bB.as<uint8_t>();
    A.R = bR.as<double>();
    A.cell = bcell.as<int32_t>();
    A.chead = bhead.as<int32_t>();
    A.E = bE.as<double>();
    A.flags = bflags.as<int>();
    RBFFD_CHECK_CUDA(cudaMemsetAsync(A.cell, 0xff, sizeof(int32_t) * ncell, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(A.chead, 0xff, sizeof(int32_t) * ncoarse, s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(A.flags, 0, sizeof(int) * 4, s));
    const int64_t side = (int64_t)Kg + 1, inner = (int64_t)Kg - 1;
    const int64_t nb = side * side * side - inner * inner * inner;
    p3_dirs<<<1, 256, 0, s>>>(K, bE.as<double>());
    const unsigned grid = (unsigned)device_sm_count() * 8;
    p3_seeds<<<grid, 256, 0, s>>>(A, Kg, nb);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    Grow gcx, gcy, gcz, gflag, gccell, gcoarse, gpos, gV, gnext, gdeg, goff, gadj, gst, grank,
        gtmp;
    int64_t lo = 0, hi = nb, N = nb, rounds = 0, passes = 0;
    int hflags[4] = {0, 0, 0, 0};
    while (hi > lo) {
        const int64_t total = (hi - lo) * K;
        if (total > INT32_MAX / 2) {
            set_error("rbffd_nodes_pds: a generation of %lld candidates is too large",
                      (long long)total);
            return RBFFD_ERR_CAPACITY;
        }
        RBFFD_CHECK_CUDA(gcx.need(total, s, &A.cx));
        RBFFD_CHECK_CUDA(gcy.need(total, s, &A.cy));
        RBFFD_CHECK_CUDA(gcz.need(total, s, &A.cz));
        RBFFD_CHECK_CUDA(gflag.need(total, s, &A.cflag));
        RBFFD_CHECK_CUDA(gccell.need(total, s, &A.ccell));
        RBFFD_CHECK_CUDA(gcoarse.need(total, s, &A.ccoarse));
        RBFFD_CHECK_CUDA(gpos.need(total + 1, s, &A.pos));
        int64_t* tmp = nullptr;
        RBFFD_CHECK_CUDA(gtmp.need(scan_tmp_elems(total + 1), s, &tmp));
        p3_gen<<<grid, 256, 0, s>>>(A, lo, total);
        RBFFD_CHECK_CUDA(exclusive_scan_i32(A.cflag, A.pos, total, tmp, s));
        int32_t nv32 = 0;
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(&nv32, A.pos + total, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s));
        RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
        const int64_t nv = nv32;
        RBFFD_CHECK_CUDA(gV.need(nv, s, &A.V));
        RBFFD_CHECK_CUDA(gnext.need(nv, s, &A.cnext));
        RBFFD_CHECK_CUDA(gst.need(nv, s, &A.st));
        RBFFD_CHECK_CUDA(gdeg.need(nv + 1, s, &A.deg));
        RBFFD_CHECK_CUDA(goff.need(nv + 1, s, &A.off));
        RBFFD_CHECK_CUDA(grank.need(nv + 1, s, &A.rank));
        int64_t nacc = 0;
        if (nv > 0) {
            p3_compact<<<grid, 256, 0, s>>>(A, total);
            p3_conflicts<false><<<grid, 256, 0, s>>>(A, nv);
            RBFFD_CHECK_CUDA(gtmp.need(scan_tmp_elems(nv + 1), s, &tmp));
            RBFFD_CHECK_CUDA(exclusive_scan_i32(A.deg, A.off, nv, tmp, s));
            int32_t nnz = 0;
            RBFFD_CHECK_CUDA(cudaMemcpyAsync(&nnz, A.off + nv, sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, s));
            RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
            RBFFD_CHECK_CUDA(gadj.need((size_t)nnz, s, &A.adj));
            p3_conflicts<true><<<grid, 256, 0, s>>>(A, nv);
            // passes until every candidate is decided (each decides at least the
            // lowest undecided one); short key ranges (a candidate is a chain of
            // dependent L2 loads), four passes per check of the undecided count
            const int per = 7;
            const int64_t T = (nv + per - 1) / per;
            const unsigned pgrid = (unsigned)((T + 127) / 128);
            for (int64_t pass = 0; pass <= nv; pass += 4) {
                for (int q = 0; q < 4; ++q) {
                    RBFFD_CHECK_CUDA(cudaMemsetAsync(A.flags, 0, sizeof(int), s));
                    p3_pass<<<pgrid, 128, 0, s>>>(A, nv, per);
                    ++passes;
                }
                int open = 0;
                RBFFD_CHECK_CUDA(cudaMemcpyAsync(&open, A.flags, sizeof(int),
                                                 cudaMemcpyDeviceToHost, s));
                RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
                if (!open) break;
            }
            p3_in_flags<<<grid, 256, 0, s>>>(A, nv);
            RBFFD_CHECK_CUDA(exclusive_scan_i32(A.deg, A.rank, nv, tmp, s));
            int32_t na32 = 0;
            RBFFD_CHECK_CUDA(cudaMemcpyAsync(&na32, A.rank + nv, sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, s));
            p3_commit<<<grid, 256, 0, s>>>(A, nv, N);
            RBFFD_CHECK_CUDA(cudaMemcpyAsync(hflags, A.flags, sizeof(hflags),
                                             cudaMemcpyDeviceToHost, s));
            RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
            RBFFD_CHECK_CUDA(cudaGetLastError());
            if (hflags[1] || hflags[2]) {
                set_error("rbffd_nodes_pds: internal error (grid cell collision or list full)");
                return RBFFD_ERR_CUDA;
            }
            nacc = na32;
        }
        ++rounds;
        lo = N;
        hi = N + nacc;
        N += nacc;
    }
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(hflags, A.flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (hflags[1]) {
        set_error("rbffd_nodes_pds: internal error (grid cell collision)");
        return RBFFD_ERR_CUDA;
    }
    *h_n = N;
    if (h_rounds) {
        h_rounds[0] = rounds;
        h_rounds[1] = passes;
    }
    if (N > cap) {
        set_error("rbffd_nodes_pds: %lld nodes, capacity %lld", (long long)N, (long long)cap);
        return RBFFD_ERR_CAPACITY;
    }
    p3_copy_out<<<grid, 256, 0, s>>>(A, N, xyz, is_bnd, cap);
    RBFFD_CHECK_CUDA(cudaGetLastError());
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    return RBFFD_OK;
}

}  // namespace rbffd
