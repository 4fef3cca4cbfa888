// rbffd_weights: batched RBF-FD Laplacian weights (Eq. 2-3), phi(r) = r^3
// augmented with every monomial of degree <= m, solved in FP64.
//
// A team of TS threads owns one local system at a time: half a warp for
// s <= 32 (two systems per warp, so the team-scalar FP64 work, one reciprocal
// and one quotient per pivot, is shared by two systems: a warp-wide FP64
// instruction costs the same pipe time however few lanes it has), one warp
// for s <= 48, five warps above: a pivot warp that runs the serial pivot
// chain one step ahead and four warps (one per SM sub-partition) that do
// the trailing update.  The (n+M) x (n+M+1)
// augmented matrix lives in shared memory (odd row pitch: column walks hit
// distinct banks).  The team assembles it (the symmetric r^3 block from its
// upper triangle), eliminates with partial pivoting, and back-substitutes by
// columns.  The trailing update is flattened over (row, column) pairs so every
// issued FP64 instruction is a useful multiply-add.  Every element sees the
// same sequence of IEEE operations as the textbook algorithm (first row of
// largest |pivot|, multiplier = entry x reciprocal pivot, update by fused
// multiply-add), so the result does not depend on how lanes split the work.
//
// FP64-ALU bound: about s^3/3 multiply-adds per stencil.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "intfp64.cuh"

namespace rbffd {

static constexpr int W_SMAX = 128;
// threads per block at most: one-warp teams up to sixteen per block (at
// s = 45, thirteen fill the shared memory of an SM only as one block: a
// second block would take its own reservation); the other team sizes keep
// 256, which leaves their register budget as it was
static constexpr int W_THREADS = 512;
__host__ __device__ constexpr int weight_max_threads(int ts) { return ts == 32 ? 512 : 256; }

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
    int op;                        // 0 Laplacian, 1 derivative along dirs[row]
    const double* dirs;            // [nc][d] unit vectors (op 1)
};

// x^e by repeated multiplication; the leading 1 * x is exact, so it is skipped
__device__ __forceinline__ double powi(double x, int e) {
    if (e == 0) return 1.0;
    double p = x;
    for (int k = 1; k < e; ++k) p = __dmul_rn(p, x);
    return p;
}

// Tests on IEEE bits with integer instructions (FP64 comparisons would occupy
// the FP64 pipe, which the elimination needs): |x| is NaN / not finite.
static constexpr long long W_INF_BITS = 0x7ff0000000000000ll;
__device__ __forceinline__ bool bits_nan(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffll) > W_INF_BITS;
}
__device__ __forceinline__ bool bits_nonfinite(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffll) >= W_INF_BITS;
}

// A team is TS threads: half a warp (two systems per warp), one warp, or five
// warps (a pivot warp and four update warps).  Lanes of a sub-warp team synchronise and shuffle under their own
// mask only, so the two halves of a warp may diverge freely; while they run
// in step, the team-scalar work (reciprocal pivot, back-substitution
// quotient) is one instruction for both systems.
template <int TS>
__device__ __forceinline__ unsigned team_mask() {
    if constexpr (TS >= 32) return 0xffffffffu;
    else return ((1u << TS) - 1u) << ((threadIdx.x & 31) & ~(TS - 1));
}

// barrier of one team: the team's lanes of a warp, or a named barrier (one
// per team of a block, id 1 + team) over the team's whole warps
template <int TS>
__device__ __forceinline__ void team_sync() {
    if constexpr (TS <= 32) {
        __syncwarp(team_mask<TS>());
    } else {
        const int id = 1 + (int)threadIdx.x / TS;
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(TS) : "memory");
    }
}

// team-wide max of a non-negative double, compared as IEEE bits (integer
// instructions: the FP64 pipe stays free for the elimination)
template <int TS>
__device__ __forceinline__ double team_max_nonneg(double v, long long* red) {
    long long b = __double_as_longlong(v);
    const unsigned mask = team_mask<TS>();
#pragma unroll
    for (int o = (TS < 32 ? TS : 32) / 2; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(mask, b, o));
    if constexpr (TS > 32) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int w0 = (int)(threadIdx.x / TS) * (TS / 32);
        if (lane == 0) red[wid] = b;
        team_sync<TS>();
        b = red[w0];
        for (int q = 1; q < TS / 32; ++q) b = max(b, red[w0 + q]);
        team_sync<TS>();
    }
    return __longlong_as_double(b);
}

// argmax of |value| as IEEE bits (non-negative doubles order like integers;
// NaN is mapped to -1 by the caller and never wins); ties -> lower index.
// Integer compares keep the FP64 pipe for the elimination's multiply-adds.
// A whole warp reduces with three warp-wide integer reductions instead of
// five shuffle rounds: keys (>= -2, so key + 2 orders as unsigned) by their
// high word, then the low word among the lanes holding the largest high word,
// then the lowest index among the lanes holding the largest key.
template <int TS>
__device__ __forceinline__ void team_argmax(long long& bv, int& bi, long long* redv, int* redi) {
    const unsigned mask = team_mask<TS>();
    if constexpr (TS == 32) {
        const unsigned long long u = (unsigned long long)(bv + 2);
        const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
        const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
        const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
        const unsigned mi =
            __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? (unsigned)bi : 0xffffffffu);
        bv = (long long)(((unsigned long long)mhi << 32) | mlo) - 2;
        bi = (int)mi;
        return;
    }
#pragma unroll
    for (int o = (TS < 32 ? TS : 32) / 2; o > 0; o >>= 1) {
        long long ov = __shfl_xor_sync(mask, bv, o);
        int oi = __shfl_xor_sync(mask, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if constexpr (TS <= 32) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int w0 = (int)(threadIdx.x / TS) * (TS / 32);
    if (lane == 0) {
        redv[wid] = bv;
        redi[wid] = bi;
    }
    team_sync<TS>();
    bv = redv[w0];
    bi = redi[w0];
    for (int q = 1; q < TS / 32; ++q)
        if (redv[w0 + q] > bv || (redv[w0 + q] == bv && redi[w0 + q] < bi)) {
            bv = redv[w0 + q];
            bi = redi[w0 + q];
        }
    team_sync<TS>();
}

__device__ __forceinline__ long long abs_key(double x) {
    long long b = __double_as_longlong(x) & 0x7fffffffffffffffll;
    return b > 0x7ff0000000000000ll ? -1ll : b;    // NaN: never the largest
}

// shared memory of one team, in doubles: the augmented matrix, the scaled
// support coordinates (d per node), and per pivot the fixed-point reciprocal
// of its significand.  At s = 45 (2D, m = 4) that is 17,760 bytes: thirteen
// teams fill an SM's shared memory.
__host__ __device__ __forceinline__ size_t weight_team_doubles(const WeightArgs& A) {
    return (size_t)A.s * A.pitch + (size_t)A.d * A.n + (size_t)A.s;
}

// the weights of stencil r of one call (all of the team's threads)
template <int TS, bool PW>
__device__ __forceinline__ void weights_one(const WeightArgs& A, int64_t r, double* G, double* xi,
                                            int tid, int team, double* redv, long long* redk,
                                            int* redi, double* bcast, int* spiv) {
    constexpr int T = TS;
    // [s] the pivots' fixed-point significand reciprocals, for the back
    // substitution's quotients (if_div)
    uint64_t* rinvY = reinterpret_cast<uint64_t*>(xi + A.d * A.n);
    const int n = A.n, M = A.M, s = A.s, P = A.pitch, d = A.d;
    do {
        const int32_t* sup = A.idx + r * n;
        const int32_t c = sup[0];
        // scale sigma = max_j |x_j - x_c| (distances are non-negative: their
        // max is taken on the IEEE bits)
        long long sigb = 0;
        for (int j = tid; j < n; j += T) {
            int32_t id = sup[j];
            double s2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double t = __dsub_rn(A.xyz[(int64_t)a * A.N + id], A.xyz[(int64_t)a * A.N + c]);
                double sq = __dmul_rn(t, t);
                s2 = a == 0 ? sq : __dadd_rn(s2, sq);
            }
            sigb = max(sigb, __double_as_longlong(if_sqrt(s2)));
        }
        const double sig = team_max_nonneg<TS>(__longlong_as_double(sigb), redk);
        if (!(sig > 0.0)) {
            for (int j = tid; j < n; j += T) A.w[r * n + j] = 0.0;
            if (tid == 0) A.status[r] = 1;
            team_sync<TS>();
            break;
        }
        uint64_t Ysig;
        if_rcp(sig, &Ysig);
        for (int j = tid; j < n; j += T) {
            int32_t id = sup[j];
            for (int a = 0; a < d; ++a) {
                double t = __dsub_rn(A.xyz[(int64_t)a * A.N + id], A.xyz[(int64_t)a * A.N + c]);
                xi[d * j + a] = if_div(t, sig, Ysig);
            }
        }
        team_sync<TS>();
        // assemble [[A P] [P^T 0]] | rhs; A from its strict upper triangle
        // (pairs j < k enumerated row by row), diagonal 0.  Each thread keeps
        // the largest |entry| (IEEE bits; NaN ignored) it writes into the
        // s x s block, for the relative pivot test.
        long long gk = 0;
        {
            const int npairs = n * (n - 1) / 2;
            // pair number e -> (j, k): row j holds the n - 1 - j pairs (j, j+1..n-1)
            int e = tid, j = 0, rowlen = n - 1, off = tid;
            while (rowlen > 0 && off >= rowlen) {
                off -= rowlen;
                ++j;
                --rowlen;
            }
            int k = j + 1 + off;
            for (; e < npairs; e += T) {
                double r2 = 0.0;
                for (int a = 0; a < d; ++a) {
                    double t = __dsub_rn(xi[d * j + a], xi[d * k + a]);
                    double sq = __dmul_rn(t, t);
                    r2 = a == 0 ? sq : __dadd_rn(r2, sq);
                }
                double rr = if_sqrt(r2);
                double v = __dmul_rn(__dmul_rn(rr, rr), rr);
                G[j * P + k] = v;
                G[k * P + j] = v;
                gk = max(gk, abs_key(v));
                // advance by T pairs (spilling into the following rows)
                k += T;
                while (j < n - 1 && k >= n) {
                    k = k - (n - 1 - j) + 1;
                    ++j;
                }
            }
        }
        for (int j = tid; j < n; j += T) G[j * P + j] = 0.0;
        // monomials: one node per thread, the monomials in one loop for all
        // threads (every lane takes the same powers at the same time)
        for (int j = tid; j < n; j += T) {
            const double x0 = xi[d * j];
            const double x1 = d >= 2 ? xi[d * j + 1] : 0.0, x2 = d >= 3 ? xi[d * j + 2] : 0.0;
            for (int al = 0; al < M; ++al) {
                // a factor x^0 = 1 multiplies exactly, so it is skipped
                double p = powi(x0, A.ex[al][0]);
                if (d >= 2 && A.ex[al][1]) p = __dmul_rn(p, powi(x1, A.ex[al][1]));
                if (d >= 3 && A.ex[al][2]) p = __dmul_rn(p, powi(x2, A.ex[al][2]));
                G[j * P + n + al] = p;
                G[(n + al) * P + j] = p;
                gk = max(gk, abs_key(p));
            }
        }
        for (int e = tid; e < M * M; e += T) {
            int a1 = e / M, a2 = e - a1 * M;
            G[(n + a1) * P + n + a2] = 0.0;
        }
        const double* dir = A.op == 1 ? A.dirs + r * d : nullptr;
        for (int j = tid; j < n; j += T) {
            double rc2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double sq = __dmul_rn(xi[d * j + a], xi[d * j + a]);
                rc2 = a == 0 ? sq : __dadd_rn(rc2, sq);
            }
            if (A.op == 0) {
                G[j * P + s] = __dmul_rn(A.lap_phi, if_sqrt(rc2));
            } else {
                // derivative of r^3 about x_j at x_c along dir: -3 |xi_j| (xi_j . dir)
                double dot = 0.0;
                for (int a = 0; a < d; ++a) {
                    double t = __dmul_rn(xi[d * j + a], dir[a]);
                    dot = a == 0 ? t : __dadd_rn(dot, t);
                }
                G[j * P + s] = -__dmul_rn(__dmul_rn(3.0, if_sqrt(rc2)), dot);
            }
        }
        for (int al = tid; al < M; al += T) {
            int e0 = A.ex[al][0], e1 = A.ex[al][1], e2 = A.ex[al][2];
            double v;
            if (A.op == 0) {
                bool pure2 = (e0 + e1 + e2 == 2) && (e0 == 2 || e1 == 2 || e2 == 2);
                v = pure2 ? 2.0 : 0.0;
            } else {
                v = (e0 + e1 + e2 == 1) ? (e0 ? dir[0] : (e1 ? dir[1] : dir[2])) : 0.0;
            }
            G[(n + al) * P + s] = v;
        }
        team_sync<TS>();
        // scale of the assembled matrix for the relative pivot test: the team's
        // max of the threads' |entry| maxima (the zeros cannot exceed them)
        long long gkb = 0;
        {
            long long bk = gk;
            int bi_dummy = 0;
            team_argmax<TS>(bk, bi_dummy, redk, redi);
            gkb = bk;
        }
        const double gmax = __longlong_as_double(gkb < 0 ? 0ll : gkb);
        const double tiny = __dmul_rn(1e-13, gmax);
        // the pivot tests on |pivot| as IEEE bits (non-negative doubles order like
        // their bits): |p| > tiny, |p| > 1e-300 and |p| finite; a key < 0 (no
        // candidate, or NaN) fails them all
        const long long key_tiny = __double_as_longlong(tiny);
        const long long key_min = __double_as_longlong(1e-300);
        // elimination with partial pivoting
        int bad = 0;
        if constexpr (!PW) {
            for (int k = 0; k < s; ++k) {
                // pivot: the first row of largest |a_ik| (NaN entries never win;
                // a NaN on the diagonal leaves no usable pivot)
                const bool diag_nan = bits_nan(G[k * P + k]);
                long long bk = -2;
                int bi = s;
                for (int i = k + tid; i < s; i += T) {
                    long long v = abs_key(G[i * P + k]);
                    if (v > bk) {
                        bk = v;
                        bi = i;
                    }
                }
                team_argmax<TS>(bk, bi, redk, redi);
                if (diag_nan || bk <= key_tiny || bk <= key_min || bk == W_INF_BITS) {
                    bad = 1;
                    break;
                }
                // reciprocal pivot: a team of at most one warp computes it in
                // every lane, from the pivot read before the swap moves it; a
                // larger team's first warp computes it and broadcasts it after
                // the swap
                double rp = 0.0;
                if constexpr (T <= 32) {
                    const double pv = G[bi * P + k];
                    team_sync<TS>();
                    uint64_t Y;
                    rp = if_rcp(pv, &Y);
                    if (tid == 0) rinvY[k] = Y;
                } else if ((tid >> 5) == 0) {
                    uint64_t Y;
                    const double t = if_rcp(G[bi * P + k], &Y);
                    if (tid == 0) {
                        bcast[team] = t;
                        rinvY[k] = Y;
                    }
                }
                if (bi != k)
                    for (int j = k + tid; j <= s; j += T) {
                        double t = G[k * P + j];
                        G[k * P + j] = G[bi * P + j];
                        G[bi * P + j] = t;
                    }
                team_sync<TS>();
                if constexpr (T > 32) rp = bcast[team];
                for (int i = k + 1 + tid; i < s; i += T) G[i * P + k] = __dmul_rn(G[i * P + k], rp);
                team_sync<TS>();
                // trailing update over (row, column) pairs: rows k+1..s-1,
                // columns k+1..s (the right-hand side included); two pairs per
                // iteration, both loaded before either is stored (they are distinct
                // elements, and column k and row k are only read here)
                const int cols = s - k;
                const int total = (s - k - 1) * cols;
                const int di = T / cols, dj = T - di * cols;
                int ii = tid / cols, jj = tid - ii * cols;
                int e = tid;
                for (; e + T < total; e += 2 * T) {
                    int ib = ii + di, jb = jj + dj;
                    if (jb >= cols) {
                        jb -= cols;
                        ++ib;
                    }
                    const int ra = (k + 1 + ii) * P, ca = k + 1 + jj;
                    const int rb = (k + 1 + ib) * P, cb = k + 1 + jb;
                    const double la = G[ra + k], ua = G[k * P + ca], ga = G[ra + ca];
                    const double lb = G[rb + k], ub = G[k * P + cb], gb = G[rb + cb];
                    G[ra + ca] = __fma_rn(-la, ua, ga);
                    G[rb + cb] = __fma_rn(-lb, ub, gb);
                    ii = ib + di;
                    jj = jb + dj;
                    if (jj >= cols) {
                        jj -= cols;
                        ++ii;
                    }
                }
                if (e < total) {
                    const int ra = (k + 1 + ii) * P, ca = k + 1 + jj;
                    G[ra + ca] = __fma_rn(-G[ra + k], G[k * P + ca], G[ra + ca]);
                }
                team_sync<TS>();
            }
        } else {
            // The team's first warp is the pivot warp.  At step k it updates
            // column k+1 (rows k+1..s-1) and at once finds the pivot of step
            // k+1 and its reciprocal, while the other warps update columns
            // k+2..s: the serial pivot chain overlaps the trailing update.
            // Every element still sees the same operations in the same order.
            const int lane = tid & 31;
            const bool pw = tid < 32;
            constexpr int UT = TS - 32;   // update threads
            const int ut = tid - 32;
            // pivot of column c over rows c..s-1 (pivot warp; result in
            // spiv[team] = row | bad << 16 and bcast[team] = reciprocal)
            auto pivot = [&](int c) {
                const bool diag_nan = bits_nan(G[c * P + c]);
                long long bk = -2;
                int bi = s;
                for (int i = c + lane; i < s; i += 32) {
                    long long v = abs_key(G[i * P + c]);
                    if (v > bk) {
                        bk = v;
                        bi = i;
                    }
                }
                team_argmax<32>(bk, bi, redk, redi);
                const int nogo =
                    diag_nan || bk <= key_tiny || bk <= key_min || bk == W_INF_BITS;
                uint64_t Y = 0;
                const double t = nogo ? 0.0 : if_rcp(G[bi * P + c], &Y);
                if (lane == 0) {
                    spiv[team] = bi | (nogo << 16);
                    bcast[team] = t;
                    rinvY[c] = Y;
                }
            };
            if (pw) pivot(0);
            team_sync<TS>();
            for (int k = 0; k < s; ++k) {
                const int pv = spiv[team];
                const double rp = bcast[team];
                if (pv >> 16) {
                    bad = 1;
                    break;
                }
                const int bi = pv & 0xffff;
                // row swap (columns k+1..s) and the multipliers of column k;
                // the thread of row bi also moves the pivot into row k
                if (bi != k)
                    for (int j = k + 1 + tid; j <= s; j += TS) {
                        double t = G[k * P + j];
                        G[k * P + j] = G[bi * P + j];
                        G[bi * P + j] = t;
                    }
                for (int i = k + 1 + tid; i < s; i += TS) {
                    if (i == bi) {
                        const double a = G[k * P + k];
                        G[k * P + k] = G[bi * P + k];
                        G[bi * P + k] = __dmul_rn(a, rp);
                    } else {
                        G[i * P + k] = __dmul_rn(G[i * P + k], rp);
                    }
                }
                team_sync<TS>();
                if (k + 1 < s) {
                    if (pw) {
                        const double ukc = G[k * P + k + 1];
                        for (int i = k + 1 + lane; i < s; i += 32)
                            G[i * P + k + 1] = __fma_rn(-G[i * P + k], ukc, G[i * P + k + 1]);
                        __syncwarp();
                        pivot(k + 1);
                    } else {
                        // rows k+1..s-1 x columns k+2..s, flattened, two
                        // pairs per iteration as above
                        const int cols = s - k - 1;
                        const int total = (s - k - 1) * cols;
                        const int di = UT / cols, dj = UT - di * cols;
                        int ii = ut / cols, jj = ut - ii * cols;
                        int e = ut;
                        for (; e + UT < total; e += 2 * UT) {
                            int ib = ii + di, jb = jj + dj;
                            if (jb >= cols) {
                                jb -= cols;
                                ++ib;
                            }
                            const int ra = (k + 1 + ii) * P, ca = k + 2 + jj;
                            const int rb = (k + 1 + ib) * P, cb = k + 2 + jb;
                            const double la = G[ra + k], ua = G[k * P + ca], ga = G[ra + ca];
                            const double lb = G[rb + k], ub = G[k * P + cb], gb = G[rb + cb];
                            G[ra + ca] = __fma_rn(-la, ua, ga);
                            G[rb + cb] = __fma_rn(-lb, ub, gb);
                            ii = ib + di;
                            jj = jb + dj;
                            if (jj >= cols) {
                                jj -= cols;
                                ++ii;
                            }
                        }
                        if (e < total) {
                            const int ra = (k + 1 + ii) * P, ca = k + 2 + jj;
                            G[ra + ca] = __fma_rn(-G[ra + k], G[k * P + ca], G[ra + ca]);
                        }
                    }
                }
                team_sync<TS>();
            }
        }
        if (!bad) {
            // back substitution by columns; x_j overwrites the rhs entry of row j
            for (int j = s - 1; j >= 0; --j) {
                double xj;
                if constexpr (T <= 32) {   // every lane divides (row j is final: the
                                           // previous column's update ended in a sync)
                    xj = if_div(G[j * P + s], G[j * P + j], rinvY[j]);
                } else {                   // one warp divides, the team reads the result
                    if ((tid >> 5) == 0) {
                        const double t = if_div(G[j * P + s], G[j * P + j], rinvY[j]);
                        if (tid == 0) bcast[team] = t;
                    }
                    team_sync<TS>();
                    xj = bcast[team];
                }
                if (bits_nonfinite(xj)) {
                    bad = 1;
                    break;
                }
                for (int i = tid; i < j; i += T)
                    G[i * P + s] = __fma_rn(-G[i * P + j], xj, G[i * P + s]);
                team_sync<TS>();
                if (tid == 0) G[j * P + s] = xj;
            }
            team_sync<TS>();
        }
        // the Laplacian scales as 1/sigma^2, a first derivative as 1/sigma
        const double scl = A.op == 0 ? __dmul_rn(sig, sig) : sig;
        uint64_t Yscl;
        if_rcp(scl, &Yscl);
        for (int j = tid; j < n; j += T) A.w[r * n + j] = bad ? 0.0 : if_div(G[j * P + s], scl, Yscl);
        if (tid == 0) A.status[r] = (int8_t)bad;
        team_sync<TS>();
    } while (0);
}

template <int TS, bool PW>
__global__ void __launch_bounds__(weight_max_threads(TS))
    weights_kernel(WeightArgs A, int teams_per_block) {
    extern __shared__ double wsm[];
    __shared__ double redv[W_THREADS / 32];
    __shared__ long long redk[W_THREADS / 32];
    __shared__ int redi[W_THREADS / 32];
    __shared__ double bcast[16];   // per-team scalar broadcast (reciprocal pivot, x_j)
    __shared__ int spiv[16];       // per-team pivot row (pivot-warp teams)
    const int tid = threadIdx.x % TS;
    const int team = threadIdx.x / TS;
    double* G = wsm + (size_t)team * weight_team_doubles(A);
    double* xi = G + (size_t)A.s * A.pitch;
    const int64_t teams = (int64_t)gridDim.x * teams_per_block;
    for (int64_t r = (int64_t)blockIdx.x * teams_per_block + team; r < A.nc; r += teams)
        weights_one<TS, PW>(A, r, G, xi, tid, team, redv, redk, redi, bcast, spiv);
}

// many calls in one launch: stencil number g of the concatenation belongs to
// the call dI with off[dI] <= g < off[dI + 1]; a team's shared memory holds
// the largest system of the launch (team_doubles)
template <int TS, bool PW>
__global__ void __launch_bounds__(weight_max_threads(TS))
    weights_multi_kernel(const WeightArgs* __restrict__ calls, const int64_t* __restrict__ off,
                         int ncalls, int teams_per_block, int64_t team_doubles) {
    extern __shared__ double wsm[];
    __shared__ double redv[W_THREADS / 32];
    __shared__ long long redk[W_THREADS / 32];
    __shared__ int redi[W_THREADS / 32];
    __shared__ double bcast[16];
    __shared__ int spiv[16];
    const int tid = threadIdx.x % TS;
    const int team = threadIdx.x / TS;
    double* G = wsm + (size_t)team * (size_t)team_doubles;
    const int64_t total = off[ncalls];
    const int64_t teams = (int64_t)gridDim.x * teams_per_block;
    for (int64_t g = (int64_t)blockIdx.x * teams_per_block + team; g < total; g += teams) {
        int lo = 0, hi = ncalls - 1;   // last call with off <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const WeightArgs& A = calls[lo];
        double* xi = G + (size_t)A.s * A.pitch;
        weights_one<TS, PW>(A, g - off[lo], G, xi, tid, team, redv, redk, redi, bcast, spiv);
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

// singular stencils per call: blockIdx.y = call
__global__ void count_bad_multi(int8_t* const* status, const int64_t* nc, int ncalls,
                                unsigned long long* cnt) {
    for (int c = blockIdx.y; c < ncalls; c += gridDim.y) {
        const int8_t* st = status[c];
        unsigned long long k = 0;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nc[c];
             r += (int64_t)gridDim.x * blockDim.x)
            k += st[r] != 0;
        if (k) atomicAdd(&cnt[c], k);
    }
}

// Launch shape of a weight build whose largest system is s x s (per_team
// bytes of shared memory per team).  Team size: half a warp up to
// W_HALF_SMAX, one warp up to 48, else a pivot warp and four update warps.
// Measured on 1M-stencil builds (all variants give identical bits):
// half-warp teams are 1.35-1.7x faster than one-warp teams at s = 18-30 but
// 6 % slower at s = 45 (twelve systems per SM then fill only six warps, too
// few to hide the shared-memory latency); at s = 45 a pivot warp plus one
// update warp is 7 % slower than one warp; at s = 84-105 the pivot warp plus
// four update warps is 12 % faster than four warps without one, which in
// turn beat two or eight warps by 14-35 %.
// Teams per block: the count that puts the most teams on an SM.
static constexpr int W_HALF_SMAX = 32;

static int weight_team_size(int s) { return s <= W_HALF_SMAX ? 16 : (s <= 48 ? 32 : 160); }

typedef void (*WeightKernel)(WeightArgs, int);
typedef void (*WeightMultiKernel)(const WeightArgs*, const int64_t*, int, int, int64_t);

// the five-warp team has a pivot warp
static WeightKernel weight_kernel_for(int ts) {
    if (ts == 16) return weights_kernel<16, false>;
    if (ts == 32) return weights_kernel<32, false>;
    return weights_kernel<160, true>;
}
static WeightMultiKernel weight_multi_kernel_for(int ts) {
    if (ts == 16) return weights_multi_kernel<16, false>;
    if (ts == 32) return weights_multi_kernel<32, false>;
    return weights_multi_kernel<160, true>;
}

struct WeightShape {
    int ts;        // threads per team
    int tpb;       // teams per block
    int threads;   // threads per block
    int per_sm;    // resident blocks per SM
    size_t smem;   // dynamic shared memory per block
};

template <class K>
static cudaError_t pick_weight_shape(K kern, int ts, size_t per_team, WeightShape* out) {
    WeightShape b{};
    b.ts = ts;
    const int max_tpb = std::min(weight_max_threads(ts) / ts, 15);   // named barriers 1..15
    const int step = ts == 16 ? 2 : 1;             // whole warps
    int best = -1;
    for (int tpb = step; tpb <= max_tpb; tpb += step) {
        const size_t smem = per_team * tpb;
        if (smem > 227 * 1024) break;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max<size_t>(smem, 48 * 1024));
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb * ts, smem);
        if (e != cudaSuccess) return e;
        if (per_sm * tpb > best) {
            best = per_sm * tpb;
            b.tpb = tpb;
            b.per_sm = per_sm;
        }
    }
    if (best <= 0) {   // a single team does not fit: let the launch report it
        b.tpb = step;
        b.per_sm = 1;
    }
    b.threads = b.tpb * ts;
    b.smem = per_team * b.tpb;
    *out = b;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(b.smem, 48 * 1024));
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

static int weights_impl(const double* xyz, int64_t N, int d, const int32_t* idx, int64_t nc,
                        int n, int m, int op, const double* dirs, double* w, int8_t* status,
                        int64_t* h_n_bad, int64_t* h_first_bad, void* stream) {
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
    A.op = op;
    A.dirs = dirs;
    const size_t per_team = sizeof(double) * weight_team_doubles(A);
    const int sms = device_sm_count();
    WeightShape ws;
    const int ts = weight_team_size(A.s);
    WeightKernel kern = weight_kernel_for(ts);
    RBFFD_CHECK_CUDA(pick_weight_shape(kern, ts, per_team, &ws));
    int64_t want = (nc + ws.tpb - 1) / ws.tpb;
    int64_t grid = std::min<int64_t>(want, (int64_t)sms * ws.per_sm);
    kern<<<(unsigned)grid, ws.threads, ws.smem, s>>>(A, ws.tpb);
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

extern "C" int rbffd_weights(const double* xyz, int64_t N, int d, const int32_t* idx, int64_t nc,
                             int n, int m, double* w, int8_t* status, int64_t* h_n_bad,
                             int64_t* h_first_bad, void* stream) {
    clear_error();
    return weights_impl(xyz, N, d, idx, nc, n, m, 0, nullptr, w, status, h_n_bad, h_first_bad,
                        stream);
}

extern "C" int rbffd_weights_dir(const double* xyz, int64_t N, int d, const int32_t* idx,
                                 int64_t nc, int n, int m, const double* dirs, double* w,
                                 int8_t* status, int64_t* h_n_bad, int64_t* h_first_bad,
                                 void* stream) {
    clear_error();
    RBFFD_ARG(dirs != nullptr || nc == 0, "rbffd_weights_dir: NULL directions");
    return weights_impl(xyz, N, d, idx, nc, n, m, 1, dirs, w, status, h_n_bad, h_first_bad,
                        stream);
}


extern "C" int rbffd_weights_batch(int ncalls, const double* const* xyz, const int64_t* N,
                                   const int* d, const int32_t* const* idx, const int64_t* nc,
                                   const int* n, const int* m, double* const* w,
                                   int8_t* const* status, int64_t* h_n_bad, void* stream) {
    clear_error();
    RBFFD_ARG(ncalls >= 1 && xyz && N && d && idx && nc && n && m && w && status,
              "rbffd_weights_batch: NULL argument");
    cudaStream_t s = as_stream(stream);
    std::vector<WeightArgs> calls(ncalls);
    for (int c = 0; c < ncalls; ++c) {
        RBFFD_ARG(d[c] >= 1 && d[c] <= 3 && m[c] >= 0 && m[c] <= 12 && n[c] >= 1 && nc[c] >= 0 &&
                      N[c] >= 1,
                  "rbffd_weights_batch: bad sizes of call %d", c);
        RBFFD_ARG(nc[c] == 0 || (xyz[c] && idx[c] && w[c] && status[c]),
                  "rbffd_weights_batch: NULL array of call %d", c);
        WeightArgs& A = calls[c];
        const int M = graded_monomials(d[c], m[c], A.ex, W_SMAX);
        RBFFD_ARG(n[c] + M <= W_SMAX, "rbffd_weights_batch: n + M = %d exceeds %d (call %d)",
                  n[c] + M, W_SMAX, c);
        A.xyz = xyz[c];
        A.N = N[c];
        A.d = d[c];
        A.idx = idx[c];
        A.nc = nc[c];
        A.n = n[c];
        A.M = M;
        A.s = n[c] + M;
        A.pitch = (A.s + 1) | 1;
        A.w = w[c];
        A.status = status[c];
        A.lap_phi = (double)(3 * (d[c] + 1));
        A.op = 0;
        A.dirs = nullptr;
    }
    const int sms = device_sm_count();
    // one launch per team size: calls with s <= 32 (half-warp teams), s <= 48
    // (one warp), and the rest (four warps)
    for (int cls = 0; cls < 3; ++cls) {
        std::vector<WeightArgs> sel;
        std::vector<int64_t> off(1, 0);
        size_t team_doubles = 0;
        for (const WeightArgs& A : calls) {
            const int c = A.s <= W_HALF_SMAX ? 0 : (A.s <= 48 ? 1 : 2);
            if (c != cls || A.nc == 0) continue;
            sel.push_back(A);
            off.push_back(off.back() + A.nc);
            team_doubles = std::max(team_doubles, weight_team_doubles(A));
        }
        if (sel.empty()) continue;
        Scratch dcalls, doff;
        RBFFD_CHECK_CUDA(dcalls.alloc(sizeof(WeightArgs) * sel.size(), s));
        RBFFD_CHECK_CUDA(doff.alloc(sizeof(int64_t) * off.size(), s));
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(dcalls.p, sel.data(), sizeof(WeightArgs) * sel.size(),
                                         cudaMemcpyHostToDevice, s));
        RBFFD_CHECK_CUDA(cudaMemcpyAsync(doff.p, off.data(), sizeof(int64_t) * off.size(),
                                         cudaMemcpyHostToDevice, s));
        const size_t per_team = sizeof(double) * team_doubles;
        int max_s = 0;
        for (const WeightArgs& A : sel) max_s = std::max(max_s, A.s);
        WeightShape ws;
        const int ts = weight_team_size(max_s);
        WeightMultiKernel kern = weight_multi_kernel_for(ts);
        RBFFD_CHECK_CUDA(pick_weight_shape(kern, ts, per_team, &ws));
        const int64_t want = (off.back() + ws.tpb - 1) / ws.tpb;
        const int64_t grid = std::min<int64_t>(want, (int64_t)sms * ws.per_sm);
        kern<<<(unsigned)grid, ws.threads, ws.smem, s>>>(dcalls.as<WeightArgs>(),
                                                         doff.as<int64_t>(), (int)sel.size(),
                                                         ws.tpb, (int64_t)team_doubles);
        RBFFD_CHECK_CUDA(cudaGetLastError());
    }
    // singular stencils per call
    Scratch dst, dnc, dcnt;
    RBFFD_CHECK_CUDA(dst.alloc(sizeof(int8_t*) * ncalls, s));
    RBFFD_CHECK_CUDA(dnc.alloc(sizeof(int64_t) * ncalls, s));
    RBFFD_CHECK_CUDA(dcnt.alloc(sizeof(unsigned long long) * ncalls, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(dst.p, status, sizeof(int8_t*) * ncalls,
                                     cudaMemcpyHostToDevice, s));
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(dnc.p, nc, sizeof(int64_t) * ncalls, cudaMemcpyHostToDevice,
                                     s));
    RBFFD_CHECK_CUDA(cudaMemsetAsync(dcnt.p, 0, sizeof(unsigned long long) * ncalls, s));
    count_bad_multi<<<dim3(16, (unsigned)std::min(ncalls, 65535)), 256, 0, s>>>(
        dst.as<int8_t*>(), dnc.as<int64_t>(), ncalls, dcnt.as<unsigned long long>());
    RBFFD_CHECK_CUDA(cudaGetLastError());
    std::vector<unsigned long long> bad(ncalls);
    RBFFD_CHECK_CUDA(cudaMemcpyAsync(bad.data(), dcnt.p, sizeof(unsigned long long) * ncalls,
                                     cudaMemcpyDeviceToHost, s));
    RBFFD_CHECK_CUDA(cudaStreamSynchronize(s));
    unsigned long long tot = 0;
    for (int c = 0; c < ncalls; ++c) {
        if (h_n_bad) h_n_bad[c] = (int64_t)bad[c];
        tot += bad[c];
    }
    if (tot) {
        set_error("rbffd_weights_batch: %llu singular stencils", tot);
        return RBFFD_ERR_SINGULAR;
    }
    return RBFFD_OK;
}
