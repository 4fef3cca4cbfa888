/*
 * Plain CPU oracle for the RBF-FD explicit Poisson solver of
 * Vehovar, Rot and Kosec, "Performance Trade-offs of High Order Meshless
 * Approximation on Distributed Memory Systems" (arXiv 2502.12878).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library; every routine below is written from the
 * paper's definitions, in the paper's order, as plainly as possible.
 *
 * Floating point: FP64 throughout (the FP32 defect-correction emulation
 * excepted).  Built with -ffp-contract=off, so every fused multiply-add in
 * this file is an explicit fma()/fmaf() call and every other operation is a
 * separately rounded IEEE operation.
 *
 * Routines and what they follow:
 *   sm64_at            SplitMix64 (Steele, Lea & Flood 2014), counter form
 *   oracle_nodes       jittered-grid stand-in for the Poisson-disc sampler
 *                      of Sec. II-C (test problem); unit d-cube or disk
 *   oracle_nodes_pds   the Poisson-disc sampler itself (Sec. II-C, last
 *                      paragraph): boundary seeds, candidates at distance h
 *                      around each node in first-in first-out order
 *   oracle_nodes_pds3  the same in the unit cube (candidates on a sphere,
 *                      randomly rotated per node)
 *   oracle_knn_brute   support = n nearest nodes incl. the centre (Sec. II,
 *                      text after Eq. 1), ties by lower index
 *   oracle_knn_kdtree  the same set, via a kd-tree (pinned to brute force)
 *   oracle_weights     RBF-FD augmented system of Eq. 2-3, phi(r)=r^3,
 *                      monomials up to order m, Gaussian elimination with
 *                      partial pivoting in FP64
 *   oracle_weights_dir the same system for a directional (normal) derivative
 *   oracle_apply       Eq. 1 (stencil operator as a weighted sum)
 *   oracle_solve_explicit  Jacobi-style explicit step, Eq. 6 (jacobi_step)
 *   oracle_solve_mixed the same with Neumann boundary nodes (Sec. II-C)
 *   oracle_solve_dc    Eq. 6 with an FP32 inner iteration on the correction
 *                      inside an FP64 defect-correction loop (paper silent)
 *   oracle_adjoint     transpose of Eq. 6 for a sensor misfit (paper silent)
 *   oracle_adjoint_w   the same, plus the gradient with respect to the weights
 *   oracle_power_rho   spectral-radius estimate for the stability bound that
 *                      Eq. 7 (cfl) only gives as a guideline
 *   oracle_gepp_dense  dense Gaussian elimination used by the pin tests
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* SplitMix64: the c-th output (c = 0, 1, ...) of the generator seeded with  */
/* `seed`.  State after c+1 increments is seed + (c+1)*golden; the output is */
/* the published two-round xor-shift-multiply finaliser of that state.       */
/* ------------------------------------------------------------------------- */
uint64_t sm64_at(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double u01(uint64_t seed, uint64_t c)
{
    /* top 53 bits -> [0, 1) */
    return (double)(sm64_at(seed, c) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------- */
/* Node generation.                                                          */
/*                                                                           */
/* The paper samples Omega with a Poisson-disc variant seeded from the       */
/* boundary (Sec. II-C, last paragraph).  The stand-in used here is a        */
/* jittered grid of spacing h = 1/Kg:                                        */
/*  shape 0 (unit d-cube): generator indices (i0..i_{d-1}) in [0,Kg]^d, the  */
/*    last axis fastest.  A node is a boundary node iff some index is 0 or   */
/*    Kg, and then sits at (i*h) exactly; otherwise each coordinate is       */
/*    i*h + (2U-1)*(jf*h) with U the (lin*d + axis)-th SplitMix64 draw.       */
/*  shape 1 (disk, d = 2, centre (1/2,1/2), R = 1/2): every grid point is    */
/*    jittered as above and kept iff |p - c|^2 < (R - h/2)^2; after them come */
/*    Nb = round(2*pi*R/h) boundary nodes at angles 2*pi*k/Nb.                */
/* ------------------------------------------------------------------------- */

/* sin and cos on [0, pi/2] by their Taylor series (terms up to x^21 / x^20),  */
/* Horner form, separately rounded operations.  Truncation < 2e-17.          */
static void taylor_sincos(double x, double* s, double* c)
{
    double x2 = x * x;
    double ps = 1.0, pc = 1.0;
    /* sin x = x (1 - x^2/(2*3) (1 - x^2/(4*5) (1 - ...))) */
    for (int k = 10; k >= 1; --k) {
        double den_s = (double)((2 * k) * (2 * k + 1));
        double den_c = (double)((2 * k - 1) * (2 * k));
        ps = 1.0 - (x2 / den_s) * ps;
        pc = 1.0 - (x2 / den_c) * pc;
    }
    *s = x * ps;
    *c = pc;
}

/* angle 2*pi*k/Nb reduced to a quadrant and an offset in [0, pi/2) */
static void disk_point(int64_t k, int64_t Nb, double R, double* px, double* py)
{
    const double two_pi = 6.283185307179586;
    const double half_pi = 1.5707963267948966;
    double a = (two_pi * (double)k) / (double)Nb;
    int q = (int)(a / half_pi);
    if (q > 3) q = 3;
    double r = a - (double)q * half_pi;
    if (r < 0.0) r = 0.0;
    double s, c;
    taylor_sincos(r, &s, &c);
    double cx, cy;
    switch (q) {
        case 0: cx = c;  cy = s;  break;
        case 1: cx = -s; cy = c;  break;
        case 2: cx = -c; cy = -s; break;
        default: cx = s; cy = -c; break;
    }
    *px = 0.5 + R * cx;
    *py = 0.5 + R * cy;
}

static int64_t disk_nb(int Kg)
{
    const double two_pi = 6.283185307179586;
    double h = 1.0 / (double)Kg;
    return (int64_t)floor((two_pi * 0.5) / h + 0.5);
}

/* shape 2 (half cube [0, 1/2]^d, the mixed-boundary variant of Sec. II-C):  */
/*   spacing h = 0.5/Kg; a node with an index 0 is a Dirichlet node (code 1)   */
/*   at (i*h); otherwise a node with an index Kg is a Neumann node (code 2),   */
/*   whose Kg coordinates are exactly 1/2 and the others i*h; interior nodes   */
/*   are jittered as in shape 0.                                               */
/* returns the node count; writes at most cap nodes (SoA, xyz[axis*cap + i]) */
int64_t oracle_nodes(int d, int shape, int Kg, double jf, uint64_t seed,
                     double* xyz, uint8_t* is_bnd, int64_t cap)
{
    if (d < 1 || d > 3 || Kg < 2 || shape < 0 || shape > 2) return -1;
    if (shape == 1 && d != 2) return -1;
    double h = (shape == 2 ? 0.5 : 1.0) / (double)Kg;
    double amp = jf * h;
    int64_t side = (int64_t)Kg + 1;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= side;

    int64_t out = 0;
    for (int64_t lin = 0; lin < total; ++lin) {
        int64_t gi[3] = {0, 0, 0};
        int64_t rem = lin;
        for (int a = d - 1; a >= 0; --a) { gi[a] = rem % side; rem /= side; }
        int bnd = 0, lo = 0;
        for (int a = 0; a < d; ++a) {
            if (gi[a] == 0 || gi[a] == Kg) bnd = 1;
            if (gi[a] == 0) lo = 1;
        }
        double p[3];
        if (shape == 0 && bnd) {
            for (int a = 0; a < d; ++a) p[a] = (double)gi[a] * h;
        } else if (shape == 2 && bnd) {
            for (int a = 0; a < d; ++a) p[a] = (gi[a] == Kg) ? 0.5 : (double)gi[a] * h;
            bnd = lo ? 1 : 2;
        } else {
            for (int a = 0; a < d; ++a) {
                double U = u01(seed, (uint64_t)lin * (uint64_t)d + (uint64_t)a);
                p[a] = (double)gi[a] * h + (2.0 * U - 1.0) * amp;
            }
        }
        if (shape == 1) {
            double dx = p[0] - 0.5, dy = p[1] - 0.5;
            double lim = 0.5 - 0.5 * h;
            if (!(dx * dx + dy * dy < lim * lim)) continue;
            bnd = 0;
        }
        if (out < cap) {
            for (int a = 0; a < d; ++a) xyz[(int64_t)a * cap + out] = p[a];
            is_bnd[out] = (uint8_t)bnd;
        }
        ++out;
    }
    if (shape == 1) {
        int64_t Nb = disk_nb(Kg);
        for (int64_t k = 0; k < Nb; ++k) {
            if (out < cap) {
                double px, py;
                disk_point(k, Nb, 0.5, &px, &py);
                xyz[out] = px;
                xyz[cap + out] = py;
                is_bnd[out] = 1;
            }
            ++out;
        }
    }
    return out;
}

/* ------------------------------------------------------------------------- */
/* Poisson-disc node placement (Sec. II-C, last paragraph, after the cited    */
/* method of Slak and Kosec), 2D, constant spacing h = 1/Kg.                  */
/*                                                                           */
/* The node list starts with the seeds, the boundary nodes:                  */
/*   shape 0 (unit square): the grid points (i*h, j*h) with i or j in {0,Kg}, */
/*     in row-major order (j fastest), as in oracle_nodes;                     */
/*   shape 1 (disk, centre (1/2,1/2), R = 1/2): Nb = round(2 pi R / h) nodes  */
/*     at angles 2 pi k / Nb, as in oracle_nodes.                             */
/* Then the list is walked in order (first in, first out; nodes appended     */
/* during the walk are walked too).  Node p proposes K candidates            */
/*   c_j = p + h u_j,  u_j = R(phi_p) e_j,  e_j at angle 2 pi j / K,         */
/* with phi_p = 2 pi U_p, U_p the p-th SplitMix64 draw of `seed` (a random   */
/* rotation of a fixed candidate set per node), j = 0..K-1 in order.  A      */
/* candidate is appended (as an interior node) when it lies inside the       */
/* domain (0 < x, y < 1 for the square; |c - centre|^2 < R^2 for the disk)   */
/* and every node in the list so far is at squared distance >= (zeta h)^2.   */
/*                                                                           */
/* Unit vectors: angle reduced to a quadrant, sin/cos by taylor_sincos; the  */
/* rotation ux = cphi ex - sphi ey, uy = sphi ex + cphi ey; then             */
/* cx = px + h ux.  Every operation separately rounded.                      */
/*                                                                           */
/* Proximity test: with brute != 0 against every node in the list; else via  */
/* a uniform grid of cells of side cs = (0.99 zeta h)/sqrt(2), which holds at */
/* most one node per cell (two nodes in one cell would be closer than zeta h),*/
/* searching the 5 x 5 cells around the candidate's (2 cs > zeta h).  Both   */
/* ways test the same set of pairs that can be closer than zeta h.           */
/* Returns N (writes min(N, cap) nodes, SoA xyz[axis*cap + i]), -1 on bad     */
/* arguments, -2 if a grid cell would hold two nodes.                         */
/* ------------------------------------------------------------------------- */
static void unit_dir(double a, double* ux, double* uy)
{
    const double half_pi = 1.5707963267948966;
    int q = (int)(a / half_pi);
    if (q > 3) q = 3;
    double r = a - (double)q * half_pi;
    if (r < 0.0) r = 0.0;
    double s, c;
    taylor_sincos(r, &s, &c);
    switch (q) {
        case 0: *ux = c;  *uy = s;  break;
        case 1: *ux = -s; *uy = c;  break;
        case 2: *ux = -c; *uy = -s; break;
        default: *ux = s; *uy = -c; break;
    }
}

static double pds_cell_side(double zeta, double h)
{
    return (0.99 * (zeta * h)) / 1.4142135623730951;
}

/* grid cells per axis on [0, 1]; also a bound on the node count per axis^2 */
int64_t oracle_nodes_pds_cap(int Kg, double zeta)
{
    if (Kg < 2 || !(zeta > 0.0 && zeta <= 1.0)) return -1;
    double cs = pds_cell_side(zeta, 1.0 / (double)Kg);
    int64_t G = (int64_t)(1.0 / cs) + 1;
    return G * G;
}

int64_t oracle_nodes_pds(int shape, int Kg, int K, double zeta, uint64_t seed, int brute,
                         double* xyz, uint8_t* is_bnd, int64_t cap)
{
    const double two_pi = 6.283185307179586;
    if ((shape != 0 && shape != 1) || Kg < 2 || K < 1 || K > 64) return -1;
    if (!(zeta > 0.0 && zeta <= 1.0)) return -1;
    const double h = 1.0 / (double)Kg;
    const double cs = pds_cell_side(zeta, h);
    const int64_t G = (int64_t)(1.0 / cs) + 1;
    const int64_t maxn = G * G;
    const double t = zeta * h;
    const double r2 = t * t;
    double* X = (double*)malloc(sizeof(double) * (size_t)maxn);
    double* Y = (double*)malloc(sizeof(double) * (size_t)maxn);
    uint8_t* B = (uint8_t*)malloc((size_t)maxn);
    int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)maxn);
    double* ex = (double*)malloc(sizeof(double) * (size_t)K);
    double* ey = (double*)malloc(sizeof(double) * (size_t)K);
    int64_t N = 0, ret = 0;
    if (!X || !Y || !B || !cell || !ex || !ey) { ret = -1; goto done; }
    for (int64_t c = 0; c < maxn; ++c) cell[c] = -1;
    for (int j = 0; j < K; ++j) unit_dir((two_pi * (double)j) / (double)K, &ex[j], &ey[j]);

    /* seeds */
    if (shape == 0) {
        for (int64_t i = 0; i <= Kg; ++i)
            for (int64_t j = 0; j <= Kg; ++j) {
                if (!(i == 0 || i == Kg || j == 0 || j == Kg)) continue;
                X[N] = (double)i * h;
                Y[N] = (double)j * h;
                B[N] = 1;
                ++N;
            }
    } else {
        int64_t Nb = disk_nb(Kg);
        for (int64_t k = 0; k < Nb; ++k) {
            disk_point(k, Nb, 0.5, &X[N], &Y[N]);
            B[N] = 1;
            ++N;
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        int64_t gx = (int64_t)(X[i] / cs), gy = (int64_t)(Y[i] / cs);
        if (cell[gx * G + gy] >= 0) { ret = -2; goto done; }
        cell[gx * G + gy] = (int32_t)i;
    }

    /* walk the list in order */
    for (int64_t p = 0; p < N; ++p) {
        double ux0, uy0;
        unit_dir(two_pi * u01(seed, (uint64_t)p), &ux0, &uy0);
        for (int j = 0; j < K; ++j) {
            double ux = ux0 * ex[j] - uy0 * ey[j];
            double uy = uy0 * ex[j] + ux0 * ey[j];
            double cx = X[p] + h * ux;
            double cy = Y[p] + h * uy;
            int inside;
            if (shape == 0) {
                inside = cx > 0.0 && cx < 1.0 && cy > 0.0 && cy < 1.0;
            } else {
                double dx = cx - 0.5, dy = cy - 0.5;
                inside = dx * dx + dy * dy < 0.25;
            }
            if (!inside) continue;
            int far = 1;
            if (brute) {
                for (int64_t q = 0; q < N && far; ++q) {
                    double dx = cx - X[q], dy = cy - Y[q];
                    if (dx * dx + dy * dy < r2) far = 0;
                }
            } else {
                int64_t gx = (int64_t)(cx / cs), gy = (int64_t)(cy / cs);
                for (int64_t a = gx - 2; a <= gx + 2 && far; ++a) {
                    if (a < 0 || a >= G) continue;
                    for (int64_t b = gy - 2; b <= gy + 2 && far; ++b) {
                        if (b < 0 || b >= G) continue;
                        int32_t q = cell[a * G + b];
                        if (q < 0) continue;
                        double dx = cx - X[q], dy = cy - Y[q];
                        if (dx * dx + dy * dy < r2) far = 0;
                    }
                }
            }
            if (!far) continue;
            if (N >= maxn) { ret = -2; goto done; }
            int64_t gx = (int64_t)(cx / cs), gy = (int64_t)(cy / cs);
            if (cell[gx * G + gy] >= 0) { ret = -2; goto done; }
            cell[gx * G + gy] = (int32_t)N;
            X[N] = cx;
            Y[N] = cy;
            B[N] = 0;
            ++N;
        }
    }
    for (int64_t i = 0; i < N && i < cap; ++i) {
        xyz[i] = X[i];
        xyz[cap + i] = Y[i];
        is_bnd[i] = B[i];
    }
    ret = N;
done:
    free(X); free(Y); free(B); free(cell); free(ex); free(ey);
    return ret;
}

/* ------------------------------------------------------------------------- */
/* Poisson-disc node placement in 3D: the unit cube, spacing h = 1/Kg.       */
/*                                                                           */
/* Seeds: the boundary grid points (i h, j h, k h) with some index 0 or Kg,   */
/* in row-major order (k fastest).  The list is walked first in, first out;  */
/* node p proposes K candidates c_j = p + h R_p e_j where                     */
/*   e_j  the j-th point of a Fibonacci sphere: z = 1 - (2j+1)/K,            */
/*        rho = sqrt(1 - z^2), angle phi = j*GA - 2 pi floor(j*GA / 2 pi)    */
/*        (GA = pi (3 - sqrt 5)), e_j = (rho cos phi, rho sin phi, z);       */
/*   R_p  the rotation of the unit quaternion (x, y, z, w) =                  */
/*        (s1 sin a2, s1 cos a2, s2 sin a3, s2 cos a3), s1 = sqrt(1 - u1),    */
/*        s2 = sqrt(u1), a2 = 2 pi u2, a3 = 2 pi u3, with u1, u2, u3 the      */
/*        (3p)-th, (3p+1)-th and (3p+2)-th SplitMix64 draws (Shoemake's       */
/*        uniform random rotation), as the usual matrix                       */
/*        [1-2(y2+z2), 2(xy-zw), 2(xz+yw); 2(xy+zw), 1-2(x2+z2), 2(yz-xw);    */
/*         2(xz-yw), 2(yz+xw), 1-2(x2+y2)], y2 = y*y etc.                     */
/* A candidate inside the open cube is appended when every node in the list  */
/* is at squared distance >= (zeta h)^2.  Grid cells of side                 */
/* (0.99 zeta h)/sqrt 3 hold at most one node; the 5x5x5 cells around a      */
/* candidate are searched (2 cs > zeta h).  Returns as oracle_nodes_pds.     */
/* ------------------------------------------------------------------------- */
static void fib_dir(int j, int K, double* ex, double* ey, double* ez)
{
    const double two_pi = 6.283185307179586;
    const double ga = 2.399963229728653;   /* pi (3 - sqrt 5) */
    double z = 1.0 - (double)(2 * j + 1) / (double)K;
    double rho = sqrt(1.0 - z * z);
    double t = (double)j * ga;
    double phi = t - floor(t / two_pi) * two_pi;
    double c, s;
    unit_dir(phi, &c, &s);
    *ex = rho * c;
    *ey = rho * s;
    *ez = z;
}

static void rand_rotation(uint64_t seed, uint64_t p, double R[9])
{
    const double two_pi = 6.283185307179586;
    double u1 = u01(seed, 3 * p), u2 = u01(seed, 3 * p + 1), u3 = u01(seed, 3 * p + 2);
    double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
    double c2, n2, c3, n3;                 /* cos and sin of a2, a3 */
    unit_dir(two_pi * u2, &c2, &n2);
    unit_dir(two_pi * u3, &c3, &n3);
    double x = s1 * n2, y = s1 * c2, z = s2 * n3, w = s2 * c3;
    double xx = x * x, yy = y * y, zz = z * z;
    double xy = x * y, xz = x * z, yz = y * z, xw = x * w, yw = y * w, zw = z * w;
    R[0] = 1.0 - 2.0 * (yy + zz); R[1] = 2.0 * (xy - zw);         R[2] = 2.0 * (xz + yw);
    R[3] = 2.0 * (xy + zw);         R[4] = 1.0 - 2.0 * (xx + zz); R[5] = 2.0 * (yz - xw);
    R[6] = 2.0 * (xz - yw);         R[7] = 2.0 * (yz + xw);         R[8] = 1.0 - 2.0 * (xx + yy);
}

static double pds3_cell_side(double zeta, double h)
{
    return (0.99 * (zeta * h)) / 1.7320508075688772;
}

int64_t oracle_nodes_pds3_cap(int Kg, double zeta)
{
    if (Kg < 2 || !(zeta > 0.0 && zeta <= 1.0)) return -1;
    double cs = pds3_cell_side(zeta, 1.0 / (double)Kg);
    int64_t G = (int64_t)(1.0 / cs) + 1;
    return G * G * G;
}

int64_t oracle_nodes_pds3(int Kg, int K, double zeta, uint64_t seed, int brute, double* xyz,
                          uint8_t* is_bnd, int64_t cap)
{
    if (Kg < 2 || K < 1 || K > 256 || !(zeta > 0.0 && zeta <= 1.0)) return -1;
    const double h = 1.0 / (double)Kg;
    const double cs = pds3_cell_side(zeta, h);
    const int64_t G = (int64_t)(1.0 / cs) + 1;
    const int64_t maxn = G * G * G;
    const double t = zeta * h;
    const double r2 = t * t;
    double* P = (double*)malloc(sizeof(double) * 3 * (size_t)maxn);
    uint8_t* B = (uint8_t*)malloc((size_t)maxn);
    int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)maxn);
    double* E = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    int64_t N = 0, ret = 0;
    if (!P || !B || !cell || !E) { ret = -1; goto done; }
    for (int64_t c = 0; c < maxn; ++c) cell[c] = -1;
    for (int j = 0; j < K; ++j) fib_dir(j, K, &E[3 * j], &E[3 * j + 1], &E[3 * j + 2]);
    for (int64_t i = 0; i <= Kg; ++i)
        for (int64_t j = 0; j <= Kg; ++j)
            for (int64_t k = 0; k <= Kg; ++k) {
                if (!(i == 0 || i == Kg || j == 0 || j == Kg || k == 0 || k == Kg)) continue;
                P[3 * N] = (double)i * h;
                P[3 * N + 1] = (double)j * h;
                P[3 * N + 2] = (double)k * h;
                B[N] = 1;
                ++N;
            }
    for (int64_t i = 0; i < N; ++i) {
        int64_t g = ((int64_t)(P[3 * i] / cs) * G + (int64_t)(P[3 * i + 1] / cs)) * G +
                    (int64_t)(P[3 * i + 2] / cs);
        if (cell[g] >= 0) { ret = -2; goto done; }
        cell[g] = (int32_t)i;
    }
    for (int64_t p = 0; p < N; ++p) {
        double R[9];
        rand_rotation(seed, (uint64_t)p, R);
        for (int j = 0; j < K; ++j) {
            const double* e = &E[3 * j];
            double c[3];
            for (int a = 0; a < 3; ++a) {
                double u = (R[3 * a] * e[0] + R[3 * a + 1] * e[1]) + R[3 * a + 2] * e[2];
                c[a] = P[3 * p + a] + h * u;
            }
            if (!(c[0] > 0.0 && c[0] < 1.0 && c[1] > 0.0 && c[1] < 1.0 && c[2] > 0.0 &&
                  c[2] < 1.0))
                continue;
            int far = 1;
            if (brute) {
                for (int64_t q = 0; q < N && far; ++q) {
                    double dx = c[0] - P[3 * q], dy = c[1] - P[3 * q + 1], dz = c[2] - P[3 * q + 2];
                    if ((dx * dx + dy * dy) + dz * dz < r2) far = 0;
                }
            } else {
                int64_t g0 = (int64_t)(c[0] / cs), g1 = (int64_t)(c[1] / cs),
                        g2 = (int64_t)(c[2] / cs);
                for (int64_t a = g0 - 2; a <= g0 + 2 && far; ++a) {
                    if (a < 0 || a >= G) continue;
                    for (int64_t b = g1 - 2; b <= g1 + 2 && far; ++b) {
                        if (b < 0 || b >= G) continue;
                        for (int64_t e2 = g2 - 2; e2 <= g2 + 2 && far; ++e2) {
                            if (e2 < 0 || e2 >= G) continue;
                            int32_t q = cell[(a * G + b) * G + e2];
                            if (q < 0) continue;
                            double dx = c[0] - P[3 * q], dy = c[1] - P[3 * q + 1],
                                   dz = c[2] - P[3 * q + 2];
                            if ((dx * dx + dy * dy) + dz * dz < r2) far = 0;
                        }
                    }
                }
            }
            if (!far) continue;
            if (N >= maxn) { ret = -2; goto done; }
            int64_t g = ((int64_t)(c[0] / cs) * G + (int64_t)(c[1] / cs)) * G +
                        (int64_t)(c[2] / cs);
            if (cell[g] >= 0) { ret = -2; goto done; }
            cell[g] = (int32_t)N;
            P[3 * N] = c[0];
            P[3 * N + 1] = c[1];
            P[3 * N + 2] = c[2];
            B[N] = 0;
            ++N;
        }
    }
    for (int64_t i = 0; i < N && i < cap; ++i) {
        xyz[i] = P[3 * i];
        xyz[cap + i] = P[3 * i + 1];
        xyz[2 * cap + i] = P[3 * i + 2];
        is_bnd[i] = B[i];
    }
    ret = N;
done:
    free(P); free(B); free(cell); free(E);
    return ret;
}

/* ------------------------------------------------------------------------- */
/* Squared distance, as both kNN routines and the weight build evaluate it:  */
/* dx = x_j - x_c per axis, then fl(fl(dx0^2) + fl(dx1^2)) [+ fl(dx2^2)].    */
/* ------------------------------------------------------------------------- */
static double dist2(const double* xyz, int64_t N, int d, int64_t j, const double* q)
{
    double s = 0.0;
    for (int a = 0; a < d; ++a) {
        double dx = xyz[(int64_t)a * N + j] - q[a];
        double sq = dx * dx;
        s = (a == 0) ? sq : s + sq;
    }
    return s;
}

/* key order (d2, j): lexicographic */
static int key_less(double da, int64_t ja, double db, int64_t jb)
{
    return da < db || (da == db && ja < jb);
}

/* insert (dd, j) into the sorted list (best first) of length *len <= n */
static void topn_insert(double* bd, int32_t* bj, int* len, int n, double dd, int64_t j)
{
    int L = *len;
    if (L == n && !key_less(dd, j, bd[n - 1], bj[n - 1])) return;
    int pos = (L < n) ? L : n - 1;
    while (pos > 0 && key_less(dd, j, bd[pos - 1], bj[pos - 1])) {
        bd[pos] = bd[pos - 1];
        bj[pos] = bj[pos - 1];
        --pos;
    }
    bd[pos] = dd;
    bj[pos] = (int32_t)j;
    if (L < n) *len = L + 1;
}

/* Support of each centre: the n nodes with the smallest (d2, index) key,    */
/* listed in increasing key order, so the centre itself comes first.          */
/* cand (may be NULL): only nodes with cand[j] != 0 are candidates, besides
 * the centre itself, which is always its own first support node */
int oracle_knn_brute_masked(const double* xyz, int64_t N, int d, const uint8_t* cand,
                            const int32_t* centres, int64_t nc, int n, int32_t* idx);

int oracle_knn_brute(const double* xyz, int64_t N, int d, const int32_t* centres,
                     int64_t nc, int n, int32_t* idx)
{
    return oracle_knn_brute_masked(xyz, N, d, NULL, centres, nc, n, idx);
}

int oracle_knn_brute_masked(const double* xyz, int64_t N, int d, const uint8_t* cand,
                            const int32_t* centres, int64_t nc, int n, int32_t* idx)
{
    if (n < 1 || n > N) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t r = 0; r < nc; ++r) {
        double q[3];
        int64_t c = centres[r];
        for (int a = 0; a < d; ++a) q[a] = xyz[(int64_t)a * N + c];
        double* bd = (double*)malloc(sizeof(double) * (size_t)n);
        int len = 0;
        if (!bd) { bad = 1; continue; }
        for (int64_t j = 0; j < N; ++j)
            if (!cand || cand[j] || j == c)
                topn_insert(bd, idx + r * n, &len, n, dist2(xyz, N, d, j, q), j);
        if (len < n) bad = 1;
        free(bd);
    }
    return bad ? -2 : 0;
}

/* ---------------------------- kd-tree ------------------------------------ */
typedef struct {
    int axis;        /* -1 for a leaf */
    double split;
    int64_t lo, hi;  /* range in perm[] for a leaf */
    int64_t left, right;
} kd_node;

typedef struct {
    const double* xyz;
    int64_t N;
    int d;
    const uint8_t* cand;
    int64_t self;
    int64_t* perm;
    kd_node* nodes;
    int64_t count;
} kd_tree;

static const double* g_sort_coord; /* used only inside the single-threaded build */
static int cmp_coord(const void* a, const void* b)
{
    int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
    double va = g_sort_coord[ia], vb = g_sort_coord[ib];
    if (va < vb) return -1;
    if (va > vb) return 1;
    return (ia < ib) ? -1 : (ia > ib);
}

static int64_t kd_build(kd_tree* t, int64_t lo, int64_t hi, int depth)
{
    int64_t me = t->count++;
    kd_node* nd = &t->nodes[me];
    if (hi - lo <= 8) {
        nd->axis = -1;
        nd->lo = lo;
        nd->hi = hi;
        return me;
    }
    int axis = depth % t->d;
    g_sort_coord = t->xyz + (int64_t)axis * t->N;
    qsort(t->perm + lo, (size_t)(hi - lo), sizeof(int64_t), cmp_coord);
    int64_t mid = lo + (hi - lo) / 2;
    double split = g_sort_coord[t->perm[mid]];
    int64_t l = kd_build(t, lo, mid, depth + 1);
    int64_t r = kd_build(t, mid, hi, depth + 1);
    nd = &t->nodes[me];
    nd->axis = axis;
    nd->split = split;
    nd->left = l;
    nd->right = r;
    return me;
}

/* Points left of the split have coordinate <= split, right ones >= split.
 * A subtree is skipped only when the squared distance to its half-space,
 * computed with the same rounded subtraction and square as dist2, exceeds
 * the current n-th key strictly: rounding is monotone, so no point of the
 * subtree can have a smaller computed d2, and ties are still visited. */
static void kd_query(const kd_tree* t, int64_t ni, const double* q, double* bd,
                     int32_t* bj, int* len, int n)
{
    const kd_node* nd = &t->nodes[ni];
    if (nd->axis < 0) {
        for (int64_t p = nd->lo; p < nd->hi; ++p) {
            int64_t j = t->perm[p];
            if (t->cand && !t->cand[j] && j != t->self) continue;
            topn_insert(bd, bj, len, n, dist2(t->xyz, t->N, t->d, j, q), j);
        }
        return;
    }
    double diff = q[nd->axis] - nd->split;
    int64_t near = diff <= 0.0 ? nd->left : nd->right;
    int64_t far = diff <= 0.0 ? nd->right : nd->left;
    kd_query(t, near, q, bd, bj, len, n);
    double lb = diff * diff;
    if (*len < n || !(lb > bd[n - 1])) kd_query(t, far, q, bd, bj, len, n);
}

int oracle_knn_kdtree_masked(const double* xyz, int64_t N, int d, const uint8_t* cand,
                             const int32_t* centres, int64_t nc, int n, int32_t* idx);

int oracle_knn_kdtree(const double* xyz, int64_t N, int d, const int32_t* centres,
                      int64_t nc, int n, int32_t* idx)
{
    return oracle_knn_kdtree_masked(xyz, N, d, NULL, centres, nc, n, idx);
}

int oracle_knn_kdtree_masked(const double* xyz, int64_t N, int d, const uint8_t* cand,
                             const int32_t* centres, int64_t nc, int n, int32_t* idx)
{
    if (n < 1 || n > N) return -1;
    kd_tree t;
    t.xyz = xyz;
    t.N = N;
    t.d = d;
    t.cand = cand;
    t.self = -1;
    t.perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    t.nodes = (kd_node*)malloc(sizeof(kd_node) * (size_t)(2 * N / 4 + 64));
    t.count = 0;
    if (!t.perm || !t.nodes) { free(t.perm); free(t.nodes); return -2; }
    for (int64_t i = 0; i < N; ++i) t.perm[i] = i;
    kd_build(&t, 0, N, 0);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int64_t r = 0; r < nc; ++r) {
        double q[3];
        int64_t c = centres[r];
        for (int a = 0; a < d; ++a) q[a] = xyz[(int64_t)a * N + c];
        double* bd = (double*)malloc(sizeof(double) * (size_t)n);
        if (!bd) { bad = 1; continue; }
        int len = 0;
        kd_tree tl = t;      /* per-centre copy: the centre is always a candidate */
        tl.self = c;
        kd_query(&tl, 0, q, bd, idx + r * n, &len, n);
        if (len < n) bad = 1;
        free(bd);
    }
    free(t.perm);
    free(t.nodes);
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------- */
/* RBF-FD weights (Eq. 2-3).                                                 */
/*                                                                           */
/* For centre x_c with support x_1..x_n (x_1 = x_c):                         */
/*  sigma = max_j ||x_j - x_c||, xi_j = (x_j - x_c)/sigma per axis.          */
/*  A_jk = phi(||xi_j - xi_k||), phi(r) = r^3 = (r*r)*r.                     */
/*  P_ja = xi_j^alpha over the M = C(m+d, d) monomials of degree <= m in     */
/*    graded order: degree ascending, then x exponent descending, then y     */
/*    exponent descending; powers by repeated multiplication, the factors    */
/*    multiplied in axis order.                                              */
/*  RHS: (L Phi)_j = Laplacian of r^3 about x_j, at x_c:                     */
/*    3(d+1) ||xi_j||;  (L p)_a = 2 for x^2, y^2, z^2 and 0 otherwise.       */
/*  Solve [[A P];[P^T 0]] [w; lambda] = [L Phi; L p] (s = n + M unknowns)     */
/*    by Gaussian elimination with partial pivoting (gepp_solve below).      */
/*  w_j = x_j / sigma^2 (the Laplacian scales as 1/sigma^2).                  */
/* ------------------------------------------------------------------------- */
int oracle_num_monomials(int d, int m)
{
    /* C(m+d, d) */
    int64_t num = 1, den = 1;
    for (int k = 1; k <= d; ++k) { num *= (m + k); den *= k; }
    return (int)(num / den);
}

/* exponents [M][3] in graded order */
int oracle_monomials(int d, int m, int* ex)
{
    int M = 0;
    for (int deg = 0; deg <= m; ++deg) {
        if (d == 1) {
            ex[3 * M + 0] = deg; ex[3 * M + 1] = 0; ex[3 * M + 2] = 0; ++M;
        } else if (d == 2) {
            for (int a = deg; a >= 0; --a) {
                ex[3 * M + 0] = a; ex[3 * M + 1] = deg - a; ex[3 * M + 2] = 0; ++M;
            }
        } else {
            for (int a = deg; a >= 0; --a)
                for (int b = deg - a; b >= 0; --b) {
                    ex[3 * M + 0] = a; ex[3 * M + 1] = b; ex[3 * M + 2] = deg - a - b; ++M;
                }
        }
    }
    return M;
}

static double ipow(double x, int e)
{
    double p = 1.0;
    for (int k = 0; k < e; ++k) p = p * x;
    return p;
}

/* Gaussian elimination with partial pivoting on the s x (s+1) row-major
 * augmented matrix G (last column = right-hand side); solution in x.
 * Elimination: for k = 0..s-1, pivot row p = first row i >= k with the
 * largest |G[i][k]|; swap rows k and p; rp = 1 / G[k][k]; for every row
 * i > k, l = G[i][k] * rp (the column scaled by the reciprocal pivot, as
 * LAPACK's unblocked LU does) and G[i][j] = fma(-l, G[k][j], G[i][j]) for j > k.
 * A pivot is unusable (status 1: numerically singular system) when it is not
 * finite or |pivot| <= 1e-13 * gmax, gmax = max |G[i][j]| over the matrix as
 * assembled (right-hand side excluded); an all-zero matrix is singular too.
 * Back substitution by columns: for j = s-1..0, x_j = G[j][s] / G[j][j],
 * then G[i][s] = fma(-G[i][j], x_j, G[i][s]) for every i < j.
 * Returns 0, or 1 when a pivot is non-finite or |pivot| <= 1e-300. */
int oracle_gepp_solve(int s, double* G, double* x)
{
    const int W = s + 1;
    double gmax = 0.0;
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) {
            double v = fabs(G[(int64_t)i * W + j]);
            if (v > gmax) gmax = v;
        }
    const double tiny = 1e-13 * gmax;
    for (int k = 0; k < s; ++k) {
        int p = k;
        double best = fabs(G[(int64_t)k * W + k]);
        for (int i = k + 1; i < s; ++i) {
            double v = fabs(G[(int64_t)i * W + k]);
            if (v > best) { best = v; p = i; }
        }
        if (!(best > tiny) || !(best > 1e-300) || !isfinite(best)) return 1;
        if (p != k)
            for (int j = 0; j < W; ++j) {
                double t = G[(int64_t)k * W + j];
                G[(int64_t)k * W + j] = G[(int64_t)p * W + j];
                G[(int64_t)p * W + j] = t;
            }
        double rp = 1.0 / G[(int64_t)k * W + k];
        for (int i = k + 1; i < s; ++i) {
            double l = G[(int64_t)i * W + k] * rp;
            for (int j = k + 1; j < W; ++j)
                G[(int64_t)i * W + j] = fma(-l, G[(int64_t)k * W + j], G[(int64_t)i * W + j]);
        }
    }
    for (int j = s - 1; j >= 0; --j) {
        double xj = G[(int64_t)j * W + s] / G[(int64_t)j * W + j];
        if (!isfinite(xj)) return 1;
        x[j] = xj;
        for (int i = 0; i < j; ++i)
            G[(int64_t)i * W + s] = fma(-G[(int64_t)i * W + j], xj, G[(int64_t)i * W + s]);
    }
    return 0;
}

/* one stencil; xyz is SoA with stride N; sup holds n node indices.
 * op 0: Laplacian (Eq. 2-3 as above).  op 1: derivative along the unit vector
 * dir (the normal derivative of a Neumann condition): (L Phi)_j = grad of
 * r^3 about x_j at x_c along dir = 3 |x_c - x_j| (x_c - x_j).dir, i.e.
 * -3 |xi_j| (xi_j . dir) in scaled coordinates; (L p)_a = dir component for
 * the degree-1 monomials, 0 otherwise; w_j = x_j / sigma. */
int oracle_weights_op(const double* xyz, int64_t N, int d, const int32_t* sup, int n, int m,
                      int op, const double* dir, double* w_out);

int oracle_weights_one(const double* xyz, int64_t N, int d, const int32_t* sup, int n,
                       int m, double* w_out)
{
    return oracle_weights_op(xyz, N, d, sup, n, m, 0, NULL, w_out);
}

int oracle_weights_op(const double* xyz, int64_t N, int d, const int32_t* sup, int n, int m,
                      int op, const double* dir, double* w_out)
{
    int ex[3 * 400];
    if (oracle_num_monomials(d, m) > 400) return 2;
    int M = oracle_monomials(d, m, ex);
    int s = n + M;
    int64_t c = sup[0];
    double* xi = (double*)malloc(sizeof(double) * (size_t)(3 * n));
    double* G = (double*)malloc(sizeof(double) * (size_t)s * (size_t)(s + 1));
    double* x = (double*)malloc(sizeof(double) * (size_t)s);
    if (!xi || !G || !x) { free(xi); free(G); free(x); return 2; }

    /* scale: sigma = max_j sqrt(d2_j) */
    double sigma = 0.0;
    for (int j = 0; j < n; ++j) {
        double s2 = 0.0;
        for (int a = 0; a < d; ++a) {
            double dx = xyz[(int64_t)a * N + sup[j]] - xyz[(int64_t)a * N + c];
            double sq = dx * dx;
            s2 = (a == 0) ? sq : s2 + sq;
        }
        double r = sqrt(s2);
        if (r > sigma) sigma = r;
    }
    if (!(sigma > 0.0)) { free(xi); free(G); free(x); return 1; }
    for (int j = 0; j < n; ++j)
        for (int a = 0; a < d; ++a) {
            double dx = xyz[(int64_t)a * N + sup[j]] - xyz[(int64_t)a * N + c];
            xi[3 * j + a] = dx / sigma;
        }

    const int W = s + 1;
    memset(G, 0, sizeof(double) * (size_t)s * (size_t)W);
    for (int j = 0; j < n; ++j) {
        for (int k = 0; k < n; ++k) {
            double r2 = 0.0;
            for (int a = 0; a < d; ++a) {
                double t = xi[3 * j + a] - xi[3 * k + a];
                double sq = t * t;
                r2 = (a == 0) ? sq : r2 + sq;
            }
            double r = sqrt(r2);
            G[(int64_t)j * W + k] = (r * r) * r;
        }
        for (int al = 0; al < M; ++al) {
            double p = ipow(xi[3 * j + 0], ex[3 * al + 0]);
            if (d >= 2) p = p * ipow(xi[3 * j + 1], ex[3 * al + 1]);
            if (d >= 3) p = p * ipow(xi[3 * j + 2], ex[3 * al + 2]);
            G[(int64_t)j * W + n + al] = p;
            G[(int64_t)(n + al) * W + j] = p;
        }
        double rc2 = 0.0;
        for (int a = 0; a < d; ++a) {
            double sq = xi[3 * j + a] * xi[3 * j + a];
            rc2 = (a == 0) ? sq : rc2 + sq;
        }
        if (op == 0) {
            G[(int64_t)j * W + s] = (double)(3 * (d + 1)) * sqrt(rc2);
        } else {
            double dot = 0.0;
            for (int a = 0; a < d; ++a) {
                double t = xi[3 * j + a] * dir[a];
                dot = (a == 0) ? t : dot + t;
            }
            G[(int64_t)j * W + s] = -((3.0 * sqrt(rc2)) * dot);
        }
    }
    for (int al = 0; al < M; ++al) {
        int deg = ex[3 * al] + ex[3 * al + 1] + ex[3 * al + 2];
        double v = 0.0;
        if (op == 0) {
            int pure2 = (deg == 2) && (ex[3 * al] == 2 || ex[3 * al + 1] == 2 || ex[3 * al + 2] == 2);
            v = pure2 ? 2.0 : 0.0;
        } else if (deg == 1) {
            for (int a = 0; a < d; ++a)
                if (ex[3 * al + a] == 1) v = dir[a];
        }
        G[(int64_t)(n + al) * W + s] = v;
    }

    int st = oracle_gepp_solve(s, G, x);
    if (st == 0) {
        double scale = (op == 0) ? sigma * sigma : sigma;
        for (int j = 0; j < n; ++j) w_out[j] = x[j] / scale;
    }
    free(xi);
    free(G);
    free(x);
    return st;
}

/* all stencils; idx[r*n..] is the support of centre r; status[r] = 0 ok,
 * 1 singular, 2 bad arguments.  Returns the number of non-zero statuses. */
int64_t oracle_weights(const double* xyz, int64_t N, int d, const int32_t* idx, int64_t nc,
                       int n, int m, double* w, int8_t* status)
{
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int64_t r = 0; r < nc; ++r) {
        int st = oracle_weights_one(xyz, N, d, idx + r * n, n, m, w + r * n);
        status[r] = (int8_t)st;
        if (st) {
            bad += 1;
            for (int j = 0; j < n; ++j) w[r * n + j] = 0.0;
        }
    }
    return bad;
}

/* directional-derivative weights for each row; dirs [nc][d] unit vectors */
int64_t oracle_weights_dir(const double* xyz, int64_t N, int d, const int32_t* idx, int64_t nc,
                           int n, int m, const double* dirs, double* w, int8_t* status)
{
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int64_t r = 0; r < nc; ++r) {
        int st = oracle_weights_op(xyz, N, d, idx + r * n, n, m, 1, dirs + r * d, w + r * n);
        status[r] = (int8_t)st;
        if (st) {
            bad += 1;
            for (int j = 0; j < n; ++j) w[r * n + j] = 0.0;
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1: (L u)(x_c) = sum_j w_j u(x_j), one row per centre, accumulated as  */
/* an fma chain in support order starting from 0.                           */
/* ------------------------------------------------------------------------- */
void oracle_apply(const double* w, const int32_t* idx, int64_t nc, int n, const double* u,
                  double* Lu)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nc; ++r) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(w[r * n + j], u[idx[r * n + j]], acc);
        Lu[r] = acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Eq. 6 (jacobi_step): u_i <- u_i + dt (Lu_i - f_i) at interior nodes,      */
/* boundary values held.  Jacobi: every row reads the previous iterate.      */
/* Per step k: r_i = (sum_j w_ij u^k_j) - f_i, u^{k+1}_i = fma(dt, r_i, u^k_i). */
/* The stop test after step k uses R_k = max_i |r_i| (the residual of u^k):  */
/* if R_k < tol the result is u^{k+1} and steps = k+1.  A non-finite R_k     */
/* stops with status 2.  u: [N] in/out (interior entries are the start       */
/* iterate, boundary entries the Dirichlet data); rows listed by interior.   */
/* Returns 0 converged, 1 step cap reached, 2 non-finite.                    */
/* ------------------------------------------------------------------------- */
int oracle_solve_explicit(const double* w, const int32_t* idx, const int32_t* interior,
                          int64_t N, int64_t NI, int n, const double* f, double* u,
                          double dt, int64_t max_steps, double tol, int64_t* steps_out,
                          double* res_out)
{
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    if (!v) return -2;
    memcpy(v, u, sizeof(double) * (size_t)N);
    double* cur = u;
    double* nxt = v;
    int status = 1;
    int64_t k = 0;
    double R = 0.0;
    for (k = 0; k < max_steps; ++k) {
        R = 0.0;
        int nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(max : R) reduction(| : nonfinite)
        for (int64_t r = 0; r < NI; ++r) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = fma(w[r * n + j], cur[idx[r * n + j]], acc);
            double ri = acc - f[r];
            int64_t i = interior[r];
            nxt[i] = fma(dt, ri, cur[i]);
            double a = fabs(ri);
            if (!isfinite(a)) nonfinite = 1;
            else if (a > R) R = a;
        }
        double* t = cur; cur = nxt; nxt = t;
        if (nonfinite) { status = 2; R = INFINITY; ++k; break; }
        if (R < tol) { status = 0; ++k; break; }
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * (size_t)N);
    free(v);
    *steps_out = k;
    *res_out = R;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Eq. 6 with Neumann boundary nodes (mixed-boundary variant, Sec. II-C).    */
/* Before each step the value of every Neumann node b is set so that its    */
/* normal-derivative stencil (support nidx[b][0..nn), nidx[b][0] = b, weights */
/* nw) meets the Neumann data g_b, using the previous iterate for the other  */
/* support nodes:  acc = fma-chain_{j>=1} nw_bj u_j,  u_b = (g_b - acc)/nw_b0 */
/* (all Neumann values from the same previous iterate).  Then the interior   */
/* step of oracle_solve_explicit runs on the updated values; the stop rule,  */
/* statuses and outputs are the same.                                        */
/* ------------------------------------------------------------------------- */
int oracle_solve_mixed(const double* w, const int32_t* idx, const int32_t* interior, int64_t N,
                       int64_t NI, int n, const double* f, const int32_t* nnode,
                       const int32_t* nidx, const double* nw, int64_t NN, int nn,
                       const double* g, double* u, double dt, int64_t max_steps, double tol,
                       int64_t* steps_out, double* res_out)
{
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    double* un = (double*)malloc(sizeof(double) * (size_t)(NN > 0 ? NN : 1));
    if (!v || !un) { free(v); free(un); return -2; }
    memcpy(v, u, sizeof(double) * (size_t)N);
    double* cur = u;
    double* nxt = v;
    int status = 1;
    int64_t k = 0;
    double R = 0.0;
    for (k = 0; k < max_steps; ++k) {
        for (int64_t b = 0; b < NN; ++b) {
            double acc = 0.0;
            for (int j = 1; j < nn; ++j) acc = fma(nw[b * nn + j], cur[nidx[b * nn + j]], acc);
            un[b] = (g[b] - acc) / nw[b * nn];
        }
        for (int64_t b = 0; b < NN; ++b) {
            cur[nnode[b]] = un[b];
            nxt[nnode[b]] = un[b];
        }
        R = 0.0;
        int nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(max : R) reduction(| : nonfinite)
        for (int64_t r = 0; r < NI; ++r) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = fma(w[r * n + j], cur[idx[r * n + j]], acc);
            double ri = acc - f[r];
            int64_t i = interior[r];
            nxt[i] = fma(dt, ri, cur[i]);
            double a = fabs(ri);
            if (!isfinite(a)) nonfinite = 1;
            else if (a > R) R = a;
        }
        double* t = cur; cur = nxt; nxt = t;
        if (nonfinite) { status = 2; R = INFINITY; ++k; break; }
        if (R < tol) { status = 0; ++k; break; }
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * (size_t)N);
    free(v);
    free(un);
    *steps_out = k;
    *res_out = R;
    return status;
}

/* ------------------------------------------------------------------------- */
/* FP32 inner iteration inside FP64 defect correction (paper silent; the    */
/* precision split is the build's).  Outer t: d = W u - f in FP64 (apply   */
/* chain, then - f); D = max|d|; stop when D < tol.  Inner, on the          */
/* correction e (float, e = 0 at start and on the boundary):                */
/*   q_i = fmaf-chain of w32_ij e_j, rho_i = q_i + d32_i,                   */
/*   e_i <- fmaf(dt32, rho_i, e_i),                                         */
/* stopping after step k when max|rho| (of e^k) < rho_in * D, or at K_in.   */
/* Then u_i += (double) e_i at interior nodes.                              */
/* w32 = (float) w, d32 = (float) d, dt32 = (float) dt.                      */
/* res_in_out (may be NULL): max|rho| of the last inner step taken.         */
/* Returns 0 converged, 1 outer cap, 2 non-finite.                          */
/* ------------------------------------------------------------------------- */
int oracle_solve_dc(const double* w, const int32_t* idx, const int32_t* interior, int64_t N,
                    int64_t NI, int n, const double* f, double* u, double dt, double tol,
                    int64_t max_outer, int64_t K_in, double rho_in, int64_t* outer_out,
                    int64_t* inner_total_out, double* res_out, double* res_in_out)
{
    float* w32 = (float*)malloc(sizeof(float) * (size_t)(NI * n));
    float* e0 = (float*)calloc((size_t)N, sizeof(float));
    float* e1 = (float*)calloc((size_t)N, sizeof(float));
    float* d32 = (float*)malloc(sizeof(float) * (size_t)NI);
    if (!w32 || !e0 || !e1 || !d32) { free(w32); free(e0); free(e1); free(d32); return -2; }
    for (int64_t q = 0; q < NI * n; ++q) w32[q] = (float)w[q];
    float dt32 = (float)dt;
    int status = 1;
    int64_t t = 0, inner_total = 0;
    double D = 0.0, R_in_last = 0.0;
    for (t = 0; t <= max_outer; ++t) {
        D = 0.0;
        int nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(max : D) reduction(| : nonfinite)
        for (int64_t r = 0; r < NI; ++r) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = fma(w[r * n + j], u[idx[r * n + j]], acc);
            double dr = acc - f[r];
            d32[r] = (float)dr;
            double a = fabs(dr);
            if (!isfinite(a)) nonfinite = 1;
            else if (a > D) D = a;
        }
        if (nonfinite) { status = 2; D = INFINITY; break; }
        if (D < tol) { status = 0; break; }
        if (t == max_outer) break;
        memset(e0, 0, sizeof(float) * (size_t)N);
        memset(e1, 0, sizeof(float) * (size_t)N);
        float* ec = e0;
        float* en = e1;
        double lim = rho_in * D;
        int inner_bad = 0;
        for (int64_t k = 0; k < K_in; ++k) {
            double Rin = 0.0;
            int nf = 0;
#pragma omp parallel for schedule(static) reduction(max : Rin) reduction(| : nf)
            for (int64_t r = 0; r < NI; ++r) {
                float acc = 0.0f;
                for (int j = 0; j < n; ++j) acc = fmaf(w32[r * n + j], ec[idx[r * n + j]], acc);
                float rho = acc + d32[r];
                int64_t i = interior[r];
                en[i] = fmaf(dt32, rho, ec[i]);
                double a = fabs((double)rho);
                if (!isfinite(a)) nf = 1;
                else if (a > Rin) Rin = a;
            }
            float* tmp = ec; ec = en; en = tmp;
            ++inner_total;
            R_in_last = nf ? INFINITY : Rin;
            if (nf) { inner_bad = 1; break; }
            if (Rin < lim) break;
        }
        if (inner_bad) { status = 2; D = INFINITY; break; }
        for (int64_t r = 0; r < NI; ++r) {
            int64_t i = interior[r];
            u[i] = u[i] + (double)ec[i];
        }
    }
    *outer_out = t;
    *inner_total_out = inner_total;
    *res_out = D;
    if (res_in_out) *res_in_out = R_in_last;
    free(w32); free(e0); free(e1); free(d32);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of K explicit steps (paper silent; derived from Eq. 6).           */
/* Forward: u^{k+1}_I = u^k_I + dt (W_II u^k_I + W_IB g - f), u^0 given.     */
/* Loss L = sum_s (u^K_s - u_obs_s)^2 over sensor rows s (interior rows).    */
/* lambda^K = dL/du^K (2 (u^K - u_obs) at sensors, 0 elsewhere);             */
/* lambda^k = lambda^{k+1} + dt W_II^T lambda^{k+1}, k = K-1..0.             */
/* dL/df = -dt sum_{k=1..K} lambda^k ;  dL/dg = dt W_IB^T sum_{k=1..K} lambda^k */
/* dL/du^0_I = lambda^0.                                                     */
/* (W^T lambda)_j is accumulated over rows i in ascending order as an fma    */
/* chain from 0; the update is fma(dt, acc_j, lambda_j).                     */
/* Input: dLdu [N] = dL/du^K over all nodes (node order).  Its interior     */
/* entries are lambda^K; a boundary entry b is the loss's direct dependence  */
/* on u^K_b = g_b, so dL/dg_b = dt (W_IB^T S)_b + dLdu_b (two roundings).    */
/* Outputs: grad_f [NI], grad_g [N] (only boundary entries non-zero),        */
/* lam0 [NI].  Sum of lambda is accumulated with plain additions in k order. */
/* ------------------------------------------------------------------------- */
int oracle_adjoint(const double* w, const int32_t* idx, const int32_t* interior, int64_t N,
                   int64_t NI, int n, const double* dLdu, int64_t K, double dt,
                   double* grad_f, double* grad_g, double* lam0)
{
    double* lam = (double*)malloc(sizeof(double) * (size_t)NI);
    double* acc = (double*)malloc(sizeof(double) * (size_t)N);
    double* S = (double*)calloc((size_t)NI, sizeof(double));
    int32_t* row_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (!lam || !acc || !S || !row_of) { free(lam); free(acc); free(S); free(row_of); return -2; }
    for (int64_t i = 0; i < N; ++i) row_of[i] = -1;
    for (int64_t r = 0; r < NI; ++r) row_of[interior[r]] = (int32_t)r;
    for (int64_t r = 0; r < NI; ++r) lam[r] = dLdu[interior[r]];
    for (int64_t k = K; k >= 1; --k) {
        /* S += lambda^k */
        for (int64_t r = 0; r < NI; ++r) S[r] = S[r] + lam[r];
        /* lambda^{k-1} = lambda^k + dt W_II^T lambda^k */
        for (int64_t i = 0; i < N; ++i) acc[i] = 0.0;
        for (int64_t r = 0; r < NI; ++r)
            for (int j = 0; j < n; ++j) {
                int64_t col = idx[r * n + j];
                acc[col] = fma(w[r * n + j], lam[r], acc[col]);
            }
        for (int64_t r = 0; r < NI; ++r) lam[r] = fma(dt, acc[interior[r]], lam[r]);
    }
    memcpy(lam0, lam, sizeof(double) * (size_t)NI);
    for (int64_t r = 0; r < NI; ++r) grad_f[r] = -dt * S[r];
    for (int64_t i = 0; i < N; ++i) acc[i] = 0.0;
    for (int64_t r = 0; r < NI; ++r)
        for (int j = 0; j < n; ++j) {
            int64_t col = idx[r * n + j];
            acc[col] = fma(w[r * n + j], S[r], acc[col]);
        }
    for (int64_t i = 0; i < N; ++i) grad_g[i] = (row_of[i] < 0) ? dt * acc[i] + dLdu[i] : 0.0;
    free(lam); free(acc); free(S); free(row_of);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient with respect to the stencil weights (paper silent; derived from   */
/* Eq. 6): u^{k+1}_i = u^k_i + dt (sum_j w_ij u^k_{idx_ij} - f_i) gives       */
/* dL/dw_ij = dt sum_{k=0..K-1} lambda^{k+1}_i u^k_{idx_ij}.  The iterates   */
/* u^0..u^{K-1} are recomputed from u0 and stored (plain, memory K x N); the */
/* sum runs k = K-1 down to 0 as G = fma(lambda^{k+1}_i, u^k_j, G), then     */
/* grad_w = dt * G.  lambda follows oracle_adjoint (same order, same S).     */
/* Also returns grad_f, grad_g, lam0 as oracle_adjoint does (dLdu [N] as    */
/* there: interior entries lambda^K, boundary entries the direct term).     */
/* ------------------------------------------------------------------------- */
int oracle_adjoint_w(const double* w, const int32_t* idx, const int32_t* interior, int64_t N,
                     int64_t NI, int n, const double* f, const double* u0, const double* dLdu,
                     int64_t K, double dt, double* grad_w, double* grad_f, double* grad_g,
                     double* lam0)
{
    double* U = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1) * (size_t)N);
    double* lam = (double*)malloc(sizeof(double) * (size_t)NI);
    double* acc = (double*)malloc(sizeof(double) * (size_t)N);
    double* S = (double*)calloc((size_t)NI, sizeof(double));
    double* G = (double*)calloc((size_t)(NI * n), sizeof(double));
    int32_t* row_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (!U || !lam || !acc || !S || !G || !row_of) {
        free(U); free(lam); free(acc); free(S); free(G); free(row_of);
        return -2;
    }
    for (int64_t i = 0; i < N; ++i) row_of[i] = -1;
    for (int64_t r = 0; r < NI; ++r) row_of[interior[r]] = (int32_t)r;
    /* forward: store u^0 .. u^{K-1} */
    if (K > 0) memcpy(U, u0, sizeof(double) * (size_t)N);
    for (int64_t k = 0; k + 1 < K; ++k) {
        const double* cur = U + (size_t)k * N;
        double* nxt = U + (size_t)(k + 1) * N;
        memcpy(nxt, cur, sizeof(double) * (size_t)N);
        for (int64_t r = 0; r < NI; ++r) {
            double a = 0.0;
            for (int j = 0; j < n; ++j) a = fma(w[r * n + j], cur[idx[r * n + j]], a);
            double ri = a - f[r];
            nxt[interior[r]] = fma(dt, ri, cur[interior[r]]);
        }
    }
    for (int64_t r = 0; r < NI; ++r) lam[r] = dLdu[interior[r]];
    for (int64_t k = K - 1; k >= 0; --k) {
        const double* uk = U + (size_t)k * N;
        /* weight gradient with lambda^{k+1} and u^k */
        for (int64_t r = 0; r < NI; ++r)
            for (int j = 0; j < n; ++j)
                G[r * n + j] = fma(lam[r], uk[idx[r * n + j]], G[r * n + j]);
        /* S += lambda^{k+1}; lambda^k = lambda^{k+1} + dt W_II^T lambda^{k+1} */
        for (int64_t r = 0; r < NI; ++r) S[r] = S[r] + lam[r];
        for (int64_t i = 0; i < N; ++i) acc[i] = 0.0;
        for (int64_t r = 0; r < NI; ++r)
            for (int j = 0; j < n; ++j) {
                int64_t col = idx[r * n + j];
                acc[col] = fma(w[r * n + j], lam[r], acc[col]);
            }
        for (int64_t r = 0; r < NI; ++r) lam[r] = fma(dt, acc[interior[r]], lam[r]);
    }
    for (int64_t q = 0; q < NI * n; ++q) grad_w[q] = dt * G[q];
    memcpy(lam0, lam, sizeof(double) * (size_t)NI);
    for (int64_t r = 0; r < NI; ++r) grad_f[r] = -dt * S[r];
    for (int64_t i = 0; i < N; ++i) acc[i] = 0.0;
    for (int64_t r = 0; r < NI; ++r)
        for (int j = 0; j < n; ++j) {
            int64_t col = idx[r * n + j];
            acc[col] = fma(w[r * n + j], S[r], acc[col]);
        }
    for (int64_t i = 0; i < N; ++i) grad_g[i] = (row_of[i] < 0) ? dt * acc[i] + dLdu[i] : 0.0;
    free(U); free(lam); free(acc); free(S); free(G); free(row_of);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Spectral radius of W_II by power iteration from v (length NI, overwritten) */
/* for `iters` steps: y = W_II v, rho = ||y||_2 / ||v||_2, v = y / ||y||_2.   */
/* Boundary columns see 0.  Returns the last rho.                             */
/* ------------------------------------------------------------------------- */
double oracle_power_rho(const double* w, const int32_t* idx, const int32_t* interior,
                        int64_t N, int64_t NI, int n, double* v, int iters)
{
    double* full = (double*)calloc((size_t)N, sizeof(double));
    double* y = (double*)malloc(sizeof(double) * (size_t)NI);
    if (!full || !y) { free(full); free(y); return -1.0; }
    double nv = 0.0;
    for (int64_t r = 0; r < NI; ++r) nv += v[r] * v[r];
    nv = sqrt(nv);
    for (int64_t r = 0; r < NI; ++r) v[r] = v[r] / nv;
    double rho = 0.0;
    for (int it = 0; it < iters; ++it) {
        for (int64_t r = 0; r < NI; ++r) full[interior[r]] = v[r];
        oracle_apply(w, idx, NI, n, full, y);
        double ny = 0.0;
        for (int64_t r = 0; r < NI; ++r) ny += y[r] * y[r];
        ny = sqrt(ny);
        rho = ny;
        if (!(ny > 0.0)) break;
        for (int64_t r = 0; r < NI; ++r) v[r] = y[r] / ny;
    }
    free(full);
    free(y);
    return rho;
}

/* dense s x s solve A x = b by the same elimination as the weight build
 * (A row-major, overwritten); used by the pin tests on tiny problems */
int oracle_gepp_dense(int s, const double* A, const double* b, double* x)
{
    double* G = (double*)malloc(sizeof(double) * (size_t)s * (size_t)(s + 1));
    if (!G) return -2;
    for (int i = 0; i < s; ++i) {
        for (int j = 0; j < s; ++j) G[(int64_t)i * (s + 1) + j] = A[(int64_t)i * s + j];
        G[(int64_t)i * (s + 1) + s] = b[i];
    }
    int st = oracle_gepp_solve(s, G, x);
    free(G);
    return st;
}

/* threads OpenMP would use for the parallel loops above */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
