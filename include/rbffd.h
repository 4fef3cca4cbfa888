/*
 * rbffd.h - C ABI of librbffd, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of the RBF-FD explicit Poisson solver of
 * Vehovar, Rot and Kosec, "Performance Trade-offs of High Order Meshless
 * Approximation on Distributed Memory Systems" (arXiv 2502.12878).
 *
 * Conventions, for every entry point:
 *  - Pointers are DEVICE pointers unless the name starts with h_ (host).
 *    All arrays are caller-owned; the library never frees them.  The only
 *    memory the library owns is inside an rbffd_plan (freed by
 *    rbffd_plan_destroy) and short-lived scratch taken from the stream-ordered
 *    allocator (cudaMallocAsync on the given stream) and returned before the
 *    call returns.
 *  - Coordinates are structure-of-arrays FP64: xyz[a * N + i] is coordinate a
 *    (a < d) of node i.  Node indices are int32.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; device outputs are valid once the stream has reached the
 *    end of the call.  Host outputs (h_*, *_out) are written before return;
 *    calls with host outputs synchronise the stream.
 *  - Return value: RBFFD_OK (0), RBFFD_NOT_CONVERGED (1, a warning), or a
 *    negative error code.  rbffd_last_error() gives a message for the last
 *    failing call on this host thread.  Invalid arguments are rejected before
 *    any device work is enqueued.
 *  - Floating point follows IEEE round-to-nearest: products and sums that the
 *    method defines as separate operations are separately rounded, and every
 *    fused multiply-add is an explicit one (the library is compiled without
 *    contraction).
 */
#ifndef RBFFD_H
#define RBFFD_H

#include <stdint.h>

#if defined(__GNUC__)
#define RBFFD_API __attribute__((visibility("default")))
#else
#define RBFFD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define RBFFD_OK 0
#define RBFFD_NOT_CONVERGED 1      /* step / outer-iteration cap reached */
#define RBFFD_ERR_ARG (-1)         /* invalid argument (nothing enqueued) */
#define RBFFD_ERR_CUDA (-2)        /* CUDA runtime error */
#define RBFFD_ERR_SINGULAR (-3)    /* a local weight system had no usable pivot */
#define RBFFD_ERR_NONFINITE (-4)   /* residual became NaN or Inf */
#define RBFFD_ERR_DIVERGED (-5)    /* residual grew 1e6-fold over its first value */
#define RBFFD_ERR_TIMEOUT (-6)     /* an in-kernel wait gave up (no progress) */
#define RBFFD_ERR_CAPACITY (-7)    /* output capacity or a compiled-in limit exceeded */

/* plan flags */
#define RBFFD_ORDER_MORTON 0       /* interior nodes first, each group in Morton order */
#define RBFFD_ORDER_INPUT 1        /* interior nodes first, each group in input order */
#define RBFFD_ORDER_RANDOM 2       /* interior nodes first, seeded random order */
#define RBFFD_LAUNCH_GRAPH 0       /* one kernel per step, replayed from a CUDA graph */
#define RBFFD_LAUNCH_PERSISTENT 16 /* one cooperative kernel runs many steps */
#define RBFFD_PACK_IDX32 32        /* keep int32 neighbour indices only (no 16-bit codes) */
#define RBFFD_LAUNCH_AUTO 64       /* the autotuner picks graph or persistent per arithmetic */
#define RBFFD_LAUNCH_RESIDENT 128  /* persistent, stencil planes resident in shared memory */
/* graph-replayed steps: the autotuner times plain and programmatic dependent
   launches (each step's blocks scheduled as the previous step drains) and
   keeps the faster; these fix the choice */
#define RBFFD_LAUNCH_PDL 256       /* graph steps as programmatic dependent launches */
#define RBFFD_LAUNCH_NO_PDL 512    /* graph steps as plain launches */
#define RBFFD_LAUNCH_FAR 2048      /* resident, with far lists: each block also stages the
                                      values outside its window that its rows read, so
                                      every gather reads shared memory */
#define RBFFD_LAUNCH_SPLIT 4096    /* persistent, one block per SM over a share of the
                                      rows: stencils streamed, the share's iterate in shared
                                      memory, the rows inside the share computed while
                                      the block waits at the step barrier */

typedef struct rbffd_plan rbffd_plan;

/* Message for the last failing call on this host thread ("" if none). */
RBFFD_API const char* rbffd_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
RBFFD_API int rbffd_version(void);

/*
 * rbffd_nodes - seeded jittered-grid node set.
 * Stands in for the Poisson-disc node generator of Sec. II-C (test problem),
 * which the paper uses to discretise the unit d-cube of Eq. 4-5.
 *   d        2 or 3 (shape 0), 2 (shape 1)
 *   shape    0: unit d-cube; grid of spacing h = 1/Kg, generator indices in
 *               [0,Kg]^d with the last axis fastest; nodes with an index 0 or
 *               Kg are boundary nodes on the exact grid position, the others
 *               get an independent offset (2U-1)*jitter_frac*h per axis, U the
 *               (lin*d+axis)-th output of SplitMix64(seed) mapped to [0,1).
 *            1: disk of radius 1/2 about (1/2,1/2); every grid point is
 *               jittered and kept iff it lies closer than 1/2 - h/2 to the
 *               centre; then round(pi/h) boundary nodes at equal angles.
 *            2: half cube [0,1/2]^d of the mixed-boundary variant (Sec. II-C,
 *               text after Eq. 5): spacing h = 0.5/Kg; nodes with an index 0
 *               are Dirichlet nodes (is_bnd 1) on the grid; other nodes with
 *               an index Kg are Neumann nodes (is_bnd 2) whose Kg coordinates
 *               are exactly 1/2; interior nodes are jittered as in shape 0.
 *   xyz      [d][cap] FP64 out, is_bnd [cap] out (0 interior, 1 Dirichlet,
 *            2 Neumann; every non-zero code is a boundary node)
 *   cap      capacity; with cap = 0 only the count is returned
 *   h_n_out  host: number of nodes.  RBFFD_ERR_CAPACITY if it exceeds cap > 0.
 */
RBFFD_API int rbffd_nodes(int d, int shape, int Kg, double jitter_frac, uint64_t seed, double* xyz,
                uint8_t* is_bnd, int64_t cap, int64_t* h_n_out, void* stream);

/*
 * rbffd_nodes_pds - Poisson-disc node placement (Sec. II-C, last paragraph:
 * the method of Slak and Kosec that the paper uses), spacing h = 1/Kg.
 * The node list starts with the boundary nodes as seeds (d = 2, shape 0, unit
 * square: the grid points (i h, j h) with i or j in {0, Kg}, row-major;
 * shape 1, disk of radius 1/2 about (1/2,1/2): round(pi/h) nodes at angles
 * 2 pi k / Nb; d = 3, unit cube: the grid points with some index 0 or Kg,
 * row-major) and is walked first in, first out: node p proposes K
 * candidates at distance h - in 2D c_j = p + h R(2 pi U_p) e_j, e_j the unit
 * vector at angle 2 pi j / K, U_p the p-th SplitMix64(seed) draw in [0,1);
 * in 3D c_j = p + h R_p e_j, e_j the j-th of K Fibonacci-sphere points
 * (z = 1 - (2j+1)/K, angle j pi (3 - sqrt 5)), R_p the rotation of
 * Shoemake's uniform quaternion from the (3p..3p+2)-th draws.  A candidate
 * inside the open domain (or |c - centre|^2 < 1/4) is appended when every
 * node already in the list is at squared distance >= (zeta h)^2.  The walk
 * ends when every node has been walked.  The GPU walks one generation at a
 * time and reproduces the sequential list bit for bit (angles from the
 * Taylor series of sin/cos, every operation separately rounded).
 *   d        2 or 3 (3: shape 0 only, Kg <= 1000)
 *   K        candidates per node, 1..64 in 2D, 1..256 in 3D (the defaults of
 *            the binding: 15 in 2D, 50 in 3D)
 *   zeta     proximity factor in (0, 1] (default 1 - 1e-10)
 *   xyz      [d][cap] FP64 device out; is_bnd [cap] device out (1 seeds,
 *            0 the rest); seeds first, then the walk's appends in order
 *   h_n_out  host: number of nodes; RBFFD_ERR_CAPACITY if it exceeds cap
 *   h_rounds host [2] (may be NULL): generations walked, and conflict-
 *            resolution passes over all generations
 * Synchronises `stream` (2D: once per 16 generations; 3D: a few times per
 * generation); scratch comes from cudaMallocAsync on `stream`.
 */
RBFFD_API int rbffd_nodes_pds(int d, int shape, int Kg, int K, double zeta, uint64_t seed,
                              double* xyz, uint8_t* is_bnd, int64_t cap, int64_t* h_n_out,
                              int64_t* h_rounds, void* stream);
/* an upper bound on the node count of rbffd_nodes_pds: d = 2, one node per
 * grid cell of side 0.99 zeta h / sqrt 2 over the unit square; d = 3, the
 * packing bound sqrt 2 (1 + zeta h)^3 / (zeta h)^3 (Hales) plus a margin */
RBFFD_API int rbffd_nodes_pds_cap(int d, int Kg, double zeta, int64_t* h_cap);

/*
 * rbffd_interior - ascending list of the interior (non-boundary) node indices.
 *   interior [N] out (first *h_ni_out entries used), h_ni_out host count.
 * The interior rows are where Eq. 6 (jacobi_step) updates u; boundary nodes
 * carry Dirichlet data (Eq. 4).
 */
RBFFD_API int rbffd_interior(const uint8_t* is_bnd, int64_t N, int32_t* interior, int64_t* h_ni_out,
                   void* stream);

/*
 * rbffd_knn - support selection (Sec. II, text after Eq. 1): for each centre,
 * the n nearest of all N nodes, the centre itself included.
 *   xyz      [d][N] coordinates; d in {1, 2, 3}; 1 <= n <= min(N, 128)
 *   centres  [nc] node indices; idx [nc][n] out, row-major.
 * Row r lists its n nodes by increasing key (d2, j), where
 * d2 = fl(fl(dx0*dx0) + fl(dx1*dx1) [+ fl(dx2*dx2)]), dx = fl(x_j - x_c), so
 * equal distances are ordered by node index and the centre comes first.
 * Uses a uniform cell grid (counting sort) and ring search; scratch comes
 * from cudaMallocAsync on `stream`.
 */
RBFFD_API int rbffd_knn(const double* xyz, int64_t N, int d, const int32_t* centres, int64_t nc, int n,
              int32_t* idx, void* stream);

/*
 * rbffd_knn_masked - rbffd_knn restricted to candidate nodes: only nodes with
 * cand[j] != 0 (device, [N]) may appear in a support, besides the centre
 * itself, which is always first.  Used for the supports of Neumann nodes,
 * whose values are set from interior nodes (Sec. II-C: "values from the last
 * step at interior nodes in the support").  RBFFD_ERR_ARG if fewer than n
 * nodes qualify.
 */
RBFFD_API int rbffd_knn_masked(const double* xyz, int64_t N, int d, const uint8_t* cand,
                               const int32_t* centres, int64_t nc, int n, int32_t* idx,
                               void* stream);

/*
 * rbffd_knn_noalloc - rbffd_knn for callers that cannot allocate device
 * memory while they run (the paper has no counterpart): for example an
 * application that reserves all of a GPU's memory up front in its own pool
 * and forbids allocation afterwards, or a latency-bound loop where an
 * allocation's cost or possible failure is not acceptable.  Same arguments
 * and the same result, bit for bit, as rbffd_knn.
 *   Working memory: one fixed array of about 6 MB in the library's device
 *   image, held on every GPU that loads the library until the process exits.
 *   It never calls cudaMalloc, cudaMallocAsync, cudaFree or any allocating
 *   library routine; memsets, copies and kernels go on `stream`.  Every call
 *   synchronises `stream` (host copies of the bounding box and of an error
 *   flag), so it must not be called while `stream` is being captured.
 *   The first call on a device, with that device current, looks up the
 *   array's device address (cudaGetSymbolAddress) and keeps it for the
 *   process; a cudaDeviceReset of that device invalidates it, so do not call
 *   this entry point on a device after resetting it.
 *   N <= RBFFD_KNN_NOALLOC_MAX_NODES, else RBFFD_ERR_CAPACITY (nothing
 *   enqueued).  All calls share the one array: calls that overlap on the GPU
 *   (other streams, other host threads) race and must be serialised by the
 *   caller.  Each call clears the parts that must start at zero.
 */
#define RBFFD_KNN_NOALLOC_MAX_NODES 262144
RBFFD_API int rbffd_knn_noalloc(const double* xyz, int64_t N, int d, const int32_t* centres,
                                int64_t nc, int n, int32_t* idx, void* stream);

/*
 * rbffd_weights - RBF-FD weights of the Laplacian (Eq. 2-3), phi(r) = r^3
 * with all monomials of degree <= m (M = C(m+d, d) of them; Sec. II).
 *   idx [nc][n] supports (first entry = centre, as rbffd_knn returns them)
 *   w   [nc][n] FP64 out; status [nc] int8 out: 0 ok, 1 singular.
 *   s = n + M <= 128.
 * Per row, in scaled coordinates xi = (x_j - x_c)/sigma, sigma the largest
 * support distance: A_jk = r_jk^3, P_ja = xi_j^alpha (graded order: degree,
 * then x exponent descending, then y descending), right-hand side
 * 3(d+1)|xi_j| and 2 for the pure squares; the (n+M)^2 system is solved in
 * FP64 by Gaussian elimination with partial pivoting (first row of largest
 * |pivot|; multiplier = entry x (1/pivot); updates by fused multiply-add; back
 * substitution by columns), and w_j = x_j / sigma^2.  A row is singular when a
 * pivot is not finite or |pivot| <= 1e-13 x max|entry| of its system.
 * Returns RBFFD_ERR_SINGULAR if any row failed; h_n_bad / h_first_bad (host,
 * may be NULL) receive the count and the first failing row.
 */
RBFFD_API int rbffd_weights(const double* xyz, int64_t N, int d, const int32_t* idx, int64_t nc, int n,
                  int m, double* w, int8_t* status, int64_t* h_n_bad, int64_t* h_first_bad,
                  void* stream);

/*
 * rbffd_weights_dir - RBF-FD weights of a directional derivative (the normal
 * derivative of a Neumann condition, Sec. II-C), the same saddle-point system
 * as rbffd_weights with the operator changed: right-hand side
 * -3 |xi_j| (xi_j . dir) for phi = r^3, the dir components for the degree-1
 * monomials, 0 for the others; w_j = x_j / sigma.  dirs [nc][d] unit vectors.
 */
RBFFD_API int rbffd_weights_dir(const double* xyz, int64_t N, int d, const int32_t* idx,
                                int64_t nc, int n, int m, const double* dirs, double* w,
                                int8_t* status, int64_t* h_n_bad, int64_t* h_first_bad,
                                void* stream);

/*
 * rbffd_weights_batch - rbffd_weights for many independent calls (domains) in
 * at most three launches, one per team size (calls whose systems s = n + M
 * are <= 32, <= 48, larger): the stencils of a launch's calls are one index
 * space, each team finding its call by binary search over the calls'
 * stencil counts.  Every
 * stencil sees the operations of rbffd_weights, so the results are the same
 * bit for bit.  Host arrays [ncalls]: xyz (device [d][N]), N, d, idx (device
 * [nc][n]), nc, n, m, w (device out [nc][n]), status (device out [nc]);
 * h_n_bad (host out [ncalls], may be NULL): singular stencils per call.
 * Returns RBFFD_ERR_SINGULAR if any stencil of any call is singular.
 */
RBFFD_API int rbffd_weights_batch(int ncalls, const double* const* xyz, const int64_t* N,
                                  const int* d, const int32_t* const* idx, const int64_t* nc,
                                  const int* n, const int* m, double* const* w,
                                  int8_t* const* status, int64_t* h_n_bad, void* stream);

/*
 * rbffd_apply - Eq. 1: Lu[r] = sum_j w[r][j] * u[idx[r][j]], accumulated as
 * a fused multiply-add chain in support order starting from 0.
 *   w, idx [nc][n] (row-major, as rbffd_weights / rbffd_knn give them),
 *   u [N], Lu [nc] out.
 */
RBFFD_API int rbffd_apply(const double* w, const int32_t* idx, int64_t nc, int n, const double* u,
                double* Lu, void* stream);

/*
 * rbffd_error - quality of a solution against a reference field u^a (both
 * [N], device): h_max = max_i |u_i - u^a_i| and h_mean = (1/N) sum_i
 * |u_i - u^a_i|, the error measure of Eq. 8 (N = all nodes of the domain).
 * Deterministic (fixed two-pass reduction).  Host outputs, may be NULL.
 */
RBFFD_API int rbffd_error(const double* u, const double* ua, int64_t N, double* h_max,
                          double* h_mean, void* stream);

/*
 * rbffd_fp64_fma_rate - measures the device's FP64 fused multiply-add rate
 * (not part of the paper's method: the roofline of the kernels the FP64 pipe
 * binds, the explicit sweep at larger stencils and the weight build).  For 4
 * and 8 independent fma chains per thread (acc <- fma(w, v, acc), v read from
 * shared memory, as the sweeps' operands come from loads), at the largest
 * resident grid of 256-thread blocks: one untimed warm-up launch, then one
 * launch of `iters` fmas per thread, timed with CUDA events on `stream`.
 * h_fma_per_s (host) receives the fastest shape's FMAs per second, h_ms (host,
 * may be NULL) its timed launch's milliseconds.  Synchronises `stream`.
 */
RBFFD_API int rbffd_fp64_fma_rate(int64_t iters, double* h_fma_per_s, double* h_ms,
                                  void* stream);

/*
 * rbffd_plan_create - device-resident solver plan for Eq. 6.
 * Reorders the nodes (interior first, then by `flags` order), packs the
 * stencils into 32-row slices (weights and neighbour indices interleaved so a
 * warp reads them as contiguous 256-byte lines), keeps an FP32 copy of the
 * weights for defect correction and the transposed interior operator for the
 * adjoint.  All inputs are copied; they may be freed afterwards.
 *   interior [NI] must list exactly the nodes with is_bnd == 0 (any order);
 *   (boundary nodes, is_bnd != 0, keep their values unless set as Neumann
 *   nodes by rbffd_plan_set_neumann);
 *   idx / w [NI][n] are the supports/weights of those rows.
 *   flags: RBFFD_ORDER_* | RBFFD_LAUNCH_* | RBFFD_PACK_IDX32; seed is used by
 *   RBFFD_ORDER_RANDOM.
 *   *plan out.
 * Unless RBFFD_PACK_IDX32 is set, the step kernels read the neighbour indices
 * of a slice as 16-bit codes against up to four window bases of 2^14 slots
 * (a slice whose supports need more windows keeps 32-bit indices); the codes
 * name the same neighbours, so the results are the same bit for bit.
 * Launch mode of the step loops: RBFFD_LAUNCH_GRAPH (default), _PERSISTENT,
 * _RESIDENT, _FAR, _SPLIT, or _AUTO, where the first solve of each
 * arithmetic (FP64 sweep, FP32 inner sweep) times the graph shapes, the
 * persistent launches and (when they fit) the resident and split launches
 * on the plan's own stencils and keeps the fastest (_PERSISTENT times the
 * grid-stride and split launches).  The split launch is a persistent launch
 * of one block per SM over a contiguous share of the slices: the stencils
 * stream from HBM every step, the share's rows' iterate stays in shared
 * memory (two buffers: 16 bytes a row in FP64, so up to about 2.2M interior
 * rows), and the share's leading slices of rows whose supports lie inside
 * it are computed while the block waits for the other SMs at the step
 * barrier; a _SPLIT plan that cannot take it returns RBFFD_ERR_CAPACITY from
 * its first solve.  The resident launch is a persistent launch of one block per SM
 * whose slices' weight and index planes (and their rows' f) are copied into
 * shared memory once per solve by TMA bulk copies, so each step reads only
 * the iterate; it fits while the plan's share per SM does (about 102,000
 * interior rows at n = 30 in FP64 with 16-bit codes, 175,000 for the FP32
 * inner sweep); a _RESIDENT plan that does not fit returns
 * RBFFD_ERR_CAPACITY from its first solve.  A Morton plan created with a
 * flag that allows the resident or split launch, whose share per SM is at
 * least two slices and fits one of them, orders each share's rows with the
 * rows whose supports lie inside the share first, each group in Morton
 * order (the plan's slot order; rbffd_plan_perm reports it); those launches
 * compute these rows while they wait for the other SMs at the step barrier.
 * A plan with Neumann nodes always replays graphs.  Every mode gives the same
 * results bit for bit.
 */
RBFFD_API int rbffd_plan_create(const double* xyz, const uint8_t* is_bnd, int64_t N, int d,
                      const int32_t* interior, const int32_t* idx, const double* w, int64_t NI,
                      int n, int flags, uint64_t seed, rbffd_plan** plan, void* stream);
RBFFD_API int rbffd_plan_destroy(rbffd_plan* plan);
/*
 * rbffd_plan_set_neumann - Neumann boundary nodes of the mixed-boundary
 * variant (Sec. II-C, text after Eq. 5).  Before every explicit step each
 * Neumann node b takes the value that meets its normal-derivative condition
 * from the previous iterate of its other support nodes:
 *   acc = fma-chain_{j>=1} w[b][j] u[idx[b][j]],  u_b = (g_b - acc) / w[b][0]
 * (all from the same previous iterate; then the interior step runs on the
 * updated values).  nodes [NN] boundary node indices, idx [NN][nn] their
 * supports with the node first (rbffd_knn_masked over interior candidates),
 * w [NN][nn] their normal-derivative weights (rbffd_weights_dir), g [NN]
 * Neumann data (NULL = 0).  NN = 0 removes the Neumann nodes.  Solves with
 * Neumann nodes run in the graph launch mode and in FP64; rbffd_stable_dt
 * then estimates the radius of the operator with the Neumann values
 * eliminated.  rbffd_solve_explicit also returns the Neumann node values.
 */
RBFFD_API int rbffd_plan_set_neumann(rbffd_plan* plan, int64_t NN, const int32_t* nodes,
                                     const int32_t* idx, const double* w, int nn,
                                     const double* g, void* stream);
/*
 * rbffd_plan_set_wait - the in-kernel waits of the persistent launch (the
 * end-of-step grid barrier): each gives up after timeout_ms (<= 0: the
 * default, about 2 s; at most 60,000), measured in SM clock cycles at the
 * device's maximum clock, and the solve then returns RBFFD_ERR_TIMEOUT.
 * held_arrivals (0..1024, normally 0) is a failure injection for testing that
 * path: the barrier waits for that many arrivals beyond the grid's, which
 * never come, so every block gives up after the timeout and returns.  Takes
 * effect from the next solve; graph-mode steps have no waits.
 */
RBFFD_API int rbffd_plan_set_wait(rbffd_plan* plan, double timeout_ms, int held_arrivals);
/*
 * rbffd_plan_set_resident_halo - the halo window of the resident launch: each
 * block stages, every step, the iterate's slots from `halo` before its first
 * row to `halo` after its last (clipped to the iterate and to the shared memory
 * left beside the stencil planes) and reads its neighbours there, the others
 * through L2.  halo = -1: no window; halo >= 0: that reach; -2: the autotuner
 * times no window, the rows alone, 256, 1024, 4096 slots and the largest that
 * fits, and keeps the fastest (the default).  Every reach gives the same
 * results bit for bit.  The launch shapes are tuned again on the next solve.
 */
RBFFD_API int rbffd_plan_set_resident_halo(rbffd_plan* plan, int64_t halo);
/*
 * rbffd_plan_set_block - block size of the resident and split launches (one
 * block per SM): 512 or 1024 threads (1024 only for the stencil sizes
 * compiled with it; a size without it leaves that launch out), or 0: the
 * autotuner times both (the default).  Every block size gives the same results
 * bit for bit.  The launch shapes are tuned again on the next solve;
 * RBFFD_ERR_ARG for any other value.
 */
RBFFD_API int rbffd_plan_set_block(rbffd_plan* plan, int threads);
/* node permutation of the plan: perm [N] out, perm[p] = original index of slot p */
RBFFD_API int rbffd_plan_perm(const rbffd_plan* plan, int32_t* perm, void* stream);

/*
 * rbffd_solve_explicit - Eq. 6 (jacobi_step): u_i <- u_i + dt (Lu_i - f_i)
 * at interior nodes, boundary values held; Jacobi order (every row reads the
 * previous iterate).  Step k computes r_i = (sum_j w_ij u^k_j) - f_i and
 * u^{k+1}_i = fma(dt, r_i, u^k_i); R_k = max_i |r_i|.  The run stops after
 * step k when R_k < tol (result u^{k+1}, steps = k+1) or at max_steps.
 *   f [NI] in the order of the plan's `interior` list; u [N] in/out: in, the
 *   start iterate with the Dirichlet data on boundary nodes; out, the result.
 *   dt: time step.  Eq. 7 (cfl) gives h^2/(2d) only as a guideline; use
 *   rbffd_stable_dt for the bound of the actual operator.
 *   precision 0: FP64.  precision 1: FP32 inner iteration inside FP64 defect
 *   correction, see rbffd_solve_dc (its K_in/rho_in from
 *   rbffd_plan_set_dc, its outer cap max(1, max_steps / K_in)).
 *   h_steps_out, h_res_out (host, may be NULL): steps taken (precision 1:
 *   inner steps in total) and the last residual max-norm.
 * Returns RBFFD_OK, RBFFD_NOT_CONVERGED, RBFFD_ERR_NONFINITE,
 * RBFFD_ERR_DIVERGED or RBFFD_ERR_TIMEOUT.
 */
RBFFD_API int rbffd_solve_explicit(rbffd_plan* plan, const double* f, double* u, double dt,
                         int64_t max_steps, double tol, int precision, int64_t* h_steps_out,
                         double* h_res_out, void* stream);

/*
 * rbffd_plan_stats - what the last solve on this plan did (host outputs, may
 * be NULL): h_loop_ms, the GPU time of its step loops measured with CUDA
 * events recorded on the caller's stream around the step launches;
 * h_loop_steps, the steps those loops took; h_launches, the kernels the solve
 * launched; h_shape[4], the autotuned launch shape (register budget, blocks
 * per SM; 0 blocks per SM = the persistent launch, -1 = the resident launch,
 * whose first entry is then its block size in units of 512 threads, + 4
 * when it stages far lists (every gather from shared memory), -2 = the split
 * launch, whose first entry is its block size in units of 512 threads;
 * blocks per SM + 16 = graph-replayed steps launched as programmatic
 * dependent launches) of the FP64 sweep and of the FP32 inner sweep.
 */
RBFFD_API int rbffd_plan_stats(const rbffd_plan* plan, double* h_loop_ms, int64_t* h_loop_steps,
                               int64_t* h_launches, int* h_shape);

/*
 * rbffd_plan_layout - the packed layout's size (host outputs, may be NULL):
 * h_nslices, 32-row slices; h_rows16, interior rows whose slice uses 16-bit
 * index codes; h_bytes64 / h_bytes32, the bytes one FP64 sweep / one FP32
 * inner sweep streams when every gathered neighbour is served from cache
 * (weights, index codes or indices, window bases, and per row f or d, the
 * row's old value and its new value).
 */
RBFFD_API int rbffd_plan_layout(const rbffd_plan* plan, int64_t* h_nslices, int64_t* h_rows16,
                                double* h_bytes64, double* h_bytes32);

/*
 * rbffd_solve_dc - defect correction (the precision split is not in the
 * paper).  Outer, FP64: d = W u - f, D = max|d|; stop when D < tol or after
 * max_outer corrections.  Inner, FP32, on the correction e (0 at the start
 * and on the boundary), w32 = (float) w, d32 = (float) d, dt32 = (float) dt:
 *   rho_i = fmaf-chain(w32_ij e_j) + d32_i,  e_i <- fmaf(dt32, rho_i, e_i),
 * stopping after step k when max|rho| (of e^k) < rho_in * D, or after K_in
 * steps.  Then u_i += (double) e_i.
 */
RBFFD_API int rbffd_solve_dc(rbffd_plan* plan, const double* f, double* u, double dt, double tol,
                   int64_t max_outer, int64_t K_in, double rho_in, int64_t* h_outer_out,
                   int64_t* h_inner_out, double* h_res_out, void* stream);
RBFFD_API int rbffd_plan_set_dc(rbffd_plan* plan, int64_t K_in, double rho_in);

/*
 * Batched solves: many independent domains (uneven node counts and stencil
 * sizes, e.g. squares and disks of 5e3..2e5 nodes with m in {2,4,6}) run
 * Eq. 6 in ONE persistent launch, replayed from a CUDA graph (batching is
 * not in the paper).  Each domain keeps its own plan; every block of the
 * persistent grid belongs to one domain's team, team sizes proportional to
 * the domains' bytes per step; each domain stops on its own (tolerance, step
 * cap, non-finite, divergence).  Domains run concurrently, so the launch
 * overhead of small domains is paid once.
 *
 * rbffd_batch_create - batch over `ndom` plans (they must outlive the batch
 *   and must not be solved separately while a batched solve runs).
 *   blocks_per_sm: blocks of the persistent grid per SM (0: 2); the grid is
 *   max(SMs x blocks_per_sm, ndom) and must fit on the device at once
 *   (else RBFFD_ERR_CAPACITY).
 * rbffd_solve_batch - one batched solve.  f[i] (device, [NI_i], the order of
 *   plan i's interior list) and u[i] (device, [N_i], in/out, Dirichlet data
 *   on boundary nodes) are host arrays of device pointers; dt, max_steps and
 *   tol are host arrays [ndom].  Per domain (host outputs, may be NULL):
 *   steps taken, last residual max-norm, status (RBFFD_OK, RBFFD_NOT_CONVERGED
 *   or an error).  Returns the most severe per-domain status.
 * rbffd_batch_set_shape - launch shape of the persistent grid (re-captures the
 *   graph): threads per block (256, 512, 768 or 1024), register budget minb
 *   (min resident blocks per SM: 1..3 at 256 threads, 1..2 at 512, 1 at 768
 *   and 1024) and
 *   blocks per SM; RBFFD_ERR_ARG for other combinations, RBFFD_ERR_CAPACITY
 *   when the grid cannot be co-resident.  The binding's autotuner times
 *   candidates through it.
 * rbffd_batch_stats - GPU ms of the last batched solve (events around the
 *   graph launch) and the shape h_shape[5] = {minb, blocks_per_sm, grid,
 *   cooperative, threads}.
 */
typedef struct rbffd_batch rbffd_batch;
RBFFD_API int rbffd_batch_create(rbffd_plan* const* plans, int ndom, int blocks_per_sm,
                                 rbffd_batch** batch, void* stream);
RBFFD_API int rbffd_batch_destroy(rbffd_batch* batch);
RBFFD_API int rbffd_solve_batch(rbffd_batch* batch, const double* const* f, double* const* u,
                                const double* dt, const int64_t* max_steps, const double* tol,
                                int64_t* h_steps, double* h_res, int* h_status, void* stream);
RBFFD_API int rbffd_batch_set_shape(rbffd_batch* batch, int minb, int blocks_per_sm, int threads,
                                    void* stream);
RBFFD_API int rbffd_batch_stats(const rbffd_batch* batch, double* h_ms, int* h_shape);
/* relative cost of one step of each domain (host [ndom], > 0), used to size the
 * domains' teams; the default is the number of memory rounds of its slices
 * (slices x (ceil(n/16) + 1)).  The binding's autotuner sets measured costs. */
RBFFD_API int rbffd_batch_set_costs(rbffd_batch* batch, const double* h_cost_per_step);
/* per domain of the last batched solve (host arrays [ndom], may be NULL): start
 * and end of its step loop in ms after the earliest start (GPU global timer), the
 * block that ran its team's rank 0, and its team size in blocks */
RBFFD_API int rbffd_batch_domain_times(const rbffd_batch* batch, double* h_start_ms,
                                       double* h_end_ms, int* h_block, int* h_team);

/*
 * rbffd_stable_dt - stability bound of the explicit step for this operator.
 * Eq. 7 (cfl) bounds dt by h^2/(2d) for regular nodes only; here the bound is
 * 2 / (safety * rho), rho the spectral radius of the interior block W_II
 * estimated by `iters` power iterations from v0 [NI] (plan's interior order):
 * y = W_II v, rho = ||y||_2, v = y / rho.
 */
RBFFD_API int rbffd_stable_dt(rbffd_plan* plan, const double* v0, int iters, double safety,
                    double* h_dt_out, double* h_rho_out, void* stream);

/*
 * rbffd_transpose - build the plan's transposed interior operator now (the
 * adjoint's W^T, derived from Eq. 6; otherwise the first rbffd_adjoint or
 * rbffd_adjoint_w builds it).  Column c of W^T lists the rows r whose support
 * holds c, in ascending interior-list order, with their weights w_rc; columns
 * are stored in 32-column slices padded with zero weights; unless the plan
 * was made with RBFFD_PACK_IDX32, every interior slice also stores 16-bit
 * codes, which the reverse step reads instead of int32 rows: offsets in up to
 * four windows of 2^14 positions where the slice's rows fit in those (same
 * rows, same bits, fewer bytes), else each entry's position in the slice,
 * through which its int32 row is read.  Owned by
 * the plan (freed by rbffd_plan_destroy); a second call does nothing.
 * Synchronises `stream`; scratch comes from cudaMallocAsync on `stream`.
 */
RBFFD_API int rbffd_transpose(rbffd_plan* plan, void* stream);

/*
 * rbffd_transpose_layout - the built transpose's size (host outputs, may be
 * NULL): h_slices, 32-column slices of interior columns; h_cols16, interior
 * columns whose slice uses 16-bit row codes; h_entries, stored entries of the
 * interior slices (padding included); h_bytes, the bytes one reverse step
 * streams when every gathered lambda is served from cache (weights, row
 * codes and the rows they point to, per slice its offset, length and window
 * bases, per column lambda and S read and written).  RBFFD_ERR_ARG before
 * rbffd_transpose.
 */
RBFFD_API int rbffd_transpose_layout(const rbffd_plan* plan, int64_t* h_slices,
                                     int64_t* h_cols16, int64_t* h_entries, double* h_bytes);

/*
 * rbffd_adjoint - gradients of a loss of the K-th iterate of Eq. 6 (the
 * adjoint is not in the paper).  With u^{k+1}_I = u^k_I + dt (W_II u^k_I +
 * W_IB g - f) and u^k_B = g for every k, from dLdu = dL/du^K [N] (caller's
 * node order, every node):
 *   lambda^K = the interior entries of dLdu,
 *   lambda^k = lambda^{k+1} + dt W_II^T lambda^{k+1}, k = K-1..0,
 *   grad_f [NI] = -dt sum_{k=1..K} lambda^k,
 *   grad_g [N]  = dt W_IB^T sum_{k=1..K} lambda^k + dLdu (boundary entries:
 *                 the loss's direct dependence on u^K_B = g; 0 inside),
 *   lam0 [NI]   = lambda^0 = dL/du^0_I (may be NULL).
 * (W^T v)_c is accumulated over rows in ascending interior-list order; the
 * boundary entry is fl(fl(dt * sum) + dLdu_b).  Builds the transpose on the
 * first call (see rbffd_transpose).
 */
RBFFD_API int rbffd_adjoint(rbffd_plan* plan, const double* dLdu, int64_t K, double dt, double* grad_f,
                  double* grad_g, double* lam0, void* stream);

/*
 * rbffd_adjoint_w - rbffd_adjoint plus the gradient with respect to the
 * stencil weights (not in the paper; derived from Eq. 6):
 *   dL/dw_ij = dt sum_{k=0..K-1} lambda^{k+1}_i u^k_{idx_ij},
 * summed for k = K-1 down to 0 as G = fma(lambda^{k+1}_i, u^k_j, G), then
 * grad_w = dt G.  The iterates come back by sqrt(K)-style checkpointing: the
 * caller keeps u^0, u^every, u^{2 every}, ... of its forward run (ckpt,
 * [ceil(K/every)][N], caller order); each segment is replayed forward from its
 * checkpoint (bit-identical to the forward sweep) into a segment buffer of
 * every x N doubles (stream-ordered scratch), then walked backward.
 *   f [NI] the source of the forward run; dLdu [N] as rbffd_adjoint;
 *   grad_w [NI][n] out (caller layout, the row order of the plan's interior
 *   list); grad_f, grad_g, lam0 as rbffd_adjoint.
 */
RBFFD_API int rbffd_adjoint_w(rbffd_plan* plan, const double* f, const double* ckpt,
                              int64_t every, const double* dLdu, int64_t K, double dt,
                              double* grad_w, double* grad_f, double* grad_g, double* lam0,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RBFFD_H */
