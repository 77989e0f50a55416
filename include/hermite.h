/*
 * hermite.h -- C ABI of the B300 (sm_103a) Hermite wave-equation library.
 *
 * The library advances u_tt = c^2 Lap u with the arbitrary-order Hermite
 * methods of Appelo, Hagstrom and Vargas, "Hermite Methods for the Scalar
 * Wave Equation": the dissipative method (Sec. 3; order 2m-1, the "full"
 * variant of Sec. 3.3 for d > 1) and the conservative method (Sec. 4;
 * order 2m), on the staggered primal/dual grids of Sec. 2.1 with periodic,
 * homogeneous Dirichlet or homogeneous Neumann boundaries (Sec. 3.1.3).
 *
 * Conventions shared by every entry point
 *   Domain       [0, N h]^d, N cells per axis.  Periodic: N primal nodes
 *                (x = i h) and N dual nodes (x = (j+1/2) h) per axis.
 *                Dirichlet/Neumann: N+1 primal and N dual nodes per axis.
 *   Host layout  row-major state[node][coef], FP64.  Nodes in C order over
 *                the axes (axis 0 slowest).  Coefficients: multi-index
 *                k = (k_0..k_{d-1}) in C order; u has k in [0,m]^d
 *                (Nu = (m+1)^d values), v has k in [0,m-1]^d (Nv = m^d).
 *                Values are the paper's scaled derivatives h^|k|/k! d^k u
 *                and h^|k|/k! d^k v (Sec. 2.2, Sec. 3.1.1).
 *   Steps        hermite_step(n) performs n full steps = 2n half-steps of
 *                dt/2 each (Sec. 2.1: primal at t_n, dual at t_{n+1/2}).
 *   Ownership    The library owns all device memory of a context; the caller
 *                owns every buffer it passes.  Host pointers are read/written
 *                synchronously; device pointers are used on the context's
 *                stream.  No C++ exception crosses this interface.
 *   Errors       Every int-returning call returns HERMITE_OK (0) or a
 *                negative HERMITE_ERR_* code; hermite_last_error() gives a
 *                message for the context.  A failed call leaves the stored
 *                state unchanged unless the code is HERMITE_ERR_CUDA.
 *   Threads      A context must not be used by two host threads at once.
 */
#ifndef HERMITE_H
#define HERMITE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hermite_ctx hermite_ctx;

/* Variants: Sec. 3.3 "full" dissipative (special interpolants I_{m,..,m-1}
 * for the first time derivative; identical to the 1-D method when d = 1),
 * Sec. 4 conservative, Sec. 3.3 plain tensor-product ("simple") dissipative. */
enum { HERMITE_DISSIPATIVE = 0, HERMITE_CONSERVATIVE = 1, HERMITE_DISSIPATIVE_SIMPLE = 2 };
/* Boundaries (Sec. 3.1.3): ghost polynomials are odd (Dirichlet) or even
 * (Neumann) reflections of the first interior dual node. */
enum { HERMITE_PERIODIC = 0, HERMITE_DIRICHLET = 1, HERMITE_NEUMANN = 2 };
/* Grids. */
enum { HERMITE_PRIMAL = 0, HERMITE_DUAL = 1 };

enum {
  HERMITE_OK = 0,
  HERMITE_ERR_ARG = -1,         /* invalid argument (sizes, CFL, pointers) */
  HERMITE_ERR_ALLOC = -2,       /* device or host allocation failed */
  HERMITE_ERR_CUDA = -3,        /* a CUDA call failed; see hermite_last_error */
  HERMITE_ERR_NONFINITE = -4,   /* NaN/Inf found in an energy reduction */
  HERMITE_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
  HERMITE_ERR_STATE = -6,       /* call not valid in the current state */
  HERMITE_ERR_UNSUPPORTED = -7  /* (d, m) outside the compiled range */
};

/* Create a problem (Sec. 2.1 grids; Sec. 3/4 methods).
 *   d in {1,2,3}; m >= 1 (dissipative) or m >= 0 (conservative); N >= 1
 *   cells per axis; c > 0 wave speed; h > 0 cell width; dt > 0 with
 *   0 < c dt / h <= 1 (the CFL bound under which the evolution of the cell
 *   polynomial at the new node is exact, Sec. 3.1.2 / 4.1).
 *   Supported (d, m): every m with 2m+1 <= 255 coefficients per node for
 *   d = 1, m <= 6 for d = 2, m <= 3 for d = 3 (else HERMITE_ERR_UNSUPPORTED).
 * Allocates both grids on the current CUDA device and builds the per-cell
 * operator (the interpolation + Taylor evolution + evaluation map of one
 * cell, Eqs. Hermcon, recursion_diss_1d_1/2, recursion_ut/vt, update) in
 * FP64 on the device.  The state is zero until set.  *out receives the
 * context (NULL on error). */
int hermite_create(int d, int m, int64_t N, double c, double h, double dt,
                   int variant, int bc, hermite_ctx **out);

/* Arithmetic of the half-step kernels.
 *   HERMITE_FP64     state and arithmetic in IEEE double precision.
 *   HERMITE_SPLIT32  state and operator as unevaluated sums of two FP32 numbers
 *                    (hi + lo, about 48 significant bits); every multiply-add
 *                    is formed from three split products (hi*hi exactly, hi*lo,
 *                    lo*hi) with error-free compensated accumulation on the
 *                    FP32 pipe.  Energies stay FP64 reductions. */
enum { HERMITE_FP64 = 0, HERMITE_SPLIT32 = 1 };

/* hermite_create with a choice of arithmetic (HERMITE_FP64 or
 * HERMITE_SPLIT32); same arguments, contracts and errors otherwise.  A split
 * context also keeps FP64 copies of both grids for I/O and energies (twice
 * the device memory of an FP64 context). */
int hermite_create_ex(int d, int m, int64_t N, double c, double h, double dt,
                      int variant, int bc, int precision, hermite_ctx **out);

/* Release all device memory of the context (NULL is ignored). */
void hermite_destroy(hermite_ctx *ctx);

/* Run subsequent device work of this context on the given cudaStream_t
 * (NULL = the legacy default stream). */
int hermite_set_stream(hermite_ctx *ctx, void *stream);

/* Initial data at t = 0 on the primal grid (Sec. 3.1.1), host buffers:
 *   u [nodes_primal][Nu], v [nodes_primal][Nv] (v may be NULL = zero).
 * Dissipative: both levels are the given data.  Conservative (Sec. 4): u is
 * the primal level at t = 0 and the dual level at t = dt/2 is generated by
 * the Taylor series of the cell interpolants of (u, v) (the paper leaves the
 * start-up open); v is ignored when m = 0.  Resets the step counter. */
int hermite_set_state(hermite_ctx *ctx, const double *u, const double *v);

/* Same with device pointers (same layout), read on the context's stream. */
int hermite_set_state_device(hermite_ctx *ctx, const double *u, const double *v);

/* Conservative only: both levels given, host buffers, u_primal at t = 0
 * [nodes_primal][Nu] and u_dual at t = dt/2 [nodes_dual][Nu]. */
int hermite_set_state2(hermite_ctx *ctx, const double *u_primal, const double *u_dual);

/* Testing hook (process-wide, no counterpart in the paper): the n-th device
 * allocation the library makes after this call fails as if the device were
 * out of memory (the call that made it returns HERMITE_ERR_ALLOC and frees
 * what it had allocated); n = 0 turns the hook off.  HERMITE_ERR_ARG if n < 0. */
int hermite_debug_fail_alloc(int n);

/* Advance n >= 0 full steps (2n half-steps), device work only, enqueued on
 * the context's stream (asynchronous with respect to the host). */
int hermite_step(hermite_ctx *ctx, int64_t nsteps);

/* Advance n >= 0 half-steps.  Dissipative: alternately primal->dual and
 * dual->primal.  Conservative: alternately update the primal level from the
 * dual one and the dual level from the primal one (Eq. update). */
int hermite_advance_half(hermite_ctx *ctx, int64_t nhalf);

/* Number of half-steps taken since the state was set. */
int64_t hermite_half_steps(const hermite_ctx *ctx);

/* Time of the primal level.  Dissipative: half-steps * dt/2 (the newest
 * level, primal after an even count).  Conservative: ((half-steps + 1) / 2) * dt
 * in integer division, i.e. half-steps * dt/2 rounded UP to a whole step: the
 * first half-step updates the primal level from t = 0 to t = dt, the second
 * the dual level from dt/2 to 3dt/2, and so on. */
double hermite_time(const hermite_ctx *ctx);

/* L2 error of the cell interpolant against an exact solution (Sec. 5.1: the
 * piecewise I_m interpolant of the u data, degree 2m+1 per axis, compared with
 * the exact solution at quadrature points), reduced in FP64 on the device.
 *   grid    grid holding the u level (cells are centred at the nodes of the
 *           other grid; ghost polynomials and half cells at non-periodic
 *           boundaries as for the energies)
 *   cells   device pointer to ncells cell indices (nodes of grid 1-grid, C
 *           order), or NULL for every cell in order (ncells must then equal
 *           hermite_nodes(ctx, 1-grid)); indices outside [0, nodes) are
 *           skipped
 *   nq, xq, wq  host arrays: nq <= 16 quadrature points per axis in cell
 *           units (xi in [-1/2, 1/2]) and weights summing to 1
 *   exact   device pointer [ncells][nq^d]: the exact u at the points
 *           centre + h (xq[i_0], .., xq[i_{d-1}]), C order over the axes
 *   out     host: out[0] = sum over the cells of the quadrature of
 *           (I_m u - exact)^2, out[1] = the same of exact^2 (both include h^d)
 * Split contexts use their hi + lo level.  Allocates a small device buffer and
 * synchronises the context's stream.  HERMITE_ERR_ARG for bad arguments. */
int hermite_l2_error(hermite_ctx *ctx, int grid, int64_t ncells, const int64_t *cells, int nq, const double *xq,
                     const double *wq, const double *exact, double out[2]);

/* Primal-grid state, host buffers [nodes_primal][Nu] / [nodes_primal][Nv]
 * (v may be NULL; ignored for the conservative method).  Dissipative: valid
 * after an even number of half-steps (HERMITE_ERR_STATE otherwise).
 * Synchronises the context's stream. */
int hermite_get_state(hermite_ctx *ctx, double *u, double *v);

/* Either grid's stored data, host buffers (v may be NULL). */
int hermite_get_grid(hermite_ctx *ctx, int grid, double *u, double *v);
/* Overwrite either grid's stored data from host buffers (v may be NULL = 0). */
int hermite_set_grid(hermite_ctx *ctx, int grid, const double *u, const double *v);
/* Copy either grid into caller-owned device buffers (same layout). */
int hermite_get_grid_device(hermite_ctx *ctx, int grid, double *u, double *v);

/* Energies of the latest level (Sec. 3.2, 3.3, 4.2), exact per-cell
 * quadrature of the piecewise interpolants, reduced on the device in the
 * context's arithmetic (FP64, or hi + lo FP32 pairs for split contexts) with
 * FP64 block sums:
 *   dissipative  out[0] = int v^2 + c^2 |grad u|^2 over the domain
 *                out[1] = c^2 sum_i |d_i I^(i) u|^2_{m,..,m} + |I_{m-1} v|^2_{m,..,m}
 *                         (Eq. stable1 for d = 1, the left side of Eq. stable2
 *                         for d > 1; non-increasing for d = 1)
 *   conservative out[0] = c^2 int |grad p^n|^2 of the primal level
 *                out[1] = G = |p^{n+1/2}|^2_{m+1,..} - <p^{n+1}, p^n>_{m+1,..},
 *                         conserved by the scheme (equals half the paper's
 *                         |P+|^2 + |P-|^2 of Eq. Vdef in 1-D)
 *   out[2] = 0 (reserved).
 * For non-periodic problems cells cut by the boundary count half per axis.
 * Returns HERMITE_ERR_NONFINITE if a result is NaN/Inf.  Synchronises. */
int hermite_energy(hermite_ctx *ctx, double out[3]);

/* Sizes: nodes on a grid, and coefficients per node. */
int64_t hermite_nodes(const hermite_ctx *ctx, int grid);
int hermite_ncoef(const hermite_ctx *ctx, int *nu, int *nv);

/* Copy the FP64 per-cell operator of the reference corner (every axis at
 * xi = -1/2), row-major: rows = outputs (u then v, or u only), columns =
 * inputs (u then v, or u only), both in the paper's scaled units.  The other
 * corners follow by reflection.  which = 0: half-step operator; 1:
 * conservative start-up operator.  rows/cols receive the sizes; out may be
 * NULL to query them. */
int hermite_operator(hermite_ctx *ctx, int which, double *out, int *rows, int *cols);

/* Allocation-free energy of a caller-provided level.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the energy -- e.g. code that runs where a
 * cudaMalloc would be illegal or would stall the device, or a host that only
 * lends the library buffers it already owns.  It performs the same reduction
 * as hermite_energy's two quadratic forms but keeps its per-block partial
 * sums in a fixed 2 MB array inside the library (held on every device that
 * uses this call until the library is unloaded) instead of allocating.
 *   ctx      an existing context (its forms and stream are used)
 *   grid     grid holding the level (HERMITE_PRIMAL or HERMITE_DUAL)
 *   level    device pointer, coefficient-major layout level[coef * ld + node]
 *            (u coefficients then v coefficients, paper units), FP64
 *   ld       plane stride in elements, ld >= hermite_nodes(ctx, grid)
 *   out_dev  device pointer to 2 doubles, written on the context's stream:
 *            dissipative: [int v^2 + c^2|grad u|^2, stable1/stable2 energy];
 *            conservative: [|p|^2_{m+1,..,m+1}, c^2 int |grad p|^2].
 * Limit: at most 2^21 cells (= nodes of the other grid); larger problems get
 * HERMITE_ERR_ARG with a message; a context without energy forms (a batch
 * problem) gets HERMITE_ERR_STATE, as from hermite_energy.  No host
 * synchronisation.  The first call
 * on a device looks up the array's device address (make that first call
 * before any stream capture).  All calls share the one array: calls whose
 * work overlaps on the GPU (other streams or threads) race and must be
 * serialised by the caller.  The context's device must be current. */
int hermite_energy_noalloc(hermite_ctx *ctx, int grid, const double *level, int64_t ld, double *out_dev);

/* Measured FMA throughput of the current device, for roofline denominators
 * (the paper has no counterpart: a measurement aid).  kind 0: FP64 FMA,
 * 1: FP32 FMA, 2: FP32 FMA on packed pairs (two per instruction, the form the
 * split-precision kernels issue).  Eight independent FMA chains per thread
 * over 8 blocks of 256 threads per SM, timed with CUDA events on a private
 * stream after one warm-up launch; *flops_per_s counts an FMA as 2 flops.
 * Allocates and frees a small device buffer; synchronises that stream.
 * HERMITE_ERR_ARG for a NULL pointer or unknown kind, HERMITE_ERR_CUDA on a
 * CUDA failure (then *flops_per_s = 0). */
int hermite_peak_probe(int kind, double *flops_per_s);

/* Engine of a split-precision context's half-step (the operator and the
 * arithmetic are the same, Sec. 3 / 4; the engines differ in how the FP32
 * hi + lo products are formed):
 *   0  CUDA cores: compensated FP32 multiply-adds on packed pairs (default);
 *   1  tensor cores (tcgen05): exact products of BF16 digits of both operands
 *      with FP32 accumulation, available where d >= 2 and every parity class
 *      of inputs and of outputs is at most 16 coefficients wide (3-D m <= 3,
 *      2-D m <= 4), for contexts of hermite_create / hermite_create_ex (not
 *      for the problems of a batch, which run the batch kernels).
 * HERMITE_ERR_STATE for an FP64 context, HERMITE_ERR_UNSUPPORTED if engine 1
 * is asked for a shape it does not cover, HERMITE_ERR_ARG otherwise bad.
 * hermite_get_split_engine returns the engine in use (-1: not a split context). */
int hermite_set_split_engine(hermite_ctx *ctx, int engine);
int hermite_get_split_engine(const hermite_ctx *ctx);

/* Tensor-core self-test (the paper has no counterpart): one CTA computes
 * D0 = A B^T and D1 = A B[0:N-16]^T with tcgen05.mma (BF16 operands in the
 * no-swizzle K-major shared-memory layout of the tensor-core half-step, FP32
 * accumulation in tensor memory, D1 at a column offset) for library-generated
 * integer operands |a|, |b| <= 256, so that every exact partial sum is an
 * integer below 2^24.  K in {16, 32, .., 128}, N in {32, 48, .., 96}.  Host
 * buffers: A [128][K] and B [N][K] receive the operands, D0 [128][N] and
 * D1 [128][N-16] the products.  HERMITE_ERR_TIMEOUT if the MMA completion wait
 * ran out (bounded), HERMITE_ERR_ARG for bad sizes.  Synchronises the device. */
int hermite_tc_selftest(int K, int N, float *A, float *B, float *D0, float *D1);

/* ------------------------------------------------------------------------
 * Ragged batches.  Many independent problems -- differing N, m, boundary
 * condition, variant and time step, one dimension d for the whole batch --
 * advanced together: every half-step of the batch is one persistent launch
 * per group of problems with similar output counts, whose blocks take
 * (problem, node range) items from a work counter (longest items first), so
 * small and large grids share the GPU in one launch.  A full step is
 * captured once as a CUDA graph and replayed.  The method per problem is the
 * same as for a single context (Sec. 3 / 4); no data moves between problems.
 * ---------------------------------------------------------------------- */
typedef struct hermite_batch hermite_batch;

/* Create nprob problems; arrays of length nprob give each problem's
 * hermite_create arguments.  precision: HERMITE_FP64 or HERMITE_SPLIT32 for
 * all problems.  Batch problems carry no energy forms (hermite_energy on them
 * returns HERMITE_ERR_STATE).  On error *out is NULL and
 * hermite_batch_last_error(NULL) names the failing problem. */
int hermite_batch_create(int nprob, const int *d, const int *m, const int64_t *N, const double *c,
                         const double *h, const double *dt, const int *variant, const int *bc,
                         int precision, hermite_batch **out);
void hermite_batch_destroy(hermite_batch *b);

/* Borrowed context of problem p (owned by the batch; do not destroy it) for
 * hermite_set_state / set_state2 / get_state / get_grid.  NULL if p is out of
 * range.  All problems must have taken the same number of half-steps when
 * hermite_batch_step is called. */
hermite_ctx *hermite_batch_problem(hermite_batch *b, int p);

/* Stream for the batch and all its problems.  Graph capture needs a
 * non-default stream; on the legacy default stream the batch launches its
 * kernels directly. */
int hermite_batch_set_stream(hermite_batch *b, void *stream);

/* Advance every problem by nsteps full steps (device work only). */
int hermite_batch_step(hermite_batch *b, int64_t nsteps);

/* Every problem's level on `grid` in one launch on the batch stream (no
 * synchronisation): u receives the [nodes][Nu] host-layout blocks of problems
 * 0, 1, ... back to back, v the [nodes][Nv] blocks (v may be NULL; nothing is
 * written to it for conservative problems).  Device pointers. */
int hermite_batch_get_states_device(hermite_batch *b, int grid, double *u, double *v);

/* Inverse for the primal level of dissipative problems (the state, as
 * hermite_set_state_device on each problem: clocks restart at 0); same
 * back-to-back layout, v may be NULL (= 0).  HERMITE_ERR_STATE if a problem is
 * conservative (its start-up level needs hermite_set_state). */
int hermite_batch_set_states_device(hermite_batch *b, const double *u, const double *v);

/* DOF-updates of one full step of the whole batch (both half-steps). */
int64_t hermite_batch_dof_per_step(const hermite_batch *b);

/* Time one full step for each candidate (item size in nodes x resident blocks
 * per SM) and keep the fastest; returns the choice and its time.  Advances the
 * loaded state by three full steps per candidate: call it before setting the
 * initial data.  Needs a non-default stream. */
int hermite_batch_autotune(hermite_batch *b, int *item_nodes, int *blocks_per_sm, double *ms_per_step);

/* Set the item size (>= 32 nodes) and resident blocks per SM (1..32) directly. */
int hermite_batch_config(hermite_batch *b, int item_nodes, int blocks_per_sm);

/* Message of the last failed call on this batch (NULL: last failed create). */
const char *hermite_batch_last_error(const hermite_batch *b);

/* Message of the last failed call on this context ("" if none).  With a NULL
 * context: the message of the last failed hermite_create in this thread. */
const char *hermite_last_error(const hermite_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HERMITE_H */
