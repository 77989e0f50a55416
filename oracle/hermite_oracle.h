/*
 * Hermite-method ORACLE: a plain, slow FP64 CPU implementation of the
 * dissipative and conservative Hermite half-steps for u_tt = c^2 Lap u
 * (Appelo, Hagstrom, Vargas, "Hermite Methods for the Scalar Wave Equation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA library: it interpolates by solving the confluent Vandermonde system
 * of Eq. (Hermcon) with partial-pivoting LU for every fibre of every cell, and
 * evolves with the paper's Taylor recursion (Eqs. recursion_diss_1d_1/2,
 * recursion_ut/vt and the special first step of Sec. 3.3) or the conservative
 * cosine series (Eq. update / convUpdate), exactly in the paper's order.
 *
 * Data layout (host, row-major): state[node][coef].
 *   node  : C order over the grid axes (axis 0 slowest).
 *   coef  : C order over the multi-index k = (k_0..k_{d-1}).
 *   u     : k in [0,m]^d,   value h^|k|/k! d^k u   (Sec. 2.2)
 *   v     : k in [0,m-1]^d, value h^|k|/k! d^k v   (Sec. 3.1.1)
 * Grids (Sec. 2.1): periodic -> N nodes per axis on both grids; Dirichlet or
 * Neumann -> primal N+1 nodes (x = i h), dual N nodes (x = (j+1/2) h).
 */
#ifndef HERMITE_ORACLE_H
#define HERMITE_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { OR_DISSIPATIVE = 0, OR_CONSERVATIVE = 1, OR_DISSIPATIVE_SIMPLE = 2 };
enum { OR_PERIODIC = 0, OR_DIRICHLET = 1, OR_NEUMANN = 2 };

typedef struct {
  int d, m, variant, bc;
  int64_t N;
  double c, h, dt;
} or_problem;

/* Nodes per axis of grid g (0 = primal, 1 = dual). */
int64_t or_npts(const or_problem *P, int g);
int64_t or_nnodes(const or_problem *P, int g);

/* 1-D confluent Vandermonde solve of Eq. (Hermcon) for data of degree q:
 * left[0..q] at xi=-1/2, right[0..q] at xi=+1/2 -> a[0..2q+1]. */
int or_interp1d(int q, const double *left, const double *right, double *a);

/* Tensor-product interpolation I_{q_0..q_{d-1}} on one cell (Eq. Hermn2).
 * corner: [2^d][prod(q_i+1)] with corner bit i = 1 meaning xi_i = +1/2
 * (bit of axis 0 is the most significant).  out: prod(2q_i+2) coefficients. */
int or_interp(int d, const int *q, const double *corner, double *out);

/* One cell of the dissipative half-step (Sec. 3.1.2 for d=1, Sec. 3.3 for d>1).
 * cu: [2^d][(m+1)^d], cv: [2^d][m^d] corner data (paper scaling);
 * nu: [(m+1)^d], nv: [m^d] data at the cell centre dt/2 later. */
int or_diss_cell(const or_problem *P, const double *cu, const double *cv,
                 double *nu, double *nv);

/* One cell of the conservative half-step (Eq. update / convUpdate and its
 * d-dimensional form, Sec. 4.3): out = 2*C(I u) - old at the cell centre. */
int or_cons_cell(const or_problem *P, const double *cu, const double *old,
                 double *out);

/* Conservative start-up (level dt/2 from u0, v0): the Taylor series of the
 * exact solution of the cell interpolants I_m u0, I_{m-1} v0 at t = dt/2. */
int or_cons_start_cell(const or_problem *P, const double *cu, const double *cv,
                       double *out);

/* Whole-grid half-step onto grid dst (0 primal, 1 dual).
 * Dissipative: reads src_u/src_v on grid 1-dst, writes dst_u/dst_v.
 * Conservative: reads src_u on grid 1-dst, updates dst_u in place
 * (dst_u holds the level dt earlier on entry); src_v/dst_v unused.
 * Returns 0 or a negative code. */
int or_half_step(const or_problem *P, int dst, const double *src_u,
                 const double *src_v, double *dst_u, double *dst_v);

/* Same, for a list of target nodes only (sampled checks).
 * dst_u/dst_v here are [nt][ncoef] outputs; for the conservative variant
 * old_u gives the earlier level at those targets ([nt][Nu]). */
int or_half_step_sample(const or_problem *P, int dst, const double *src_u,
                        const double *src_v, const int64_t *targets, int64_t nt,
                        const double *old_u, double *dst_u, double *dst_v);

/* Conservative start-up over the whole dual grid. */
int or_cons_start(const or_problem *P, const double *u0, const double *v0,
                  double *dual_u);

/* Dissipative energies of a level held on grid g (Sec. 3.2, Eq. stable1/stable2):
 * out[0] = int v^2 + c^2 |grad u|^2 over the domain,
 * out[1] = c^2 sum_i |d_i I^(i) u|^2_{m..m} + |I_{m-1} v|^2_{m..m}. */
int or_diss_energy(const or_problem *P, int g, const double *u,
                   const double *v, double out[2]);

/* Conservative quadratic forms on grid g:
 * out[0] = <p_a, p_b>_{m+1,..,m+1}, out[1] = c^2 int grad p_a . grad p_b. */
int or_cons_forms(const or_problem *P, int g, const double *ua,
                  const double *ub, double out[2]);

/* L2 error of the I_m interpolant of grid-g u data against an exact function
 * sampled at Gauss-Legendre points: the caller passes the point values
 * exact[cell][npts^d] for the points returned by or_gauss_points. */
int or_gauss_points(int n, double *x, double *w);
int or_l2_error(const or_problem *P, int g, const double *u, int nq,
                const double *exact, double *err2);

#ifdef __cplusplus
}
#endif
#endif
