/*
 * Hermite-method ORACLE (test infrastructure only; see hermite_oracle.h).
 *
 * Plain FP64 loops written from the paper's text, in the paper's order:
 *   interpolation   Sec. 2.2, Eqs. (Hermn), (Hermcon), (Hermn2), (Hermcon2)
 *   dissipative     Sec. 3.1.2 (recursions recursion_diss_1d_1/2, truncation
 *                   kappa_u/kappa_v, evaluation Taylorsum1/2) and Sec. 3.3
 *                   (recursion_ut/vt with the special first step)
 *   boundaries      Sec. 3.1.3 (odd/even ghost polynomials)
 *   conservative    Sec. 4, Eq. (update) / (convUpdate) and Sec. 4.3
 *   energies        Sec. 3.2 (stable1, Energyeq), Sec. 3.3 (stable2), Sec. 4.2
 * Readings where the paper is silent or inconsistent are stated inline.
 */
#include "hermite_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 3
#define OR_EARG (-1)
#define OR_EALLOC (-2)
#define OR_ESING (-3)

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

static int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

/* C-order strides of a box with extents e[0..d-1]. */
static int64_t box_strides(int d, const int *e, int64_t *st) {
  int64_t s = 1;
  for (int i = d - 1; i >= 0; --i) {
    st[i] = s;
    s *= e[i];
  }
  return s;
}

static void box_unravel(int d, const int *e, int64_t idx, int *a) {
  for (int i = d - 1; i >= 0; --i) {
    a[i] = (int)(idx % e[i]);
    idx /= e[i];
  }
}

/* ------------------------------------------------------------------------- */
/* Grids (Sec. 2.1).                                                          */
int64_t or_npts(const or_problem *P, int g) {
  if (P->bc == OR_PERIODIC) return P->N;
  return g == 0 ? P->N + 1 : P->N;
}

int64_t or_nnodes(const or_problem *P, int g) {
  int64_t n = 1;
  for (int i = 0; i < P->d; ++i) n *= or_npts(P, g);
  return n;
}

static int check_problem(const or_problem *P) {
  if (!P || P->d < 1 || P->d > OR_MAXD || P->N < 1) return OR_EARG;
  if (P->variant == OR_CONSERVATIVE) {
    if (P->m < 0) return OR_EARG;
  } else if (P->m < 1) {
    return OR_EARG;
  }
  if (P->bc != OR_PERIODIC && P->bc != OR_DIRICHLET && P->bc != OR_NEUMANN)
    return OR_EARG;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. (Hermcon) in the scaled variable xi = (x - x_centre)/h: the degree-
 * (2q+1) polynomial sum_j a_j xi^j must satisfy (1/l!) d^l p/dxi^l = c_l at
 * xi = -1/2 (rows 0..q) and xi = +1/2 (rows q+1..2q+1).  Row (s,l), column j:
 * binom(j,l) xi_s^(j-l). */
static void hermite_system(int q, double *A) {
  int n = 2 * q + 2;
  for (int s = 0; s < 2; ++s) {
    double xi = s == 0 ? -0.5 : 0.5;
    for (int l = 0; l <= q; ++l) {
      int row = s * (q + 1) + l;
      for (int j = 0; j < n; ++j)
        A[row * n + j] = j < l ? 0.0 : binom(j, l) * pow(xi, (double)(j - l));
    }
  }
}

/* LU factorisation with partial pivoting, in place (row-major n x n). */
static int lu_factor(int n, double *A, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) {
        best = fabs(A[i * n + k]);
        p = i;
      }
    if (best == 0.0) return OR_ESING;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      A[i * n + k] = f;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
    }
  }
  return 0;
}

static void lu_solve(int n, const double *LU, const int *piv, double *b) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) {
      double t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
  }
  for (int i = 1; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
    b[i] /= LU[i * n + i];
  }
}

int or_interp1d(int q, const double *left, const double *right, double *a) {
  if (q < 0 || q > 30) return OR_EARG;
  int n = 2 * q + 2;
  double *A = (double *)malloc(sizeof(double) * n * n);
  int *piv = (int *)malloc(sizeof(int) * n);
  if (!A || !piv) {
    free(A);
    free(piv);
    return OR_EALLOC;
  }
  hermite_system(q, A);
  int rc = lu_factor(n, A, piv);
  if (rc == 0) {
    for (int l = 0; l <= q; ++l) {
      a[l] = left[l];
      a[q + 1 + l] = right[l];
    }
    lu_solve(n, A, piv, a);
  }
  free(A);
  free(piv);
  return rc;
}

/* Tensor-product interpolation, Eq. (Hermn2)/(Hermcon2) with degrees q_i:
 * solve the 1-D system of Eq. (Hermcon) along every fibre, axis by axis. */
int or_interp(int d, const int *q, const double *corner, double *out) {
  if (d < 1 || d > OR_MAXD) return OR_EARG;
  int e[OR_MAXD], eb[OR_MAXD];
  int64_t st[OR_MAXD], stb[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    if (q[i] < 0) return OR_EARG;
    e[i] = 2 * q[i] + 2;
    eb[i] = q[i] + 1;
  }
  int64_t size = box_strides(d, e, st);
  int64_t nb = box_strides(d, eb, stb);
  int nc = 1 << d;
  /* Place corner data: along axis i the index is bit_i*(q_i+1) + beta_i, which
   * is the row order of the Eq. (Hermcon) system. */
  for (int s = 0; s < nc; ++s) {
    for (int64_t b = 0; b < nb; ++b) {
      int beta[OR_MAXD];
      box_unravel(d, eb, b, beta);
      int64_t pos = 0;
      for (int i = 0; i < d; ++i) {
        int bit = (s >> (d - 1 - i)) & 1;
        pos += (int64_t)(bit * (q[i] + 1) + beta[i]) * st[i];
      }
      out[pos] = corner[s * nb + b];
    }
  }
  for (int ax = 0; ax < d; ++ax) {
    int n = e[ax];
    double *A = (double *)malloc(sizeof(double) * n * n);
    int *piv = (int *)malloc(sizeof(int) * n);
    double *rhs = (double *)malloc(sizeof(double) * n);
    if (!A || !piv || !rhs) {
      free(A);
      free(piv);
      free(rhs);
      return OR_EALLOC;
    }
    hermite_system(q[ax], A);
    int rc = lu_factor(n, A, piv);
    if (rc) {
      free(A);
      free(piv);
      free(rhs);
      return rc;
    }
    for (int64_t f = 0; f < size; ++f) {
      int a[OR_MAXD];
      box_unravel(d, e, f, a);
      if (a[ax] != 0) continue; /* one visit per fibre */
      for (int j = 0; j < n; ++j) rhs[j] = out[f + j * st[ax]];
      lu_solve(n, A, piv, rhs);
      for (int j = 0; j < n; ++j) out[f + j * st[ax]] = rhs[j];
    }
    free(A);
    free(piv);
    free(rhs);
  }
  return 0;
}

/* Copy a box with extents es into a (larger or equal) box with extents ed,
 * zero elsewhere. */
static void box_embed(int d, const int *es, const double *src, const int *ed,
                      double *dst) {
  int64_t sts[OR_MAXD], std_[OR_MAXD];
  int64_t ns = box_strides(d, es, sts);
  int64_t nd = box_strides(d, ed, std_);
  memset(dst, 0, sizeof(double) * nd);
  for (int64_t k = 0; k < ns; ++k) {
    int a[OR_MAXD];
    box_unravel(d, es, k, a);
    int64_t p = 0;
    for (int i = 0; i < d; ++i) p += (int64_t)a[i] * std_[i];
    dst[p] = src[k];
  }
}

/* Corner data of degree q (all axes) restricted to degrees qr_i <= q. */
static void restrict_corner(int d, int q, const int *qr, const double *cu,
                            double *out) {
  int e[OR_MAXD], er[OR_MAXD];
  int64_t st[OR_MAXD], str[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    e[i] = q + 1;
    er[i] = qr[i] + 1;
  }
  int64_t n = box_strides(d, e, st);
  int64_t nr = box_strides(d, er, str);
  for (int s = 0; s < (1 << d); ++s)
    for (int64_t k = 0; k < nr; ++k) {
      int a[OR_MAXD];
      box_unravel(d, er, k, a);
      int64_t p = 0;
      for (int i = 0; i < d; ++i) p += (int64_t)a[i] * st[i];
      out[s * nr + k] = cu[s * n + p];
    }
}

/* ------------------------------------------------------------------------- */
/* Dissipative half-step on one cell.                                         */

/* d = 1: Sec. 3.1.2 verbatim.  c_{l,s} = dt/s d_{l,s-1},
 * d_{l,s} = c^2 (l+2)(l+1)/s dt/h^2 c_{l+2,s-1}, truncated at
 * kappa_v(l) = 2m-1-2 floor(l/2), kappa_u = kappa_v + 1, then the Taylor
 * series in (t - t0)/dt is summed at 1/2 (Eqs. Taylorsum1/2). */
static int diss_cell_1d(const or_problem *P, const double *cu, const double *cv,
                        double *nu, double *nv) {
  int m = P->m;
  int nu_c = 2 * m + 2, nv_c = 2 * m, S = 2 * m + 2;
  double *c = (double *)calloc((size_t)nu_c * (S + 1), sizeof(double));
  double *dd = (double *)calloc((size_t)nu_c * (S + 1), sizeof(double));
  double a[64], b[64];
  if (!c || !dd || m > 30) {
    free(c);
    free(dd);
    return OR_EALLOC;
  }
  int rc = or_interp1d(m, cu, cu + (m + 1), a);
  if (!rc) rc = or_interp1d(m - 1, cv, cv + m, b);
  if (rc) {
    free(c);
    free(dd);
    return rc;
  }
#define C(l, s) c[(l) * (S + 1) + (s)]
#define D(l, s) dd[(l) * (S + 1) + (s)]
  for (int l = 0; l < nu_c; ++l) C(l, 0) = a[l];
  for (int l = 0; l < nv_c; ++l) D(l, 0) = b[l];
  double k2 = P->c * P->c * P->dt / (P->h * P->h);
  for (int s = 1; s <= S; ++s) {
    for (int l = 0; l < nu_c; ++l) {
      int kv = 2 * m - 1 - 2 * (l / 2);
      int ku = kv + 1;
      if (s <= ku) C(l, s) = P->dt / s * D(l, s - 1);
      if (l < nv_c && s <= kv)
        D(l, s) = k2 * (double)((l + 2) * (l + 1)) / s * C(l + 2, s - 1);
    }
  }
  for (int l = 0; l <= m; ++l) {
    int ku = 2 * m - 2 * (l / 2);
    double acc = 0.0, w = 1.0;
    for (int s = 0; s <= ku; ++s, w *= 0.5) acc += C(l, s) * w;
    nu[l] = acc;
  }
  for (int l = 0; l < m; ++l) {
    int kv = 2 * m - 1 - 2 * (l / 2);
    double acc = 0.0, w = 1.0;
    for (int s = 0; s <= kv; ++s, w *= 0.5) acc += D(l, s) * w;
    nv[l] = acc;
  }
#undef C
#undef D
  free(c);
  free(dd);
  return 0;
}

/* d > 1: Sec. 3.3.  c_{a,0} from I_{m..m} u, d_{a,0} from I_{m-1..m-1} v.
 * First step: "full" variant uses the special interpolants, i.e.
 * d_{a,1} = c^2 sum_i (a_i+2)(a_i+1) dt/h^2 c^(i)_{a+2e_i} with c^(i) the
 * coefficients of I with degree m in axis i and m-1 in the others (the 3-D
 * form with five interpolants is the direct extension of the printed 2-D
 * one); the "simple" variant uses the plain recursion from s = 1.  Later
 * steps: Eqs. (recursion_ut), (recursion_vt) on the (2m+2)^d box, run until
 * s = d(2m+1)+2, past which every coefficient vanishes. */
static int diss_cell_nd(const or_problem *P, const double *cu, const double *cv,
                        double *nu, double *nv) {
  int d = P->d, m = P->m;
  int E[OR_MAXD], Ev[OR_MAXD], qu[OR_MAXD], qv[OR_MAXD];
  int64_t st[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    E[i] = 2 * m + 2;
    Ev[i] = 2 * m;
    qu[i] = m;
    qv[i] = m - 1;
  }
  int64_t B = box_strides(d, E, st);
  int64_t Bv = 1;
  for (int i = 0; i < d; ++i) Bv *= Ev[i];
  int S = d * (2 * m + 1) + 2;
  double *buf = (double *)calloc((size_t)B * 8 + (size_t)Bv * 2, sizeof(double));
  double *corner_r = (double *)calloc((size_t)(1 << d) * B, sizeof(double));
  if (!buf || !corner_r) {
    free(buf);
    free(corner_r);
    return OR_EALLOC;
  }
  double *cprev = buf, *dprev = buf + B, *ccur = buf + 2 * B, *dcur = buf + 3 * B;
  double *uacc = buf + 4 * B, *vacc = buf + 5 * B, *tmp = buf + 6 * B;
  double *vsmall = buf + 8 * B;
  int rc = or_interp(d, qu, cu, cprev);
  if (!rc) rc = or_interp(d, qv, cv, vsmall);
  if (rc) goto done;
  box_embed(d, Ev, vsmall, E, dprev);
  memcpy(uacc, cprev, sizeof(double) * B);
  memcpy(vacc, dprev, sizeof(double) * B);
  double k2 = P->c * P->c * P->dt / (P->h * P->h);
  double w = 1.0;
  for (int s = 1; s <= S; ++s) {
    w *= 0.5;
    if (s == 1 && P->variant == OR_DISSIPATIVE) {
      /* special first step */
      memset(ccur, 0, sizeof(double) * B);
      memset(dcur, 0, sizeof(double) * B);
      for (int64_t k = 0; k < B; ++k) {
        int a[OR_MAXD];
        box_unravel(d, E, k, a);
        int inside = 1;
        for (int i = 0; i < d; ++i) inside &= a[i] <= 2 * m - 1;
        if (inside) ccur[k] = P->dt * dprev[k];
      }
      for (int ax = 0; ax < d; ++ax) {
        int qi[OR_MAXD], Ei[OR_MAXD];
        int64_t sti[OR_MAXD];
        for (int i = 0; i < d; ++i) {
          qi[i] = i == ax ? m : m - 1;
          Ei[i] = 2 * qi[i] + 2;
        }
        box_strides(d, Ei, sti);
        restrict_corner(d, m, qi, cu, corner_r);
        rc = or_interp(d, qi, corner_r, tmp);
        if (rc) goto done;
        for (int64_t k = 0; k < B; ++k) {
          int a[OR_MAXD];
          box_unravel(d, E, k, a);
          int inside = 1;
          for (int i = 0; i < d; ++i) inside &= a[i] <= 2 * m - 1;
          if (!inside) continue;
          int64_t p = 0;
          for (int i = 0; i < d; ++i) p += (int64_t)(a[i] + (i == ax ? 2 : 0)) * sti[i];
          dcur[k] += k2 * (double)((a[ax] + 2) * (a[ax] + 1)) * tmp[p];
        }
      }
    } else {
      for (int64_t k = 0; k < B; ++k) {
        int a[OR_MAXD];
        box_unravel(d, E, k, a);
        ccur[k] = P->dt / s * dprev[k];
        double acc = 0.0;
        for (int i = 0; i < d; ++i)
          if (a[i] + 2 < E[i])
            acc += (double)((a[i] + 2) * (a[i] + 1)) * cprev[k + 2 * st[i]];
        dcur[k] = k2 / s * acc;
      }
    }
    for (int64_t k = 0; k < B; ++k) {
      uacc[k] += ccur[k] * w;
      vacc[k] += dcur[k] * w;
    }
    double *t1 = cprev;
    cprev = ccur;
    ccur = t1;
    t1 = dprev;
    dprev = dcur;
    dcur = t1;
  }
  /* evaluation at the cell centre: keep degrees <= m (u), <= m-1 (v) */
  {
    int eu[OR_MAXD], ev[OR_MAXD];
    for (int i = 0; i < d; ++i) {
      eu[i] = m + 1;
      ev[i] = m;
    }
    int64_t su[OR_MAXD], sv[OR_MAXD];
    int64_t nuc = box_strides(d, eu, su), nvc = box_strides(d, ev, sv);
    for (int64_t k = 0; k < nuc; ++k) {
      int a[OR_MAXD];
      box_unravel(d, eu, k, a);
      int64_t p = 0;
      for (int i = 0; i < d; ++i) p += (int64_t)a[i] * st[i];
      nu[k] = uacc[p];
    }
    for (int64_t k = 0; k < nvc; ++k) {
      int a[OR_MAXD];
      box_unravel(d, ev, k, a);
      int64_t p = 0;
      for (int i = 0; i < d; ++i) p += (int64_t)a[i] * st[i];
      nv[k] = vacc[p];
    }
  }
done:
  free(buf);
  free(corner_r);
  return rc;
}

int or_diss_cell(const or_problem *P, const double *cu, const double *cv,
                 double *nu, double *nv) {
  int rc = check_problem(P);
  if (rc) return rc;
  if (P->variant == OR_CONSERVATIVE) return OR_EARG;
  if (P->d == 1) return diss_cell_1d(P, cu, cv, nu, nv);
  return diss_cell_nd(P, cu, cv, nu, nv);
}

/* ------------------------------------------------------------------------- */
/* Conservative half-step on one cell.                                        */

/* Laplacian of a polynomial in xi = (x - X)/h held as a coefficient box:
 * (Lap f)_a = h^-2 sum_i (a_i+2)(a_i+1) f_{a+2e_i}. */
static void laplacian(int d, const int *E, const int64_t *st, int64_t B,
                      double h, const double *f, double *out) {
  for (int64_t k = 0; k < B; ++k) {
    int a[OR_MAXD];
    box_unravel(d, E, k, a);
    double acc = 0.0;
    for (int i = 0; i < d; ++i)
      if (a[i] + 2 < E[i]) acc += (double)((a[i] + 2) * (a[i] + 1)) * f[k + 2 * st[i]];
    out[k] = acc / (h * h);
  }
}

/* Eq. (update): u(t+dt/2) + u(t-dt/2) = 2 sum_l (c dt/2)^{2l}/(2l)! Lap^l u(t),
 * applied to the cell interpolant centred at the target node; the scaled
 * derivatives at the node are the coefficients of the resulting polynomial.
 * Reading: "(2l!)" of Eq. (update) is (2l)!; the d-dimensional weights are
 * these Taylor weights (c dt/(2h))^{2r}, so the printed Pascal-matrix form of
 * Sec. 4.3 is read with the factor 2^{-2r} that its 1-D form carries. */
int or_cons_cell(const or_problem *P, const double *cu, const double *old,
                 double *out) {
  int rc = check_problem(P);
  if (rc) return rc;
  int d = P->d, m = P->m;
  int E[OR_MAXD], q[OR_MAXD], eo[OR_MAXD];
  int64_t st[OR_MAXD], so[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    E[i] = 2 * m + 2;
    q[i] = m;
    eo[i] = m + 1;
  }
  int64_t B = box_strides(d, E, st);
  int64_t no = box_strides(d, eo, so);
  double *a = (double *)calloc((size_t)B * 4, sizeof(double));
  if (!a) return OR_EALLOC;
  double *term = a + B, *W = a + 2 * B, *t2 = a + 3 * B;
  rc = or_interp(d, q, cu, a);
  if (rc) {
    free(a);
    return rc;
  }
  memcpy(term, a, sizeof(double) * B);
  memcpy(W, a, sizeof(double) * B);
  double half = 0.5 * P->c * P->dt;
  int R = (d * (2 * m + 1)) / 2 + 1;
  for (int r = 1; r <= R; ++r) {
    laplacian(d, E, st, B, P->h, term, t2);
    memcpy(term, t2, sizeof(double) * B);
    double wr = pow(half, 2.0 * r) / fact(2 * r);
    for (int64_t k = 0; k < B; ++k) W[k] += wr * term[k];
  }
  for (int64_t k = 0; k < no; ++k) {
    int al[OR_MAXD];
    box_unravel(d, eo, k, al);
    int64_t p = 0;
    for (int i = 0; i < d; ++i) p += (int64_t)al[i] * st[i];
    out[k] = 2.0 * W[p] - old[k];
  }
  free(a);
  return 0;
}

/* Start-up of the conservative scheme (the paper only asks for accurate
 * initial data at the second level).  Reading: the exact Taylor series in
 * time of the cell interpolants at t = dt/2,
 *   sum_r tau^{2r} c^{2r}/(2r)! Lap^r I_m u0 + tau^{2r+1} c^{2r}/(2r+1)! Lap^r I_{m-1} v0,
 * tau = dt/2, evaluated at the dual node. */
int or_cons_start_cell(const or_problem *P, const double *cu, const double *cv,
                       double *out) {
  int rc = check_problem(P);
  if (rc) return rc;
  int d = P->d, m = P->m;
  int E[OR_MAXD], Ev[OR_MAXD], q[OR_MAXD], qv[OR_MAXD], eo[OR_MAXD];
  int64_t st[OR_MAXD], so[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    E[i] = 2 * m + 2;
    Ev[i] = 2 * m;
    q[i] = m;
    qv[i] = m - 1;
    eo[i] = m + 1;
  }
  int64_t B = box_strides(d, E, st);
  int64_t no = box_strides(d, eo, so);
  double *a = (double *)calloc((size_t)B * 6, sizeof(double));
  if (!a) return OR_EALLOC;
  double *b = a + B, *ta = a + 2 * B, *tb = a + 3 * B, *W = a + 4 * B, *t2 = a + 5 * B;
  rc = or_interp(d, q, cu, a);
  if (!rc && m >= 1 && cv) {
    double *vs = (double *)calloc((size_t)B, sizeof(double));
    if (!vs) {
      free(a);
      return OR_EALLOC;
    }
    rc = or_interp(d, qv, cv, vs);
    if (!rc) box_embed(d, Ev, vs, E, b);
    free(vs);
  }
  if (rc) {
    free(a);
    return rc;
  }
  double tau = 0.5 * P->dt;
  memcpy(ta, a, sizeof(double) * B);
  memcpy(tb, b, sizeof(double) * B);
  for (int64_t k = 0; k < B; ++k) W[k] = a[k] + tau * b[k];
  int R = (d * (2 * m + 1)) / 2 + 1;
  for (int r = 1; r <= R; ++r) {
    laplacian(d, E, st, B, P->h, ta, t2);
    memcpy(ta, t2, sizeof(double) * B);
    laplacian(d, E, st, B, P->h, tb, t2);
    memcpy(tb, t2, sizeof(double) * B);
    double c2r = pow(P->c, 2.0 * r);
    double wa = pow(tau, 2.0 * r) * c2r / fact(2 * r);
    double wb = pow(tau, 2.0 * r + 1) * c2r / fact(2 * r + 1);
    for (int64_t k = 0; k < B; ++k) W[k] += wa * ta[k] + wb * tb[k];
  }
  for (int64_t k = 0; k < no; ++k) {
    int al[OR_MAXD];
    box_unravel(d, eo, k, al);
    int64_t p = 0;
    for (int i = 0; i < d; ++i) p += (int64_t)al[i] * st[i];
    out[k] = W[p];
  }
  free(a);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Grid gather with ghost polynomials (Sec. 3.1.3).                           */

/* Corner sigma of the cell centred at target node t of grid dst: along each
 * axis, dst dual -> source primal indices t and t+1; dst primal -> source
 * dual indices t-1 and t.  Periodic: wrap.  Otherwise a source dual index -1
 * or N is a ghost: the mirror image of dual node 0 or N-1 (reflection about
 * the boundary).  Reading (the worked example of Sec. 5.1 uses an even
 * extension on the left and an odd one on the right for the same Dirichlet
 * problem): Dirichlet ghosts are odd extensions at both ends,
 * ghost_k = (-1)^{k_i+1} mirror_k; Neumann ghosts are even, (-1)^{k_i}
 * mirror_k; a corner ghosted in several axes takes the product. */
static void gather(const or_problem *P, int dst, const int *t, const double *src,
                   int q, double *corner) {
  int d = P->d;
  int64_t ns = or_npts(P, 1 - dst);
  int eb[OR_MAXD];
  int64_t stb[OR_MAXD];
  for (int i = 0; i < d; ++i) eb[i] = q + 1;
  int64_t nb = box_strides(d, eb, stb);
  for (int s = 0; s < (1 << d); ++s) {
    int64_t node = 0;
    int ghost[OR_MAXD];
    for (int i = 0; i < d; ++i) {
      int bit = (s >> (d - 1 - i)) & 1;
      int64_t si = dst == 1 ? (int64_t)t[i] + bit : (int64_t)t[i] - 1 + bit;
      ghost[i] = 0;
      if (P->bc == OR_PERIODIC) {
        si = ((si % ns) + ns) % ns;
      } else if (si < 0) {
        si = 0;
        ghost[i] = 1;
      } else if (si >= ns) {
        si = ns - 1;
        ghost[i] = 1;
      }
      node = node * ns + si;
    }
    for (int64_t k = 0; k < nb; ++k) {
      int kk[OR_MAXD];
      box_unravel(d, eb, k, kk);
      double sign = 1.0;
      for (int i = 0; i < d; ++i)
        if (ghost[i]) {
          double odd = (kk[i] & 1) ? -1.0 : 1.0;
          sign *= P->bc == OR_DIRICHLET ? -odd : odd;
        }
      corner[s * nb + k] = sign * src[node * nb + k];
    }
  }
}

static int ncoef_box(int d, int q) { return q < 0 ? 0 : ipow(q + 1, d); }

static int half_step_impl(const or_problem *P, int dst, const double *src_u,
                          const double *src_v, const int64_t *targets,
                          int64_t nt, const double *old_u, double *out_u,
                          double *out_v, int inplace) {
  int rc = check_problem(P);
  if (rc) return rc;
  if (dst != 0 && dst != 1) return OR_EARG;
  int d = P->d, m = P->m;
  int Nu = ncoef_box(d, m), Nv = ncoef_box(d, m - 1);
  int nc = 1 << d;
  double *cu = (double *)malloc(sizeof(double) * (nc * (Nu + Nv) + 2 * Nu + 1));
  if (!cu) return OR_EALLOC;
  double *cv = cu + nc * Nu;
  double *tmp = cv + nc * Nv;
  int64_t nd = or_npts(P, dst);
  int64_t total = targets ? nt : or_nnodes(P, dst);
  for (int64_t it = 0; it < total && !rc; ++it) {
    int64_t node = targets ? targets[it] : it;
    int t[OR_MAXD];
    int64_t r = node;
    for (int i = d - 1; i >= 0; --i) {
      t[i] = (int)(r % nd);
      r /= nd;
    }
    gather(P, dst, t, src_u, m, cu);
    int64_t ou = inplace ? node : it;
    if (P->variant == OR_CONSERVATIVE) {
      const double *old = inplace ? out_u + node * Nu : old_u + it * Nu;
      rc = or_cons_cell(P, cu, old, tmp);
      memcpy(out_u + ou * Nu, tmp, sizeof(double) * Nu);
    } else {
      gather(P, dst, t, src_v, m - 1, cv);
      rc = or_diss_cell(P, cu, cv, out_u + ou * Nu, out_v + ou * Nv);
    }
  }
  free(cu);
  return rc;
}

int or_half_step(const or_problem *P, int dst, const double *src_u,
                 const double *src_v, double *dst_u, double *dst_v) {
  return half_step_impl(P, dst, src_u, src_v, NULL, 0, NULL, dst_u, dst_v, 1);
}

int or_half_step_sample(const or_problem *P, int dst, const double *src_u,
                        const double *src_v, const int64_t *targets, int64_t nt,
                        const double *old_u, double *dst_u, double *dst_v) {
  if (!targets || nt < 0) return OR_EARG;
  if (P->variant == OR_CONSERVATIVE && !old_u) return OR_EARG;
  return half_step_impl(P, dst, src_u, src_v, targets, nt, old_u, dst_u, dst_v, 0);
}

int or_cons_start(const or_problem *P, const double *u0, const double *v0,
                  double *dual_u) {
  int rc = check_problem(P);
  if (rc) return rc;
  int d = P->d, m = P->m;
  int Nu = ncoef_box(d, m), Nv = ncoef_box(d, m - 1);
  int nc = 1 << d;
  double *cu = (double *)malloc(sizeof(double) * (nc * (Nu + Nv) + 1));
  if (!cu) return OR_EALLOC;
  double *cv = cu + nc * Nu;
  int64_t nd = or_npts(P, 1), total = or_nnodes(P, 1);
  for (int64_t node = 0; node < total && !rc; ++node) {
    int t[OR_MAXD];
    int64_t r = node;
    for (int i = d - 1; i >= 0; --i) {
      t[i] = (int)(r % nd);
      r /= nd;
    }
    gather(P, 1, t, u0, m, cu);
    if (v0 && m >= 1) gather(P, 1, t, v0, m - 1, cv);
    rc = or_cons_start_cell(P, cu, (v0 && m >= 1) ? cv : NULL, dual_u + node * Nu);
  }
  free(cu);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Quadratic forms by exact integration of polynomial products over the cell */
/* [-1/2,1/2]^d in xi; d/dx = h^-1 d/dxi, dx = h^d dxi.                        */

static double moment(int n) { return (n & 1) ? 0.0 : pow(0.5, (double)n) / (n + 1); }

static double integrate_product(int d, const int *E, const double *f,
                                const double *g) {
  int64_t st[OR_MAXD];
  int64_t B = box_strides(d, E, st);
  double acc = 0.0;
  for (int64_t i = 0; i < B; ++i) {
    if (f[i] == 0.0) continue;
    int a[OR_MAXD];
    box_unravel(d, E, i, a);
    for (int64_t j = 0; j < B; ++j) {
      int b[OR_MAXD];
      box_unravel(d, E, j, b);
      double w = 1.0;
      for (int k = 0; k < d && w != 0.0; ++k) w *= moment(a[k] + b[k]);
      acc += f[i] * g[j] * w;
    }
  }
  return acc;
}

/* out = d^ord/dxi_ax^ord f (same box). */
static void deriv(int d, const int *E, const double *f, int ax, int ord,
                  double *out) {
  int64_t st[OR_MAXD];
  int64_t B = box_strides(d, E, st);
  for (int64_t k = 0; k < B; ++k) {
    int a[OR_MAXD];
    box_unravel(d, E, k, a);
    if (a[ax] + ord >= E[ax]) {
      out[k] = 0.0;
      continue;
    }
    double fct = 1.0;
    for (int j = 1; j <= ord; ++j) fct *= (double)(a[ax] + j);
    out[k] = fct * f[k + ord * st[ax]];
  }
}

/* Cells of a level held on grid g are centred at the nodes of grid 1-g; the
 * corners come from the same gather as a half-step (ghosts included).  For
 * non-periodic problems a cell centred on a boundary primal node straddles
 * the boundary and only its inner half lies in the domain: by the odd/even
 * symmetry of the ghost it contributes half its integral per such axis. */
static double cell_weight(const or_problem *P, int g, const int *t) {
  if (P->bc == OR_PERIODIC || g == 0) return 1.0;
  double w = 1.0;
  for (int i = 0; i < P->d; ++i)
    if (t[i] == 0 || t[i] == P->N) w *= 0.5;
  return w;
}

int or_diss_energy(const or_problem *P, int g, const double *u, const double *v,
                   double out[2]) {
  int rc = check_problem(P);
  if (rc) return rc;
  if (P->variant == OR_CONSERVATIVE) return OR_EARG;
  int d = P->d, m = P->m;
  int Nu = ncoef_box(d, m), Nv = ncoef_box(d, m - 1), nc = 1 << d;
  int E[OR_MAXD], Ev[OR_MAXD], q[OR_MAXD], qv[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    E[i] = 2 * m + 2;
    Ev[i] = 2 * m;
    q[i] = m;
    qv[i] = m - 1;
  }
  int64_t st[OR_MAXD];
  int64_t B = box_strides(d, E, st);
  double *cu = (double *)malloc(sizeof(double) * nc * (Nu + Nv));
  double *w = (double *)calloc((size_t)B * 6 + (size_t)nc * B, sizeof(double));
  if (!cu || !w) {
    free(cu);
    free(w);
    return OR_EALLOC;
  }
  double *cv = cu + nc * Nu;
  double *a = w, *b = w + B, *t1 = w + 2 * B, *t2 = w + 3 * B, *ai = w + 4 * B,
         *bs = w + 5 * B, *cr = w + 6 * B;
  int64_t nt = or_npts(P, 1 - g), total = or_nnodes(P, 1 - g);
  double hd = pow(P->h, (double)d), c2 = P->c * P->c;
  double plain = 0.0, inv = 0.0;
  for (int64_t node = 0; node < total && !rc; ++node) {
    int t[OR_MAXD];
    int64_t r = node;
    for (int i = d - 1; i >= 0; --i) {
      t[i] = (int)(r % nt);
      r /= nt;
    }
    double wc = cell_weight(P, g, t);
    gather(P, 1 - g, t, u, m, cu);
    gather(P, 1 - g, t, v, m - 1, cv);
    rc = or_interp(d, q, cu, a);
    if (!rc) rc = or_interp(d, qv, cv, bs);
    if (rc) break;
    box_embed(d, Ev, bs, E, b);
    /* plain energy: int v^2 + c^2 |grad u|^2 */
    double e = integrate_product(d, E, b, b);
    for (int i = 0; i < d; ++i) {
      deriv(d, E, a, i, 1, t1);
      e += c2 / (P->h * P->h) * integrate_product(d, E, t1, t1);
    }
    plain += wc * hd * e;
    /* invariant: c^2 sum_i |d_i I^(i) u|^2_{m..m} + |I_{m-1} v|^2_{m..m} */
    double ei = 0.0;
    for (int ax = 0; ax < d; ++ax) {
      int qi[OR_MAXD], Ei[OR_MAXD];
      for (int i = 0; i < d; ++i) {
        qi[i] = (d == 1 || i == ax) ? m : m - 1;
        Ei[i] = 2 * qi[i] + 2;
      }
      restrict_corner(d, m, qi, cu, cr);
      rc = or_interp(d, qi, cr, t2);
      if (rc) break;
      box_embed(d, Ei, t2, E, ai);
      memcpy(t1, ai, sizeof(double) * B);
      for (int i = 0; i < d; ++i) {
        deriv(d, E, t1, i, m + (i == ax ? 1 : 0), t2);
        memcpy(t1, t2, sizeof(double) * B);
      }
      ei += c2 * pow(P->h, -2.0 * (d * m + 1)) * integrate_product(d, E, t1, t1);
    }
    memcpy(t1, b, sizeof(double) * B);
    for (int i = 0; i < d; ++i) {
      deriv(d, E, t1, i, m, t2);
      memcpy(t1, t2, sizeof(double) * B);
    }
    ei += pow(P->h, -2.0 * d * m) * integrate_product(d, E, t1, t1);
    inv += wc * hd * ei;
  }
  out[0] = plain;
  out[1] = inv;
  free(cu);
  free(w);
  return rc;
}

int or_cons_forms(const or_problem *P, int g, const double *ua, const double *ub,
                  double out[2]) {
  int rc = check_problem(P);
  if (rc) return rc;
  int d = P->d, m = P->m;
  int Nu = ncoef_box(d, m), nc = 1 << d;
  int E[OR_MAXD], q[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    E[i] = 2 * m + 2;
    q[i] = m;
  }
  int64_t st[OR_MAXD];
  int64_t B = box_strides(d, E, st);
  double *ca = (double *)malloc(sizeof(double) * nc * Nu * 2);
  double *w = (double *)calloc((size_t)B * 6, sizeof(double));
  if (!ca || !w) {
    free(ca);
    free(w);
    return OR_EALLOC;
  }
  double *cb = ca + nc * Nu;
  double *pa = w, *pb = w + B, *ta = w + 2 * B, *tb = w + 3 * B, *t2 = w + 4 * B;
  int64_t nt = or_npts(P, 1 - g), total = or_nnodes(P, 1 - g);
  double hd = pow(P->h, (double)d), c2 = P->c * P->c;
  double semi = 0.0, grad = 0.0;
  for (int64_t node = 0; node < total && !rc; ++node) {
    int t[OR_MAXD];
    int64_t r = node;
    for (int i = d - 1; i >= 0; --i) {
      t[i] = (int)(r % nt);
      r /= nt;
    }
    double wc = cell_weight(P, g, t);
    gather(P, 1 - g, t, ua, m, ca);
    gather(P, 1 - g, t, ub, m, cb);
    rc = or_interp(d, q, ca, pa);
    if (!rc) rc = or_interp(d, q, cb, pb);
    if (rc) break;
    memcpy(ta, pa, sizeof(double) * B);
    memcpy(tb, pb, sizeof(double) * B);
    for (int i = 0; i < d; ++i) {
      deriv(d, E, ta, i, m + 1, t2);
      memcpy(ta, t2, sizeof(double) * B);
      deriv(d, E, tb, i, m + 1, t2);
      memcpy(tb, t2, sizeof(double) * B);
    }
    semi += wc * hd * pow(P->h, -2.0 * d * (m + 1)) * integrate_product(d, E, ta, tb);
    double gsum = 0.0;
    for (int i = 0; i < d; ++i) {
      deriv(d, E, pa, i, 1, ta);
      deriv(d, E, pb, i, 1, tb);
      gsum += integrate_product(d, E, ta, tb);
    }
    grad += wc * hd * c2 / (P->h * P->h) * gsum;
  }
  out[0] = semi;
  out[1] = grad;
  free(ca);
  free(w);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre points on [-1/2,1/2] (Newton on P_n), weights summing to 1. */
int or_gauss_points(int n, double *x, double *w) {
  if (n < 1 || n > 64) return OR_EARG;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), p0 = 1.0, p1 = z, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      p0 = 1.0;
      p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    p0 = 1.0;
    p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = 0.5 * z;
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp); /* 2/(..) on [-1,1], /2 */
  }
  return 0;
}

int or_l2_error(const or_problem *P, int g, const double *u, int nq,
                const double *exact, double *err2) {
  int rc = check_problem(P);
  if (rc) return rc;
  int d = P->d, m = P->m;
  int Nu = ncoef_box(d, m), nc = 1 << d;
  int E[OR_MAXD], q[OR_MAXD], eq[OR_MAXD];
  for (int i = 0; i < d; ++i) {
    E[i] = 2 * m + 2;
    q[i] = m;
    eq[i] = nq;
  }
  int64_t st[OR_MAXD], sq[OR_MAXD];
  int64_t B = box_strides(d, E, st);
  int64_t NQ = box_strides(d, eq, sq);
  double xq[64], wq[64];
  rc = or_gauss_points(nq, xq, wq);
  if (rc) return rc;
  double *cu = (double *)malloc(sizeof(double) * nc * Nu);
  double *a = (double *)malloc(sizeof(double) * B);
  if (!cu || !a) {
    free(cu);
    free(a);
    return OR_EALLOC;
  }
  int64_t nt = or_npts(P, 1 - g), total = or_nnodes(P, 1 - g);
  double hd = pow(P->h, (double)d), acc = 0.0;
  for (int64_t node = 0; node < total && !rc; ++node) {
    int t[OR_MAXD];
    int64_t r = node;
    for (int i = d - 1; i >= 0; --i) {
      t[i] = (int)(r % nt);
      r /= nt;
    }
    double wc = cell_weight(P, g, t);
    gather(P, 1 - g, t, u, m, cu);
    rc = or_interp(d, q, cu, a);
    if (rc) break;
    for (int64_t pq = 0; pq < NQ; ++pq) {
      int iq[OR_MAXD];
      box_unravel(d, eq, pq, iq);
      double val = 0.0;
      for (int64_t k = 0; k < B; ++k) {
        int al[OR_MAXD];
        box_unravel(d, E, k, al);
        double mono = 1.0;
        for (int i = 0; i < d; ++i) mono *= pow(xq[iq[i]], (double)al[i]);
        val += a[k] * mono;
      }
      double wt = 1.0;
      for (int i = 0; i < d; ++i) wt *= wq[iq[i]];
      double e = val - exact[node * NQ + pq];
      acc += wc * hd * wt * e * e;
    }
  }
  *err2 = acc;
  free(cu);
  free(a);
  return rc;
}
