// FP64 device set-up of a Hermite context: the per-cell operator (the
// interpolation of Sec. 2.2 composed with the exact Taylor evolution of
// Sec. 3.1.2 / 3.3 / 4.1 and the evaluation at the cell centre) and the
// per-parity-class quadratic forms of the energies of Sec. 3.2 / 3.3 / 4.2.
//
// Derivation used here (independent of the recursion form the paper prints):
// in xi = (x - X)/h the cell interpolant of unit data at the reference corner
// (every axis at xi = -1/2) is a tensor product of 1-D two-point Hermite basis
// polynomials.  With D = sum_i d^2/dxi_i^2, tau = c dt / (2h) and the velocity
// stored as (h/c) v, the exact solution of the wave equation started from
// the cell polynomials (a_u, b_v) and first-derivative term L1 is, after dt/2,
//   u+ = a_u + sum_{j>=1} tau^{2j}/(2j)! D^{j-1} L1 + sum_{j>=0} tau^{2j+1}/(2j+1)! D^j b_v
//   v+ =       sum_{j>=1} tau^{2j-1}/(2j-1)! D^{j-1} L1 + sum_{j>=0} tau^{2j}/(2j)! D^j b_v
// (L1 = D a_u, or sum_i d_i^2 I^(i) u for the d > 1 full variant of Sec. 3.3),
// and for the conservative update (Eq. update) 2 sum_r tau^{2r}/(2r)! D^r a_u.
// The series stop when D^j annihilates the polynomial.  The new nodal data
// are the coefficients of degree <= m (u) and <= m-1 (v) at xi = 0.
#include <cmath>
#include <vector>

#include "hermite_internal.h"

namespace hermite {
namespace {

__device__ inline void unravel(int d, int E, int idx, int *a) {
  for (int i = d - 1; i >= 0; --i) {
    a[i] = idx % E;
    idx /= E;
  }
}

__device__ inline int ravel(int d, int E, const int *a) {
  int p = 0;
  for (int i = 0; i < d; ++i) p = p * E + a[i];
  return p;
}

__device__ inline double dbinom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

// 1-D two-point Hermite basis for data of degree q given at the left corner
// (s = xi + 1/2 = 0):  phi_l(s) = s^l (1-s)^{q+1} sum_{k=0}^{q-l} binom(q+k,k) s^k.
// Its Taylor coefficients at s = 0 are delta_{jl} (j <= q), and it vanishes
// to order q at s = 1, which are the conditions of Eq. (Hermcon).
// H[j*(q+1)+l] = coefficient of xi^j, j in [0, 2q+1].
__global__ void basis_kernel(int q, double *H) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || q < 0) return;
  const int n = 2 * q + 2;
  double s[64];
  for (int l = 0; l <= q; ++l) {
    for (int i = 0; i < n; ++i) s[i] = 0.0;
    for (int k = 0; k <= q - l; ++k) s[l + k] = dbinom(q + k, k);
    for (int r = 0; r <= q; ++r)  // multiply by (1 - s), q+1 times
      for (int i = n - 1; i >= 1; --i) s[i] -= s[i - 1];
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int i = j; i < n; ++i) acc += s[i] * dbinom(i, j) * ldexp(1.0, -(i - j));  // exact 2^-(i-j)
      H[j * (q + 1) + l] = acc;
    }
  }
}

struct PolySpace {
  int d, m, E, B;
  const double *Hm;   // basis for degree-m data
  const double *Hm1;  // basis for degree-(m-1) data (unused when m = 0)
};

// Interpolant of unit data at the reference corner, data multi-index b, data
// degree q[i] per axis; zero when b exceeds the degree in some axis.
__device__ void interp_unit(const PolySpace &P, const int *q, const int *b, double *out) {
  for (int k = 0; k < P.B; ++k) out[k] = 0.0;
  for (int i = 0; i < P.d; ++i)
    if (b[i] > q[i]) return;
  for (int k = 0; k < P.B; ++k) {
    int a[kMaxDim];
    unravel(P.d, P.E, k, a);
    double v = 1.0;
    for (int i = 0; i < P.d && v != 0.0; ++i) {
      if (a[i] >= 2 * q[i] + 2) {
        v = 0.0;
        break;
      }
      const double *H = q[i] == P.m ? P.Hm : P.Hm1;
      v *= H[a[i] * (q[i] + 1) + b[i]];
    }
    out[k] = v;
  }
}

// out = d^ord/dxi_ax^ord f (same box); out may not alias f.
__device__ void deriv(const PolySpace &P, const double *f, int ax, int ord, double *out) {
  for (int k = 0; k < P.B; ++k) {
    int a[kMaxDim];
    unravel(P.d, P.E, k, a);
    if (a[ax] + ord >= P.E) {
      out[k] = 0.0;
      continue;
    }
    double fct = 1.0;
    for (int j = 1; j <= ord; ++j) fct *= (double)(a[ax] + j);
    a[ax] += ord;
    out[k] = fct * f[ravel(P.d, P.E, a)];
  }
}

// out = D f (sum of second derivatives); out may not alias f.
__device__ void lap(const PolySpace &P, const double *f, double *out) {
  for (int k = 0; k < P.B; ++k) {
    int a[kMaxDim];
    unravel(P.d, P.E, k, a);
    double acc = 0.0;
    for (int i = 0; i < P.d; ++i) {
      if (a[i] + 2 >= P.E) continue;
      int b[kMaxDim] = {a[0], P.d > 1 ? a[1] : 0, P.d > 2 ? a[2] : 0};
      b[i] += 2;
      acc += (double)((a[i] + 2) * (a[i] + 1)) * f[ravel(P.d, P.E, b)];
    }
    out[k] = acc;
  }
}

__device__ double taylor_weight(double tau, int k) {
  double w = 1.0;
  for (int i = 1; i <= k; ++i) w *= tau / (double)i;
  return w;
}

struct OpParams {
  PolySpace P;
  int variant, startup, Nu, Nv, nci, nco;
  double tau;
  double vscale;  // h/c: the series act on (h/c) v; columns of v inputs are
                  // multiplied by h/c and rows of v outputs by c/h so that the
                  // operator maps the paper's (u, v) data directly
  double *work;  // [nci][8][B]
  double *out;   // [nco][nci]
};

__global__ void operator_kernel(OpParams p) {
  const int beta = blockIdx.x * blockDim.x + threadIdx.x;
  if (beta >= p.nci) return;
  const PolySpace &P = p.P;
  const int B = P.B, d = P.d, m = P.m;
  double *w = p.work + (size_t)beta * 8 * B;
  double *au = w, *L1 = w + B, *bv = w + 2 * B, *U = w + 3 * B, *V = w + 4 * B;
  double *T = w + 5 * B, *T2 = w + 6 * B, *tmp = w + 7 * B;
  for (int k = 0; k < 5 * B; ++k) w[k] = 0.0;
  const bool cons = (p.variant == HERMITE_CONSERVATIVE) && !p.startup;
  const bool is_u = beta < p.Nu;
  const double colscale = is_u ? 1.0 : p.vscale;
  int b[kMaxDim] = {0, 0, 0};
  unravel(d, is_u ? m + 1 : m, is_u ? beta : beta - p.Nu, b);
  int qm[kMaxDim] = {m, m, m}, qv[kMaxDim] = {m - 1, m - 1, m - 1};
  if (is_u) {
    interp_unit(P, qm, b, au);
    if (!cons) {
      if (p.variant == HERMITE_DISSIPATIVE && d > 1 && !p.startup) {
        // special interpolants I^(i): degree m in axis i, m-1 elsewhere
        for (int ax = 0; ax < d; ++ax) {
          int qi[kMaxDim];
          for (int i = 0; i < kMaxDim; ++i) qi[i] = (i == ax) ? m : m - 1;
          interp_unit(P, qi, b, tmp);
          deriv(P, tmp, ax, 2, T);
          for (int k = 0; k < B; ++k) L1[k] += T[k];
        }
      } else {
        lap(P, au, L1);
      }
    }
  } else {
    interp_unit(P, qv, b, bv);
  }
  const int J = (d * (2 * m + 1)) / 2 + 2;
  if (cons) {
    for (int k = 0; k < B; ++k) {
      U[k] = au[k];
      T[k] = au[k];
    }
    for (int r = 1; r <= J; ++r) {
      lap(P, T, T2);
      const double wr = taylor_weight(p.tau, 2 * r);
      for (int k = 0; k < B; ++k) {
        T[k] = T2[k];
        U[k] += wr * T[k];
      }
    }
    for (int row = 0; row < p.Nu; ++row) {
      int a[kMaxDim] = {0, 0, 0};
      unravel(d, m + 1, row, a);
      p.out[(size_t)row * p.nci + beta] = 2.0 * U[ravel(d, P.E, a)];
    }
    return;
  }
  for (int k = 0; k < B; ++k) {
    U[k] = au[k];
    T[k] = L1[k];
  }
  for (int j = 1; j <= J; ++j) {
    const double wu = taylor_weight(p.tau, 2 * j), wv = taylor_weight(p.tau, 2 * j - 1);
    for (int k = 0; k < B; ++k) {
      U[k] += wu * T[k];
      V[k] += wv * T[k];
    }
    lap(P, T, T2);
    for (int k = 0; k < B; ++k) T[k] = T2[k];
  }
  for (int k = 0; k < B; ++k) T[k] = bv[k];
  for (int j = 0; j <= J; ++j) {
    const double wu = taylor_weight(p.tau, 2 * j + 1), wv = taylor_weight(p.tau, 2 * j);
    for (int k = 0; k < B; ++k) {
      U[k] += wu * T[k];
      V[k] += wv * T[k];
    }
    lap(P, T, T2);
    for (int k = 0; k < B; ++k) T[k] = T2[k];
  }
  for (int row = 0; row < p.Nu; ++row) {
    int a[kMaxDim] = {0, 0, 0};
    unravel(d, m + 1, row, a);
    p.out[(size_t)row * p.nci + beta] = colscale * U[ravel(d, P.E, a)];
  }
  if (!p.startup)
    for (int row = 0; row < p.Nv; ++row) {
      int a[kMaxDim] = {0, 0, 0};
      unravel(d, m, row, a);
      p.out[(size_t)(p.Nu + row) * p.nci + beta] = (colscale / p.vscale) * V[ravel(d, P.E, a)];
    }
}

// ---------------------------------------------------------------------------
// Energy quadratic forms.  Writing the corner data of a cell through the
// Walsh-Hadamard transform over corners, z_q[beta] = sum_s (-1)^{|q & s|} x_s[beta],
// the cell interpolant is p = sum_c sum_beta z_{c ^ par(beta)}[beta] * (a_beta
// restricted to the monomials of parity class c), a_beta being the interpolant
// of unit data at the reference corner.  Energies are integrals invariant
// under reflection of each axis, so classes do not mix and each cell's energy
// is sum_c y_c^T Q_c y_c with y_c[beta] = z_{c ^ par(beta)}[beta].

enum FormKind { kDissPlain = 0, kDissInvariant = 1, kConsSemi = 2, kConsGrad = 3 };

struct FormParams {
  PolySpace P;
  int kind, Nu, Nv, nq, ncomp, nclass;
  double vscale;  // h/c: v data enter the forms as (h/c) v
  double *F;   // [nclass][nq][ncomp][B] component polynomials
  double *HF;  // same with the monomial Gram matrix applied per axis
  double *work;  // [nclass*nq][4][B]
};

__device__ inline int parity_bits(int d, const int *a) {
  int p = 0;
  for (int i = 0; i < d; ++i) p = (p << 1) | (a[i] & 1);
  return p;
}

__device__ void restrict_class(const PolySpace &P, int c, double *f) {
  for (int k = 0; k < P.B; ++k) {
    int a[kMaxDim];
    unravel(P.d, P.E, k, a);
    if (parity_bits(P.d, a) != c) f[k] = 0.0;
  }
}

// int_{-1/2}^{1/2} xi^n dxi
__device__ inline double moment(int n) { return (n & 1) ? 0.0 : ldexp(1.0, -n) / (n + 1); }

__device__ void gram_apply(const PolySpace &P, const double *f, double *out, double *tmp) {
  for (int k = 0; k < P.B; ++k) out[k] = f[k];
  for (int ax = 0; ax < P.d; ++ax) {
    for (int k = 0; k < P.B; ++k) {
      int a[kMaxDim];
      unravel(P.d, P.E, k, a);
      double acc = 0.0;
      const int keep = a[ax];
      for (int j = 0; j < P.E; ++j) {
        a[ax] = j;
        acc += moment(keep + j) * out[ravel(P.d, P.E, a)];
      }
      tmp[k] = acc;
    }
    for (int k = 0; k < P.B; ++k) out[k] = tmp[k];
  }
}

__global__ void form_components_kernel(FormParams p) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= p.nclass * p.nq) return;
  const int c = id / p.nq, beta = id % p.nq;
  const PolySpace &P = p.P;
  const int B = P.B, d = P.d, m = P.m;
  double *w = p.work + (size_t)id * 4 * B;
  double *a = w, *t1 = w + B, *t3 = w + 3 * B;
  const bool is_u = beta < p.Nu;
  int b[kMaxDim] = {0, 0, 0};
  unravel(d, is_u ? m + 1 : m, is_u ? beta : beta - p.Nu, b);
  int qm[kMaxDim] = {m, m, m}, qv[kMaxDim] = {m - 1, m - 1, m - 1};
  for (int comp = 0; comp < p.ncomp; ++comp) {
    double *F = p.F + (((size_t)c * p.nq + beta) * p.ncomp + comp) * B;
    double *HF = p.HF + (((size_t)c * p.nq + beta) * p.ncomp + comp) * B;
    for (int k = 0; k < B; ++k) F[k] = 0.0;
    const bool v_comp = (p.kind == kDissPlain || p.kind == kDissInvariant) && comp == d;
    if (v_comp != !is_u) {
      // this input does not feed this component
    } else if (p.kind == kDissPlain || p.kind == kConsGrad) {
      if (v_comp) {
        interp_unit(P, qv, b, F);
        restrict_class(P, c, F);
      } else {
        interp_unit(P, qm, b, a);
        restrict_class(P, c, a);
        deriv(P, a, comp, 1, F);
      }
    } else if (p.kind == kDissInvariant) {
      if (v_comp) {
        interp_unit(P, qv, b, a);
      } else {
        int qi[kMaxDim];
        for (int i = 0; i < kMaxDim; ++i) qi[i] = (d == 1 || i == comp) ? m : m - 1;
        interp_unit(P, qi, b, a);
      }
      restrict_class(P, c, a);
      for (int ax = 0; ax < d; ++ax) {
        deriv(P, a, ax, m + ((!v_comp && ax == comp) ? 1 : 0), t1);
        for (int k = 0; k < B; ++k) a[k] = t1[k];
      }
      for (int k = 0; k < B; ++k) F[k] = a[k];
    } else {  // kConsSemi
      interp_unit(P, qm, b, a);
      restrict_class(P, c, a);
      for (int ax = 0; ax < d; ++ax) {
        deriv(P, a, ax, m + 1, t1);
        for (int k = 0; k < B; ++k) a[k] = t1[k];
      }
      for (int k = 0; k < B; ++k) F[k] = a[k];
    }
    if (!is_u)
      for (int k = 0; k < B; ++k) F[k] *= p.vscale;
    gram_apply(P, F, HF, t3);
  }
}

// Cholesky factor (upper, G = R^T R) of the 1-D monomial Gram matrix
// G[a][b] = int_{-1/2}^{1/2} xi^{a+b} dxi, a, b < E.  Its zero pattern follows
// the parity of a + b, so odd and even exponents stay separate.
__global__ void gram_cholesky_kernel(int E, double *R) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < E * E; ++i) R[i] = 0.0;
  for (int j = 0; j < E; ++j) {
    double s = moment(2 * j);
    for (int k = 0; k < j; ++k) s -= R[k * E + j] * R[k * E + j];
    const double rjj = sqrt(s);
    R[j * E + j] = rjj;
    for (int i = j + 1; i < E; ++i) {
      double t = moment(i + j);
      for (int k = 0; k < j; ++k) t -= R[k * E + j] * R[k * E + i];
      R[j * E + i] = t / rjj;
    }
  }
}

// RF = (R x ... x R) F for every component polynomial: |RF|^2 = int F^2
__global__ void form_cholesky_apply_kernel(const double *F, int64_t npoly, int d, int E, int B, const double *R,
                                           double *RF, double *work) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npoly) return;
  const double *f = F + id * B;
  double *out = RF + id * B, *tmp = work + id * B;
  for (int k = 0; k < B; ++k) out[k] = f[k];
  for (int ax = 0; ax < d; ++ax) {
    for (int k = 0; k < B; ++k) {
      int a[kMaxDim];
      unravel(d, E, k, a);
      const int row = a[ax];
      double acc = 0.0;
      for (int b = row; b < E; ++b) {
        a[ax] = b;
        acc += R[row * E + b] * out[ravel(d, E, a)];
      }
      tmp[k] = acc;
    }
    for (int k = 0; k < B; ++k) out[k] = tmp[k];
  }
}

// Pivoted Cholesky of each class matrix Q_c (symmetric positive semidefinite):
// Q_c[perm][perm] = L^T L with L upper triangular in the permuted order, rows
// beyond the numerical rank dropped (remaining diagonal <= 1e-15 of the
// largest).  One thread per class.  L_out[c][r][k] holds row r against the
// permuted column k; perm_out[c][k] is the original column.
__global__ void pivoted_cholesky_kernel(const double *Q, int nclass, int nq, double *work, double *L_out,
                                        int16_t *perm_out, int *rank_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nclass) return;
  double *A = work + (size_t)c * nq * nq;
  for (int i = 0; i < nq * nq; ++i) A[i] = Q[(size_t)c * nq * nq + i];
  int16_t *perm = perm_out + (size_t)c * nq;
  double *L = L_out + (size_t)c * nq * nq;
  for (int i = 0; i < nq; ++i) perm[i] = (int16_t)i;
  for (int i = 0; i < nq * nq; ++i) L[i] = 0.0;
  double dmax0 = 0.0;
  for (int i = 0; i < nq; ++i) dmax0 = fmax(dmax0, A[i * nq + i]);
  int r = 0;
  for (; r < nq; ++r) {
    // pivot: largest remaining diagonal
    int p = r;
    for (int i = r + 1; i < nq; ++i)
      if (A[perm[i] * nq + perm[i]] > A[perm[p] * nq + perm[p]]) p = i;
    const int16_t tp = perm[r];
    perm[r] = perm[p];
    perm[p] = tp;
    for (int k = 0; k < r; ++k) {  // keep earlier rows aligned with the permuted columns
      const double t = L[k * nq + r];
      L[k * nq + r] = L[k * nq + p];
      L[k * nq + p] = t;
    }
    const double piv = A[perm[r] * nq + perm[r]];
    if (!(piv > 1e-15 * dmax0)) break;
    const double lrr = sqrt(piv);
    L[r * nq + r] = lrr;
    for (int j = r + 1; j < nq; ++j) L[r * nq + j] = A[perm[r] * nq + perm[j]] / lrr;
    // Schur complement on the remaining (original-index) entries
    for (int i = r + 1; i < nq; ++i)
      for (int j = r + 1; j < nq; ++j) A[perm[i] * nq + perm[j]] -= L[r * nq + i] * L[r * nq + j];
  }
  rank_out[c] = r;
}

__global__ void form_gram_kernel(const double *F, const double *HF, int nclass, int nq, int ncomp,
                                 int B, double *Q) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)nclass * nq * nq;
  if (id >= total) return;
  const int c = (int)(id / ((int64_t)nq * nq));
  const int r = (int)(id % ((int64_t)nq * nq));
  const int b1 = r / nq, b2 = r % nq;
  double acc = 0.0;
  for (int comp = 0; comp < ncomp; ++comp) {
    const double *f = F + (((size_t)c * nq + b1) * ncomp + comp) * B;
    const double *g = HF + (((size_t)c * nq + b2) * ncomp + comp) * B;
    for (int k = 0; k < B; ++k) acc += f[k] * g[k];
  }
  Q[id] = acc;
}

struct Basis {
  double *Hm = nullptr, *Hm1 = nullptr;
};

int make_basis(hermite_ctx *ctx, Basis &bs) {
  const int m = ctx->m;
  if (!cuda_ok(ctx, device_alloc(&bs.Hm, sizeof(double) * (2 * m + 2) * (m + 1)), "cudaMalloc basis"))
    return HERMITE_ERR_ALLOC;
  basis_kernel<<<1, 1, 0, ctx->stream>>>(m, bs.Hm);
  if (m >= 1) {
    if (!cuda_ok(ctx, device_alloc(&bs.Hm1, sizeof(double) * (2 * m) * m), "cudaMalloc basis"))
      return HERMITE_ERR_ALLOC;
    basis_kernel<<<1, 1, 0, ctx->stream>>>(m - 1, bs.Hm1);
  }
  if (!cuda_ok(ctx, cudaGetLastError(), "basis_kernel")) return HERMITE_ERR_CUDA;
  return HERMITE_OK;
}

void free_basis(Basis &bs) {
  cudaFree(bs.Hm);
  cudaFree(bs.Hm1);
}

// Factor of a form with many monomials per class: pivoted Cholesky of Q_c.
int build_cholesky_factor(hermite_ctx *ctx, int f, int nclass, int nq) {
  double *work = nullptr;
  int *rank = nullptr;
  int rc = HERMITE_OK;
  const size_t n2 = (size_t)nclass * nq * nq;
  if (!cuda_ok(ctx, device_alloc(&work, sizeof(double) * n2), "cudaMalloc chol work") ||
      !cuda_ok(ctx, device_alloc(&rank, sizeof(int) * nclass), "cudaMalloc rank") ||
      !cuda_ok(ctx, device_alloc(&ctx->L[f], sizeof(double) * n2), "cudaMalloc L") ||
      !cuda_ok(ctx, device_alloc(&ctx->lperm[f], sizeof(int16_t) * nclass * nq), "cudaMalloc perm")) {
    rc = HERMITE_ERR_ALLOC;
  } else {
    pivoted_cholesky_kernel<<<1, 32, 0, ctx->stream>>>(ctx->Q[f], nclass, nq, work, ctx->L[f], ctx->lperm[f], rank);
    std::vector<int> rh(nclass);
    if (!cuda_ok(ctx, cudaGetLastError(), "pivoted_cholesky_kernel") ||
        !cuda_ok(ctx, cudaMemcpyAsync(rh.data(), rank, sizeof(int) * nclass, cudaMemcpyDeviceToHost, ctx->stream),
                 "rank copy") ||
        !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "cholesky sync")) {
      rc = HERMITE_ERR_CUDA;
    } else {
      int rmax = 0;
      for (int c = 0; c < nclass; ++c) rmax = std::max(rmax, rh[c]);
      ctx->rmax[f] = rmax;
      ctx->lrows[f] = nq;
      ctx->ltri[f] = 1;
    }
  }
  cudaFree(work);
  cudaFree(rank);
  return rc;
}

// Low-rank factor of a form: rows (component k, monomial mu) of
// (R x .. x R) F_{c,beta,k} that are non-zero for some input beta.  Kept only
// when every class has at most nq/2 rows (then r*nq < nq^2/2 multiply-adds).
int build_lowrank_factor(hermite_ctx *ctx, int f, const double *F, int nclass, int nq, int ncomp,
                         const PolySpace &P) {
  const int64_t npoly = (int64_t)nclass * nq * ncomp;
  const size_t nF = (size_t)npoly * P.B;
  double *R = nullptr, *RF = nullptr, *work = nullptr;
  int rc = HERMITE_OK;
  if (!cuda_ok(ctx, device_alloc(&R, sizeof(double) * P.E * P.E), "cudaMalloc R") ||
      !cuda_ok(ctx, device_alloc(&RF, sizeof(double) * nF), "cudaMalloc RF") ||
      !cuda_ok(ctx, device_alloc(&work, sizeof(double) * nF), "cudaMalloc work")) {
    rc = HERMITE_ERR_ALLOC;
  } else {
    gram_cholesky_kernel<<<1, 1, 0, ctx->stream>>>(P.E, R);
    form_cholesky_apply_kernel<<<(unsigned)((npoly + 63) / 64), 64, 0, ctx->stream>>>(F, npoly, P.d, P.E, P.B, R,
                                                                                       RF, work);
    std::vector<double> h(nF);
    if (!cuda_ok(ctx, cudaGetLastError(), "cholesky kernels") ||
        !cuda_ok(ctx, cudaMemcpyAsync(h.data(), RF, sizeof(double) * nF, cudaMemcpyDeviceToHost, ctx->stream),
                 "RF copy") ||
        !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "RF sync")) {
      rc = HERMITE_ERR_CUDA;
    } else {
      // support rows per class
      std::vector<std::vector<std::pair<int, int>>> rows(nclass);
      int rmax = 0;
      for (int c = 0; c < nclass; ++c) {
        for (int k = 0; k < ncomp; ++k)
          for (int mu = 0; mu < P.B; ++mu) {
            bool nz = false;
            for (int b = 0; b < nq && !nz; ++b) nz = h[(((size_t)c * nq + b) * ncomp + k) * P.B + mu] != 0.0;
            if (nz) rows[c].push_back({k, mu});
          }
        rmax = std::max<int>(rmax, (int)rows[c].size());
      }
      if (2 * rmax <= nq) {
        std::vector<double> Lh((size_t)nclass * rmax * nq, 0.0);
        for (int c = 0; c < nclass; ++c)
          for (size_t r = 0; r < rows[c].size(); ++r)
            for (int b = 0; b < nq; ++b)
              Lh[((size_t)c * rmax + r) * nq + b] =
                  h[(((size_t)c * nq + b) * ncomp + rows[c][r].first) * P.B + rows[c][r].second];
        std::vector<int16_t> ident((size_t)nclass * nq);
        for (size_t i = 0; i < ident.size(); ++i) ident[i] = (int16_t)(i % nq);
        if (!cuda_ok(ctx, device_alloc(&ctx->L[f], sizeof(double) * Lh.size()), "cudaMalloc L") ||
            !cuda_ok(ctx, device_alloc(&ctx->lperm[f], sizeof(int16_t) * ident.size()), "cudaMalloc perm")) {
          rc = HERMITE_ERR_ALLOC;
        } else if (!cuda_ok(ctx, cudaMemcpy(ctx->L[f], Lh.data(), sizeof(double) * Lh.size(), cudaMemcpyHostToDevice),
                            "L copy") ||
                   !cuda_ok(ctx, cudaMemcpy(ctx->lperm[f], ident.data(), sizeof(int16_t) * ident.size(),
                                            cudaMemcpyHostToDevice),
                            "perm copy")) {
          rc = HERMITE_ERR_CUDA;
        } else {
          ctx->rmax[f] = rmax;
          ctx->lrows[f] = rmax;
          ctx->ltri[f] = 0;
        }
      }
    }
  }
  cudaFree(R);
  cudaFree(RF);
  cudaFree(work);
  if (rc == HERMITE_OK && !ctx->L[f]) rc = build_cholesky_factor(ctx, f, nclass, nq);
  return rc;
}

PolySpace make_space(const hermite_ctx *ctx, const Basis &bs) {
  PolySpace P;
  P.d = ctx->d;
  P.m = ctx->m;
  P.E = 2 * ctx->m + 2;
  P.B = 1;
  for (int i = 0; i < ctx->d; ++i) P.B *= P.E;
  P.Hm = bs.Hm;
  P.Hm1 = bs.Hm1;
  return P;
}

}  // namespace

int build_operator(hermite_ctx *ctx, bool startup, double *out, int rows, int cols) {
  Basis bs;
  int rc = make_basis(ctx, bs);
  double *work = nullptr;
  if (rc == HERMITE_OK) {
    OpParams p;
    p.P = make_space(ctx, bs);
    p.variant = ctx->variant;
    p.startup = startup ? 1 : 0;
    p.Nu = ctx->Nu;
    p.Nv = ctx->Nv;
    p.nci = cols;
    p.nco = rows;
    p.tau = 0.5 * ctx->lam;
    p.vscale = ctx->h / ctx->c;
    p.out = out;
    if (!cuda_ok(ctx, device_alloc(&work, sizeof(double) * (size_t)cols * 8 * p.P.B), "cudaMalloc work")) {
      rc = HERMITE_ERR_ALLOC;
    } else {
      p.work = work;
      operator_kernel<<<(cols + 63) / 64, 64, 0, ctx->stream>>>(p);
      if (!cuda_ok(ctx, cudaGetLastError(), "operator_kernel") ||
          !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "operator_kernel sync"))
        rc = HERMITE_ERR_CUDA;
    }
  }
  cudaFree(work);
  free_basis(bs);
  return rc;
}

int build_energy_forms(hermite_ctx *ctx) {
  const bool cons = ctx->variant == HERMITE_CONSERVATIVE;
  const int kinds[2] = {cons ? kConsSemi : kDissPlain, cons ? kConsGrad : kDissInvariant};
  {
    // physical scale of each form (xi-integrals times powers of h and c)
    const int d = ctx->d, m = ctx->m;
    const double hd = pow(ctx->h, (double)d), c2 = ctx->c * ctx->c;
    for (int f = 0; f < kNumForms; ++f) {
      if (kinds[f] == kDissPlain || kinds[f] == kConsGrad)
        ctx->formscale[f] = c2 * hd / (ctx->h * ctx->h);
      else if (kinds[f] == kDissInvariant)
        ctx->formscale[f] = c2 * hd * pow(ctx->h, -2.0 * (d * m + 1));
      else
        ctx->formscale[f] = hd * pow(ctx->h, -2.0 * d * (m + 1));
    }
  }
  // the sum-factorised kernel covers these energies without the class forms
  if (energy_tp_supported(ctx->d, ctx->m, ctx->variant)) return HERMITE_OK;
  Basis bs;
  int rc = make_basis(ctx, bs);
  if (rc) {
    free_basis(bs);
    return rc;
  }
  const PolySpace P = make_space(ctx, bs);
  const int nclass = 1 << ctx->d;
  const int nq = cons ? ctx->Nu : ctx->Nu + ctx->Nv;
  for (int f = 0; f < kNumForms && rc == HERMITE_OK; ++f) {
    const int kind = kinds[f];
    const int ncomp = (kind == kConsSemi) ? 1 : (kind == kConsGrad ? ctx->d : ctx->d + 1);
    double *F = nullptr, *HF = nullptr, *work = nullptr;
    const size_t nF = (size_t)nclass * nq * ncomp * P.B;
    if (!cuda_ok(ctx, device_alloc(&F, sizeof(double) * nF), "cudaMalloc F") ||
        !cuda_ok(ctx, device_alloc(&HF, sizeof(double) * nF), "cudaMalloc HF") ||
        !cuda_ok(ctx, device_alloc(&work, sizeof(double) * (size_t)nclass * nq * 4 * P.B), "cudaMalloc work") ||
        !cuda_ok(ctx, device_alloc(&ctx->Q[f], sizeof(double) * (size_t)nclass * nq * nq), "cudaMalloc Q")) {
      rc = HERMITE_ERR_ALLOC;
    } else {
      FormParams p;
      p.P = P;
      p.kind = kind;
      p.Nu = ctx->Nu;
      p.Nv = ctx->Nv;
      p.nq = nq;
      p.ncomp = ncomp;
      p.nclass = nclass;
      p.vscale = ctx->h / ctx->c;
      p.F = F;
      p.HF = HF;
      p.work = work;
      const int n1 = nclass * nq;
      form_components_kernel<<<(n1 + 63) / 64, 64, 0, ctx->stream>>>(p);
      const int64_t n2 = (int64_t)nclass * nq * nq;
      form_gram_kernel<<<(unsigned)((n2 + 127) / 128), 128, 0, ctx->stream>>>(F, HF, nclass, nq, ncomp, P.B,
                                                                                ctx->Q[f]);
      if (!cuda_ok(ctx, cudaGetLastError(), "energy form kernels") ||
          !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "energy form sync"))
        rc = HERMITE_ERR_CUDA;
      ctx->nq[f] = nq;
      if (rc == HERMITE_OK) rc = build_lowrank_factor(ctx, f, F, nclass, nq, ncomp, P);
    }
    cudaFree(F);
    cudaFree(HF);
    cudaFree(work);
  }
  free_basis(bs);
  return rc;
}

int build_parity_tables(hermite_ctx *ctx) {
  // parity bits (axis 0 most significant) of each coefficient multi-index:
  // u indices [0,m]^d first, then v indices [0,m-1]^d
  const int d = ctx->d, m = ctx->m;
  std::vector<int8_t> par;
  for (int box = 0; box < 2; ++box) {
    const int E = box == 0 ? m + 1 : m;
    const int n = box == 0 ? ctx->Nu : ctx->Nv;
    for (int k = 0; k < n; ++k) {
      int r = k, bits = 0;
      int a[kMaxDim] = {0, 0, 0};
      for (int i = d - 1; i >= 0; --i) {
        a[i] = r % E;
        r /= E;
      }
      for (int i = 0; i < d; ++i) bits = (bits << 1) | (a[i] & 1);
      par.push_back((int8_t)bits);
    }
  }
  if (!cuda_ok(ctx, device_alloc(&ctx->par_in, par.size() + 1), "cudaMalloc parity")) return HERMITE_ERR_ALLOC;
  if (!cuda_ok(ctx, cudaMemcpy(ctx->par_in, par.data(), par.size(), cudaMemcpyHostToDevice), "parity copy"))
    return HERMITE_ERR_CUDA;
  ctx->par_out = ctx->par_in;
  return HERMITE_OK;
}

}  // namespace hermite
