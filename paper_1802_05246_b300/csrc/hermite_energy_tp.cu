// Energies by sum factorisation, FP64 or double-FP32: the dissipative
// method's (Sec. 3.2 Eq. stable1/Energyeq, Sec. 3.3 Eq. stable2) and the
// conservative method's seminorm and gradient forms (Sec. 4.2).
//
// In the reference coordinate xi of a cell the interpolant is a tensor
// product of 1-D two-point Hermite bases, and after the Walsh-Hadamard
// transform over the corners each axis's basis splits into functions of
// even and of odd parity (psi^e_k, k = 0..q, e = the class bit of the axis).
// Every integrand of the energies is then a sum of tensor products of 1-D
// Gram matrices G^(j)_{q,e}[k][l] = int D^j psi^e_k D^j psi^e_l dxi, so per
// cell and parity class (y = the class's u and v tensors):
//   plain:      int |grad_xi I_m u|^2 = sum_abc (lam_a + lam_b + lam_c) w_abc^2,
//               w = (W x W x W) y_u with W = Q^T L^T from M = L L^T and
//               L^-1 K L^-T = Q diag(lam) Q^T (simultaneous diagonalisation
//               of the mass and stiffness matrices of the u basis);
//               int (I_{m-1} v)^2 = |(F x F x F) y_v|^2, F^T F the v mass matrix;
//   invariant:  sum_ax |(R_ax x S_others) y_u restricted|^2 + |(S x S x S) y_v|^2,
//               R^T R = G^(m+1)_{m,e}, S^T S = G^(m)_{m-1,e}, the restriction
//               keeping orders <= m along ax and <= m-1 elsewhere (the
//               interpolant I^(ax) of Sec. 3.3);
//   conservative: |(R x R x R) y_u|^2 and the gradient term as above.
// The 1-D matrices are built once per context on the host in long double.
// A block takes 32 cells and all 2^d classes (warp = class, lane = cell):
// its warps gather and transform the corner data into the class tensors in
// shared memory, then each thread evaluates its (cell, class) terms, one
// output row of the first axis at a time.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hermite_device.cuh"
#include "hermite_internal.h"

namespace hermite {
namespace {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

struct ArF64 {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ void mac(T &acc, T a, T b) { acc = fma(a, b, acc); }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T scale(T a, float w) { return a * (double)w; }  // w a power of two
  static __device__ __forceinline__ T norm(T a) { return a; }
  static __device__ __forceinline__ double to_double(T a) { return a; }
};

struct ArSplit {
  using T = float2;
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void mac(T &acc, T a, T b) { dev::df_fma(acc, a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return dev::df_add(a, b); }
  static __device__ __forceinline__ T neg(T a) { return dev::df_neg(a); }
  static __device__ __forceinline__ T mul(T a, T b) { return dev::df_mul(a, b); }
  static __device__ __forceinline__ T scale(T a, float w) { return make_float2(a.x * w, a.y * w); }
  // an accumulated hi + lo pair can carry |lo| > |hi| after cancellation; a
  // product drops lo * lo, so squares take the renormalised pair
  static __device__ __forceinline__ T norm(T a) { return dev::df_norm(a); }
  static __device__ __forceinline__ double to_double(T a) { return (double)a.x + (double)a.y; }
};

// Sizes of the per-axis matrices for data degree m: u basis n = m+1 functions
// per class bit, v basis nv = m; ranks of the seminorm factors R and S.
template <int MM>
struct Shape {
  static constexpr int n = MM + 1, nv = MM;
  static constexpr int RR = (MM + 2) / 2, RS = (MM + 1) / 2;
  static constexpr int oW = 0, oL = n * n, oF = oL + n, oR = oF + nv * nv, oS = oR + RR * n;
  static constexpr int EB = oS + RS * nv;  // entries per class bit
};

// |(A_0 x .. x A_{D-1}) y|^2, or with WEIGHTED the sum over the transformed
// entries of lamsum[(i0 * NB + i1) * NB + i2] times their squares, for the
// class tensor y of extents E_i (axis i; coefficient (i0, i1, i2) of the
// NB^D box at y[b * 32], the lane's column of the block's class tensors).
// A_i is K_i x E_i row-major.  The first axis is done one output row a at a
// time (a rolled loop, so the code stays small): t = A_0[a] . y, then the
// remaining axes on t in registers.
template <class Ar, int D, int NB, int E0, int E1, int E2, int K0, int K1, int K2, bool WEIGHTED>
__device__ __forceinline__ typename Ar::T kron_norm2(const typename Ar::T *y, const typename Ar::T *A0,
                                                     const typename Ar::T *A1, const typename Ar::T *A2,
                                                     const typename Ar::T *lamsum) {
  using T = typename Ar::T;
  T acc = Ar::zero();
  if constexpr (D == 1) {
#pragma unroll 1
    for (int a = 0; a < K0; ++a) {
      T s = Ar::zero();
#pragma unroll
      for (int i = 0; i < E0; ++i) Ar::mac(s, A0[a * E0 + i], y[i * 32]);
      s = Ar::norm(s);
      Ar::mac(acc, WEIGHTED ? Ar::mul(s, lamsum[a]) : s, s);
    }
  } else if constexpr (D == 2) {
#pragma unroll 1
    for (int a = 0; a < K0; ++a) {
      T t[E1];
#pragma unroll
      for (int k = 0; k < E1; ++k) t[k] = Ar::zero();
#pragma unroll 1
      for (int i = 0; i < E0; ++i) {
        const T f = A0[a * E0 + i];
#pragma unroll
        for (int k = 0; k < E1; ++k) Ar::mac(t[k], f, y[(i * NB + k) * 32]);
      }
#pragma unroll
      for (int cc = 0; cc < K1; ++cc) {
        T u = Ar::zero();
#pragma unroll
        for (int k = 0; k < E1; ++k) Ar::mac(u, A1[cc * E1 + k], t[k]);
        u = Ar::norm(u);
        Ar::mac(acc, WEIGHTED ? Ar::mul(u, lamsum[a * NB + cc]) : u, u);
      }
    }
  } else {
#pragma unroll 1
    for (int a = 0; a < K0; ++a) {
      T t[E1][E2];
#pragma unroll
      for (int j = 0; j < E1; ++j)
#pragma unroll
        for (int k = 0; k < E2; ++k) t[j][k] = Ar::zero();
#pragma unroll 1
      for (int i = 0; i < E0; ++i) {
        const T f = A0[a * E0 + i];
#pragma unroll
        for (int j = 0; j < E1; ++j)
#pragma unroll
          for (int k = 0; k < E2; ++k) Ar::mac(t[j][k], f, y[((i * NB + j) * NB + k) * 32]);
      }
#pragma unroll
      for (int bb = 0; bb < K1; ++bb) {
        T s[E2];
#pragma unroll
        for (int k = 0; k < E2; ++k) {
          s[k] = Ar::zero();
#pragma unroll
          for (int j = 0; j < E1; ++j) Ar::mac(s[k], A1[bb * E1 + j], t[j][k]);
        }
#pragma unroll
        for (int cc = 0; cc < K2; ++cc) {
          T u = Ar::zero();
#pragma unroll
          for (int k = 0; k < E2; ++k) Ar::mac(u, A2[cc * E2 + k], s[k]);
          u = Ar::norm(u);
          Ar::mac(acc, WEIGHTED ? Ar::mul(u, lamsum[(a * NB + bb) * NB + cc]) : u, u);
        }
      }
    }
  }
  return acc;
}

// Invariant u term of axis AX: R along AX (all n orders), S elsewhere (the
// first nv orders); in 1-D the single axis takes R.
template <class Ar, int D, int MM, int AX>
__device__ __forceinline__ typename Ar::T inv_u_term(const typename Ar::T *yu, const typename Ar::T *const *mb) {
  using Sh = Shape<MM>;
  constexpr int n = Sh::n, nv = Sh::nv;
  constexpr int E0 = (AX == 0 || D == 1) ? n : nv, E1 = AX == 1 ? n : nv, E2 = AX == 2 ? n : nv;
  constexpr int K0 = (AX == 0 || D == 1) ? Sh::RR : Sh::RS, K1 = AX == 1 ? Sh::RR : Sh::RS,
                K2 = AX == 2 ? Sh::RR : Sh::RS;
  const typename Ar::T *A0 = mb[0] + ((AX == 0 || D == 1) ? Sh::oR : Sh::oS);
  const typename Ar::T *A1 = mb[1] + (AX == 1 ? Sh::oR : Sh::oS);
  const typename Ar::T *A2 = mb[2] + (AX == 2 ? Sh::oR : Sh::oS);
  return kron_norm2<Ar, D, n, E0, E1, E2, K0, K1, K2, false>(yu, A0, A1, A2, nullptr);
}

// CONS = false: the dissipative forms of the level src (plain, invariant).
// CONS = true: the conservative forms (Sec. 4.2) of the u level
// src + sigma * srcB, sigma in {0, 1, -1}: the seminorm |p|^2_{m+1,..,m+1}
// and int |grad p|^2 (the bilinear form of two levels follows by
// polarisation from sigma = +-1).
template <class Ar, int D, int MM, bool CONS>
__global__ void __launch_bounds__(32 << D) energy_tp_kernel(Geometry g, const typename Ar::T *__restrict__ mats,
                                                            const typename Ar::T *__restrict__ src,
                                                            const typename Ar::T *__restrict__ srcB, float sigma,
                                                            double vs2, double *__restrict__ partials) {
  using T = typename Ar::T;
  using Sh = Shape<MM>;
  constexpr int NC = 1 << D, NT = 32 * NC;
  constexpr int n = Sh::n, nv = Sh::nv;
  constexpr int NU = ipow(n, D), NV = CONS ? 0 : ipow(nv, D), NCI = NU + NV;
  extern __shared__ __align__(16) unsigned char tp_smem[];
  T *ms = reinterpret_cast<T *>(tp_smem);  // [2][EB]
  T *lamsum = ms + 2 * Sh::EB;            // [NC][NU]
  T *Ty = lamsum + NC * NU;               // [NC class][NCI coefficient][32 cell]
  __shared__ double red[2][NC];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 2 * Sh::EB; i += NT) ms[i] = mats[i];
  __syncthreads();
  // lam_a + lam_b + lam_c of each class's diagonalised stiffness
  for (int i = threadIdx.x; i < NC * NU; i += NT) {
    const int c = i / NU;
    int k = i % NU;
    T s = Ar::zero();
    for (int ax = D - 1; ax >= 0; --ax) {
      const int e = (c >> (D - 1 - ax)) & 1;
      s = Ar::add(s, ms[e * Sh::EB + Sh::oL + k % n]);
      k /= n;
    }
    lamsum[i] = s;
  }
  const int c = w;  // this thread's parity class
  const T *mb[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) mb[ax] = ms + (ax < D ? ((c >> (D - 1 - ax)) & 1) : 0) * Sh::EB;
  T pu = Ar::zero(), pv = Ar::zero(), iu = Ar::zero(), iv = Ar::zero();
  const int64_t ntiles = (g.nodes_dst + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t = tile * 32 + lane;
    const bool valid = t < g.nodes_dst;
    int64_t idx[NC];
    int gm[NC];
    if (valid) {
      dev::cell_corners<D>(g, t, idx, gm);
    } else {
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        idx[s] = 0;
        gm[s] = 0;
      }
    }
    const float cw = valid ? dev::cell_weight<D>(g, t) : 0.0f;
    // Phase A: warp w gathers coefficients b = w, w + 2^d, ... of its lane's
    // cell, applies the ghost signs and the corner transform, and stores
    // z_q[b] as the class-(q ^ par(b)) entry b (the next coefficient's loads
    // are issued before this one is transformed).
    T x[NC], xn[NC];
    auto load = [&](int b, T *dst) {
#pragma unroll
      for (int s = 0; s < NC; ++s) dst[s] = (b < NCI && valid) ? src[(size_t)b * g.ld_src + idx[s]] : Ar::zero();
      if (CONS && sigma != 0.0f && b < NCI && valid) {
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          const T vb = srcB[(size_t)b * g.ld_src + idx[s]];
          dst[s] = Ar::add(dst[s], sigma > 0.0f ? vb : Ar::neg(vb));
        }
      }
    };
    load(w, x);
#pragma unroll 1
    for (int b = w; b < NCI; b += NC) {
      load(b + NC, xn);
      const bool isu = b < NU;
      const int E = isu ? n : nv;
      int kk = isu ? b : b - NU, pb = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        pb |= (kk % E & 1) << i;
        kk /= E;
      }
#pragma unroll
      for (int s = 0; s < NC; ++s)
        if (gm[s] && dev::ghost_negates(g.bc, gm[s], pb)) x[s] = Ar::neg(x[s]);
#pragma unroll
      for (int bm = 1; bm < NC; bm <<= 1)
#pragma unroll
        for (int i = 0; i < NC; ++i)
          if (!(i & bm)) {
            const T a = x[i], d = x[i | bm];
            x[i] = Ar::add(a, d);
            x[i | bm] = Ar::add(a, Ar::neg(d));
          }
#pragma unroll
      for (int q = 0; q < NC; ++q) Ty[((size_t)(q ^ pb) * NCI + b) * 32 + lane] = x[q];
#pragma unroll
      for (int s = 0; s < NC; ++s) x[s] = xn[s];
    }
    __syncthreads();
    // Phase B: this thread's (cell, class) terms
    const T *yu = Ty + (size_t)c * NCI * 32 + lane;
    // plain / gradient: the stiffness diagonalised along every axis, weighted by lam sums
    const T pl = kron_norm2<Ar, D, n, n, n, n, n, n, n, true>(yu, mb[0] + Sh::oW, mb[1] + Sh::oW, mb[2] + Sh::oW,
                                                              lamsum + c * NU);
    if constexpr (CONS) {
      // seminorm: the (m+1)-th derivative in every axis
      const T sm = kron_norm2<Ar, D, n, n, n, n, Sh::RR, Sh::RR, Sh::RR, false>(yu, mb[0] + Sh::oR, mb[1] + Sh::oR,
                                                                              mb[2] + Sh::oR, nullptr);
      iu = Ar::add(iu, Ar::scale(sm, cw));
      pu = Ar::add(pu, Ar::scale(pl, cw));
    } else {
      const T *yv = yu + NU * 32;
      const T pvc = kron_norm2<Ar, D, nv, nv, nv, nv, nv, nv, nv, false>(yv, mb[0] + Sh::oF, mb[1] + Sh::oF,
                                                                         mb[2] + Sh::oF, nullptr);
      const T ivc = kron_norm2<Ar, D, nv, nv, nv, nv, Sh::RS, Sh::RS, Sh::RS, false>(
          yv, mb[0] + Sh::oS, mb[1] + Sh::oS, mb[2] + Sh::oS, nullptr);
      T inv = inv_u_term<Ar, D, MM, 0>(yu, mb);
      if constexpr (D > 1) inv = Ar::add(inv, inv_u_term<Ar, D, MM, 1>(yu, mb));
      if constexpr (D > 2) inv = Ar::add(inv, inv_u_term<Ar, D, MM, 2>(yu, mb));
      pv = Ar::add(pv, Ar::scale(pvc, cw));
      iv = Ar::add(iv, Ar::scale(ivc, cw));
      pu = Ar::add(pu, Ar::scale(pl, cw));
      iu = Ar::add(iu, Ar::scale(inv, cw));
    }
    __syncthreads();  // the next tile's phase A overwrites the class tensors
  }
  // block sums: dissipative [plain, invariant] (v terms carry (h/c)^2),
  // conservative [seminorm, gradient]
  double e[2];
  if constexpr (CONS) {
    e[0] = Ar::to_double(iu);
    e[1] = Ar::to_double(pu);
  } else {
    e[0] = Ar::to_double(pu) + vs2 * Ar::to_double(pv);
    e[1] = Ar::to_double(iu) + vs2 * Ar::to_double(iv);
  }
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    double v = e[f];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[f][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int i = 0; i < NC; ++i) s += red[threadIdx.x][i];
    partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void reduce_tp_kernel(const double *partials, int64_t n, double scale, double *out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * red[0];
}

// ---------------------------------------------------------------------------
// Host construction of the 1-D matrices (long double).
using LD = long double;
using Poly = std::vector<LD>;  // coefficients of xi^j

LD binom(int n, int k) {
  if (k < 0 || k > n) return 0.0L;
  LD r = 1.0L;
  for (int i = 1; i <= k; ++i) r = r * (LD)(n - k + i) / (LD)i;
  return r;
}

// Parity-e part of the left-corner basis function of order k for data degree
// q: with s = xi + 1/2, phi_k(s) = s^k (1-s)^{q+1} sum_{j<=q-k} binom(q+j,j) s^j
// (Taylor data delta_{jk} at s = 0, vanishing to order q at s = 1).  Since the
// right-corner functions are the reflections of the left ones, the class-e
// function of order k after the corner transform is this parity part.
Poly psi(int q, int e, int k) {
  const int n = 2 * q + 2;
  Poly sp(n, 0.0L), xp(n, 0.0L);
  for (int j = 0; j <= q - k; ++j) sp[k + j] = binom(q + j, j);
  for (int r = 0; r <= q; ++r)  // times (1 - s), q+1 times
    for (int i = n - 1; i >= 1; --i) sp[i] -= sp[i - 1];
  for (int j = 0; j < n; ++j) {
    LD acc = 0.0L;
    for (int i = j; i < n; ++i) acc += sp[i] * binom(i, j) * ldexpl(1.0L, -(i - j));
    xp[j] = ((j & 1) == e) ? acc : 0.0L;
  }
  return xp;
}

Poly deriv(const Poly &f, int j) {
  Poly g(f.size(), 0.0L);
  for (size_t p = j; p < f.size(); ++p) {
    LD c = f[p];
    for (int i = 0; i < j; ++i) c *= (LD)(p - i);
    g[p - j] = c;
  }
  return g;
}

// G[a][b] = int_{-1/2}^{1/2} D^j psi^e_a D^j psi^e_b dxi, a, b = 0..q
std::vector<LD> gram(int q, int e, int j) {
  const int n = q + 1;
  std::vector<Poly> f(n);
  for (int k = 0; k < n; ++k) f[k] = deriv(psi(q, e, k), j);
  std::vector<LD> G((size_t)n * n, 0.0L);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      LD acc = 0.0L;
      for (size_t p = 0; p < f[a].size(); ++p)
        for (size_t r = 0; r < f[b].size(); ++r)
          if (((p + r) & 1) == 0) acc += f[a][p] * f[b][r] * ldexpl(1.0L, -(int)(p + r)) / (LD)(p + r + 1);
      G[(size_t)a * n + b] = acc;
    }
  return G;
}

// Symmetric eigenproblem by cyclic Jacobi rotations: A = V diag(w) V^T,
// eigenpairs sorted by decreasing eigenvalue (V column i <-> w[i]).
void jacobi_eigen(int n, std::vector<LD> A, std::vector<LD> &w, std::vector<LD> &V) {
  V.assign((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0L;
  for (int sweep = 0; sweep < 100; ++sweep) {
    LD off = 0.0L, tot = 0.0L;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (i != j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
      }
    if (off <= 1e-38L * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const LD apq = A[(size_t)p * n + q];
        if (apq == 0.0L) continue;
        const LD theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0L * apq);
        const LD t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
        const LD cs = 1.0L / sqrtl(t * t + 1.0L), sn = t * cs;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const LD akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = cs * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const LD apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = cs * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const LD vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = cs * vkp - sn * vkq;
          V[(size_t)k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
  std::vector<LD> Vs((size_t)n * n);
  w.assign(n, 0.0L);
  for (int i = 0; i < n; ++i) {
    w[i] = A[(size_t)ord[i] * n + ord[i]];
    for (int k = 0; k < n; ++k) Vs[(size_t)k * n + i] = V[(size_t)k * n + ord[i]];
  }
  V = Vs;
}

// rows x n factor F (F^T F = G) from the top `rank` eigenpairs; rows beyond
// the rank are zero
void psd_factor(int n, const std::vector<LD> &G, int rank, int rows, double *F) {
  std::vector<LD> w, V;
  jacobi_eigen(n, G, w, V);
  for (int i = 0; i < rows; ++i)
    for (int a = 0; a < n; ++a)
      F[(size_t)i * n + a] = i < rank ? (double)(sqrtl(std::max(w[i], 0.0L)) * V[(size_t)a * n + i]) : 0.0;
}

int count_parity(int lo, int hi, int e) {
  int k = 0;
  for (int p = lo; p <= hi; ++p) k += (p & 1) == e;
  return k;
}

bool tp_supported(int d, int m) { return m >= 1 && m <= (d == 3 ? 3 : (d == 2 ? 6 : 8)); }

template <class Ar, int D, int MM, bool CONS>
int launch_tp(hermite_ctx *ctx, int grid, const typename Ar::T *A, const typename Ar::T *B, float sigma, int64_t ld,
              const typename Ar::T *mats, double *partials, int64_t partials_len, double *out) {
  using T = typename Ar::T;
  using Sh = Shape<MM>;
  constexpr int NC = 1 << D;
  constexpr int NU = ipow(MM + 1, D);
  constexpr int NCI = NU + (CONS ? 0 : ipow(MM, D));
  auto kern = energy_tp_kernel<Ar, D, MM, CONS>;
  const size_t smem = sizeof(T) * (2 * Sh::EB + NC * NU + (size_t)NC * NCI * 32);
  static thread_local int configured_dev = -1;
  if (configured_dev != ctx->device) {
    if (!cuda_ok(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                 "cudaFuncSetAttribute energy_tp"))
      return HERMITE_ERR_CUDA;
    configured_dev = ctx->device;
  }
  // cells of a level held on grid g are centred at the nodes of grid 1-g
  Geometry g = make_geometry(ctx, 1 - grid);
  g.ld_src = ld;
  const int64_t ntiles = (g.nodes_dst + 31) / 32;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>({ntiles, 148 * 8, partials_len / 2}));
  const double vs = ctx->h / ctx->c;
  kern<<<(unsigned)blocks, 32 * NC, smem, ctx->stream>>>(g, mats, A, B ? B : A, B ? sigma : 0.0f, vs * vs,
                                                          partials);
  for (int f = 0; f < 2; ++f)
    reduce_tp_kernel<<<1, 256, 0, ctx->stream>>>(partials + f * blocks, blocks, ctx->formscale[f], out + f);
  return cuda_ok(ctx, cudaGetLastError(), "energy_tp_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

template <class Ar>
int launch_tp_any(hermite_ctx *ctx, int grid, const typename Ar::T *A, const typename Ar::T *B, float sigma,
                  int64_t ld, const typename Ar::T *mats, double *partials, int64_t plen, double *out) {
  const bool cons = ctx->variant == HERMITE_CONSERVATIVE;
#define HERMITE_TP_CASE(D_, M_)                                                                         \
  case D_ * 8 + M_:                                                                                     \
    return cons ? launch_tp<Ar, D_, M_, true>(ctx, grid, A, B, sigma, ld, mats, partials, plen, out)   \
                : launch_tp<Ar, D_, M_, false>(ctx, grid, A, B, sigma, ld, mats, partials, plen, out);
  switch (ctx->d * 8 + ctx->m) {
    HERMITE_TP_CASE(1, 1)
    HERMITE_TP_CASE(1, 2)
    HERMITE_TP_CASE(1, 3)
    HERMITE_TP_CASE(1, 4)
    HERMITE_TP_CASE(1, 5)
    HERMITE_TP_CASE(1, 6)
    HERMITE_TP_CASE(1, 7)
    HERMITE_TP_CASE(1, 8)
    HERMITE_TP_CASE(2, 1)
    HERMITE_TP_CASE(2, 2)
    HERMITE_TP_CASE(2, 3)
    HERMITE_TP_CASE(2, 4)
    HERMITE_TP_CASE(2, 5)
    HERMITE_TP_CASE(2, 6)
    HERMITE_TP_CASE(3, 1)
    HERMITE_TP_CASE(3, 2)
    HERMITE_TP_CASE(3, 3)
  }
#undef HERMITE_TP_CASE
  return HERMITE_ERR_UNSUPPORTED;
}

__global__ void split_copy_kernel(const double *a, int n, float2 *out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float hi = __double2float_rn(a[i]);
    out[i] = make_float2(hi, __double2float_rn(a[i] - (double)hi));
  }
}

// The matrices of both class bits for data degree m, laid out as Shape<m>
// (W, lam, F, R, S per class bit); empty if the mass matrix is not positive
// definite (not reached for m >= 1).
std::vector<double> tp_matrices(int m) {
  const int n = m + 1, nv = m;
  const int RR = (m + 2) / 2, RS = (m + 1) / 2;
  const int oL = n * n, oF = oL + n, oR = oF + nv * nv, oS = oR + RR * n, EB = oS + RS * nv;
  std::vector<double> h(2 * (size_t)EB, 0.0);
  for (int e = 0; e < 2; ++e) {
    double *b = h.data() + (size_t)e * EB;
    // plain u: simultaneous diagonalisation of the mass and stiffness matrices
    const std::vector<LD> M = gram(m, e, 0), K = gram(m, e, 1);
    std::vector<LD> L((size_t)n * n, 0.0L);  // M = L L^T
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j) {
        LD s = M[(size_t)i * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
        if (i == j) {
          if (!(s > 0.0L)) return {};
          L[(size_t)i * n + i] = sqrtl(s);
        } else {
          L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
        }
      }
    // C = L^-1 K L^-T by forward substitution on rows, then on columns
    std::vector<LD> X = K, C((size_t)n * n);
    for (int col = 0; col < n; ++col)
      for (int i = 0; i < n; ++i) {
        LD s = X[(size_t)i * n + col];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * n + col];
        X[(size_t)i * n + col] = s / L[(size_t)i * n + i];
      }
    for (int row = 0; row < n; ++row)
      for (int i = 0; i < n; ++i) {
        LD s = X[(size_t)row * n + i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * C[(size_t)row * n + k];
        C[(size_t)row * n + i] = s / L[(size_t)i * n + i];
      }
    for (int i = 0; i < n; ++i)  // symmetrise rounding
      for (int j = 0; j < i; ++j) C[(size_t)i * n + j] = C[(size_t)j * n + i] = 0.5L * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
    std::vector<LD> lam, Q;
    jacobi_eigen(n, C, lam, Q);
    for (int r = 0; r < n; ++r) {  // W = Q^T L^T
      for (int a = 0; a < n; ++a) {
        LD s = 0.0L;
        for (int i = 0; i <= a; ++i) s += Q[(size_t)i * n + r] * L[(size_t)a * n + i];
        b[r * n + a] = (double)s;
      }
      b[oL + r] = (double)std::max(lam[r], 0.0L);
    }
    psd_factor(nv, gram(m - 1, e, 0), nv, nv, b + oF);
    psd_factor(n, gram(m, e, m + 1), count_parity(m + 1, 2 * m + 1, e), RR, b + oR);
    psd_factor(nv, gram(m - 1, e, m), count_parity(m, 2 * m - 1, e), RS, b + oS);
  }
  return h;
}

}  // namespace

bool energy_tp_supported(int d, int m, int variant) {
  (void)variant;  // both methods (the conservative one for m >= 1 as well)
  return tp_supported(d, m);
}

int build_energy_tp(hermite_ctx *ctx) {
  if (!energy_tp_supported(ctx->d, ctx->m, ctx->variant)) return HERMITE_OK;
  const std::vector<double> h = tp_matrices(ctx->m);
  if (h.empty()) {
    ctx->err = "energy mass matrix not positive definite";
    return HERMITE_ERR_ARG;
  }
  if (!cuda_ok(ctx, device_alloc(&ctx->tpm, sizeof(double) * h.size()), "cudaMalloc tp matrices"))
    return HERMITE_ERR_ALLOC;
  if (!cuda_ok(ctx, cudaMemcpy(ctx->tpm, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice), "tp copy"))
    return HERMITE_ERR_CUDA;
  if (ctx->precision == HERMITE_SPLIT32) {
    if (!cuda_ok(ctx, device_alloc(&ctx->tpmf, sizeof(float2) * h.size()), "cudaMalloc tp matrices"))
      return HERMITE_ERR_ALLOC;
    split_copy_kernel<<<1, 256, 0, ctx->stream>>>(ctx->tpm, (int)h.size(), ctx->tpmf);
    if (!cuda_ok(ctx, cudaGetLastError(), "split_copy_kernel")) return HERMITE_ERR_CUDA;
  }
  return HERMITE_OK;
}

int launch_energy_tp(hermite_ctx *ctx, int grid, double *out) {
  return launch_energy_tp_pair(ctx, grid, nullptr, nullptr, 0.0f, out);
}

int launch_energy_tp_pair(hermite_ctx *ctx, int grid, const void *A, const void *B, float sigma, double *out) {
  if (!ctx->tpm) return HERMITE_ERR_UNSUPPORTED;
  if (ctx->precision == HERMITE_SPLIT32)
    return launch_tp_any<ArSplit>(ctx, grid, A ? static_cast<const float2 *>(A) : ctx->fgrid[grid],
                                  static_cast<const float2 *>(B), sigma, ctx->ld[grid], ctx->tpmf, ctx->partials,
                                  ctx->partials_len, out);
  return launch_tp_any<ArF64>(ctx, grid, A ? static_cast<const double *>(A) : ctx->grid[grid],
                              static_cast<const double *>(B), sigma, ctx->ld[grid], ctx->tpm, ctx->partials,
                              ctx->partials_len, out);
}

int launch_energy_tp_level(hermite_ctx *ctx, int grid, const double *level, int64_t ld, double *partials,
                           int64_t partials_len, double *out) {
  if (!ctx->tpm) return HERMITE_ERR_UNSUPPORTED;
  return launch_tp_any<ArF64>(ctx, grid, level, nullptr, 0.0f, ld, ctx->tpm, partials, partials_len, out);
}

}  // namespace hermite
