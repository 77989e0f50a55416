// L2 error of the cell interpolant I_m u against an exact solution (the error
// measure of Sec. 5.1: the piecewise interpolant of the nodal data compared
// with the exact solution at quadrature points "on a sufficiently fine grid"),
// reduced in FP64 on the device over a caller's list of cells.
//
// The interpolant of one cell is written in the 1-D two-point Hermite bases of
// Sec. 2.2: for data of degree m given at the left end (s = xi + 1/2 = 0),
//   phi_l(s) = s^l (1-s)^{m+1} sum_{k=0}^{m-l} binom(m+k, k) s^k,
// whose Taylor coefficients at s = 0 are delta_{jl} for j <= m and which
// vanishes to order m at s = 1; the right-end function of order l is
// (-1)^l phi_l(1 - s).  The value at a tensor quadrature point is then
//   I u(p) = sum_corners sum_k x_corner[k] prod_i B_i(p_i, corner bit i, k_i).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hermite_device.cuh"
#include "hermite_internal.h"

namespace hermite {
namespace {

constexpr int kErrThreads = 128;
constexpr int kMaxQ = 16;  // quadrature points per axis

template <int D>
__global__ void __launch_bounds__(kErrThreads) l2_error_kernel(Geometry g, const double *__restrict__ level,
                                                               int m, int Nu, const int8_t *__restrict__ par,
                                                               int64_t ncells, const int64_t *__restrict__ cells,
                                                               int nq, const double *__restrict__ basis,
                                                               const double *__restrict__ wq,
                                                               const double *__restrict__ exact, double *partials) {
  constexpr int NC = 1 << D;
  extern __shared__ double sm[];
  const int E = m + 1;
  double *xs = sm;                       // [NC][Nu] corner data with ghost signs
  double *B = xs + NC * Nu;              // [nq][2][E] basis values
  double *W = B + nq * 2 * E;            // [nq] weights
  __shared__ double red[2][kErrThreads];
  for (int i = threadIdx.x; i < nq * 2 * E; i += kErrThreads) B[i] = basis[i];
  for (int i = threadIdx.x; i < nq; i += kErrThreads) W[i] = wq[i];
  int npts = 1;
  for (int i = 0; i < D; ++i) npts *= nq;
  double err2 = 0.0, norm2 = 0.0;
  for (int64_t ci = blockIdx.x; ci < ncells; ci += gridDim.x) {
    const int64_t t = cells ? cells[ci] : ci;
    if (t < 0 || t >= g.nodes_dst) continue;  // not a cell of this level (same for the whole block)
    int64_t idx[NC];
    int gm[NC];
    dev::cell_corners<D>(g, t, idx, gm);
    const double wc = (double)dev::cell_weight<D>(g, t);
    __syncthreads();  // previous cell's corner data no longer in use
    for (int e = threadIdx.x; e < NC * Nu; e += kErrThreads) {
      const int s = e / Nu, k = e % Nu;
      double v = level[(size_t)k * g.ld_src + idx[s]];
      if (gm[s] && dev::ghost_negates(g.bc, gm[s], par[k])) v = -v;
      xs[e] = v;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < npts; p += kErrThreads) {
      int pi[D];
      double wt = 1.0;
      int r = p;
#pragma unroll
      for (int i = D - 1; i >= 0; --i) {
        pi[i] = r % nq;
        r /= nq;
        wt *= W[pi[i]];
      }
      double val = 0.0;
      for (int s = 0; s < NC; ++s) {
        const double *xc = xs + s * Nu;
        for (int k = 0; k < Nu; ++k) {
          int kr = k;
          double prod = xc[k];
#pragma unroll
          for (int i = D - 1; i >= 0; --i) {
            const int ki = kr % E;
            kr /= E;
            const int bit = (s >> (D - 1 - i)) & 1;
            prod *= B[(pi[i] * 2 + bit) * E + ki];
          }
          val += prod;
        }
      }
      const double ex = exact[(size_t)ci * npts + p];
      const double e = val - ex;
      err2 += wc * wt * e * e;
      norm2 += wc * wt * ex * ex;
    }
  }
  red[0][threadIdx.x] = err2;
  red[1][threadIdx.x] = norm2;
  __syncthreads();
  for (int off = kErrThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      red[0][threadIdx.x] += red[0][threadIdx.x + off];
      red[1][threadIdx.x] += red[1][threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = red[0][0];
    partials[2 * blockIdx.x + 1] = red[1][0];
  }
}

double hermite_left_basis(int m, int l, double s) {
  double sum = 0.0, bin = 1.0;  // binom(m + k, k)
  for (int k = 0; k <= m - l; ++k) {
    sum += bin * std::pow(s, k);
    bin = bin * (double)(m + k + 1) / (double)(k + 1);
  }
  return std::pow(s, l) * std::pow(1.0 - s, m + 1) * sum;
}

}  // namespace

int launch_l2_error(hermite_ctx *ctx, int grid, int64_t ncells, const int64_t *cells, int nq, const double *xq,
                    const double *wq, const double *exact, double out[2]) {
  if (nq < 1 || nq > kMaxQ) {
    ctx->err = "hermite_l2_error: nq must be in [1, 16]";
    return HERMITE_ERR_ARG;
  }
  const Geometry g0 = make_geometry(ctx, 1 - grid);
  if (ncells < 0 || (!cells && ncells != g0.nodes_dst)) {
    ctx->err = "hermite_l2_error: without a cell list ncells must be the number of cells";
    return HERMITE_ERR_ARG;
  }
  out[0] = out[1] = 0.0;
  if (ncells == 0) return HERMITE_OK;
  const int E = ctx->m + 1;
  std::vector<double> basis((size_t)nq * 2 * E);
  for (int p = 0; p < nq; ++p)
    for (int l = 0; l < E; ++l) {
      basis[(p * 2 + 0) * E + l] = hermite_left_basis(ctx->m, l, xq[p] + 0.5);
      basis[(p * 2 + 1) * E + l] = ((l & 1) ? -1.0 : 1.0) * hermite_left_basis(ctx->m, l, 0.5 - xq[p]);
    }
  const int blocks = (int)std::min<int64_t>(ncells, 148 * 8);
  double *dbuf = nullptr;
  const size_t nb = basis.size() + nq + 2 * (size_t)blocks;
  if (!cuda_ok(ctx, device_alloc(&dbuf, sizeof(double) * nb), "cudaMalloc l2 error")) return HERMITE_ERR_ALLOC;
  double *dbasis = dbuf, *dw = dbuf + basis.size(), *dpart = dw + nq;
  std::vector<double> part(2 * (size_t)blocks);
  int rc = HERMITE_OK;
  if (!cuda_ok(ctx, cudaMemcpyAsync(dbasis, basis.data(), sizeof(double) * basis.size(), cudaMemcpyHostToDevice,
                                    ctx->stream), "copy basis") ||
      !cuda_ok(ctx, cudaMemcpyAsync(dw, wq, sizeof(double) * nq, cudaMemcpyHostToDevice, ctx->stream), "copy w")) {
    rc = HERMITE_ERR_CUDA;
  } else {
    Geometry g = g0;
    const size_t smem = sizeof(double) * ((size_t)(1 << ctx->d) * ctx->Nu + (size_t)nq * 2 * E + nq);
    const double *lev = ctx->grid[grid];
    switch (ctx->d) {
      case 1:
        l2_error_kernel<1><<<blocks, kErrThreads, smem, ctx->stream>>>(g, lev, ctx->m, ctx->Nu, ctx->par_in, ncells,
                                                                       cells, nq, dbasis, dw, exact, dpart);
        break;
      case 2:
        l2_error_kernel<2><<<blocks, kErrThreads, smem, ctx->stream>>>(g, lev, ctx->m, ctx->Nu, ctx->par_in, ncells,
                                                                       cells, nq, dbasis, dw, exact, dpart);
        break;
      default:
        l2_error_kernel<3><<<blocks, kErrThreads, smem, ctx->stream>>>(g, lev, ctx->m, ctx->Nu, ctx->par_in, ncells,
                                                                       cells, nq, dbasis, dw, exact, dpart);
        break;
    }
    if (!cuda_ok(ctx, cudaGetLastError(), "l2_error_kernel") ||
        !cuda_ok(ctx, cudaMemcpyAsync(part.data(), dpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                                      ctx->stream), "copy partials") ||
        !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "l2 error sync"))
      rc = HERMITE_ERR_CUDA;
  }
  cudaFree(dbuf);
  if (rc) return rc;
  long double e2 = 0, n2 = 0;
  for (int b = 0; b < blocks; ++b) {
    e2 += part[2 * b];
    n2 += part[2 * b + 1];
  }
  const double hd = std::pow(ctx->h, ctx->d);
  out[0] = (double)(e2 * hd);
  out[1] = (double)(n2 * hd);
  return HERMITE_OK;
}

}  // namespace hermite
