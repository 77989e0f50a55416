// FP64 fused half-step kernel: gather of the 2^d corner nodes of each cell
// (with the odd/even ghost polynomials of Sec. 3.1.3 applied on the fly),
// Walsh-Hadamard transform over the corners, and the per-cell operator that
// composes Hermite interpolation (Sec. 2.2), exact Taylor evolution
// (Sec. 3.1.2 / 3.3 / 4.1) and evaluation at the cell centre.
//
// Reflection symmetry of a cell gives M_s[a][b] = sign_s(a) sign_s(b) M_0[a][b]
// for corner s, so with z_q[b] = sum_s (-1)^{|q & s|} x_s[b] one operator row
// suffices:  out[a] = sum_b M_0[a][b] z_{par(a) ^ par(b)}[b].
#include <algorithm>

#include "hermite_device.cuh"
#include "hermite_internal.h"

namespace hermite {
namespace {

constexpr int kThreads = 128;

// Ghost polynomial sign for a coefficient with parity bits pb when the corner
// is a ghost in the axes of mask (Sec. 3.1.3).
__device__ __forceinline__ double ghost_sign(int bc, int mask, int pb) {
  return dev::ghost_negates(bc, mask, pb) ? -1.0 : 1.0;
}

template <int D>
__device__ __forceinline__ void wht(double *x) {
#pragma unroll
  for (int bm = 1; bm < (1 << D); bm <<= 1)
#pragma unroll
    for (int i = 0; i < (1 << D); ++i)
      if (!(i & bm)) {
        const double a = x[i], b = x[i | bm];
        x[i] = a + b;
        x[i | bm] = a - b;
      }
}

template <int D, int CH>
__global__ void __launch_bounds__(kThreads) half_step_f64_kernel(Geometry g, const double *__restrict__ M,
                                                                 int nci, int nco,
                                                                 const int8_t *__restrict__ par,
                                                                 const double *__restrict__ src,
                                                                 double *__restrict__ dst, int subtract_old) {
  extern __shared__ double smem[];
  constexpr int NC = 1 << D;
  const int chunk0 = blockIdx.y * CH;
  double *Ms = smem;                              // [nci][CH]
  double *zb = Ms + (size_t)nci * CH;             // [NC][kThreads]
  int8_t *pin = reinterpret_cast<int8_t *>(zb + NC * kThreads);
  for (int i = threadIdx.x; i < nci * CH; i += kThreads) {
    const int b = i / CH, j = i % CH, row = chunk0 + j;
    Ms[i] = row < nco ? M[(size_t)row * nci + b] : 0.0;
  }
  for (int i = threadIdx.x; i < nci; i += kThreads) pin[i] = par[i];
  int po[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) po[j] = (chunk0 + j < nco) ? par[chunk0 + j] : 0;
  __syncthreads();
  double *myz = zb + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < g.nodes_dst; t += stride) {
    int64_t idx[NC];
    int gm[NC];
    dev::cell_corners<D>(g, t, idx, gm);
    double acc[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) acc[j] = 0.0;
    for (int b = 0; b < nci; ++b) {
      const double *plane = src + (size_t)b * g.ld_src;
      const int pb = pin[b];
      double x[NC];
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        double v = __ldg(plane + idx[s]);
        if (gm[s]) v *= ghost_sign(g.bc, gm[s], pb);
        x[s] = v;
      }
      wht<D>(x);
#pragma unroll
      for (int s = 0; s < NC; ++s) myz[s * kThreads] = x[s];
      const double *mrow = Ms + (size_t)b * CH;
#pragma unroll
      for (int j = 0; j < CH; ++j) acc[j] = fma(mrow[j], myz[(po[j] ^ pb) * kThreads], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int row = chunk0 + j;
      if (row < nco) {
        double *o = dst + (size_t)row * g.ld_dst + t;
        *o = subtract_old ? acc[j] - *o : acc[j];
      }
    }
  }
}

template <int D, int CH>
int launch_dch(hermite_ctx *ctx, const Geometry &g, const double *M, int nci, int nco, const double *src,
               double *dst, bool sub) {
  auto kern = half_step_f64_kernel<D, CH>;
  const size_t smem = sizeof(double) * ((size_t)nci * CH + (1 << D) * kThreads) + nci + 16;
  static thread_local int configured_dev = -1;
  if (configured_dev != ctx->device) {
    if (!cuda_ok(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                 "cudaFuncSetAttribute"))
      return HERMITE_ERR_CUDA;
    configured_dev = ctx->device;
  }
  if (g.nodes_dst == 0) return HERMITE_OK;
  const int chunks = (nco + CH - 1) / CH;
  int64_t blocks = (g.nodes_dst + kThreads - 1) / kThreads;
  blocks = std::min<int64_t>(blocks, 148 * 64);
  dim3 grid((unsigned)blocks, (unsigned)chunks);
  kern<<<grid, kThreads, smem, ctx->stream>>>(g, M, nci, nco, ctx->par_in, src, dst, sub ? 1 : 0);
  return cuda_ok(ctx, cudaGetLastError(), "half_step_f64_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

template <int D>
int launch_d(hermite_ctx *ctx, const Geometry &g, const double *M, int nci, int nco, const double *src,
             double *dst, bool sub) {
  if (nco <= 8) return launch_dch<D, 8>(ctx, g, M, nci, nco, src, dst, sub);
  if (nco <= 16) return launch_dch<D, 16>(ctx, g, M, nci, nco, src, dst, sub);
  if (nco <= 32) return launch_dch<D, 32>(ctx, g, M, nci, nco, src, dst, sub);
  if (nco <= 64) return launch_dch<D, 64>(ctx, g, M, nci, nco, src, dst, sub);
  if (nco <= 92) return launch_dch<D, 92>(ctx, g, M, nci, nco, src, dst, sub);  // 3-D m = 3: 91 outputs
  return launch_dch<D, 96>(ctx, g, M, nci, nco, src, dst, sub);
}

// host layout [node][coef] (u block then v block) <-> SoA planes [coef][ld]
// (values copied unchanged: the device holds the paper's scaled data).
// Layout conversions through a shared-memory tile of 32 nodes x all
// coefficients: the node-major side is read or written as one contiguous run
// per tile, the coefficient-major side as 32-node runs per plane.
constexpr int kTileNodes = 32;

__global__ void to_soa_kernel(const double *__restrict__ hu, const double *__restrict__ hv, int64_t nodes,
                              int nu, int nv, double vscale, double *__restrict__ soa, int64_t ld) {
  extern __shared__ double tile[];  // [kTileNodes][nu + nv + 1]
  const int nc = nu + nv, pitch = nc + 1;
  for (int64_t n0 = (int64_t)blockIdx.x * kTileNodes; n0 < nodes; n0 += (int64_t)gridDim.x * kTileNodes) {
    const int cnt = (int)(nodes - n0 < kTileNodes ? nodes - n0 : kTileNodes);
    for (int e = threadIdx.x; e < cnt * nu; e += blockDim.x) tile[(e / nu) * pitch + e % nu] = hu[n0 * nu + e];
    for (int e = threadIdx.x; e < cnt * nv; e += blockDim.x)
      tile[(e / nv) * pitch + nu + e % nv] = hv ? vscale * hv[n0 * nv + e] : 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < nc * kTileNodes; e += blockDim.x) {
      const int k = e / kTileNodes, r = e % kTileNodes;
      if (r < cnt) soa[(int64_t)k * ld + n0 + r] = tile[r * pitch + k];
    }
    __syncthreads();
  }
}

__global__ void from_soa_kernel(const double *__restrict__ soa, int64_t ld, int64_t nodes, int nu, int nv,
                                double vscale, double *__restrict__ hu, double *__restrict__ hv) {
  extern __shared__ double tile[];  // [kTileNodes][nu + nv + 1]
  const int nc = nu + nv, pitch = nc + 1;
  for (int64_t n0 = (int64_t)blockIdx.x * kTileNodes; n0 < nodes; n0 += (int64_t)gridDim.x * kTileNodes) {
    const int cnt = (int)(nodes - n0 < kTileNodes ? nodes - n0 : kTileNodes);
    for (int e = threadIdx.x; e < nc * kTileNodes; e += blockDim.x) {
      const int k = e / kTileNodes, r = e % kTileNodes;
      if (r < cnt) tile[r * pitch + k] = soa[(int64_t)k * ld + n0 + r];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * nu; e += blockDim.x) hu[n0 * nu + e] = tile[(e / nu) * pitch + e % nu];
    for (int e = threadIdx.x; e < cnt * nv; e += blockDim.x)
      hv[n0 * nv + e] = vscale * tile[(e / nv) * pitch + nu + e % nv];
    __syncthreads();
  }
}

}  // namespace

Geometry make_geometry(const hermite_ctx *ctx, int dst) {
  Geometry g;
  g.d = ctx->d;
  g.bc = ctx->bc;
  g.dst = dst;
  g.n_dst = ctx->npts[dst];
  g.n_src = ctx->npts[1 - dst];
  g.nodes_dst = ctx->nodes[dst];
  g.ld_src = ctx->ld[1 - dst];
  g.ld_dst = ctx->ld[dst];
  return g;
}

int launch_half_step(hermite_ctx *ctx, int dst, const double *M, int nci, int nco, const double *src,
                     double *dst_arr, bool subtract_old) {
  const Geometry g = make_geometry(ctx, dst);
  switch (ctx->d) {
    case 1: return launch_d<1>(ctx, g, M, nci, nco, src, dst_arr, subtract_old);
    case 2: return launch_d<2>(ctx, g, M, nci, nco, src, dst_arr, subtract_old);
    case 3: return launch_d<3>(ctx, g, M, nci, nco, src, dst_arr, subtract_old);
  }
  return HERMITE_ERR_ARG;
}

int launch_to_device_layout(hermite_ctx *ctx, const double *hu, const double *hv, int grid, int64_t nodes,
                            double *soa, int64_t ld, int nu_count, bool has_v) {
  (void)grid;
  const int nv = has_v ? ctx->Nv : 0;
  const int64_t total = nodes * (nu_count + nv);
  if (total == 0) return HERMITE_OK;
  const int64_t blocks = std::min<int64_t>((nodes + kTileNodes - 1) / kTileNodes, 148 * 16);
  const size_t smem = sizeof(double) * kTileNodes * (nu_count + nv + 1);
  to_soa_kernel<<<(unsigned)blocks, 256, smem, ctx->stream>>>(hu, hv, nodes, nu_count, nv, 1.0, soa, ld);
  return cuda_ok(ctx, cudaGetLastError(), "to_soa_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

int launch_to_host_layout(hermite_ctx *ctx, const double *soa, int64_t ld, int64_t nodes, double *hu,
                          double *hv, bool want_v) {
  const int nv = want_v ? ctx->Nv : 0;
  const int64_t total = nodes * (ctx->Nu + nv);
  if (total == 0) return HERMITE_OK;
  const int64_t blocks = std::min<int64_t>((nodes + kTileNodes - 1) / kTileNodes, 148 * 16);
  const size_t smem = sizeof(double) * kTileNodes * (ctx->Nu + nv + 1);
  from_soa_kernel<<<(unsigned)blocks, 256, smem, ctx->stream>>>(soa, ld, nodes, ctx->Nu, nv, 1.0, hu, hv);
  return cuda_ok(ctx, cudaGetLastError(), "from_soa_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

}  // namespace hermite
