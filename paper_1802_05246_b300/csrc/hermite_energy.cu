// FP64 energy reduction (Sec. 3.2 Eq. stable1, Sec. 3.3 Eq. stable2,
// Sec. 4.2).  Each cell's energy is an exact integral of products of its
// interpolant polynomials, i.e. a quadratic (or bilinear) form in the corner
// data.  After the Walsh-Hadamard transform over corners the form splits into
// 2^d parity classes:  E_cell = sum_c y_c(A)^T Q_c y_c(B),
// y_c[b] = z_{c ^ par(b)}[b].  Q_c is built once per context by the set-up
// kernels.  Block partial sums are reduced in a fixed order (bit-reproducible).
#include <algorithm>
#include <mutex>
#include <string>

#include "hermite_device.cuh"
#include "hermite_internal.h"

namespace hermite {
namespace {

constexpr int kEThreads = 64;

// corners of the cell centred at target node t and its weight in the sum
template <int D>
__device__ __forceinline__ void cell_corners_e(const Geometry &g, int64_t t, int64_t *idx, int *gmask,
                                               double *weight) {
  dev::cell_corners<D>(g, t, idx, gmask);
  *weight = dev::cell_weight<D>(g, t);
}

__device__ __forceinline__ double gsign(int bc, int mask, int pb) {
  return dev::ghost_negates(bc, mask, pb) ? -1.0 : 1.0;
}

// class-c component of the corner Walsh-Hadamard transform of coefficient b
template <int D>
__device__ __forceinline__ double class_value(const double *__restrict__ plane, const int64_t *idx, const int *gm,
                                              int bc, int pb, int q, int stride = 1) {
  double acc = 0.0;
#pragma unroll
  for (int s = 0; s < (1 << D); ++s) {
    double v = __ldg(plane + idx[s * stride]);
    const int gs = gm[s * stride];
    if (gs) v *= gsign(bc, gs, pb);
    acc += (__popc(q & s) & 1) ? -v : v;
  }
  return acc;
}

template <int D>
__global__ void __launch_bounds__(kEThreads) energy_kernel(Geometry g, const double *__restrict__ Q, int nq,
                                                           const int8_t *__restrict__ par,
                                                           const double *__restrict__ A,
                                                           const double *__restrict__ B, double *partials) {
  extern __shared__ double sm[];
  const int c = blockIdx.y;
  double *Qs = sm;                              // [nq][nq]
  double *yb = Qs + (size_t)nq * nq;            // [nq][kEThreads]
  int8_t *pin = reinterpret_cast<int8_t *>(yb + (size_t)nq * kEThreads);
  __shared__ double red[kEThreads];
  const double *Qc = Q + (size_t)c * nq * nq;
  for (int i = threadIdx.x; i < nq * nq; i += kEThreads) Qs[i] = Qc[i];
  for (int i = threadIdx.x; i < nq; i += kEThreads) pin[i] = par[i];
  __syncthreads();
  double total = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kEThreads;
  for (int64_t t = (int64_t)blockIdx.x * kEThreads + threadIdx.x; t < g.nodes_dst; t += stride) {
    int64_t idx[1 << D];
    int gm[1 << D];
    double w;
    cell_corners_e<D>(g, t, idx, gm, &w);
    for (int b = 0; b < nq; ++b)
      yb[b * kEThreads + threadIdx.x] =
          class_value<D>(B + (size_t)b * g.ld_src, idx, gm, g.bc, pin[b], c ^ pin[b]);
    double cell = 0.0;
    for (int b = 0; b < nq; ++b) {
      const bool quad = (A == B);
      const double ya =
          quad ? yb[b * kEThreads + threadIdx.x]
               : class_value<D>(A + (size_t)b * g.ld_src, idx, gm, g.bc, pin[b], c ^ pin[b]);
      if (ya == 0.0) continue;
      const double *qrow = Qs + (size_t)b * nq;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      // a quadratic form needs only the upper triangle of the symmetric Q_c:
      // y^T Q y = sum_b y_b (Q_bb y_b + 2 sum_{k>b} Q_bk y_k)
      int k = quad ? b + 1 : 0;
      for (; k + 3 < nq; k += 4) {
        s0 = fma(qrow[k], yb[k * kEThreads + threadIdx.x], s0);
        s1 = fma(qrow[k + 1], yb[(k + 1) * kEThreads + threadIdx.x], s1);
        s2 = fma(qrow[k + 2], yb[(k + 2) * kEThreads + threadIdx.x], s2);
        s3 = fma(qrow[k + 3], yb[(k + 3) * kEThreads + threadIdx.x], s3);
      }
      for (; k < nq; ++k) s0 = fma(qrow[k], yb[k * kEThreads + threadIdx.x], s0);
      const double off = (s0 + s1) + (s2 + s3);
      cell = quad ? fma(ya, fma(qrow[b], ya, 2.0 * off), cell) : fma(ya, off, cell);
    }
    total = fma(w, cell, total);
  }
  red[threadIdx.x] = total;
  __syncthreads();
  for (int off = kEThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// Factored form Q_c = L_c^T L_c (L_c upper triangular in a permuted column
// order, or a short dense low-rank factor): a block takes a tile of 64 cells
// and one class, stages their class vectors y_c (columns permuted) in shared
// memory, and thread (cell group cg, row group rg) forms z = L_r . y for four
// cells and rows r = rg, rg+16, ... starting at column r when L is
// triangular.  E_cell = sum_r z_r(A) z_r(B).
constexpr int kFTile = 64;
constexpr int kFThreads = 256;

template <int D>
__global__ void __launch_bounds__(kFThreads) energy_factored_kernel(
    Geometry g, const double *__restrict__ L, int lrows, int rmax, int tri, const int16_t *__restrict__ perm, int nq,
    const int8_t *__restrict__ par, const double *__restrict__ A, const double *__restrict__ B, double *partials) {
  constexpr int NC = 1 << D;
  extern __shared__ double sm[];
  const int c = blockIdx.y;
  const bool quad = (A == B);
  const int ld = nq | 1;  // odd row stride: conflict-free column reads
  double *Ls = sm;                                    // [rmax][nq]
  double *YA = Ls + (size_t)rmax * nq;                // [kFTile][ld]
  double *YB = quad ? YA : YA + (size_t)kFTile * ld;  // [kFTile][ld]
  double *cw = YA + (size_t)(quad ? 1 : 2) * kFTile * ld;  // [kFTile]
  int64_t *cidx = reinterpret_cast<int64_t *>(cw + kFTile);  // [NC][kFTile]: lanes of a warp read consecutive words
  int *cgm = reinterpret_cast<int *>(cidx + kFTile * NC);    // [NC][kFTile]
  int16_t *ps = reinterpret_cast<int16_t *>(cgm + kFTile * NC);  // [nq]
  int8_t *pin = reinterpret_cast<int8_t *>(ps + nq);             // [nq]
  __shared__ double red[kFThreads];
  const double *Lc = L + (size_t)c * lrows * nq;
  for (int i = threadIdx.x; i < rmax * nq; i += kFThreads) Ls[i] = Lc[i];
  for (int i = threadIdx.x; i < nq; i += kFThreads) {
    ps[i] = perm[(size_t)c * nq + i];
    pin[i] = par[i];
  }
  const int cg = threadIdx.x & 15, rg = threadIdx.x >> 4;
  double total = 0.0;
  const int64_t ntiles = (g.nodes_dst + kFTile - 1) / kFTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < kFTile) {
      const int64_t t = tile * kFTile + threadIdx.x;
      int64_t li[NC];
      int lg[NC];
      double w = 0.0;
      if (t < g.nodes_dst) {
        cell_corners_e<D>(g, t, li, lg, &w);
      } else {
        for (int s = 0; s < NC; ++s) {
          li[s] = 0;
          lg[s] = 0;
        }
      }
      for (int s = 0; s < NC; ++s) {
        cidx[s * kFTile + threadIdx.x] = li[s];
        cgm[s * kFTile + threadIdx.x] = lg[s];
      }
      cw[threadIdx.x] = w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kFTile * nq; e += kFThreads) {
      // consecutive lanes take consecutive cells of one coefficient plane so
      // that their corner gathers coalesce
      const int i = e % kFTile, k = e / kFTile, b = ps[k];
      YA[i * ld + k] = class_value<D>(A + (size_t)b * g.ld_src, cidx + i, cgm + i, g.bc, pin[b], c ^ pin[b], kFTile);
      if (!quad)
        YB[i * ld + k] = class_value<D>(B + (size_t)b * g.ld_src, cidx + i, cgm + i, g.bc, pin[b], c ^ pin[b], kFTile);
    }
    __syncthreads();
    double e4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = rg; r < rmax; r += 16) {
      const double *lrow = Ls + (size_t)r * nq;
      double za[4] = {0.0, 0.0, 0.0, 0.0}, zb[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = tri ? r : 0; k < nq; ++k) {
        const double l = lrow[k];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          za[i] = fma(l, YA[(cg + 16 * i) * ld + k], za[i]);
          if (!quad) zb[i] = fma(l, YB[(cg + 16 * i) * ld + k], zb[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) e4[i] = fma(za[i], quad ? za[i] : zb[i], e4[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) total = fma(cw[cg + 16 * i], e4[i], total);
  }
  red[threadIdx.x] = total;
  __syncthreads();
  for (int off = kFThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// single-block fixed-order sum of n partials, scaled
__global__ void reduce_kernel(const double *partials, int64_t n, double scale, double *out) {
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

// The quadratic form `form` of levels A, B over the cells of geometry g: the
// factored kernel (sums of squares, no cancellation) where the context has
// the factors, else the dense per-class form.  Block partial sums go to
// `partials` (at most partials_len doubles).
template <int D>
int launch_energy_d(hermite_ctx *ctx, const Geometry &g, int form, const double *A, const double *B,
                    double *result_slot, double *partials, int64_t partials_len) {
  const int nq = ctx->nq[form];
  const size_t smem = sizeof(double) * ((size_t)nq * nq + (size_t)nq * kEThreads) + nq + 16;
  static thread_local int configured_dev = -1;
  if (configured_dev != ctx->device) {
    if (!cuda_ok(ctx,
                 cudaFuncSetAttribute(energy_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024),
                 "cudaFuncSetAttribute energy"))
      return HERMITE_ERR_CUDA;
    configured_dev = ctx->device;
  }
  const int nclass = 1 << D;
  int64_t blocks = std::max<int64_t>(1, (g.nodes_dst + kEThreads - 1) / kEThreads);
  blocks = std::min<int64_t>(blocks, partials_len / nclass);
  dim3 grid((unsigned)blocks, (unsigned)nclass);
  if (ctx->L[form]) {
    static thread_local int configured_f = -1;
    if (configured_f != ctx->device) {
      if (!cuda_ok(ctx,
                   cudaFuncSetAttribute(energy_factored_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        220 * 1024),
                   "cudaFuncSetAttribute energy factored"))
        return HERMITE_ERR_CUDA;
      configured_f = ctx->device;
    }
    const int rmax = ctx->rmax[form];
    const int ld = nq | 1;
    const size_t smem_f = sizeof(double) * ((size_t)rmax * nq + (A == B ? 1 : 2) * (size_t)kFTile * ld + kFTile) +
                          sizeof(int64_t) * kFTile * nclass + sizeof(int) * kFTile * nclass + 3 * nq + 16;
    int64_t fblocks = std::max<int64_t>(1, (g.nodes_dst + kFTile - 1) / kFTile);
    fblocks = std::min<int64_t>(fblocks, partials_len / nclass);
    dim3 fgrid((unsigned)fblocks, (unsigned)nclass);
    energy_factored_kernel<D><<<fgrid, kFThreads, smem_f, ctx->stream>>>(
        g, ctx->L[form], ctx->lrows[form], rmax, ctx->ltri[form], ctx->lperm[form], nq, ctx->par_in, A, B,
        partials);
    reduce_kernel<<<1, 256, 0, ctx->stream>>>(partials, fblocks * nclass, ctx->formscale[form], result_slot);
    return cuda_ok(ctx, cudaGetLastError(), "energy_factored_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
  } else {
    energy_kernel<D><<<grid, kEThreads, smem, ctx->stream>>>(g, ctx->Q[form], nq, ctx->par_in, A, B, partials);
  }
  reduce_kernel<<<1, 256, 0, ctx->stream>>>(partials, blocks * nclass, ctx->formscale[form], result_slot);
  return cuda_ok(ctx, cudaGetLastError(), "energy_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

}  // namespace

int launch_energy_form(hermite_ctx *ctx, int form, int g, const double *A, const double *B, double *result_slot) {
  // cells of a level held on grid g are centred at the nodes of grid 1-g
  const Geometry geo = make_geometry(ctx, 1 - g);
  switch (ctx->d) {
    case 1: return launch_energy_d<1>(ctx, geo, form, A, B, result_slot, ctx->partials, ctx->partials_len);
    case 2: return launch_energy_d<2>(ctx, geo, form, A, B, result_slot, ctx->partials, ctx->partials_len);
    case 3: return launch_energy_d<3>(ctx, geo, form, A, B, result_slot, ctx->partials, ctx->partials_len);
  }
  return HERMITE_ERR_ARG;
}

}  // namespace hermite

// ---------------------------------------------------------------------------
// Allocation-free energy entry point.  Callers that must not allocate device
// memory at the point of the call (for example code running inside a region
// where cudaMalloc is forbidden or would synchronise the device, or a host
// that only hands the library pre-existing buffers) get the same reduction
// with its block partial sums in this file-scope array instead of the
// context's own scratch buffer.  The array lives for as long as the library
// is loaded, on every device that uses this entry point.
namespace hermite {
namespace {

constexpr int64_t kNoAllocMaxCells = int64_t(1) << 21;  // 2,097,152 cells
constexpr int64_t kNoAllocPartials = (kNoAllocMaxCells / kEThreads) * 8;  // 2 MB of doubles

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
double *noalloc_scratch(hermite_ctx *ctx, int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (!cuda_ok(ctx, cudaGetSymbolAddress(&p, g_noalloc_partials), "cudaGetSymbolAddress")) return nullptr;
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace
}  // namespace hermite

extern "C" int hermite_energy_noalloc(hermite_ctx *ctx, int grid, const double *level, int64_t ld,
                                      double *out_dev) {
  using namespace hermite;
  if (!ctx) return HERMITE_ERR_ARG;
  if ((grid != 0 && grid != 1) || !level || !out_dev || ld < ctx->nodes[grid]) {
    ctx->err = "hermite_energy_noalloc: bad grid, NULL pointer or ld < nodes";
    return HERMITE_ERR_ARG;
  }
  if (!ctx->has_energy) {
    ctx->err = "this context was created without energy forms";
    return HERMITE_ERR_STATE;
  }
  // cells of a level held on grid g are centred at the nodes of grid 1-g
  const int64_t cells = ctx->nodes[1 - grid];
  if (cells > kNoAllocMaxCells) {
    ctx->err = "hermite_energy_noalloc: " + std::to_string(cells) + " cells exceed the maximum of " +
               std::to_string(kNoAllocMaxCells) + " supported without allocation";
    return HERMITE_ERR_ARG;
  }
  int dev = -1;
  if (!cuda_ok(ctx, cudaGetDevice(&dev), "cudaGetDevice")) return HERMITE_ERR_CUDA;
  if (dev != ctx->device || dev < 0 || dev >= kMaxDevices) {
    ctx->err = "hermite_energy_noalloc: the context's device must be current";
    return HERMITE_ERR_ARG;
  }
  double *partials = noalloc_scratch(ctx, dev);
  if (!partials) return HERMITE_ERR_CUDA;
  // dissipative contexts: the sum-factorised kernel, both forms in one pass
  const int tp = launch_energy_tp_level(ctx, grid, level, ld, partials, kNoAllocPartials, out_dev);
  if (tp != HERMITE_ERR_UNSUPPORTED) return tp;
  Geometry g = make_geometry(ctx, 1 - grid);
  g.ld_src = ld;
  for (int f = 0; f < kNumForms; ++f) {
    int rc;
    switch (ctx->d) {
      case 1: rc = launch_energy_d<1>(ctx, g, f, level, level, out_dev + f, partials, kNoAllocPartials); break;
      case 2: rc = launch_energy_d<2>(ctx, g, f, level, level, out_dev + f, partials, kNoAllocPartials); break;
      default: rc = launch_energy_d<3>(ctx, g, f, level, level, out_dev + f, partials, kNoAllocPartials); break;
    }
    if (rc) return rc;
  }
  return HERMITE_OK;
}
