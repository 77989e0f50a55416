// Split-precision half-step: state and operator held as unevaluated sums of
// two FP32 numbers (hi + lo, ~48 significant bits), every multiply-add formed
// from three split products -- hi*hi exactly (FMA residual), hi*lo, lo*hi --
// and accumulated with an error-free two-sum.  Same algorithm as the FP64
// kernel (corner gather with ghost signs, Walsh-Hadamard transform over the
// 2^d corners, one operator row per output), run on the FP32 pipe.
//
// Work split inside a block of 32 target nodes and 2^d warps: in phase A warp
// w transforms input coefficient b0+w for the 32 nodes and writes its 2^d
// class components to shared memory; in phase B warp w accumulates S output
// slots, the first P of one parity class and the rest of a second one (the
// classes differ in size, so packing two per warp keeps the warps' slot
// counts, and the padding multiply-adds, small).  Each corner value is loaded
// and transformed once per node.
#include <algorithm>
#include <vector>

#include "hermite_device.cuh"
#include "hermite_internal.h"

namespace hermite {
namespace {

using dev::df_add;
using dev::df_fma;
using dev::df_neg;
using dev::df_norm;
using dev::ghost_negates;

template <int D, int S, int P, int NBUF>
__device__ __forceinline__ void half_step_split_body(
    const Geometry &g, const float2 *__restrict__ Mp, const int16_t *__restrict__ prow,
    const int8_t *__restrict__ pcls, int nci, const int8_t *__restrict__ par, const float2 *__restrict__ src,
    float2 *__restrict__ dst, int subtract_old) {
  static_assert(S % 2 == 0 && P % 2 == 0 && P > 0 && P <= S, "slot layout: slot pairs never straddle the classes");
  constexpr int NC = 1 << D;
  constexpr int NT = 32 * NC;
  constexpr int YSZ = NC * NC * 32;
  extern __shared__ float2 sm2[];
  float2 *Ms = sm2;                           // [NC warp][nci][S]
  float2 *Ybuf = Ms + (size_t)NC * nci * S;   // NBUF x [NC beta slot][NC class][32]
  int8_t *pin = reinterpret_cast<int8_t *>(Ybuf + NBUF * YSZ);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < NC * nci * S; i += NT) Ms[i] = Mp[i];
  for (int i = threadIdx.x; i < nci; i += NT) pin[i] = par[i];
  // one class per warp (P = S): warp w holds class w
  const int cA = P == S ? w : pcls[2 * w], cB = P == S ? w : pcls[2 * w + 1];
  __syncthreads();
  const int64_t nblk = (g.nodes_dst + 31) / 32;
  const int nchunks = (nci + NC - 1) / NC;
  for (int64_t nb = blockIdx.x; nb < nblk; nb += gridDim.x) {
    const int64_t t = nb * 32 + lane;
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
    // phase A is split in two so that corner loads run ahead: load() fetches
    // coefficient b0 + w of the chunk into registers, transform() applies the
    // ghost signs and the corner transform and writes the class components
    float2 x[NC];
    auto load = [&](int b0) {
      const int b = b0 + w;
      if (b >= nci) return;
      const float2 *plane = src + (size_t)b * g.ld_src;
#pragma unroll
      for (int s = 0; s < NC; ++s) x[s] = plane[idx[s]];
    };
    auto transform = [&](int b0, float2 *Y) {
      const int b = b0 + w;
      if (b >= nci) return;
      const int pb = pin[b];
#pragma unroll
      for (int s = 0; s < NC; ++s)
        if (gm[s] && ghost_negates(g.bc, gm[s], pb)) x[s] = df_neg(x[s]);
#pragma unroll
      for (int bm = 1; bm < NC; bm <<= 1)
#pragma unroll
        for (int i = 0; i < NC; ++i)
          if (!(i & bm)) {
            const float2 a = x[i], c = x[i | bm];
            x[i] = df_add(a, c);
            x[i | bm] = df_add(a, df_neg(c));
          }
#pragma unroll
      for (int q = 0; q < NC; ++q) Y[(w * NC + q) * 32 + lane] = x[q];
    };
    // slot pairs (2k, 2k+1): hi parts in ahi[k], lo parts in alo[k]
    float2 ahi[S / 2], alo[S / 2];
#pragma unroll
    for (int k = 0; k < S / 2; ++k) ahi[k] = alo[k] = make_float2(0.f, 0.f);
    load(0);
    transform(0, Ybuf);
    if (nchunks > 1) load(NC);
    __syncthreads();
    for (int ch = 0; ch < nchunks; ++ch) {
      const float2 *Y = Ybuf + (NBUF == 2 ? (ch & 1) * YSZ : 0);
      const int b0 = ch * NC;
      const int kmax = min(NC, nci - b0);
      // every slot runs (unused slots multiply zeros) so that the S
      // independent accumulator chains interleave; a slot pair's operator
      // entries (hi, hi, lo, lo) are read 16 bytes at a time
      auto consume = [&](int k) {
        const int bb = b0 + k;
        const int pb = pin[bb];
        const float2 ya = Y[(k * NC + (cA ^ pb)) * 32 + lane];
        const float2 yb = P < S ? Y[(k * NC + (cB ^ pb)) * 32 + lane] : ya;
        const float2 yah = make_float2(ya.x, ya.x), yal = make_float2(ya.y, ya.y), yan = make_float2(-ya.x, -ya.x);
        const float2 ybh = make_float2(yb.x, yb.x), ybl = make_float2(yb.y, yb.y), ybn = make_float2(-yb.x, -yb.x);
        const float4 *mrow = reinterpret_cast<const float4 *>(Ms + ((size_t)w * nci + bb) * S);
#pragma unroll
        for (int j = 0; j < S / 2; ++j) {
          const float4 mm = mrow[j];
          if constexpr (S == 2) {
            // one slot pair: forming the packed copies of y would cost as much
            // as the packing saves (measured), so the scalar form
            float2 a0 = make_float2(ahi[j].x, alo[j].x), a1 = make_float2(ahi[j].y, alo[j].y);
            df_fma(a0, make_float2(mm.x, mm.z), ya);
            df_fma(a1, make_float2(mm.y, mm.w), ya);
            ahi[j] = make_float2(a0.x, a1.x);
            alo[j] = make_float2(a0.y, a1.y);
          } else if (2 * j < P) {
            dev::df_fma_x2(ahi[j], alo[j], make_float2(mm.x, mm.y), make_float2(mm.z, mm.w), yah, yal, yan);
          } else {
            dev::df_fma_x2(ahi[j], alo[j], make_float2(mm.x, mm.y), make_float2(mm.z, mm.w), ybh, ybl, ybn);
          }
        }
      };
      if (kmax == NC) {
#pragma unroll
        for (int k = 0; k < NC; ++k) consume(k);
      } else {
        for (int k = 0; k < kmax; ++k) consume(k);
      }
      // the next chunk (already loaded) goes into the other buffer, or, with
      // one buffer, replaces this one once every warp has consumed it; the
      // loads of the chunk after are issued before the barrier.  One buffer is
      // used where it is what lets two blocks share an SM (3-D, m = 3: 110 KB
      // instead of 125 KB), so that they cover each other's barriers.
      if (NBUF == 1) __syncthreads();
      if (ch + 1 < nchunks) {
        transform((ch + 1) * NC, Ybuf + (NBUF == 2 ? ((ch + 1) & 1) * YSZ : 0));
        if (ch + 2 < nchunks) load((ch + 2) * NC);
      }
      __syncthreads();
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const int row = prow[w * S + j];
        if (row >= 0) {
          float2 *o = dst + (size_t)row * g.ld_dst + t;
          const float2 a = (j & 1) ? make_float2(ahi[j / 2].y, alo[j / 2].y) : make_float2(ahi[j / 2].x, alo[j / 2].x);
          float2 r = df_norm(a);
          if (subtract_old) r = df_norm(df_add(r, df_neg(*o)));
          *o = r;
        }
      }
    }
  }
}

// Two entry points: two exchange buffers with the compiler's own register
// budget, and one buffer with a budget that keeps two blocks per SM.
template <int D, int S, int P>
__global__ void __launch_bounds__(32 << D) half_step_split_kernel(
    Geometry g, const float2 *__restrict__ Mp, const int16_t *__restrict__ prow, const int8_t *__restrict__ pcls,
    int nci, const int8_t *__restrict__ par, const float2 *__restrict__ src, float2 *__restrict__ dst,
    int subtract_old) {
  half_step_split_body<D, S, P, 2>(g, Mp, prow, pcls, nci, par, src, dst, subtract_old);
}

template <int D, int S, int P>
__global__ void __launch_bounds__(32 << D, 2) half_step_split_1buf_kernel(
    Geometry g, const float2 *__restrict__ Mp, const int16_t *__restrict__ prow, const int8_t *__restrict__ pcls,
    int nci, const int8_t *__restrict__ par, const float2 *__restrict__ src, float2 *__restrict__ dst,
    int subtract_old) {
  half_step_split_body<D, S, P, 1>(g, Mp, prow, pcls, nci, par, src, dst, subtract_old);
}

template <int D, int S, int P, int NBUF>
int launch_split_dnb(hermite_ctx *ctx, const Geometry &g, const float2 *src, float2 *dst, bool sub, size_t smem) {
  auto kern = [] {
    if constexpr (NBUF == 2)
      return half_step_split_kernel<D, S, P>;
    else
      return half_step_split_1buf_kernel<D, S, P>;
  }();
  static thread_local int configured_dev = -1;
  if (configured_dev != ctx->device) {
    if (!cuda_ok(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024),
                 "cudaFuncSetAttribute split"))
      return HERMITE_ERR_CUDA;
    configured_dev = ctx->device;
  }
  if (g.nodes_dst == 0) return HERMITE_OK;
  const int64_t nblk = (g.nodes_dst + 31) / 32;
  const int64_t blocks = std::min<int64_t>(nblk, 148 * 16);
  kern<<<(unsigned)blocks, 32 << D, smem, ctx->stream>>>(g, ctx->Mp, ctx->prow, ctx->pcls, ctx->nci, ctx->par_in,
                                                          src, dst, sub ? 1 : 0);
  return cuda_ok(ctx, cudaGetLastError(), "half_step_split_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

// Two exchange buffers, unless a single one is what lets two blocks share an
// SM (3-D, m = 3 with one class per warp: 110 KB instead of 125 KB); then the
// blocks cover each other's extra barrier.
template <int D, int S, int P>
int launch_split_dn(hermite_ctx *ctx, const Geometry &g, const float2 *src, float2 *dst, bool sub) {
  constexpr int NC = 1 << D;
  const size_t base = sizeof(float2) * (size_t)NC * ctx->nci * S + ctx->nci + 16;
  const size_t ybytes = sizeof(float2) * NC * NC * 32;
  if constexpr (D == 3) {
    constexpr size_t kTwoBlocks = 112 * 1024;
    if (base + 2 * ybytes > kTwoBlocks && base + ybytes <= kTwoBlocks)
      return launch_split_dnb<D, S, P, 1>(ctx, g, src, dst, sub, base + ybytes);
  }
  return launch_split_dnb<D, S, P, 2>(ctx, g, src, dst, sub, base + 2 * ybytes);
}

// Slot layouts (S slots per warp, the first P of one class) with a compiled
// kernel: one class per warp (P = S), and for d > 1 two classes per warp.
constexpr int kOneClassLayouts[] = {2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};
constexpr int kTwoClassLayouts[][2] = {{4, 2},   {6, 4},   {8, 6},   {10, 8},  {12, 10}, {14, 12},
                                       {16, 14}, {20, 16}, {24, 20}, {28, 24}, {32, 28}};

template <int D>
int launch_split_d(hermite_ctx *ctx, const Geometry &g, const float2 *src, float2 *dst, bool sub) {
  const int S = ctx->pslots, P = ctx->psplit;
#define HERMITE_SPLIT_LAYOUT(S_, P_) \
  if (S == S_ && P == P_) return launch_split_dn<D, S_, P_>(ctx, g, src, dst, sub);
  HERMITE_SPLIT_LAYOUT(2, 2)
  HERMITE_SPLIT_LAYOUT(4, 4)
  HERMITE_SPLIT_LAYOUT(6, 6)
  HERMITE_SPLIT_LAYOUT(8, 8)
  HERMITE_SPLIT_LAYOUT(10, 10)
  HERMITE_SPLIT_LAYOUT(12, 12)
  HERMITE_SPLIT_LAYOUT(14, 14)
  HERMITE_SPLIT_LAYOUT(16, 16)
  HERMITE_SPLIT_LAYOUT(20, 20)
  HERMITE_SPLIT_LAYOUT(24, 24)
  HERMITE_SPLIT_LAYOUT(28, 28)
  HERMITE_SPLIT_LAYOUT(32, 32)
  if constexpr (D > 1) {
    HERMITE_SPLIT_LAYOUT(4, 2)
    HERMITE_SPLIT_LAYOUT(6, 4)
    HERMITE_SPLIT_LAYOUT(8, 6)
    HERMITE_SPLIT_LAYOUT(10, 8)
    HERMITE_SPLIT_LAYOUT(12, 10)
    HERMITE_SPLIT_LAYOUT(14, 12)
    HERMITE_SPLIT_LAYOUT(16, 14)
    HERMITE_SPLIT_LAYOUT(20, 16)
    HERMITE_SPLIT_LAYOUT(24, 20)
    HERMITE_SPLIT_LAYOUT(28, 24)
    HERMITE_SPLIT_LAYOUT(32, 28)
  }
#undef HERMITE_SPLIT_LAYOUT
  return HERMITE_ERR_ARG;
}

// Energy forms on split-precision levels: the factored form of the FP64
// kernel (Q_c = L_c^T L_c, tile of 64 cells per block, class vectors staged in
// shared memory) with the class vectors, the factor and every product in
// hi + lo arithmetic; block partial sums are returned as FP64 hi + lo.
constexpr int kSFTile = 64;
constexpr int kSFThreads = 256;

template <int D>
__global__ void __launch_bounds__(kSFThreads) energy_factored_split_kernel(
    Geometry g, const float2 *__restrict__ L, int lrows, int rmax, int tri, const int16_t *__restrict__ perm, int nq,
    const int8_t *__restrict__ par, const float2 *__restrict__ A, const float2 *__restrict__ B, double *partials) {
  constexpr int NC = 1 << D;
  extern __shared__ float2 smf[];
  const int c = blockIdx.y;
  const bool quad = (A == B);
  const int ld = nq | 1;
  float2 *Ls = smf;                                    // [rmax][nq]
  float2 *YA = Ls + (size_t)rmax * nq;                 // [kSFTile][ld]
  float2 *YB = quad ? YA : YA + (size_t)kSFTile * ld;
  double *cw = reinterpret_cast<double *>(YA + (size_t)(quad ? 1 : 2) * kSFTile * ld);  // [kSFTile]
  int64_t *cidx = reinterpret_cast<int64_t *>(cw + kSFTile);
  int *cgm = reinterpret_cast<int *>(cidx + kSFTile * NC);
  int16_t *ps = reinterpret_cast<int16_t *>(cgm + kSFTile * NC);
  int8_t *pin = reinterpret_cast<int8_t *>(ps + nq);
  __shared__ double red[kSFThreads];
  const float2 *Lc = L + (size_t)c * lrows * nq;
  for (int i = threadIdx.x; i < rmax * nq; i += kSFThreads) Ls[i] = Lc[i];
  for (int i = threadIdx.x; i < nq; i += kSFThreads) {
    ps[i] = perm[(size_t)c * nq + i];
    pin[i] = par[i];
  }
  const int cg = threadIdx.x & 15, rg = threadIdx.x >> 4;
  float2 total = make_float2(0.f, 0.f);
  const int64_t ntiles = (g.nodes_dst + kSFTile - 1) / kSFTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < kSFTile) {
      const int64_t t = tile * kSFTile + threadIdx.x;
      double w = 0.0;
      int64_t li[NC];
      int lg[NC];
      if (t < g.nodes_dst) {
        dev::cell_corners<D>(g, t, li, lg);
        w = dev::cell_weight<D>(g, t);
      } else {
        for (int s = 0; s < NC; ++s) {
          li[s] = 0;
          lg[s] = 0;
        }
      }
      // corner-major ([NC][kSFTile]): the lanes of a warp read consecutive words
      for (int s = 0; s < NC; ++s) {
        cidx[s * kSFTile + threadIdx.x] = li[s];
        cgm[s * kSFTile + threadIdx.x] = lg[s];
      }
      cw[threadIdx.x] = w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kSFTile * nq; e += kSFThreads) {
      // consecutive lanes take consecutive cells of one coefficient plane so
      // that their corner gathers coalesce
      const int i = e % kSFTile, k = e / kSFTile, b = ps[k], q = c ^ pin[b];
      const int64_t *idx = cidx + i;
      const int *gm = cgm + i;
      float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        const int gs = gm[s * kSFTile];
        const int64_t is = idx[s * kSFTile];
        const bool neg = ((__popc(q & s) & 1) != 0) != (gs && ghost_negates(g.bc, gs, pin[b]));
        float2 v = A[(size_t)b * g.ld_src + is];
        ya = df_add(ya, neg ? df_neg(v) : v);
        if (!quad) {
          v = B[(size_t)b * g.ld_src + is];
          yb = df_add(yb, neg ? df_neg(v) : v);
        }
      }
      YA[i * ld + k] = df_norm(ya);
      if (!quad) YB[i * ld + k] = df_norm(yb);
    }
    __syncthreads();
    float2 e4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) e4[i] = make_float2(0.f, 0.f);
    for (int r = rg; r < rmax; r += 16) {
      const float2 *lrow = Ls + (size_t)r * nq;
      float2 za[4], zb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        za[i] = make_float2(0.f, 0.f);
        zb[i] = make_float2(0.f, 0.f);
      }
      for (int k = tri ? r : 0; k < nq; ++k) {
        const float2 l = lrow[k];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          df_fma(za[i], l, YA[(cg + 16 * i) * ld + k]);
          if (!quad) df_fma(zb[i], l, YB[(cg + 16 * i) * ld + k]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 a = df_norm(za[i]);
        df_fma(e4[i], a, quad ? a : df_norm(zb[i]));
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // weights are 1, 1/2, 1/4 or 1/8: exact in FP32
      const float w = (float)cw[cg + 16 * i];
      const float2 e = df_norm(e4[i]);
      total = df_add(total, make_float2(w * e.x, w * e.y));
    }
  }
  red[threadIdx.x] = (double)total.x + (double)total.y;
  __syncthreads();
  for (int off = kSFThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__global__ void split_factor_kernel(const double *L, int64_t n, float2 *Lf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = L[i];
    const float hi = __double2float_rn(x);
    Lf[i] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}

__global__ void reduce_partials_kernel(const double *partials, int64_t n, double scale, double *out) {
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

template <int D>
int launch_energy_split_d(hermite_ctx *ctx, int form, int grid, const float2 *A, const float2 *B, double *out) {
  const Geometry g = make_geometry(ctx, 1 - grid);
  const int nclass = 1 << D, nq = ctx->nq[form], rmax = ctx->rmax[form], ld = nq | 1;
  static thread_local int configured = -1;
  if (configured != ctx->device) {
    if (!cuda_ok(ctx,
                 cudaFuncSetAttribute(energy_factored_split_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024),
                 "cudaFuncSetAttribute split energy"))
      return HERMITE_ERR_CUDA;
    configured = ctx->device;
  }
  const size_t smem = sizeof(float2) * ((size_t)rmax * nq + (A == B ? 1 : 2) * (size_t)kSFTile * ld) +
                      sizeof(double) * kSFTile + sizeof(int64_t) * kSFTile * nclass + sizeof(int) * kSFTile * nclass +
                      3 * nq + 16;
  int64_t blocks = std::max<int64_t>(1, (g.nodes_dst + kSFTile - 1) / kSFTile);
  blocks = std::min<int64_t>(blocks, ctx->partials_len / nclass);
  dim3 grd((unsigned)blocks, (unsigned)nclass);
  energy_factored_split_kernel<D><<<grd, kSFThreads, smem, ctx->stream>>>(
      g, ctx->Lf[form], ctx->lrows[form], rmax, ctx->ltri[form], ctx->lperm[form], nq, ctx->par_in, A, B,
      ctx->partials);
  reduce_partials_kernel<<<1, 256, 0, ctx->stream>>>(ctx->partials, blocks * nclass, ctx->formscale[form], out);
  return cuda_ok(ctx, cudaGetLastError(), "energy_factored_split_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

// operator rows in a warp slot layout, each entry split hi + lo; the entries
// of slots 2k and 2k+1 for one input are stored (hi, hi, lo, lo)
__global__ void split_operator_kernel(const double *M, int nci, const int16_t *prow, int nwarps, int S,
                                      float2 *Mp) {
  const int64_t n = (int64_t)nwarps * nci * S;
  float *f = reinterpret_cast<float *>(Mp);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % S);
    const int b = (int)((i / S) % nci);
    const int w = (int)(i / ((int64_t)S * nci));
    const int row = prow[w * S + j];
    const double m = row >= 0 ? M[(size_t)row * nci + b] : 0.0;
    const float hi = __double2float_rn(m);
    const int64_t base = 2 * (i - j) + 4 * (j / 2) + (j & 1);
    f[base] = hi;
    f[base + 2] = __double2float_rn(m - (double)hi);
  }
}

// plane-wise conversions (grid.y = coefficient plane, no division per element)
__global__ void to_split_kernel(const double *__restrict__ a, int64_t ld, int planes, int64_t nodes,
                                float2 *__restrict__ out) {
  const double *src = a + (int64_t)blockIdx.y * ld;
  float2 *dst = out + (int64_t)blockIdx.y * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = src[i];
    const float hi = __double2float_rn(x);
    dst[i] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}

__global__ void from_split_kernel(const float2 *__restrict__ a, int64_t ld, int planes, int64_t nodes,
                                  double *__restrict__ out) {
  const float2 *src = a + (int64_t)blockIdx.y * ld;
  double *dst = out + (int64_t)blockIdx.y * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    dst[i] = (double)v.x + (double)v.y;
  }
}

// Can warps of S slots, the first P for one parity class and the other S - P
// for one more, hold counts[c] outputs of every class?  Each class takes some
// number of P-slot bins and then enough (S - P)-slot bins for the rest; a
// dynamic programme over the classes finds an assignment using at most one
// bin of each kind per warp.  On success bins[w] and bins[nclass + w] are the
// classes of warp w's two bins (-1: unused).
bool pack_two_classes(const std::vector<int> &counts, int S, int P, std::vector<int> *bins) {
  const int nclass = (int)counts.size(), s = S - P;
  // reach[c][big][small]: classes < c placed with that many bins used; choice
  // records the big-bin count of class c - 1
  std::vector<std::vector<std::vector<int>>> choice(
      nclass + 1, std::vector<std::vector<int>>(nclass + 1, std::vector<int>(nclass + 1, -1)));
  choice[0][0][0] = 0;
  for (int c = 0; c < nclass; ++c)
    for (int bu = 0; bu <= nclass; ++bu)
      for (int su = 0; su <= nclass; ++su) {
        if (choice[c][bu][su] < 0) continue;
        for (int b = 0; bu + b <= nclass; ++b) {
          const int rest = std::max(0, counts[c] - b * P);
          const int k = rest == 0 ? 0 : (s > 0 ? (rest + s - 1) / s : nclass + 1);
          if (su + k <= nclass && choice[c + 1][bu + b][su + k] < 0) choice[c + 1][bu + b][su + k] = b;
        }
      }
  for (int bu = 0; bu <= nclass; ++bu)
    for (int su = 0; su <= nclass; ++su) {
      if (choice[nclass][bu][su] < 0) continue;
      bins->assign(2 * nclass, -1);
      int wb = 0, ws = 0, b_left = bu, s_left = su;
      for (int c = nclass - 1; c >= 0; --c) {
        const int b = choice[c + 1][b_left][s_left];
        const int rest = std::max(0, counts[c] - b * P);
        const int k = rest == 0 ? 0 : (rest + s - 1) / s;
        for (int i = 0; i < b; ++i) (*bins)[wb++] = c;
        for (int i = 0; i < k; ++i) (*bins)[nclass + ws++] = c;
        b_left -= b;
        s_left -= k;
      }
      return true;
    }
  return false;
}

}  // namespace

int build_split_operator(hermite_ctx *ctx) {
  const int nclass = 1 << ctx->d;
  // output rows by parity class
  std::vector<int8_t> parh(ctx->Nu + ctx->Nv);
  if (!cuda_ok(ctx, cudaMemcpy(parh.data(), ctx->par_in, parh.size(), cudaMemcpyDeviceToHost), "parity copy"))
    return HERMITE_ERR_CUDA;
  std::vector<std::vector<int>> rows(nclass);
  for (int r = 0; r < ctx->nco; ++r) rows[parh[r]].push_back(r);
  std::vector<int> counts(nclass);
  for (int c = 0; c < nclass; ++c) counts[c] = (int)rows[c].size();
  const int cmax = *std::max_element(counts.begin(), counts.end());
  if (cmax > 32) return HERMITE_ERR_UNSUPPORTED;
  // one class per warp: the smallest even slot count that holds the largest
  // class (up to 16; then 24 or 32) ...
  const int one = cmax <= 16 ? std::max(2, (cmax + 1) / 2 * 2) : (cmax <= 24 ? 24 : 32);
  std::vector<int> bins(2 * nclass, -1);  // class of warp w's first P / last S - P slots
  for (int w = 0; w < nclass; ++w) bins[w] = w;
  int S = one, P = one;
  // ... unless a layout with fewer slots holds the classes, two per warp
  for (int cand = 2; cand < one && S == one; cand += 2) {
    if (cmax <= cand && std::find(std::begin(kOneClassLayouts), std::end(kOneClassLayouts), cand) !=
                            std::end(kOneClassLayouts)) {
      S = P = cand;
    } else if (nclass > 1) {
      std::vector<int> packed;
      for (const auto &l : kTwoClassLayouts)
        if (l[0] == cand && pack_two_classes(counts, l[0], l[1], &packed)) {
          S = l[0];
          P = l[1];
          bins = packed;
          break;
        }
    }
  }
  std::vector<int8_t> cls(2 * nclass);
  std::vector<int16_t> prow((size_t)nclass * S, -1);
  std::vector<size_t> next(nclass, 0);
  for (int part = 0; part < 2; ++part)
    for (int w = 0; w < nclass; ++w) {
      const int c = bins[part * nclass + w];
      const int j0 = part ? P : 0, j1 = part ? S : P;
      cls[2 * w + part] = (int8_t)(c < 0 ? (part ? cls[2 * w] : 0) : c);
      for (int j = j0; j < j1 && c >= 0 && next[c] < rows[c].size(); ++j)
        prow[(size_t)w * S + j] = (int16_t)rows[c][next[c]++];
    }
  for (int c = 0; c < nclass; ++c)
    if (next[c] != rows[c].size()) return HERMITE_ERR_UNSUPPORTED;  // not reached: the layout holds every row
  if (!cuda_ok(ctx, device_alloc(&ctx->prow, sizeof(int16_t) * prow.size()), "cudaMalloc prow") ||
      !cuda_ok(ctx, device_alloc(&ctx->pcls, 2 * nclass), "cudaMalloc pcls") ||
      !cuda_ok(ctx, device_alloc(&ctx->Mp, sizeof(float2) * (size_t)nclass * ctx->nci * S), "cudaMalloc Mp"))
    return HERMITE_ERR_ALLOC;
  if (!cuda_ok(ctx, cudaMemcpy(ctx->prow, prow.data(), sizeof(int16_t) * prow.size(), cudaMemcpyHostToDevice),
               "prow copy") ||
      !cuda_ok(ctx, cudaMemcpy(ctx->pcls, cls.data(), cls.size(), cudaMemcpyHostToDevice), "pcls copy"))
    return HERMITE_ERR_CUDA;
  split_operator_kernel<<<64, 256, 0, ctx->stream>>>(ctx->M, ctx->nci, ctx->prow, nclass, S, ctx->Mp);
  ctx->pslots = S;
  ctx->psplit = P;
  if (!cuda_ok(ctx, cudaGetLastError(), "split_operator_kernel") ||
      !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "split operator sync"))
    return HERMITE_ERR_CUDA;
  return HERMITE_OK;
}

int build_split_forms(hermite_ctx *ctx) {
  for (int f = 0; f < kNumForms; ++f) {
    const int64_t n = (int64_t)(1 << ctx->d) * ctx->lrows[f] * ctx->nq[f];
    if (!cuda_ok(ctx, device_alloc(&ctx->Lf[f], sizeof(float2) * std::max<int64_t>(n, 1)), "cudaMalloc Lf"))
      return HERMITE_ERR_ALLOC;
    split_factor_kernel<<<64, 256, 0, ctx->stream>>>(ctx->L[f], n, ctx->Lf[f]);
  }
  return cuda_ok(ctx, cudaGetLastError(), "split_factor_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

int launch_energy_form_split(hermite_ctx *ctx, int form, int grid, const float2 *A, const float2 *B,
                             double *result_slot) {
  switch (ctx->d) {
    case 1: return launch_energy_split_d<1>(ctx, form, grid, A, B, result_slot);
    case 2: return launch_energy_split_d<2>(ctx, form, grid, A, B, result_slot);
    case 3: return launch_energy_split_d<3>(ctx, form, grid, A, B, result_slot);
  }
  return HERMITE_ERR_ARG;
}

int launch_half_step_split_into(hermite_ctx *ctx, int dst, const float2 *src, float2 *out, bool subtract_old) {
  if (ctx->tc_ready && ctx->split_engine == 1) return launch_half_step_tc(ctx, dst, src, out, subtract_old);
  const Geometry g = make_geometry(ctx, dst);
  switch (ctx->d) {
    case 1: return launch_split_d<1>(ctx, g, src, out, subtract_old);
    case 2: return launch_split_d<2>(ctx, g, src, out, subtract_old);
    case 3: return launch_split_d<3>(ctx, g, src, out, subtract_old);
  }
  return HERMITE_ERR_ARG;
}

int launch_half_step_split(hermite_ctx *ctx, int dst, bool subtract_old) {
  const Geometry g = make_geometry(ctx, dst);
  const float2 *src = ctx->fgrid[1 - dst];
  float2 *out = ctx->fgrid[dst];
  if (ctx->tc_ready && ctx->split_engine == 1) return launch_half_step_tc(ctx, dst, src, out, subtract_old);
  switch (ctx->d) {
    case 1: return launch_split_d<1>(ctx, g, src, out, subtract_old);
    case 2: return launch_split_d<2>(ctx, g, src, out, subtract_old);
    case 3: return launch_split_d<3>(ctx, g, src, out, subtract_old);
  }
  return HERMITE_ERR_ARG;
}

// blocks per plane: about 8 waves of 256-thread blocks over the whole grid
static dim3 plane_grid(const hermite_ctx *ctx, int grid) {
  const int64_t per_plane = std::max<int64_t>(1, std::min<int64_t>((ctx->nodes[grid] + 255) / 256,
                                                                    (148 * 64 + ctx->ncoef - 1) / ctx->ncoef));
  return dim3((unsigned)per_plane, (unsigned)ctx->ncoef);
}

int split_from_fp64(hermite_ctx *ctx, int grid) {
  if (ctx->nodes[grid] == 0) return HERMITE_OK;
  to_split_kernel<<<plane_grid(ctx, grid), 256, 0, ctx->stream>>>(ctx->grid[grid], ctx->ld[grid], ctx->ncoef,
                                                                  ctx->nodes[grid], ctx->fgrid[grid]);
  return cuda_ok(ctx, cudaGetLastError(), "to_split_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

int split_to_fp64(hermite_ctx *ctx, int grid) {
  if (ctx->nodes[grid] == 0) return HERMITE_OK;
  from_split_kernel<<<plane_grid(ctx, grid), 256, 0, ctx->stream>>>(ctx->fgrid[grid], ctx->ld[grid], ctx->ncoef,
                                                                    ctx->nodes[grid], ctx->grid[grid]);
  return cuda_ok(ctx, cudaGetLastError(), "from_split_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

}  // namespace hermite
