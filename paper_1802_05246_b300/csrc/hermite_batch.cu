// Ragged batches: many problems (differing N, m, boundary condition and
// variant, one dimension d per batch) advanced together.  Each half-step of
// the whole batch is one persistent launch per output-size group: blocks take
// (problem, node range) items from an atomic counter until the list is empty,
// so large and small problems share the GPU without one launch per problem
// and without any inter-block waiting.  Items are ordered longest first.  A
// full step (two half-steps) is captured once as a CUDA graph and replayed.
// A small autotuner times the item size and the number of resident blocks.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hermite_device.cuh"
#include "hermite_internal.h"

namespace hermite {
namespace {

struct BatchItem {
  int prob;
  int64_t n0, n1;
};

struct BatchDesc {
  Geometry g;
  const void *src;
  void *dst;
  const double *M;
  const float2 *Mp;     // split operator in the context's slot layout
  const int16_t *prow;  // output row of each slot (-1 unused)
  const int8_t *pcls;   // parity classes of each warp's two slot ranges
  const int8_t *par;
  int nci, nco, sub;
};

// ---------------------------------------------------------------- FP64
constexpr int kBT = 128;

// One item = a node range of one problem; the block first copies that
// problem's operator (all nco <= CH outputs, transposed to [input][output])
// into shared memory, then each thread takes nodes: corner gather, transform,
// and every output from the staged rows in one pass.
template <int D, int CH>
__global__ void __launch_bounds__(kBT) batch_f64_kernel(const BatchDesc *__restrict__ descs,
                                                        const BatchItem *__restrict__ items, int nitems,
                                                        unsigned *counter) {
  constexpr int NC = 1 << D;
  extern __shared__ __align__(16) double fsm[];
  double *Ms = fsm;              // [nci][CH]
  double *zb = Ms + CH * CH;     // [NC][kBT]  (nci <= nco <= CH)
  // parity class of each output, beside the staged rows (in registers, CH of
  // them pushed the 96-output instantiation past the register file)
  int8_t *po = reinterpret_cast<int8_t *>(zb + NC * kBT);  // [CH]
  __shared__ int item_s;
  __shared__ int staged;         // problem whose operator Ms holds (-1: none)
  double *myz = zb + threadIdx.x;
  if (threadIdx.x == 0) staged = -1;
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = item_s;
    if (it >= nitems) break;
    const BatchItem I = items[it];
    const BatchDesc P = descs[I.prob];
    if (staged != I.prob) {  // uniform: every thread read the same item
      for (int e = threadIdx.x; e < P.nci * CH; e += kBT) {
        const int bb = e / CH, j = e % CH;
        Ms[e] = j < P.nco ? P.M[(size_t)j * P.nci + bb] : 0.0;
      }
      for (int j = threadIdx.x; j < CH; j += kBT) po[j] = j < P.nco ? P.par[j] : 0;
      __syncthreads();
      if (threadIdx.x == 0) staged = I.prob;
    }
    const double *src = static_cast<const double *>(P.src);
    double *dst = static_cast<double *>(P.dst);
    for (int64_t t = I.n0 + threadIdx.x; t < I.n1; t += kBT) {
      int64_t idx[NC];
      int gm[NC];
      dev::cell_corners<D>(P.g, t, idx, gm);
      double acc[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) acc[j] = 0.0;
      for (int b = 0; b < P.nci; ++b) {
        const double *plane = src + (size_t)b * P.g.ld_src;
        const int pb = P.par[b];
        double x[NC];
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          double v = __ldg(plane + idx[s]);
          if (gm[s] && dev::ghost_negates(P.g.bc, gm[s], pb)) v = -v;
          x[s] = v;
        }
#pragma unroll
        for (int bm = 1; bm < NC; bm <<= 1)
#pragma unroll
          for (int i = 0; i < NC; ++i)
            if (!(i & bm)) {
              const double a = x[i], c = x[i | bm];
              x[i] = a + c;
              x[i | bm] = a - c;
            }
#pragma unroll
        for (int s = 0; s < NC; ++s) myz[s * kBT] = x[s];
        const double *mrow = Ms + (size_t)b * CH;
#pragma unroll
        for (int j = 0; j < CH; ++j) acc[j] = fma(mrow[j], myz[(po[j] ^ pb) * kBT], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        if (j < P.nco) {
          double *o = dst + (size_t)j * P.g.ld_dst + t;
          *o = P.sub ? acc[j] - *o : acc[j];
        }
      }
    }
    __syncthreads();  // item_s and the staged rows are rewritten next
  }
}

// ---------------------------------------------------------------- split
// one item = a range of target nodes processed 32 at a time by 2^d warps;
// warp w accumulates NS output slots, the first NP of parity class pcls[2w]
// and the rest of class pcls[2w+1] (the contexts' slot layout)
// 16-byte asynchronous copy global -> shared (completion tracked in groups)
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Shared memory of the split batch kernel: the operator rows of the current
// and the next chunk per warp (copied one chunk ahead), then the exchange
// buffer of the transformed corner data.
template <int D, int NS>
constexpr size_t batch_split_smem() {
  return sizeof(float2) * (2 * (1 << D) * (1 << D) * NS + (1 << D) * (1 << D) * 32);
}

template <int D, int NS, int NP>
__global__ void __launch_bounds__(32 << D) batch_split_kernel(const BatchDesc *__restrict__ descs,
                                                              const BatchItem *__restrict__ items, int nitems,
                                                              unsigned *counter) {
  static_assert(NS % 2 == 0 && NP % 2 == 0, "slot pairs never straddle the two classes");
  constexpr int NC = 1 << D;
  extern __shared__ __align__(16) float2 bsm[];
  float2 *Ms = bsm;                     // [2 buffers][NC warps][NC rows][NS]
  float2 *Y = Ms + 2 * NC * NC * NS;    // [NC][NC][32]
  __shared__ int item_s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = item_s;
    __syncthreads();
    if (it >= nitems) break;
    const BatchItem I = items[it];
    const BatchDesc P = descs[I.prob];
    const float2 *src = static_cast<const float2 *>(P.src);
    float2 *dst = static_cast<float2 *>(P.dst);
    const int cA = P.pcls[2 * w], cB = P.pcls[2 * w + 1];
    for (int64_t base = I.n0; base < I.n1; base += 32) {
      const int64_t t = base + lane;
      const bool valid = t < I.n1;
      int64_t idx[NC];
      int gm[NC];
      if (valid) {
        dev::cell_corners<D>(P.g, t, idx, gm);
      } else {
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          idx[s] = 0;
          gm[s] = 0;
        }
      }
      // slot pairs (2k, 2k+1): hi parts in ahi[k], lo parts in alo[k]
      float2 ahi[NS / 2], alo[NS / 2];
#pragma unroll
      for (int k = 0; k < NS / 2; ++k) ahi[k] = alo[k] = make_float2(0.f, 0.f);
      // this warp's operator rows b0 .. b0+NC-1 (contiguous) into buffer buf
      auto stage = [&](int b0, int buf) {
        const int kc = min(NC, P.nci - b0);
        const float2 *g = P.Mp + ((size_t)w * P.nci + b0) * NS;
        float2 *sdst = Ms + ((size_t)buf * NC + w) * NC * NS;
        for (int e = lane; e < kc * NS / 2; e += 32) cp_async16(sdst + 2 * e, g + 2 * e);
      };
      stage(0, 0);
      cp_async_commit();
      for (int b0 = 0, ch = 0; b0 < P.nci; b0 += NC, ++ch) {
        // the next chunk's rows are in flight while this one is used
        if (b0 + NC < P.nci) stage(b0 + NC, (ch + 1) & 1);
        cp_async_commit();
        const int b = b0 + w;
        if (b < P.nci) {
          const float2 *plane = src + (size_t)b * P.g.ld_src;
          const int pb = P.par[b];
          float2 x[NC];
#pragma unroll
          for (int s = 0; s < NC; ++s) {
            float2 v = plane[idx[s]];
            if (gm[s] && dev::ghost_negates(P.g.bc, gm[s], pb)) v = dev::df_neg(v);
            x[s] = v;
          }
#pragma unroll
          for (int bm = 1; bm < NC; bm <<= 1)
#pragma unroll
            for (int i = 0; i < NC; ++i)
              if (!(i & bm)) {
                const float2 a = x[i], c = x[i | bm];
                x[i] = dev::df_add(a, c);
                x[i | bm] = dev::df_add(a, dev::df_neg(c));
              }
#pragma unroll
          for (int q = 0; q < NC; ++q) Y[(w * NC + q) * 32 + lane] = x[q];
        }
        __syncthreads();
        cp_async_wait_prev();  // this chunk's rows have landed (each warp reads its own)
        __syncwarp();
        const float2 *mbuf = Ms + ((size_t)(ch & 1) * NC + w) * NC * NS;
        const int kmax = min(NC, P.nci - b0);
        for (int k = 0; k < kmax; ++k) {
          const int bb = b0 + k;
          const int pb = P.par[bb];
          const float2 ya = Y[(k * NC + (cA ^ pb)) * 32 + lane];
          const float2 yb = NP < NS ? Y[(k * NC + (cB ^ pb)) * 32 + lane] : ya;
          const float2 yah = make_float2(ya.x, ya.x), yal = make_float2(ya.y, ya.y), yan = make_float2(-ya.x, -ya.x);
          const float2 ybh = make_float2(yb.x, yb.x), ybl = make_float2(yb.y, yb.y), ybn = make_float2(-yb.x, -yb.x);
          const float4 *mrow = reinterpret_cast<const float4 *>(mbuf + k * NS);
#pragma unroll
          for (int j = 0; j < NS / 2; ++j) {
            const float4 mm = mrow[j];  // (hi, hi, lo, lo) of slots 2j, 2j+1
            if constexpr (NS == 2) {
              // one slot pair: forming the packed copies of y costs what the
              // packing saves (measured), so the scalar form
              float2 a0 = make_float2(ahi[j].x, alo[j].x), a1 = make_float2(ahi[j].y, alo[j].y);
              dev::df_fma(a0, make_float2(mm.x, mm.z), 2 * j < NP ? ya : yb);
              dev::df_fma(a1, make_float2(mm.y, mm.w), 2 * j < NP ? ya : yb);
              ahi[j] = make_float2(a0.x, a1.x);
              alo[j] = make_float2(a0.y, a1.y);
            } else if (2 * j < NP) {
              dev::df_fma_x2(ahi[j], alo[j], make_float2(mm.x, mm.y), make_float2(mm.z, mm.w), yah, yal, yan);
            } else {
              dev::df_fma_x2(ahi[j], alo[j], make_float2(mm.x, mm.y), make_float2(mm.z, mm.w), ybh, ybl, ybn);
            }
          }
        }
        __syncthreads();
      }
      if (valid) {
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          const int row = P.prow[w * NS + j];
          if (row >= 0) {
            float2 *o = dst + (size_t)row * P.g.ld_dst + t;
            const float2 a = (j & 1) ? make_float2(ahi[j / 2].y, alo[j / 2].y) : make_float2(ahi[j / 2].x, alo[j / 2].x);
            float2 r = dev::df_norm(a);
            if (P.sub) r = dev::df_norm(dev::df_add(r, dev::df_neg(*o)));
            *o = r;
          }
        }
      }
    }
  }
}

}  // namespace
}  // namespace hermite

struct hermite_batch {
  int d = 0, precision = 0, nprob = 0;
  std::vector<hermite_ctx *> probs;
  cudaStream_t stream = nullptr;
  hermite::BatchDesc *d_desc[2] = {nullptr, nullptr};
  struct Group {
    int tmpl;  // CH (FP64), or 64 * slots + split (split)
    hermite::BatchItem *d_items;
    int nitems;
  };
  std::vector<Group> groups[2];
  unsigned *d_counters = nullptr;
  int ncounters = 0;
  int item_nodes = 1024, blocks_per_sm = 2, nsm = 148;
  cudaGraphExec_t graph = nullptr;
  int64_t half = 0;
  void *d_state[2] = {nullptr, nullptr};  // per-grid StateDesc arrays of the batched state transfers
  std::string err;
};

namespace hermite {
namespace {

thread_local std::string g_batch_error;

bool bok(hermite_batch *b, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  b->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

int half_dst(const hermite_ctx *ctx, int64_t half) {
  if (ctx->variant == HERMITE_CONSERVATIVE) return (half % 2 == 0) ? HERMITE_PRIMAL : HERMITE_DUAL;
  return (half % 2 == 0) ? HERMITE_DUAL : HERMITE_PRIMAL;
}

void free_items(hermite_batch *b) {
  for (int k = 0; k < 2; ++k) {
    for (auto &gr : b->groups[k]) cudaFree(gr.d_items);
    b->groups[k].clear();
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

int group_key(const hermite_batch *b, const hermite_ctx *ctx) {
  if (b->precision == HERMITE_SPLIT32) return ctx->pslots * 64 + ctx->psplit;
  // FP64: the output count rounded up to a compiled chunk (all outputs in one)
  return ctx->nco <= 8 ? 8 : (ctx->nco <= 16 ? 16 : (ctx->nco <= 32 ? 32 : (ctx->nco <= 48 ? 48 : 96)));
}

int build_items(hermite_batch *b) {
  free_items(b);
  for (int k = 0; k < 2; ++k) {
    std::vector<int> keys;
    for (auto *c : b->probs) {
      const int key = group_key(b, c);
      if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
    }
    for (int key : keys) {
      struct HostItem {
        BatchItem it;
        double cost;
      };
      std::vector<HostItem> h;
      for (int p = 0; p < b->nprob; ++p) {
        const hermite_ctx *c = b->probs[p];
        if (group_key(b, c) != key) continue;
        const int dst = half_dst(c, k);
        const int64_t n = c->nodes[dst];
        for (int64_t n0 = 0; n0 < n; n0 += b->item_nodes) {
          HostItem hi;
          hi.it.prob = p;
          hi.it.n0 = n0;
          hi.it.n1 = std::min<int64_t>(n, n0 + b->item_nodes);
          hi.cost = (double)(hi.it.n1 - hi.it.n0) * c->nci * c->nco;
          h.push_back(hi);
        }
      }
      std::stable_sort(h.begin(), h.end(), [](const HostItem &a, const HostItem &c) { return a.cost > c.cost; });
      std::vector<BatchItem> items(h.size());
      for (size_t i = 0; i < h.size(); ++i) items[i] = h[i].it;
      hermite_batch::Group gr{key, nullptr, (int)items.size()};
      if (!bok(b, device_alloc(&gr.d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)), "cudaMalloc items") ||
          !bok(b, cudaMemcpy(gr.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice),
               "items copy"))
        return HERMITE_ERR_CUDA;
      b->groups[k].push_back(gr);
    }
  }
  const int need = (int)(b->groups[0].size() + b->groups[1].size());
  if (need > b->ncounters) {
    cudaFree(b->d_counters);
    b->d_counters = nullptr;
    if (!bok(b, device_alloc(&b->d_counters, sizeof(unsigned) * need), "cudaMalloc counters")) return HERMITE_ERR_ALLOC;
    b->ncounters = need;
  }
  return HERMITE_OK;
}

int build_descs(hermite_batch *b) {
  for (int k = 0; k < 2; ++k) {
    std::vector<BatchDesc> h(b->nprob);
    for (int p = 0; p < b->nprob; ++p) {
      const hermite_ctx *c = b->probs[p];
      const int dst = half_dst(c, k);
      BatchDesc &ds = h[p];
      ds.g = make_geometry(c, dst);
      if (b->precision == HERMITE_SPLIT32) {
        ds.src = c->fgrid[1 - dst];
        ds.dst = c->fgrid[dst];
      } else {
        ds.src = c->grid[1 - dst];
        ds.dst = c->grid[dst];
      }
      ds.M = c->M;
      ds.Mp = c->Mp;
      ds.prow = c->prow;
      ds.pcls = c->pcls;
      ds.par = c->par_in;
      ds.nci = c->nci;
      ds.nco = c->nco;
      ds.sub = c->variant == HERMITE_CONSERVATIVE ? 1 : 0;
    }
    if (!bok(b, device_alloc(&b->d_desc[k], sizeof(BatchDesc) * b->nprob), "cudaMalloc descs") ||
        !bok(b, cudaMemcpy(b->d_desc[k], h.data(), sizeof(BatchDesc) * b->nprob, cudaMemcpyHostToDevice),
             "descs copy"))
      return HERMITE_ERR_CUDA;
  }
  return HERMITE_OK;
}

template <int D>
int launch_group(hermite_batch *b, int k, const hermite_batch::Group &gr, unsigned *counter) {
  const unsigned blocks = (unsigned)(b->nsm * b->blocks_per_sm);
  if (b->precision == HERMITE_SPLIT32) {
    // the template must equal the contexts' slot layout: it is the stride of their split operators
#define HERMITE_BATCH_LAYOUT(S_, P_)                                                                          \
  if (gr.tmpl == S_ * 64 + P_) {                                                                              \
    constexpr size_t smem = batch_split_smem<D, S_>();                                                        \
    if (smem > 40 * 1024 && /* the block also holds a little static shared memory */                        \
        !bok(b, cudaFuncSetAttribute(batch_split_kernel<D, S_, P_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)smem),                                                              \
             "batch kernel shared memory"))                                                                   \
      return HERMITE_ERR_CUDA;                                                                                \
    batch_split_kernel<D, S_, P_><<<blocks, 32 << D, smem, b->stream>>>(b->d_desc[k], gr.d_items, gr.nitems,  \
                                                                        counter);                             \
    return bok(b, cudaGetLastError(), "batch kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;                      \
  }
    HERMITE_BATCH_LAYOUT(2, 2)
    HERMITE_BATCH_LAYOUT(4, 4)
    HERMITE_BATCH_LAYOUT(6, 6)
    HERMITE_BATCH_LAYOUT(8, 8)
    HERMITE_BATCH_LAYOUT(10, 10)
    HERMITE_BATCH_LAYOUT(12, 12)
    HERMITE_BATCH_LAYOUT(14, 14)
    HERMITE_BATCH_LAYOUT(16, 16)
    HERMITE_BATCH_LAYOUT(20, 20)
    HERMITE_BATCH_LAYOUT(24, 24)
    HERMITE_BATCH_LAYOUT(28, 28)
    HERMITE_BATCH_LAYOUT(32, 32)
    if constexpr (D > 1) {
      HERMITE_BATCH_LAYOUT(4, 2)
      HERMITE_BATCH_LAYOUT(6, 4)
      HERMITE_BATCH_LAYOUT(8, 6)
      HERMITE_BATCH_LAYOUT(10, 8)
      HERMITE_BATCH_LAYOUT(12, 10)
      HERMITE_BATCH_LAYOUT(14, 12)
      HERMITE_BATCH_LAYOUT(16, 14)
      HERMITE_BATCH_LAYOUT(20, 16)
      HERMITE_BATCH_LAYOUT(24, 20)
      HERMITE_BATCH_LAYOUT(28, 24)
      HERMITE_BATCH_LAYOUT(32, 28)
    }
#undef HERMITE_BATCH_LAYOUT
    return HERMITE_ERR_ARG;
  } else {
#define HERMITE_BATCH_F64(CH_)                                                                              \
  if (gr.tmpl == CH_) {                                                                                     \
    const size_t smem = sizeof(double) * ((size_t)CH_ * CH_ + (1 << D) * kBT) + CH_;                        \
    if (smem > 40 * 1024 &&                                                                                 \
        !bok(b, cudaFuncSetAttribute(batch_f64_kernel<D, CH_>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                     (int)smem),                                                            \
             "batch kernel shared memory"))                                                                 \
      return HERMITE_ERR_CUDA;                                                                              \
    batch_f64_kernel<D, CH_><<<blocks, kBT, smem, b->stream>>>(b->d_desc[k], gr.d_items, gr.nitems, counter); \
    return bok(b, cudaGetLastError(), "batch kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;                    \
  }
    HERMITE_BATCH_F64(8)
    HERMITE_BATCH_F64(16)
    HERMITE_BATCH_F64(32)
    HERMITE_BATCH_F64(48)
    HERMITE_BATCH_F64(96)
#undef HERMITE_BATCH_F64
    return HERMITE_ERR_ARG;
  }
  return bok(b, cudaGetLastError(), "batch kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

// enqueue one half-step of every problem (parity k): per group, reset its
// work counter and launch the persistent kernel
int enqueue_half(hermite_batch *b, int k) {
  int ci = (k == 0) ? 0 : (int)b->groups[0].size();
  for (const auto &gr : b->groups[k]) {
    unsigned *counter = b->d_counters + ci++;
    if (!bok(b, cudaMemsetAsync(counter, 0, sizeof(unsigned), b->stream), "counter reset")) return HERMITE_ERR_CUDA;
    int rc;
    switch (b->d) {
      case 1: rc = launch_group<1>(b, k, gr, counter); break;
      case 2: rc = launch_group<2>(b, k, gr, counter); break;
      default: rc = launch_group<3>(b, k, gr, counter); break;
    }
    if (rc) return rc;
  }
  return HERMITE_OK;
}

// Batched state transfer: every problem's level, host layout [node][coef],
// problems back to back in one device buffer (u and v separately).
struct StateDesc {
  double *g;      // FP64 SoA grid [ncoef][ld]
  float2 *fg;     // split SoA grid (NULL for FP64 contexts)
  int64_t ld, nodes, off_u, off_v;
  int Nu, Nv;     // Nv = 0 for the conservative method
};

__global__ void batch_get_states_kernel(const StateDesc *__restrict__ d, double *__restrict__ u,
                                        double *__restrict__ v) {
  const StateDesc D = d[blockIdx.y];
  const int nc = D.Nu + D.Nv;
  const int64_t total = D.nodes * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = e / nc;
    const int c = (int)(e % nc);
    const int64_t i = (int64_t)c * D.ld + node;
    const double val = D.fg ? (double)D.fg[i].x + (double)D.fg[i].y : D.g[i];
    if (c < D.Nu)
      u[D.off_u + node * D.Nu + c] = val;
    else if (v)
      v[D.off_v + node * D.Nv + (c - D.Nu)] = val;
  }
}

__global__ void batch_set_states_kernel(const StateDesc *__restrict__ d, const double *__restrict__ u,
                                        const double *__restrict__ v) {
  const StateDesc D = d[blockIdx.y];
  const int nc = D.Nu + D.Nv;
  const int64_t total = D.nodes * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = e / nc;
    const int c = (int)(e % nc);
    const int64_t i = (int64_t)c * D.ld + node;
    const double val = c < D.Nu ? u[D.off_u + node * D.Nu + c] : (v ? v[D.off_v + node * D.Nv + (c - D.Nu)] : 0.0);
    D.g[i] = val;
    if (D.fg) {
      const float hi = __double2float_rn(val);
      D.fg[i] = make_float2(hi, __double2float_rn(val - (double)hi));
    }
  }
}

int state_descs(hermite_batch *b, int grid, const StateDesc **out, int64_t *max_elems) {
  int64_t ou = 0, ov = 0, mx = 0;
  std::vector<StateDesc> h(b->nprob);
  for (int p = 0; p < b->nprob; ++p) {
    hermite_ctx *c = b->probs[p];
    StateDesc &D = h[p];
    D.g = c->grid[grid];
    D.fg = c->precision == HERMITE_SPLIT32 ? c->fgrid[grid] : nullptr;
    D.ld = c->ld[grid];
    D.nodes = c->nodes[grid];
    D.Nu = c->Nu;
    D.Nv = c->variant == HERMITE_CONSERVATIVE ? 0 : c->Nv;
    D.off_u = ou;
    D.off_v = ov;
    ou += D.nodes * D.Nu;
    ov += D.nodes * D.Nv;
    mx = std::max<int64_t>(mx, D.nodes * (D.Nu + D.Nv));
  }
  if (!b->d_state[grid]) {
    if (!bok(b, device_alloc(&b->d_state[grid], sizeof(StateDesc) * b->nprob), "cudaMalloc state descs"))
      return HERMITE_ERR_ALLOC;
    if (!bok(b, cudaMemcpy(b->d_state[grid], h.data(), sizeof(StateDesc) * b->nprob, cudaMemcpyHostToDevice),
             "state descs copy")) {
      cudaFree(b->d_state[grid]);
      b->d_state[grid] = nullptr;
      return HERMITE_ERR_CUDA;
    }
  }
  *out = static_cast<const StateDesc *>(b->d_state[grid]);
  *max_elems = mx;
  return HERMITE_OK;
}

int sync_half(hermite_batch *b) {
  const int64_t h0 = b->probs[0]->half;
  for (auto *c : b->probs)
    if (c->half != h0) {
      b->err = "problems of a batch must have taken the same number of half-steps";
      return HERMITE_ERR_STATE;
    }
  b->half = h0;
  return HERMITE_OK;
}

void set_half(hermite_batch *b) {
  for (auto *c : b->probs) c->half = b->half;
}

}  // namespace
}  // namespace hermite

using namespace hermite;

extern "C" {

int hermite_batch_create(int nprob, const int *d, const int *m, const int64_t *N, const double *c, const double *h,
                         const double *dt, const int *variant, const int *bc, int precision, hermite_batch **out) {
  if (!out || nprob < 1 || !d || !m || !N || !c || !h || !dt || !variant || !bc) {
    g_batch_error = "invalid argument to hermite_batch_create";
    return HERMITE_ERR_ARG;
  }
  *out = nullptr;
  for (int p = 1; p < nprob; ++p)
    if (d[p] != d[0]) {
      g_batch_error = "all problems of a batch must have the same dimension";
      return HERMITE_ERR_ARG;
    }
  hermite_batch *b = new hermite_batch;
  b->d = d[0];
  b->precision = precision;
  b->nprob = nprob;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  int rc = HERMITE_OK;
  for (int p = 0; p < nprob && rc == HERMITE_OK; ++p) {
    hermite_ctx *ctx = nullptr;
    rc = create_context(d[p], m[p], N[p], c[p], h[p], dt[p], variant[p], bc[p], precision, false, &ctx);
    if (rc) {
      g_batch_error = "problem " + std::to_string(p) + ": " + hermite_last_error(nullptr);
      break;
    }
    b->probs.push_back(ctx);
  }
  if (rc == HERMITE_OK) rc = build_descs(b);
  if (rc == HERMITE_OK) rc = build_items(b);
  if (rc != HERMITE_OK) {
    if (g_batch_error.empty()) g_batch_error = b->err;
    hermite_batch_destroy(b);
    return rc;
  }
  *out = b;
  return HERMITE_OK;
}

void hermite_batch_destroy(hermite_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_items(b);
  for (int k = 0; k < 2; ++k) {
    cudaFree(b->d_desc[k]);
    cudaFree(b->d_state[k]);
  }
  cudaFree(b->d_counters);
  for (auto *c : b->probs) hermite_destroy(c);
  delete b;
}

hermite_ctx *hermite_batch_problem(hermite_batch *b, int p) {
  if (!b || p < 0 || p >= b->nprob) return nullptr;
  return b->probs[p];
}

int hermite_batch_set_stream(hermite_batch *b, void *stream) {
  if (!b) return HERMITE_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  for (auto *c : b->probs) c->stream = b->stream;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return HERMITE_OK;
}

int hermite_batch_get_states_device(hermite_batch *b, int grid, double *u, double *v) {
  if (!b) return HERMITE_ERR_ARG;
  if ((grid != 0 && grid != 1) || !u) {
    b->err = "bad grid or NULL u";
    return HERMITE_ERR_ARG;
  }
  const StateDesc *d = nullptr;
  int64_t mx = 0;
  if (int rc = state_descs(b, grid, &d, &mx)) return rc;
  const int64_t blocks = std::min<int64_t>(std::max<int64_t>((mx + 255) / 256, 1), 64);
  batch_get_states_kernel<<<dim3((unsigned)blocks, (unsigned)b->nprob), 256, 0, b->stream>>>(d, u, v);
  return bok(b, cudaGetLastError(), "batch_get_states_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}

int hermite_batch_set_states_device(hermite_batch *b, const double *u, const double *v) {
  if (!b) return HERMITE_ERR_ARG;
  if (!u) {
    b->err = "NULL u";
    return HERMITE_ERR_ARG;
  }
  for (auto *c : b->probs)
    if (c->variant == HERMITE_CONSERVATIVE) {
      b->err = "hermite_batch_set_states_device is for the dissipative methods";
      return HERMITE_ERR_STATE;
    }
  const StateDesc *d = nullptr;
  int64_t mx = 0;
  if (int rc = state_descs(b, HERMITE_PRIMAL, &d, &mx)) return rc;
  const int64_t blocks = std::min<int64_t>(std::max<int64_t>((mx + 255) / 256, 1), 64);
  batch_set_states_kernel<<<dim3((unsigned)blocks, (unsigned)b->nprob), 256, 0, b->stream>>>(d, u, v);
  if (!bok(b, cudaGetLastError(), "batch_set_states_kernel")) return HERMITE_ERR_CUDA;
  b->half = 0;
  set_half(b);
  return HERMITE_OK;
}

int hermite_batch_step(hermite_batch *b, int64_t nsteps) {
  if (!b) return HERMITE_ERR_ARG;
  if (nsteps < 0) {
    b->err = "nsteps < 0";
    return HERMITE_ERR_ARG;
  }
  int rc = sync_half(b);
  if (rc) return rc;
  if (b->half % 2 != 0 || b->stream == nullptr) {
    // direct launches (odd start, or the legacy stream, which cannot be captured)
    for (int64_t i = 0; i < 2 * nsteps; ++i) {
      rc = enqueue_half(b, (int)(b->half % 2));
      if (rc) return rc;
      b->half += 1;
    }
    set_half(b);
    return HERMITE_OK;
  }
  if (!b->graph && nsteps > 0) {
    cudaGraph_t g = nullptr;
    if (!bok(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture"))
      return HERMITE_ERR_CUDA;
    int rc1 = enqueue_half(b, 0);
    int rc2 = rc1 ? rc1 : enqueue_half(b, 1);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc2) {
      if (g) cudaGraphDestroy(g);
      return rc2;
    }
    if (!bok(b, e, "end capture")) return HERMITE_ERR_CUDA;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (!bok(b, e, "graph instantiate")) return HERMITE_ERR_CUDA;
  }
  for (int64_t i = 0; i < nsteps; ++i)
    if (!bok(b, cudaGraphLaunch(b->graph, b->stream), "graph launch")) return HERMITE_ERR_CUDA;
  b->half += 2 * nsteps;
  set_half(b);
  return HERMITE_OK;
}

int64_t hermite_batch_dof_per_step(const hermite_batch *b) {
  if (!b) return -1;
  int64_t s = 0;
  for (auto *c : b->probs) s += (c->nodes[0] + c->nodes[1]) * (int64_t)c->nco;
  return s;
}

int hermite_batch_autotune(hermite_batch *b, int *item_nodes, int *blocks_per_sm, double *ms_per_step) {
  if (!b) return HERMITE_ERR_ARG;
  if (!b->stream) {
    b->err = "set a non-default stream before autotuning";
    return HERMITE_ERR_STATE;
  }
  const int cand_items[] = {256, 1024, 4096};
  const int cand_blocks[] = {1, 2, 4, 8};
  double best = 1e30;
  int bi = b->item_nodes, bb = b->blocks_per_sm;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = HERMITE_OK;
  for (int in : cand_items) {
    for (int bp : cand_blocks) {
      b->item_nodes = in;
      b->blocks_per_sm = bp;
      rc = build_items(b);
      if (rc) break;
      rc = hermite_batch_step(b, 1);  // warm-up, builds the graph
      if (rc) break;
      cudaEventRecord(e0, b->stream);
      rc = hermite_batch_step(b, 2);
      if (rc) break;
      cudaEventRecord(e1, b->stream);
      if (!bok(b, cudaEventSynchronize(e1), "autotune sync")) {
        rc = HERMITE_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 2 < best) {
        best = ms / 2;
        bi = in;
        bb = bp;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->item_nodes = bi;
  b->blocks_per_sm = bb;
  rc = build_items(b);
  if (item_nodes) *item_nodes = bi;
  if (blocks_per_sm) *blocks_per_sm = bb;
  if (ms_per_step) *ms_per_step = best;
  return rc;
}

int hermite_batch_config(hermite_batch *b, int item_nodes, int blocks_per_sm) {
  if (!b || item_nodes < 32 || blocks_per_sm < 1 || blocks_per_sm > 32) return HERMITE_ERR_ARG;
  b->item_nodes = item_nodes;
  b->blocks_per_sm = blocks_per_sm;
  return build_items(b);
}

const char *hermite_batch_last_error(const hermite_batch *b) {
  if (!b) return g_batch_error.c_str();
  return b->err.c_str();
}

}  // extern "C"
