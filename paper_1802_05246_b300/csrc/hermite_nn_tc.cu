// Tensor-core (tcgen05) forward convolution of the learned super-stepper, for
// 64 input channels and 32 or 64 output channels.
//
// One CTA owns one output image row at a time (persistent, rows round robin).
// The three input rows a dilated 3x3 kernel touches, (y - dil, y, y + dil)
// mod H, arrive UNSHIFTED by TMA (one 128 x 64 BF16 box each, 128-byte
// swizzle) in a four-stage ring.  The column shift of the taps is moved to
// the output: for each kernel column kx an accumulator in tensor memory
// collects D_kx[q] = sum_ky X_ky[q] W_{ky,kx}^T, and the epilogue forms
// y[p] = D_0[p - dil] + D_1[p] + D_2[p + dil] (indices mod 128), exchanging
// D_0 and D_2 through shared memory with 16-byte accesses (dilations up to 8;
// larger ones use the mma.sync kernel).  A shifted operand tile
// cannot be described by a tensor-core shared-memory descriptor (its rows
// would not start on the 8-row swizzle atoms), an output shift needs no copy.
//
// Roles (320 threads): warp 0 issues the TMA loads, warp 1 owns the tensor
// memory and issues the MMAs (one elected thread, tcgen05.mma kind::f16,
// M = 128, N = 3 Cout, K = 16, BF16 in, FP32 accumulate), warps 2-9 drain the
// accumulators (tcgen05.ld; two warps per 32-lane quarter of tensor memory,
// each with half of the channels), add bias, apply ReLU and the optional mask
// and store.  Accumulators are double buffered so the epilogue of one row
// overlaps the MMAs of the next.  Every wait is bounded: a wait that runs out
// records an error, the CTA drains what it issued and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hermite.h"
#include "hermite_nn.h"
#include "hermite_nn_internal.h"
#include "hermite_tc.cuh"

namespace hermite_nn {
namespace {

typedef __nv_bfloat16 bf16;

constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait polls before a wait is declared failed
constexpr int kMaxTcDil = 8;               // largest dilation of the tensor-core kernel (boundary rows)

using hermite::tc::saddr;

// ---- mbarrier ----------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  return hermite::tc::mbar_wait(b, parity, kWaitLimit);
}
using hermite::tc::mbar_fence_init;
using hermite::tc::mbar_init;

// ---- TMA ------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
      : "memory");
}

// ---- tcgen05 ------------------------------------------------------------------------
namespace tc = hermite::tc;

// three 32-column loads under one wait (the epilogue's D_0, D_2 and D_1)
__device__ __forceinline__ void tc_ld32x3(uint32_t t0, uint32_t t1, uint32_t t2, float (&a)[32], float (&b)[32],
                                          float (&c)[32]) {
  uint32_t r[96];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%96];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%97];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79,%80,%81,%82,%83,%84,%85,%86,%87,%88,%89,%90,%91,%92,%93,%94,%95}, [%98];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]), "=r"(r[72]), "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79]), "=r"(r[80]), "=r"(r[81]), "=r"(r[82]), "=r"(r[83]), "=r"(r[84]), "=r"(r[85]), "=r"(r[86]), "=r"(r[87]), "=r"(r[88]), "=r"(r[89]), "=r"(r[90]), "=r"(r[91]), "=r"(r[92]), "=r"(r[93]), "=r"(r[94]), "=r"(r[95])
      : "r"(t0), "r"(t1), "r"(t2)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[32 + i]);
    c[i] = __uint_as_float(r[64 + i]);
  }
}

// Shared-memory matrix descriptor: K-major rows of 128 bytes (64 BF16), 128-byte
// swizzle, 8-row atoms 1024 bytes apart; the tile must start on a 1024-byte boundary.
// Bits: start address >> 4 [0,14), leading offset >> 4 [16,30) (unused here),
// stride offset >> 4 [32,46), descriptor version 1 [46,48), layout 2 = 128B swizzle [61,64).
__device__ __forceinline__ uint64_t sw128_desc(const void *tile) {
  uint64_t d = (uint64_t)((saddr(tile) >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

using hermite::tc::idesc_bf16;

// the 16-byte chunk c of row r of a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128_offset(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}
// barrier among nthreads threads that also returns the OR of every thread's flag (a uniform decision)
__device__ __forceinline__ int named_sync_or(int id, int nthreads, int flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(flag), "r"(id), "r"(nthreads)
      : "memory");
  return (int)r;
}
__device__ __forceinline__ int read_flag(const int *f) { return *reinterpret_cast<const volatile int *>(f); }

__device__ int g_tc_status;  // set to 1 by a tensor-core kernel whose bounded wait ran out

// ---------------------------------------------------------------------------
// Self-test GEMM: D[128][N] = A[128][64] B[N][64]^T on one CTA
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) tc_gemm_selftest_kernel(const bf16 *__restrict__ A, const bf16 *__restrict__ B,
                                                               float *__restrict__ D, int *status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char *As = base;
  unsigned char *Bs = As + 128 * 128;
  uint64_t *bar = reinterpret_cast<uint64_t *>(Bs + N * 128);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 128 * 8; i += 128) {
    const int r = i >> 3, c = i & 7;
    *reinterpret_cast<uint4 *>(As + sw128_offset(r, c)) = *reinterpret_cast<const uint4 *>(A + r * 64 + c * 8);
  }
  for (int i = tid; i < N * 8; i += 128) {
    const int r = i >> 3, c = i & 7;
    *reinterpret_cast<uint4 *>(Bs + sw128_offset(r, c)) = *reinterpret_cast<const uint4 *>(B + r * 64 + c * 8);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy writes -> tensor core
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tc::alloc(slot, 64);
    tc::relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    const uint64_t da = sw128_desc(As), db = sw128_desc(Bs);
#pragma unroll
    for (int k = 0; k < 4; ++k) tc::mma(tmem, da + 2 * k, db + 2 * k, idesc_bf16(128, N), k > 0 ? 1u : 0u);
    tc::commit(bar);
  }
  const bool ok = mbar_wait(bar, 0);
  tc::fence_after();
  if (ok) {
    const int row = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) D[row * N + c0 + j] = v[j];
    }
  } else if (lane == 0) {
    atomicExch(status, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------
// Forward convolution, Cin = 64
// ---------------------------------------------------------------------------
template <int COUT>
struct TcCfg {
  static constexpr int STAGES = COUT == 64 ? 5 : 8;
  static constexpr int A_BYTES = 128 * 128;            // one input row: 128 nodes x 64 channels BF16
  static constexpr int W_BYTES = 9 * COUT * 128;       // [tap][co] rows of 64 BF16
  static constexpr int CH = COUT / 2;                  // channels per epilogue thread
  static constexpr int XLD = COUT + 4;                 // exchange row stride in floats: 16-byte accesses
                                                       // of 8 consecutive rows hit distinct banks
  static constexpr int X_BYTES = 2 * 128 * XLD * 4;    // D_0 and D_2 of all 128 rows
  static constexpr int ACC = 3 * COUT;                 // tensor-memory columns of one accumulator set
  static constexpr uint32_t TMEM_COLS = 2 * ACC <= 256 ? 256 : 512;
  static constexpr size_t SMEM = 1024 + W_BYTES + STAGES * A_BYTES + X_BYTES + 256;
  // one MMA covers the three kernel columns of a kernel row: N = 3 * Cout (their
  // weight blocks are consecutive rows in shared memory, their accumulators
  // consecutive tensor-memory columns)
  static constexpr uint32_t IDESC = idesc_bf16(128, 3 * COUT);
  static constexpr int EPI = 256;          // epilogue threads (warps 2-9)
  static constexpr int THREADS = 64 + EPI;
};

template <int COUT>
__global__ void __launch_bounds__(320, 1)
    conv_fwd_tc_kernel(const __grid_constant__ CUtensorMap tmX, const bf16 *__restrict__ w,
                       const float *__restrict__ bias, const bf16 *__restrict__ mask, int rows, int H, int dil,
                       int relu, bf16 *__restrict__ y16, float *__restrict__ y32) {
  using C = TcCfg<COUT>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char *Ws = base;                            // 1024-aligned (W_BYTES is a multiple of 1024)
  unsigned char *As = Ws + C::W_BYTES;                 // STAGES x A_BYTES, each 1024-aligned
  float *xch = reinterpret_cast<float *>(As + C::STAGES * C::A_BYTES);
  uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(xch) + C::X_BYTES);
  uint64_t *empty = full + C::STAGES;
  uint64_t *tfull = empty + C::STAGES;  // [2]
  uint64_t *tempty = tfull + 2;         // [2]
  uint64_t *drain = tempty + 2;
  uint32_t *slot = reinterpret_cast<uint32_t *>(drain + 1);
  __shared__ int s_err;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // weights [co][tap][ci] -> shared [tap][co] swizzled rows
  for (int i = tid; i < 9 * COUT * 8; i += C::THREADS) {
    const int c = i & 7, row = i >> 3;  // row = co * 9 + tap
    const int co = row / 9, tap = row % 9;
    *reinterpret_cast<uint4 *>(Ws + tap * COUT * 128 + sw128_offset(co, c)) =
        *reinterpret_cast<const uint4 *>(w + (size_t)row * 64 + c * 8);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (tid == 0) {
    s_err = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull + a, 1);
      mbar_init(tempty + a, C::EPI);
    }
    mbar_init(drain, 1);
    mbar_fence_init();
  }
  if (warp == 1) {
    tc::alloc(slot, C::TMEM_COLS);
    tc::relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int it = 0;
      for (int r = blockIdx.x; r < rows && !read_flag(&s_err); r += gridDim.x) {
        const int b = r / H, yy = r % H;
        for (int ky = 0; ky < 3; ++ky, ++it) {
          const int s = it % C::STAGES, use = it / C::STAGES;
          if (use > 0 && !mbar_wait(empty + s, (use - 1) & 1)) {
            atomicExch(&s_err, 1);
            break;
          }
          int ys = (yy + (ky - 1) * dil) % H;
          if (ys < 0) ys += H;
          mbar_expect_tx(full + s, C::A_BYTES);
          tma_load_3d(As + s * C::A_BYTES, &tmX, 0, 0, b * H + ys, full + s);
        }
      }
      // loads still in flight land before the CTA may exit: wait for the last use of every stage
      for (int s = 0; s < C::STAGES && s < it; ++s) {
        const int last = ((it - 1 - s) / C::STAGES) * C::STAGES + s;  // last load issued into stage s
        mbar_wait(full + s, (last / C::STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int it = 0, ri = 0;
      for (int r = blockIdx.x; r < rows && !read_flag(&s_err); r += gridDim.x, ++ri) {
        const int a = ri & 1, use = ri >> 1;
        if (use > 0 && !mbar_wait(tempty + a, (use - 1) & 1)) {
          atomicExch(&s_err, 1);
          break;
        }
        tc::fence_after();
        const uint32_t dacc = tmem + (uint32_t)(a * C::ACC);
        bool ok = true;
        for (int ky = 0; ky < 3; ++ky, ++it) {
          const int s = it % C::STAGES;
          if (!mbar_wait(full + s, (it / C::STAGES) & 1)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint64_t da = sw128_desc(As + s * C::A_BYTES);
          const uint64_t dw = sw128_desc(Ws + 3 * ky * COUT * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) tc::mma(dacc, da + 2 * kk, dw + 2 * kk, C::IDESC, (ky | kk) ? 1u : 0u);
          tc::commit(empty + s);  // the stage is free once these MMAs have read it
        }
        if (!ok) {
          atomicExch(&s_err, 1);
          break;
        }
        tc::commit(tfull + a);
      }
      // every MMA this thread issued has completed before tensor memory is released
      tc::commit(drain);
      if (!mbar_wait(drain, 0)) atomicExch(&s_err, 1);
    }
  } else {
    // ---------------- epilogue: warps 2-9; tensor-memory lane quarter = warp % 4,
    // channel half = (warp - 2) / 4
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int p = q * 32 + lane;     // output node of this thread
    const int cb = half * C::CH;     // first channel of this thread
    float *x0 = xch, *x2 = xch + 128 * C::XLD;
    float bz[C::CH];  // this thread's biases, loaded once
#pragma unroll
    for (int j = 0; j < C::CH; ++j) bz[j] = bias ? bias[cb + j] : 0.f;
    int ri = 0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x, ++ri) {
      const int a = ri & 1, use = ri >> 1;
      const bool ok = mbar_wait(tfull + a, use & 1);
      if (!ok) atomicExch(&s_err, 1);
      // all epilogue warps leave together; this barrier also orders the previous
      // row's exchange reads before this row's exchange writes
      if (named_sync_or(1, C::EPI, !ok || read_flag(&s_err))) break;
      tc::fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * C::ACC + cb);
      float acc[C::CH], d0[C::CH], d2[C::CH];
      if constexpr (C::CH == 32) {
        tc_ld32x3(tbase, tbase + 2 * COUT, tbase + COUT, d0, d2, acc);
      } else {
        tc::ld16(tbase, d0);
        tc::ld16(tbase + 2 * COUT, d2);
        tc::ld16(tbase + COUT, acc);
      }
      tc::fence_before();
      mbar_arrive(tempty + a);
#pragma unroll
      for (int j = 0; j < C::CH; j += 4) {
        *reinterpret_cast<float4 *>(x0 + p * C::XLD + cb + j) = make_float4(d0[j], d0[j + 1], d0[j + 2], d0[j + 3]);
        *reinterpret_cast<float4 *>(x2 + p * C::XLD + cb + j) = make_float4(d2[j], d2[j + 1], d2[j + 2], d2[j + 3]);
      }
      named_sync(1, C::EPI);
      const float *r0 = x0 + ((p - dil) & 127) * C::XLD + cb;
      const float *r2 = x2 + ((p + dil) & 127) * C::XLD + cb;
#pragma unroll
      for (int j = 0; j < C::CH; j += 4) {
        const float4 u = *reinterpret_cast<const float4 *>(r0 + j);
        const float4 v = *reinterpret_cast<const float4 *>(r2 + j);
        acc[j] += u.x + v.x;
        acc[j + 1] += u.y + v.y;
        acc[j + 2] += u.z + v.z;
        acc[j + 3] += u.w + v.w;
      }
      const size_t o = ((size_t)r * 128 + p) * COUT + cb;
#pragma unroll
      for (int j = 0; j < C::CH; j += 8) {
        float t8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float t = acc[j + i] + bz[j + i];
          if (relu) t = fmaxf(t, 0.f);
          t8[i] = t;
        }
        if (mask) {
          const uint4 mk = *reinterpret_cast<const uint4 *>(mask + o + j);
          const bf16 *mb = reinterpret_cast<const bf16 *>(&mk);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (!(__bfloat162float(mb[i]) > 0.f)) t8[i] = 0.f;
        }
        if (y16) {
          uint4 pk;
          __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
          for (int i = 0; i < 4; ++i) h2[i] = __floats2bfloat162_rn(t8[2 * i], t8[2 * i + 1]);
          *reinterpret_cast<uint4 *>(y16 + o + j) = pk;
        }
        if (y32) {
          *reinterpret_cast<float4 *>(y32 + o + j) = make_float4(t8[0], t8[1], t8[2], t8[3]);
          *reinterpret_cast<float4 *>(y32 + o + j + 4) = make_float4(t8[4], t8[5], t8[6], t8[7]);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::dealloc(tmem, C::TMEM_COLS);
  if (tid == 0 && read_flag(&s_err)) atomicExch(&g_tc_status, 1);
}

// Failure-path self-test: one block waits on an mbarrier that nothing arrives
// at; the bounded wait gives up and records the error.
__global__ void wait_selftest_kernel() {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicExch(&g_tc_status, 1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode;
}

int g_sms = 0;
std::once_flag g_sms_once;
int sm_count() {
  std::call_once(g_sms_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 148;
  });
  return g_sms;
}

template <int COUT>
int launch_tc(const bf16 *x, const bf16 *w, const float *bias, const bf16 *mask, int rows, int H, int dil, int relu,
              bf16 *y16, float *y32, cudaStream_t s) {
  using C = TcCfg<COUT>;
  auto enc = encoder();
  if (!enc) return HERMITE_ERR_CUDA;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(conv_fwd_tc_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  });
  if (attr != cudaSuccess) return HERMITE_ERR_CUDA;
  // x viewed as [rows][128 nodes][64 channels]: innermost channel, then node, then row
  CUtensorMap tm;
  const cuuint64_t dims[3] = {64, 128, (cuuint64_t)rows};
  const cuuint64_t strides[2] = {64 * sizeof(bf16), 128 * 64 * sizeof(bf16)};
  const cuuint32_t box[3] = {64, 128, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(x), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HERMITE_ERR_CUDA;
  const int grid = rows < sm_count() ? rows : sm_count();
  conv_fwd_tc_kernel<COUT><<<grid, C::THREADS, C::SMEM, s>>>(tm, w, bias, mask, rows, H, dil, relu, y16, y32);
  return cudaGetLastError() == cudaSuccess ? HERMITE_OK : HERMITE_ERR_CUDA;
}

int g_engine = 0;  // 0: tensor-core kernels where supported, 1: mma.sync kernels only

}  // namespace

int conv_engine() { return g_engine; }

bool tc_conv_supported(int Cin, int Cout, int dil) {
  return g_engine == 0 && Cin == 64 && (Cout == 64 || Cout == 32) && dil >= 1 && dil <= kMaxTcDil;
}

int tc_conv_fwd(const bf16 *x, const bf16 *w, const float *bias, const bf16 *mask, int rows, int H, int dil,
                int relu, bf16 *y16, float *y32, int Cout, cudaStream_t s) {
  if (((uintptr_t)x & 15) || ((uintptr_t)w & 15) || (y16 && ((uintptr_t)y16 & 15)) || (y32 && ((uintptr_t)y32 & 15)) ||
      (mask && ((uintptr_t)mask & 15)))
    return HERMITE_ERR_ARG;
  if (Cout == 64) return launch_tc<64>(x, w, bias, mask, rows, H, dil, relu, y16, y32, s);
  return launch_tc<32>(x, w, bias, mask, rows, H, dil, relu, y16, y32, s);
}

}  // namespace hermite_nn

using namespace hermite_nn;

extern "C" {

int hnn_set_conv_engine(int engine) {
  if (engine != 0 && engine != 1) return HERMITE_ERR_ARG;
  g_engine = engine;
  return HERMITE_OK;
}

int hnn_conv_status(void) {
  int v = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return HERMITE_ERR_CUDA;
  if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) return HERMITE_ERR_CUDA;
  if (v) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int)) != cudaSuccess) return HERMITE_ERR_CUDA;
    return HERMITE_ERR_TIMEOUT;
  }
  return HERMITE_OK;
}

int hnn_wait_selftest(void *stream) {
  wait_selftest_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>();
  return cudaGetLastError() == cudaSuccess ? HERMITE_OK : HERMITE_ERR_CUDA;
}

int hnn_tc_gemm_selftest(const uint16_t *A, const uint16_t *B, float *D, int N, int *status, void *stream) {
  if (!A || !B || !D || !status || (N != 32 && N != 64)) return HERMITE_ERR_ARG;
  const size_t smem = 1024 + 128 * 128 + (size_t)N * 128 + 64;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto a = reinterpret_cast<const bf16 *>(A);
  auto b = reinterpret_cast<const bf16 *>(B);
  if (N == 64)
    tc_gemm_selftest_kernel<64><<<1, 128, smem, s>>>(a, b, D, status);
  else
    tc_gemm_selftest_kernel<32><<<1, 128, smem, s>>>(a, b, D, status);
  return cudaGetLastError() == cudaSuccess ? HERMITE_OK : HERMITE_ERR_CUDA;
}

}  // extern "C"
