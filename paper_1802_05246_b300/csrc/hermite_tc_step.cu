// Tensor-core (tcgen05) building blocks of the split-precision half-step.
//
// hermite_tc_selftest checks, on the device it runs on, the two properties the
// tensor-core half-step rests on:
//  * the shared-memory operand layout of tc::desc_kmajor (K-major, no swizzle,
//    16-column tiles), B operands cut to their first N rows and accumulators
//    placed at a column offset in tensor memory;
//  * exact FP32 accumulation of products of integer-valued BF16 operands
//    (|a|, |b| <= 256, K <= 128): every partial sum is an integer below 2^24.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hermite_device.cuh"

#include "hermite_internal.h"
#include "hermite_tc.cuh"

namespace hermite {
namespace {

constexpr int kSelfMaxK = 128, kSelfMaxN = 96;

__global__ void __launch_bounds__(128) tc_selftest_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                          int K, int N, float *__restrict__ D0,
                                                          float *__restrict__ D1, int *status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int nch = K / 16;
  unsigned char *As = sm;                       // [chunk][4096 B]
  unsigned char *Bs = As + nch * 4096;          // [chunk][N rows x 32 B]
  uint64_t *bar = reinterpret_cast<uint64_t *>(Bs + nch * N * 32);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 128 * K; i += 128) {
    const int r = i / K, k = i % K;
    *reinterpret_cast<__nv_bfloat16 *>(As + (k / 16) * 4096 + tc::kmajor16_offset(r, k % 16)) =
        __float2bfloat16_rn(A[i]);
  }
  for (int i = tid; i < N * K; i += 128) {
    const int r = i / K, k = i % K;
    *reinterpret_cast<__nv_bfloat16 *>(Bs + (k / 16) * N * 32 + tc::kmajor16_offset(r, k % 16)) =
        __float2bfloat16_rn(B[i]);
  }
  tc::fence_async_smem();
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::alloc(slot, 256);
    tc::relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    for (int ch = 0; ch < nch; ++ch) {
      const uint64_t da = tc::desc_kmajor(As + ch * 4096, 128, 256);
      const uint64_t db = tc::desc_kmajor(Bs + ch * N * 32, 128, 256);
      // D0 = A B^T at columns [0, N); D1 = A B[0:N-16]^T at columns [128 + 16, 128 + N)
      tc::mma(tmem, da, db, tc::idesc_bf16(128, N), ch > 0);
      tc::mma(tmem + 128 + 16, da, db, tc::idesc_bf16(128, N - 16), ch > 0);
    }
    tc::commit(bar);
  }
  const bool ok = tc::mbar_wait(bar, 0);
  tc::fence_after();
  if (ok) {
    const int row = tid;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      for (int j = 0; j < 16; ++j) D0[row * N + c0 + j] = v[j];
    }
    for (int c0 = 16; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + 128 + c0, v);
      for (int j = 0; j < 16; ++j) D1[row * (N - 16) + c0 - 16 + j] = v[j];
    }
  } else if ((tid & 31) == 0) {
    atomicExch(status, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 256);
}

// deterministic integer test values in [-256, 256], mostly of full size with
// some small ones; the sign is a row sign times a column sign shared by A and
// B, so that every product of a row pair has the same sign and the sums come
// close to 2^23 (exactness is tested near the top and at the bottom bit)
uint32_t selftest_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

float selftest_value(uint32_t row, uint32_t k, uint32_t salt) {
  const uint32_t h = selftest_hash(row * 1315423911u + k * 2654435761u + salt * 97u);
  const int sign = ((selftest_hash(row * 7919u + salt) ^ selftest_hash(k + 12345u)) & 1) ? -1 : 1;
  const uint32_t kind = h % 8;
  const int mag = kind < 6 ? 256 - (int)((h >> 4) % 3) : (int)((h >> 4) % 7) + 1;
  return (float)(sign * mag);
}

}  // namespace
}  // namespace hermite

extern "C" int hermite_tc_selftest(int K, int N, float *A, float *B, float *D0, float *D1) {
  using namespace hermite;
  if (K < 16 || K > kSelfMaxK || K % 16 || N < 32 || N > kSelfMaxN || N % 16 || !A || !B || !D0 || !D1)
    return HERMITE_ERR_ARG;
  for (int i = 0; i < 128 * K; ++i) A[i] = selftest_value(i / K, i % K, 1);
  for (int i = 0; i < N * K; ++i) B[i] = selftest_value(i / K, i % K, 2);
  float *dA = nullptr;
  const size_t nA = 128 * (size_t)K, nB = (size_t)N * K, n0 = 128 * (size_t)N, n1 = 128 * (size_t)(N - 16);
  if (device_alloc(&dA, sizeof(float) * (nA + nB + n0 + n1) + 16) != cudaSuccess) return HERMITE_ERR_ALLOC;
  float *dB = dA + nA, *dD0 = dB + nB, *dD1 = dD0 + n0;
  int *dstatus = reinterpret_cast<int *>(dD1 + n1);
  int status = 0, rc = HERMITE_OK;
  const size_t smem = (size_t)(K / 16) * (4096 + N * 32) + 64;
  if (cudaMemcpy(dA, A, sizeof(float) * nA, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dB, B, sizeof(float) * nB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(dstatus, 0, sizeof(int)) != cudaSuccess ||
      cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    rc = HERMITE_ERR_CUDA;
  } else {
    tc_selftest_kernel<<<1, 128, smem>>>(dA, dB, K, N, dD0, dD1, dstatus);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(D0, dD0, sizeof(float) * n0, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(D1, dD1, sizeof(float) * n1, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&status, dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = HERMITE_ERR_CUDA;
    else if (status)
      rc = HERMITE_ERR_TIMEOUT;
  }
  cudaFree(dA);
  return rc;
}

// ---------------------------------------------------------------------------
// Split-precision half-step on the tensor cores.
//
// The map is the one of the CUDA-core kernels: corner gather with the ghost
// signs of Sec. 3.1.3, Walsh-Hadamard transform over the 2^d corners
// (z_q[b] = sum_s (-1)^{|q & s|} x_s[b]) and, for every output a of parity
// class c = par(a), out[a] = sum_b M0[a][b] Y_c[b] with Y_c[b] = z_{c ^ par(b)}[b].
// Per output class this is a product (nodes x inputs) . (inputs x outputs),
// done here on tcgen05 with an exact digit split (the fixed-point slicing of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication", 2012):
//  * data side: per node and class, Y_c scaled by 2^(8 - E_c), with 2^E_c
//    above max |Y_c| (a bound from an FP32 pre-pass), split into six signed
//    8-bit digits A_0..A_5 (|A_0| <= 256, the rest <= 128, each exact in BF16);
//  * operator side: M' = M0 with its velocity columns divided by 2^vexp (the
//    data side multiplies velocity inputs by 2^vexp, which balances u and v),
//    each row scaled by 2^(8 - er[a]) and split into seven digits B_0..B_6;
//  * every product A_i . B_j with i + j <= 6 is formed by tcgen05.mma in FP32:
//    all terms are integers and every partial sum stays below 2^24 (at most
//    91 inputs), so each is exact; the products of one diagonal k = i + j
//    share an accumulator, seven diagonals per class in tensor memory;
//  * out[a] = 2^(E_c + er[a] - 16) sum_k 2^(-8k) D_k[a], summed in FP32 hi + lo.
// What is dropped: data digits below 2^-48 of the class maximum and the digit
// products below 2^-56 of the row and class maxima.
//
// Work split: a CTA owns 128 consecutive target nodes at a time (one per
// tensor-memory lane); 256 threads, thread t and t + 128 share a node and
// take K slots 0-7 and 8-15 of each 16-wide parity-class chunk (a class's
// inputs are dealt to the two halves in pairs, in turn: see k_slot).
// Per tile, one FP32 pre-pass over the corner data bounds max |Y_c| for all
// classes.  Output classes then go in groups of four (3-D: two groups), so
// that a group's accumulators (4 classes x 7 diagonals x 16 columns) fit in
// tensor memory.  Per input parity class p (a 16-wide K chunk, whose inputs
// share their parity and so their ghost signs), the threads write the digits
// of their inputs to one of two shared-memory A buffers while the tensor core
// works on the other; each thread handles two inputs per packed FP32 lane
// pair (transform, digits and BF16x2 packing without lane shuffles).  Every
// thread arrives on the buffer's mbarrier when its digits are stored; lane 0
// of warp (chunk % 8) waits for all of them, for the operator chunk (a bulk
// copy it started) and for the previous chunk's MMAs, then issues 24 MMAs
// (4 classes x 6 data digits, N = 16 (7 - i) operator digits each) and
// commits them to the buffer's mbarrier, which frees the buffer two chunks
// later.  The epilogue reads the diagonals with tcgen05.ld and arrives on a
// barrier that the next group's first MMA waits for.  Every wait is bounded.
// ---------------------------------------------------------------------------
namespace hermite {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcDigits = 6;                         // data digits
constexpr int kTcMDigits = 7;                        // operator digits = diagonals
constexpr int kTcClasses = 4;                        // output classes per group
constexpr int kTcCols = kTcMDigits * 16;             // tensor-memory columns per class
constexpr int kTcTileA = 4096;                       // 128 rows x 16 K, BF16
constexpr int kTcTileB = kTcCols * 32;               // 112 rows x 16 K, BF16
constexpr int kTcBufA = kTcClasses * kTcDigits * kTcTileA;
constexpr int kTcBufB = kTcClasses * kTcTileB;
constexpr int kTcMaxNC = 8;
constexpr size_t kTcSmem = 2 * (size_t)kTcBufA + 2 * (size_t)kTcBufB + kTcMaxNC * 128 * 4 + 6 * kTcMaxNC * 16 + 64;

struct TcArgs {
  Geometry g;
  const float2 *src;
  float2 *dst;
  int subtract_old;
  const uint4 *Bimg;     // [group][input class][class in group][112 x 16 K-major BF16 tile]
  const int16_t *inb;    // [2^d][16] input coefficient at (input class, position), -1 = none
  const int16_t *orow;   // [2^d][16] output row at (output class, position), -1 = none
  const int8_t *er;      // [nco] operator row exponents
  int nu;                // inputs b >= nu are velocity coefficients
  int vexp;              // velocity inputs are multiplied by 2^vexp
  int *status;           // set by a bounded wait that ran out
};

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // e in [-126, 127]

// 2^e for e in [-252, 252] as a product of two normal powers of two
__device__ __forceinline__ float2 pow2_split(int e) {
  const int e1 = e / 2;
  return make_float2(pow2f(e1), pow2f(e - e1));
}

// FP32 transform over all 2^d corners for two inputs at once (packed lanes;
// butterflies in the order of the corner bits): z[q] = sum_s (-1)^{|q & s|} x[s]
template <int D>
__device__ __forceinline__ void transform_f32_x2(float2 *x) {
#pragma unroll
  for (int bm = 1; bm < (1 << D); bm <<= 1)
#pragma unroll
    for (int i = 0; i < (1 << D); ++i)
      if (!(i & bm)) {
        const float2 a = x[i], c = x[i | bm];
        x[i] = __fadd2_rn(a, c);
        x[i | bm] = __ffma2_rn(c, make_float2(-1.f, -1.f), a);
      }
}

// (ah, al) += sg * (bh, bl) for two independent values in packed lanes, in
// FP32 hi + lo (Knuth's two-sum of the hi parts, the lo parts added to its
// error); sg = +-1 (exact), so a - b costs the same as a + b.
__device__ __forceinline__ void df_axpy_x2(float2 &ah, float2 &al, const float2 sg, const float2 bh, const float2 bl) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __ffma2_rn(sg, bh, ah);                 // fl(a + sg b)
  const float2 bb = __ffma2_rn(ah, m1, s);                 // s - a
  const float2 t1 = __ffma2_rn(bb, m1, s);                 // s - bb
  const float2 e1 = __ffma2_rn(t1, m1, ah);                // a - (s - bb)
  const float2 e2 = __ffma2_rn(bb, m1, __fmul2_rn(sg, bh));  // sg b - bb
  const float2 e = __fadd2_rn(__fadd2_rn(e1, e2), __ffma2_rn(sg, bl, al));
  ah = s;
  al = e;
}

// Corner transform restricted to one group of four output classes, for two
// inputs of the same input class at once (lane x: one input, lane y: the
// next), in FP32 hi + lo: (zh[j], zl[j]) = z_q with q & 3 = j and the top
// corner bit of q (3-D) fixed by group gi and input class p.
template <int D>
__device__ __forceinline__ void group_transform_pair(const float2 *h, const float2 *l, int gi, int p, float2 (&zh)[4],
                                                     float2 (&zl)[4]) {
  const float2 P1 = make_float2(1.f, 1.f), M1 = make_float2(-1.f, -1.f);
  float2 yh[4], yl[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    yh[i] = h[i];
    yl[i] = l[i];
  }
  if constexpr (D == 3) {
    const float2 sg = ((gi ^ (p >> 2)) & 1) ? M1 : P1;
#pragma unroll
    for (int i = 0; i < 4; ++i) df_axpy_x2(yh[i], yl[i], sg, h[i + 4], l[i + 4]);
  }
  // corner bit 0: (y0 + y1, y0 - y1, y2 + y3, y2 - y3)
  float2 ah[4] = {yh[0], yh[0], yh[2], yh[2]}, al[4] = {yl[0], yl[0], yl[2], yl[2]};
  df_axpy_x2(ah[0], al[0], P1, yh[1], yl[1]);
  df_axpy_x2(ah[1], al[1], M1, yh[1], yl[1]);
  df_axpy_x2(ah[2], al[2], P1, yh[3], yl[3]);
  df_axpy_x2(ah[3], al[3], M1, yh[3], yl[3]);
  // corner bit 1: z0 = a0 + a2, z1 = a1 + a3, z2 = a0 - a2, z3 = a1 - a3
  zh[0] = ah[0]; zl[0] = al[0];
  zh[1] = ah[1]; zl[1] = al[1];
  zh[2] = ah[0]; zl[2] = al[0];
  zh[3] = ah[1]; zl[3] = al[1];
  df_axpy_x2(zh[0], zl[0], P1, ah[2], al[2]);
  df_axpy_x2(zh[1], zl[1], P1, ah[3], al[3]);
  df_axpy_x2(zh[2], zl[2], M1, ah[2], al[2]);
  df_axpy_x2(zh[3], zl[3], M1, ah[3], al[3]);
}

// Six signed 8-bit digits of two values of one class at once (packed lanes),
// each v = (hi + lo) * sc with |v| <= 256: v = sum_i d_i 2^(-8 i) up to a
// remainder below 2^-41; d[i] holds digit i of both values.  Each digit is the
// nearest integer to the rounded sum of the remainder pair (1.5 * 2^23
// shift), the remainder itself is kept exactly as hi and lo parts, so
// |d_0| <= 256 and |d_i| <= 128 for i > 0 (every digit exact in BF16).
__device__ __forceinline__ void six_digits_pair(float2 h, float2 l, float2 sc, float2 (&d)[kTcDigits]) {
  // digit i is taken at granularity 2^(-8 i) (shift constant 1.5 * 2^(23 - 8 i))
  // and only the digit is scaled back to an integer: the same roundings as
  // scaling the remainder by 256 before every digit, one multiply fewer
  const float2 M1 = make_float2(-1.0f, -1.0f);
  float2 rh = __fmul2_rn(h, sc), rl = __fmul2_rn(l, sc);
  float ci = 12582912.0f, si = 1.0f;  // 1.5 * 2^(23 - 8 i) and 2^(8 i), exact
#pragma unroll
  for (int i = 0; i < kTcDigits; ++i) {
    const float2 C = make_float2(ci, ci);
    const float2 q = __ffma2_rn(C, M1, __fadd2_rn(__fadd2_rn(rh, rl), C));  // a multiple of 2^(-8 i)
    rh = __ffma2_rn(q, M1, rh);
    d[i] = i == 0 ? q : __fmul2_rn(q, make_float2(si, si));
    ci *= 0.00390625f;
    si *= 256.0f;
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&b);
}

// smallest E with 2^E > m (m >= 0), clamped to the range the scalings use
__device__ __forceinline__ int bound_exponent(float m) {
  if (!(m > 0.0f)) return -100;
  const int e = ((__float_as_int(m) >> 23) & 0xFF) - 127;
  return max(-100, min(100, e + 1));
}

}  // namespace
}  // namespace hermite

namespace hermite {
namespace {

template <int D>
__global__ void __launch_bounds__(kTcThreads, 1) half_step_tc_kernel(const TcArgs a) {
  constexpr int NC = 1 << D;
  constexpr int NG = NC / kTcClasses;  // groups of four output classes
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char *Abuf = tsm;                                           // [2][class][digit][4096]
  unsigned char *Bbuf = Abuf + 2 * kTcBufA;                            // [2][class][112 x 16]
  float *mxs = reinterpret_cast<float *>(Bbuf + 2 * kTcBufB);          // [class][128]
  int16_t *s_inb = reinterpret_cast<int16_t *>(mxs + kTcMaxNC * 128);  // [NC][16]
  int16_t *s_orow = s_inb + kTcMaxNC * 16;                             // [NC][16]
  int8_t *s_er = reinterpret_cast<int8_t *>(s_orow + kTcMaxNC * 16);    // [NC][16] row exponent by (class, position)
  int8_t *s_sh = s_er + kTcMaxNC * 16;                                 // [NC][16]
  uint64_t *bar = reinterpret_cast<uint64_t *>(s_sh + kTcMaxNC * 16);   // [2] MMAs of a buffer done
  uint64_t *bar_b = bar + 2;                                            // [2] operator chunk arrived
  uint64_t *full = bar + 4;                                             // [2] every thread wrote its digits
  uint64_t *tfree = bar + 6;                                            // every thread read the accumulators
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 7);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int node = tid & 127, half = tid >> 7;
  const Geometry &g = a.g;
  for (int i = tid; i < NC * 16; i += kTcThreads) {
    const int b = a.inb[i];
    s_inb[i] = (int16_t)b;
    s_sh[i] = (int8_t)(b >= a.nu ? a.vexp : 0);
    const int row = a.orow[i];
    s_orow[i] = (int16_t)row;
    s_er[i] = row >= 0 ? a.er[row] : (int8_t)0;
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_init(&bar_b[0], 1);
    tc::mbar_init(&bar_b[1], 1);
    tc::mbar_init(&full[0], kTcThreads);
    tc::mbar_init(&full[1], kTcThreads);
    tc::mbar_init(tfree, kTcThreads);
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::alloc(slot, 512);
    tc::relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint64_t desc_a0 = tc::desc_kmajor(Abuf, 128, 256), desc_b0 = tc::desc_kmajor(Bbuf, 128, 256);
  uint32_t it = 0;      // K chunks this CTA has produced
  uint32_t groups = 0;  // class groups whose accumulators this CTA has read
  // A wait that runs out marks this thread failed: from then on it skips its
  // waits (so nothing waits on it for long) and the CTA stops at the next tile.
  bool failed = false;
  auto wait = [&](uint64_t *b, uint32_t parity) {
    if (!failed && !tc::mbar_wait(b, parity)) failed = true;
  };
  const int64_t ntiles = (g.nodes_dst + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (__syncthreads_or(failed)) break;
    const int64_t t = tile * 128 + node;
    const bool valid = t < g.nodes_dst;
    int idx[NC];
    uint64_t negm = 0;  // byte p: corners whose ghost image flips inputs of parity p
    {
      int64_t li[NC];
      int gm[NC];
      if (valid) {
        dev::cell_corners<D>(g, t, li, gm);
      } else {
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          li[s] = 0;
          gm[s] = 0;
        }
      }
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        idx[s] = (int)li[s];
        if (gm[s])
#pragma unroll
          for (int p = 0; p < NC; ++p)
            if (dev::ghost_negates(g.bc, gm[s], p)) negm |= (uint64_t)1 << (8 * p + s);
      }
    }
    // ---- pre-pass: bound max |Y_c| for every output class (FP32 transform of
    // the hi parts; the lo parts and the roundings are covered by 2^-20 sum |x|)
    // Two inputs per packed lane pair, the corners of the pair after next
    // loaded while this one is transformed.
    float mx[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) mx[c] = 0.f;
    // the input-class loop stays rolled (code size): maxima are kept by q and
    // moved to the classes c = q ^ p once per input class
#pragma unroll 1
    for (int p = 0; p < NC; ++p) {
      const uint32_t neg = (uint32_t)(negm >> (8 * p)) & 0xFF;
      const int16_t *pin = s_inb + p * 16 + half * 8;
      float tq[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) tq[q] = 0.f;
      float2 nx[2][NC];
      auto load_pair = [&](int j) {
        const int b0 = pin[2 * j], b1 = pin[2 * j + 1];
        if (b0 < 0) return;
        const float2 *p0 = a.src + (size_t)b0 * g.ld_src;
        const float2 *p1 = a.src + (size_t)(b1 >= 0 ? b1 : b0) * g.ld_src;
#pragma unroll
        for (int s = 0; s < NC; ++s) nx[j & 1][s] = make_float2(p0[idx[s]].x, p1[idx[s]].x);
      };
      load_pair(0);
      load_pair(1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b0 = pin[2 * j], b1 = pin[2 * j + 1];
        if (b0 < 0) break;  // a class's inputs come first, the padding after
        float2 x[NC];
#pragma unroll
        for (int s = 0; s < NC; ++s) x[s] = nx[j & 1][s];
        if (b1 < 0) {
#pragma unroll
          for (int s = 0; s < NC; ++s) x[s].y = 0.f;
        }
        if (j < 2) load_pair(j + 2);
        float2 S = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < NC; ++s) {
          S.x += fabsf(x[s].x);
          S.y += fabsf(x[s].y);
        }
        if (neg) {
#pragma unroll
          for (int s = 0; s < NC; ++s)
            if ((neg >> s) & 1) x[s] = make_float2(-x[s].x, -x[s].y);
        }
        transform_f32_x2<D>(x);
        const float2 sc = make_float2(pow2f(s_sh[p * 16 + half * 8 + 2 * j]), pow2f(s_sh[p * 16 + half * 8 + 2 * j + 1]));
        const float2 sl = make_float2(S.x * 9.5367431640625e-07f * sc.x, S.y * 9.5367431640625e-07f * sc.y);
#pragma unroll
        for (int q = 0; q < NC; ++q)
          tq[q] = fmaxf(tq[q], fmaxf(__fmaf_rn(fabsf(x[q].x), sc.x, sl.x), __fmaf_rn(fabsf(x[q].y), sc.y, sl.y)));
      }
      // tq[q] -> class q ^ p: exchange the halves of every pair of entries
      // that differ in a set bit of p
#pragma unroll
      for (int bm = 1; bm < NC; bm <<= 1)
        if (p & bm)
#pragma unroll
          for (int q = 0; q < NC; ++q)
            if (!(q & bm)) {
              const float t0 = tq[q];
              tq[q] = tq[q | bm];
              tq[q | bm] = t0;
            }
#pragma unroll
      for (int c = 0; c < NC; ++c) mx[c] = fmaxf(mx[c], tq[c]);
    }
    // combine the two halves of each node's inputs
    if (half) {
#pragma unroll
      for (int c = 0; c < NC; ++c) mxs[c * 128 + node] = mx[c];
    }
    __syncthreads();
    if (!half) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        mx[c] = fmaxf(mx[c], mxs[c * 128 + node]);
        mxs[c * 128 + node] = mx[c];
      }
    }
    __syncthreads();
    int E[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) E[c] = bound_exponent(mxs[c * 128 + node]);
    // the group loop stays rolled: its body is large enough that two copies
    // miss the instruction cache
#pragma unroll 1
    for (int gi = 0; gi < NG; ++gi) {
      // this group's four exponents (a select, not a run-time register index)
      int Eg[kTcClasses];
#pragma unroll
      for (int cc = 0; cc < kTcClasses; ++cc) Eg[cc] = (NG > 1 && gi) ? E[(NG > 1 ? kTcClasses : 0) + cc] : E[cc];
      // per-class digit scales of u and (balanced) v inputs
      float scu[kTcClasses], scv[kTcClasses];
#pragma unroll
      for (int cc = 0; cc < kTcClasses; ++cc) {
        scu[cc] = pow2f(8 - Eg[cc]);
        scv[cc] = pow2f(a.vexp + 8 - Eg[cc]);
      }
      // ---- K loop over input parity classes
      for (int p = 0; p < NC; ++p, ++it) {
        const int buf = it & 1;
        // the chunk's MMAs are issued by one thread, warp it % 8 in turn, so
        // the other warps go on with the next chunk meanwhile
        const bool issuer = warp == (int)(it & 7) && lane == 0;
        if (it >= 2) wait(&bar[buf], ((it >> 1) - 1) & 1);  // MMAs of chunk it - 2 done: buffers free
        // this chunk's operator digits arrive asynchronously while the
        // threads produce the data digits; only the issuer waits for them
        if (issuer && !failed) {
          tc::mbar_expect_tx(&bar_b[buf], kTcBufB);
          tc::bulk_g2s(Bbuf + buf * kTcBufB, a.Bimg + (size_t)(gi * NC + p) * (kTcBufB / 16), kTcBufB, &bar_b[buf]);
        }
        const uint32_t neg = (uint32_t)(negm >> (8 * p)) & 0xFF;
        // digit scales in the order of q: z_q goes to class cc = q ^ (p & 3)
        float squ[kTcClasses], sqv[kTcClasses];
#pragma unroll
        for (int q = 0; q < kTcClasses; ++q) {
          const int cc = q ^ (p & 3);
          squ[q] = cc == 0 ? scu[0] : cc == 1 ? scu[1] : cc == 2 ? scu[2] : scu[3];
          sqv[q] = cc == 0 ? scv[0] : cc == 1 ? scv[1] : cc == 2 ? scv[2] : scv[3];
        }
        // two inputs per packed lane pair: positions (2j, 2j + 1) of this
        // thread's eight; the corner data of pair j + 1 are loaded while pair j
        // is transformed.  Positions past the class's inputs are zero padding
        // (the same for the whole warp) and skip all arithmetic.
        uint32_t pk[kTcClasses][kTcDigits][2];  // two pairs of digits: one 8-byte word per class and digit
        float2 nh[NC], nl[NC];
        const int16_t *pin = s_inb + p * 16 + half * 8;
        unsigned char *Ab = Abuf + buf * kTcBufA + tc::kmajor16_offset(node, half * 8);
        auto load_pair = [&](int j) {
          const int b0 = pin[2 * j], b1 = pin[2 * j + 1];
          if (b0 < 0) return;
          const float2 *p0 = a.src + (size_t)b0 * g.ld_src;
          const float2 *p1 = a.src + (size_t)(b1 >= 0 ? b1 : b0) * g.ld_src;
#pragma unroll
          for (int s = 0; s < NC; ++s) {
            const float2 v0 = p0[idx[s]], v1 = p1[idx[s]];
            nh[s] = make_float2(v0.x, v1.x);
            nl[s] = make_float2(v0.y, v1.y);
          }
        };
        load_pair(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int b0 = pin[2 * j], b1 = pin[2 * j + 1];
          if (b0 < 0) {
#pragma unroll
            for (int q = 0; q < kTcClasses; ++q)
#pragma unroll
              for (int i = 0; i < kTcDigits; ++i) pk[q][i][j & 1] = 0u;
          } else {
            float2 xh[NC], xl[NC];
#pragma unroll
            for (int s = 0; s < NC; ++s) {
              xh[s] = nh[s];
              xl[s] = nl[s];
            }
            if (b1 < 0) {  // an odd class size: the second lane is padding
#pragma unroll
              for (int s = 0; s < NC; ++s) {
                xh[s].y = 0.f;
                xl[s].y = 0.f;
              }
            }
            if (neg) {  // ghost images (non-periodic boundaries only)
#pragma unroll
              for (int s = 0; s < NC; ++s)
                if ((neg >> s) & 1) {
                  xh[s] = make_float2(-xh[s].x, -xh[s].y);
                  xl[s] = make_float2(-xl[s].x, -xl[s].y);
                }
            }
            if (j < 3) load_pair(j + 1);
            float2 zh[4], zl[4];
            group_transform_pair<D>(xh, xl, gi, p, zh, zl);
            const bool v0 = s_sh[p * 16 + half * 8 + 2 * j] != 0, v1 = s_sh[p * 16 + half * 8 + 2 * j + 1] != 0;
#pragma unroll
            for (int q = 0; q < kTcClasses; ++q) {
              float2 d[kTcDigits];
              six_digits_pair(zh[q], zl[q], make_float2(v0 ? sqv[q] : squ[q], v1 ? sqv[q] : squ[q]), d);
#pragma unroll
              for (int i = 0; i < kTcDigits; ++i) pk[q][i][j & 1] = pack_bf16x2(d[i].x, d[i].y);
            }
          }
          if (j & 1) {  // positions 4 (j >> 1) .. + 3 of this thread's eight
#pragma unroll
            for (int q = 0; q < kTcClasses; ++q) {
              unsigned char *Aq = Ab + (q ^ (p & 3)) * kTcDigits * kTcTileA + 8 * (j >> 1);
#pragma unroll
              for (int i = 0; i < kTcDigits; ++i)
                *reinterpret_cast<uint2 *>(Aq + i * kTcTileA) = make_uint2(pk[q][i][0], pk[q][i][1]);
            }
          }
        }
        tc::fence_async_smem();
        tc::mbar_arrive(&full[buf]);
        if (issuer) {
          wait(&full[buf], (it >> 1) & 1);    // every thread's digits
          wait(&bar_b[buf], (it >> 1) & 1);   // the operator digits
          if (it >= 1) wait(&bar[(it - 1) & 1], ((it - 1) >> 1) & 1);  // chunk it - 1 first (another thread's MMAs)
          if (p == 0 && groups > 0) wait(tfree, (groups - 1) & 1);     // accumulators read before they restart
        }
        if (issuer && !failed) {
          tc::fence_after();
          // digit-major order: consecutive MMAs go to different classes'
          // accumulators, which do not depend on one another.  Descriptors are
          // the buffer's base descriptor plus the tile offset in 16-byte units
          // (shared-memory addresses stay below 2^18, inside the 14-bit field).
          const uint64_t da0 = desc_a0 + (uint64_t)((buf * kTcBufA) >> 4);
          const uint64_t db0 = desc_b0 + (uint64_t)((buf * kTcBufB) >> 4);
#pragma unroll
          for (int i = 0; i < kTcDigits; ++i)
#pragma unroll
            for (int cc = 0; cc < kTcClasses; ++cc)
              tc::mma(tmem + cc * kTcCols + 16 * i, da0 + (uint64_t)(((cc * kTcDigits + i) * kTcTileA) >> 4),
                      db0 + (uint64_t)((cc * kTcTileB) >> 4), tc::idesc_bf16(128, 16 * (kTcMDigits - i)),
                      (p > 0 || i > 0) ? 1u : 0u);
          tc::commit(&bar[buf]);
        }
        __syncwarp();
      }
      // ---- epilogue: the seven diagonals of each class -> FP32 hi + lo outputs
      wait(&bar[(it - 1) & 1], ((it - 1) >> 1) & 1);  // the group's last MMAs (issued after all others)
      tc::fence_after();
#pragma unroll 1
      for (int cq = 0; cq < 2; ++cq) {
        const int cc = half * 2 + cq, c = gi * kTcClasses + cc;
        const int Ec = half ? (cq ? Eg[3] : Eg[2]) : (cq ? Eg[1] : Eg[0]);
        float acc[kTcMDigits][16];
#pragma unroll
        for (int k = 0; k < kTcMDigits; ++k) tc::ld16(tmem + lane_base + cc * kTcCols + 16 * k, acc[k]);
#pragma unroll
        for (int n = 0; n < 16; ++n) {
          const int row = s_orow[c * 16 + n];
          if (row < 0) continue;
          float2 r = make_float2(acc[kTcMDigits - 1][n] * pow2f(-8 * (kTcMDigits - 1)), 0.f);
#pragma unroll
          for (int k = kTcMDigits - 2; k >= 0; --k) r = dev::df_add(r, make_float2(acc[k][n] * pow2f(-8 * k), 0.f));
          const float2 sc = pow2_split(Ec + s_er[c * 16 + n] - 16);
          r = make_float2(__fmul_rn(__fmul_rn(r.x, sc.x), sc.y), __fmul_rn(__fmul_rn(r.y, sc.x), sc.y));
          if (valid) {
            float2 *o = a.dst + (size_t)row * g.ld_dst + t;
            if (a.subtract_old) r = dev::df_add(r, dev::df_neg(*o));
            *o = dev::df_norm(r);
          }
        }
      }
      tc::fence_before();
      tc::mbar_arrive(tfree);  // the next group's first MMA may overwrite the accumulators
      ++groups;
    }
  }
  if (failed) atomicExch(a.status, 1);
  // the last MMAs and operator copies (in flight only after a failure) end,
  // bounded, before the tensor and shared memory go
  if (it > 0) {
    (void)tc::mbar_wait(&bar[(it - 1) & 1], ((it - 1) >> 1) & 1);
    (void)tc::mbar_wait(&bar_b[(it - 1) & 1], ((it - 1) >> 1) & 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 512);
}

}  // namespace
}  // namespace hermite

namespace hermite {

// Host side of the tensor-core half-step: the operator's digit image.
// M' = M0 with velocity columns divided by 2^vexp; row a scaled by
// 2^(8 - er[a]) (2^er[a] > max_b |M'[a][b]|) and split, in FP64 (exact), into
// seven digits by rounding to the nearest integer, remainder times 256.  Tile
// (group, input class p, class cc of the group) holds rows j * 16 + n (digit
// j of output n of class 4 group + cc) and K columns k (input k of class p),
// zero where a class has fewer than 16 members.
namespace {
// K slot of the k-th input of a parity class: consecutive input pairs go to
// the two halves of the 16 slots in turn (slots 0-7 are read by the first
// thread of each node, 8-15 by the second), so that both threads of a node
// get about half of a class's 9-16 inputs; each half keeps its real inputs
// first and its padding after.
int k_slot(int k) {
  const int pair = k >> 1;
  return (pair & 1) * 8 + (pair >> 1) * 2 + (k & 1);
}
}  // namespace

int build_tc_operator(hermite_ctx *ctx) {
  ctx->tc_ready = false;
  ctx->split_engine = 0;
  const int d = ctx->d, NC = 1 << d;
  // every partial sum of a diagonal stays below 2^24 for at most 127 inputs;
  // node indices and planes are addressed with 32-bit offsets
  if (d < 2 || ctx->nci > 127 || ctx->nodes[0] >= (int64_t(1) << 31) || ctx->nodes[1] >= (int64_t(1) << 31))
    return HERMITE_OK;
  std::vector<double> M((size_t)ctx->nco * ctx->nci);
  std::vector<int8_t> par(ctx->nci);
  if (!cuda_ok(ctx, cudaMemcpy(M.data(), ctx->M, sizeof(double) * M.size(), cudaMemcpyDeviceToHost), "copy M") ||
      !cuda_ok(ctx, cudaMemcpy(par.data(), ctx->par_in, par.size(), cudaMemcpyDeviceToHost), "copy parity"))
    return HERMITE_ERR_CUDA;
  std::vector<std::vector<int>> in_cls(NC), out_cls(NC);
  for (int b = 0; b < ctx->nci; ++b) in_cls[par[b]].push_back(b);
  for (int a = 0; a < ctx->nco; ++a) out_cls[par[a]].push_back(a);
  for (int c = 0; c < NC; ++c)
    if (in_cls[c].size() > 16 || out_cls[c].size() > 16) return HERMITE_OK;  // CUDA-core kernel only
  const bool has_v = ctx->variant != HERMITE_CONSERVATIVE && ctx->Nv > 0;
  const int vexp = has_v ? std::max(-15, std::min(15, (int)std::lround(std::log2(ctx->h / ctx->c)))) : 0;
  std::vector<int8_t> er(ctx->nco, 0);
  std::vector<double> Mp(M.size());
  for (int a = 0; a < ctx->nco; ++a) {
    double mx = 0.0;
    for (int b = 0; b < ctx->nci; ++b) {
      const double v = M[(size_t)a * ctx->nci + b] * (b >= ctx->Nu ? std::ldexp(1.0, -vexp) : 1.0);
      Mp[(size_t)a * ctx->nci + b] = v;
      mx = std::max(mx, std::fabs(v));
    }
    int e = 0;
    if (mx > 0) std::frexp(mx, &e);  // mx < 2^e
    if (e < -60 || e > 60) return HERMITE_OK;
    er[a] = (int8_t)e;
  }
  const int NG = NC / 4;
  const size_t tile_bytes = kTcTileB;
  std::vector<uint16_t> img((size_t)NG * NC * 4 * tile_bytes / 2, 0);
  for (int gi = 0; gi < NG; ++gi)
    for (int p = 0; p < NC; ++p)
      for (int cc = 0; cc < 4; ++cc) {
        const int c = gi * 4 + cc;
        uint16_t *tile = img.data() + ((size_t)(gi * NC + p) * 4 + cc) * (tile_bytes / 2);
        for (size_t n = 0; n < out_cls[c].size(); ++n)
          for (size_t k = 0; k < in_cls[p].size(); ++k) {
            const int a = out_cls[c][n], b = in_cls[p][k];
            double r = std::ldexp(Mp[(size_t)a * ctx->nci + b], 8 - er[a]);
            for (int j = 0; j < kTcMDigits; ++j) {
              const double dg = std::nearbyint(r);
              r = (r - dg) * 256.0;
              const float f = (float)dg;  // an integer of at most 9 bits: its BF16 is the top half
              uint32_t bits;
              std::memcpy(&bits, &f, 4);
              tile[tc::kmajor16_offset(j * 16 + (int)n, k_slot((int)k)) / 2] = (uint16_t)(bits >> 16);
            }
          }
      }
  std::vector<int16_t> inb((size_t)NC * 16, -1), orow((size_t)NC * 16, -1);
  for (int c = 0; c < NC; ++c) {
    for (size_t k = 0; k < in_cls[c].size(); ++k) inb[c * 16 + k_slot((int)k)] = (int16_t)in_cls[c][k];
    for (size_t n = 0; n < out_cls[c].size(); ++n) orow[c * 16 + n] = (int16_t)out_cls[c][n];
  }
  if (!cuda_ok(ctx, device_alloc(&ctx->tc_B, img.size() * 2), "cudaMalloc tc_B") ||
      !cuda_ok(ctx, device_alloc(&ctx->tc_inb, inb.size() * 2), "cudaMalloc tc_inb") ||
      !cuda_ok(ctx, device_alloc(&ctx->tc_orow, orow.size() * 2), "cudaMalloc tc_orow") ||
      !cuda_ok(ctx, device_alloc(&ctx->tc_er, er.size()), "cudaMalloc tc_er") ||
      !cuda_ok(ctx, device_alloc(&ctx->tc_status, sizeof(int)), "cudaMalloc tc_status"))
    return HERMITE_ERR_ALLOC;
  if (!cuda_ok(ctx, cudaMemcpy(ctx->tc_B, img.data(), img.size() * 2, cudaMemcpyHostToDevice), "copy tc_B") ||
      !cuda_ok(ctx, cudaMemcpy(ctx->tc_inb, inb.data(), inb.size() * 2, cudaMemcpyHostToDevice), "copy inb") ||
      !cuda_ok(ctx, cudaMemcpy(ctx->tc_orow, orow.data(), orow.size() * 2, cudaMemcpyHostToDevice), "copy orow") ||
      !cuda_ok(ctx, cudaMemcpy(ctx->tc_er, er.data(), er.size(), cudaMemcpyHostToDevice), "copy er") ||
      !cuda_ok(ctx, cudaMemset(ctx->tc_status, 0, sizeof(int)), "clear tc_status"))
    return HERMITE_ERR_CUDA;
  ctx->tc_vexp = vexp;
  ctx->tc_ready = true;
  return HERMITE_OK;
}

namespace {
template <int D>
int launch_tc_d(hermite_ctx *ctx, const TcArgs &a) {
  static thread_local int configured_dev = -1;
  if (configured_dev != ctx->device) {
    if (!cuda_ok(ctx, cudaFuncSetAttribute(half_step_tc_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kTcSmem),
                 "cudaFuncSetAttribute tc"))
      return HERMITE_ERR_CUDA;
    configured_dev = ctx->device;
  }
  static thread_local int sms = 0, sms_dev = -1;
  if (sms_dev != ctx->device) {
    if (!cuda_ok(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "SM count"))
      return HERMITE_ERR_CUDA;
    sms_dev = ctx->device;
  }
  const int64_t ntiles = (a.g.nodes_dst + 127) / 128;
  const int blocks = (int)std::min<int64_t>(ntiles, sms);
  half_step_tc_kernel<D><<<blocks, kTcThreads, kTcSmem, ctx->stream>>>(a);
  return cuda_ok(ctx, cudaGetLastError(), "half_step_tc_kernel") ? HERMITE_OK : HERMITE_ERR_CUDA;
}
}  // namespace

int launch_half_step_tc(hermite_ctx *ctx, int dst, const float2 *src, float2 *out, bool subtract_old) {
  TcArgs a;
  a.g = make_geometry(ctx, dst);
  if (a.g.nodes_dst == 0) return HERMITE_OK;
  a.src = src;
  a.dst = out;
  a.subtract_old = subtract_old ? 1 : 0;
  a.Bimg = ctx->tc_B;
  a.inb = ctx->tc_inb;
  a.orow = ctx->tc_orow;
  a.er = ctx->tc_er;
  a.nu = ctx->Nu;
  a.vexp = ctx->tc_vexp;
  a.status = ctx->tc_status;
  switch (ctx->d) {
    case 2: return launch_tc_d<2>(ctx, a);
    case 3: return launch_tc_d<3>(ctx, a);
  }
  return HERMITE_ERR_ARG;
}

int tc_check_status(hermite_ctx *ctx) {
  if (!ctx->tc_status) return HERMITE_OK;
  int st = 0;
  if (!cuda_ok(ctx, cudaMemcpy(&st, ctx->tc_status, sizeof(int), cudaMemcpyDeviceToHost), "read tc status"))
    return HERMITE_ERR_CUDA;
  if (st == 0) return HERMITE_OK;
  cudaMemset(ctx->tc_status, 0, sizeof(int));
  ctx->err = "tensor-core half-step: a bounded wait for the tensor core ran out";
  return HERMITE_ERR_TIMEOUT;
}

}  // namespace hermite

extern "C" int hermite_set_split_engine(hermite_ctx *ctx, int engine) {
  using namespace hermite;
  if (!ctx || (engine != 0 && engine != 1)) return HERMITE_ERR_ARG;
  if (ctx->precision != HERMITE_SPLIT32) {
    ctx->err = "hermite_set_split_engine: not a split-precision context";
    return HERMITE_ERR_STATE;
  }
  if (engine == 1 && !ctx->tc_ready) {
    ctx->err = "hermite_set_split_engine: no tensor-core kernel for this shape (d = 1 or a parity class wider than 16)";
    return HERMITE_ERR_UNSUPPORTED;
  }
  ctx->split_engine = engine;
  return HERMITE_OK;
}

extern "C" int hermite_get_split_engine(const hermite_ctx *ctx) {
  if (!ctx || ctx->precision != HERMITE_SPLIT32) return -1;
  return ctx->split_engine;
}
