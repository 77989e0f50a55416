// Learned super-stepper kernels: a dilated 3x3 convolution network on NHWC
// BF16 tensors with FP32 accumulation on the tensor cores (forward, input
// gradient via flipped weights, weight and bias gradients), the loss, the
// Adam update and the conversions between solver states and network tensors.
//
// Convolution as implicit GEMM.  One CTA owns one output image row (128
// nodes) and all output channels; it stages the three input rows that the
// 3x3 taps touch, (y - dil, y, y + dil) mod H, in shared memory and reads the
// column shift (x + (kx-1) dil) mod 128 through per-lane ldmatrix row
// addresses, so circular padding costs nothing.  The weights of the layer stay
// in shared memory for the CTA's lifetime (persistent CTAs, rows handed out
// round robin) and the next row's inputs are fetched with cp.async while the
// current row is multiplied (double buffer).  Tiles are multiplied with
// mma.sync m16n8k16 (BF16 in, FP32 accumulate); rows are padded by 16 bytes so
// that every ldmatrix phase touches 32 distinct banks.
//
// The weight gradient is the same contraction with the pixel index as the
// reduction: CTAs take rows round robin for one kernel-row ky (gridDim.y = 3),
// accumulate dW[co][3 ky + kx][ci] over their rows in registers, and add
// their partial sums to global memory once at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hermite.h"
#include "hermite_nn.h"
#include "hermite_nn_internal.h"

namespace hermite_nn {
namespace {

constexpr int kW = 128;        // nodes per image row (one CTA row tile)
constexpr int kThreads = 256;  // 8 warps per CTA

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap_row(int y, int s, int H) {
  int r = (y + s) % H;
  return r < 0 ? r + H : r;
}

// ---------------------------------------------------------------------------
// Forward convolution (also the input gradient with flipped weights)
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct FwdCfg {
  static constexpr int LD = CIN + 8;              // padded smem row, BF16 elements
  static constexpr int WARPS_N = COUT / 32;       // each warp: 32 output channels
  static constexpr int WARPS_M = 8 / WARPS_N;
  static constexpr int MT = kW / (16 * WARPS_M);  // m16 tiles (of nodes) per warp
  static constexpr int W_ELEMS = 9 * COUT * LD;
  static constexpr int ROW_ELEMS = kW * LD;
  static constexpr size_t SMEM = sizeof(bf16) * (size_t)(W_ELEMS + 2 * 3 * ROW_ELEMS);
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
    conv_fwd_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w, const float *__restrict__ bias,
                    const bf16 *__restrict__ mask, int rows, int H, int dil, int relu, bf16 *__restrict__ y16,
                    float *__restrict__ y32) {
  using C = FwdCfg<CIN, COUT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *Ws = reinterpret_cast<bf16 *>(smem_raw);  // [tap][co][LD]
  bf16 *Xs = Ws + C::W_ELEMS;                     // [buf][ky][px][LD]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % C::WARPS_M, wn = warp / C::WARPS_M;
  constexpr int CH = CIN / 8;  // 16-byte chunks per node

  // weights, global [co][tap][ci] -> shared [tap][co][ci]
  for (int i = tid; i < 9 * COUT * CH; i += kThreads) {
    const int row = i / CH, ch = i % CH;  // row = co * 9 + tap
    const int co = row / 9, tap = row % 9;
    cp_async16(Ws + (tap * COUT + co) * C::LD + ch * 8, w + (size_t)row * CIN + ch * 8);
  }
  auto load_rows = [&](int r, int buf) {
    const int b = r / H, yy = r % H;
    for (int i = tid; i < 3 * kW * CH; i += kThreads) {
      const int ky = i / (kW * CH), rem = i % (kW * CH), px = rem / CH, ch = rem % CH;
      const int ys = wrap_row(yy, (ky - 1) * dil, H);
      cp_async16(Xs + ((buf * 3 + ky) * kW + px) * C::LD + ch * 8,
                 x + (((size_t)b * H + ys) * kW + px) * CIN + ch * 8);
    }
  };

  int r = blockIdx.x;
  if (r < rows) load_rows(r, 0);
  cp_async_commit();
  int buf = 0;
  for (; r < rows; r += gridDim.x) {
    const int rn = r + gridDim.x;
    if (rn < rows) load_rows(rn, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    float acc[C::MT][4][4];
#pragma unroll
    for (int i = 0; i < C::MT; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap % 3;
      const int shift = (kx - 1) * dil;
      const bf16 *Xrow = Xs + (buf * 3 + ky) * C::ROW_ELEMS;
      uint32_t a_addr[C::MT];
#pragma unroll
      for (int mt = 0; mt < C::MT; ++mt) {
        const int px = wm * (C::MT * 16) + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int src = (px + shift) & (kW - 1);
        a_addr[mt] = smem_addr(Xrow + src * C::LD + (lane >> 4) * 8);
      }
      const bf16 *Wt = Ws + tap * COUT * C::LD;
      uint32_t b_addr[2];
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int n = wn * 32 + np * 16 + (lane & 7) + (lane >> 4) * 8;
        b_addr[np] = smem_addr(Wt + n * C::LD + ((lane >> 3) & 1) * 8);
      }
#pragma unroll
      for (int kc = 0; kc < CIN / 16; ++kc) {
        uint32_t a[C::MT][4], b[4][2];
#pragma unroll
        for (int mt = 0; mt < C::MT; ++mt) ldsm_x4(a[mt][0], a[mt][1], a[mt][2], a[mt][3], a_addr[mt] + kc * 32);
#pragma unroll
        for (int np = 0; np < 2; ++np)
          ldsm_x4(b[2 * np][0], b[2 * np][1], b[2 * np + 1][0], b[2 * np + 1][1], b_addr[np] + kc * 32);
#pragma unroll
        for (int mt = 0; mt < C::MT; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt], b[nt][0], b[nt][1]);
      }
    }

    // epilogue: bias, ReLU, mask, BF16 / FP32 stores (two channels per store)
#pragma unroll
    for (int mt = 0; mt < C::MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int co = wn * 32 + nt * 8 + (lane & 3) * 2;
        float b0 = 0.f, b1 = 0.f;
        if (bias) {
          b0 = bias[co];
          b1 = bias[co + 1];
        }
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int px = wm * (C::MT * 16) + mt * 16 + (lane >> 2) + hf * 8;
          float v0 = acc[mt][nt][2 * hf] + b0, v1 = acc[mt][nt][2 * hf + 1] + b1;
          if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          const size_t o = ((size_t)r * kW + px) * COUT + co;
          if (mask) {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + o);
            if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
          }
          if (y16) *reinterpret_cast<__nv_bfloat162 *>(y16 + o) = __floats2bfloat162_rn(v0, v1);
          if (y32) *reinterpret_cast<float2 *>(y32 + o) = make_float2(v0, v1);
        }
      }
    __syncthreads();  // buffer buf is refilled by the next iteration's prefetch
    buf ^= 1;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Weight gradient
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct WgCfg {
  static constexpr int LDX = CIN + 8;
  static constexpr int LDY = COUT + 8;
  static constexpr int WARPS_M = COUT / 32;  // each warp: 32 output channels (2 m16 tiles)
  static constexpr int WARPS_N = 8 / WARPS_M;
  static constexpr int NTOT = 3 * CIN / 8;  // n8 tiles over (kx, ci)
  static constexpr int NT = NTOT / WARPS_N;
  static_assert(NTOT % WARPS_N == 0, "n tiles must split evenly over warps");
  static constexpr size_t SMEM = sizeof(bf16) * (size_t)2 * kW * (LDX + LDY);
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads)
    conv_wgrad_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ dy, int rows, int H, int dil,
                      float *__restrict__ dw) {
  using C = WgCfg<CIN, COUT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *Xs = reinterpret_cast<bf16 *>(smem_raw);  // [buf][px][LDX]
  bf16 *Ys = Xs + 2 * kW * C::LDX;                // [buf][px][LDY]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % C::WARPS_M, wn = warp / C::WARPS_M;
  const int ky = blockIdx.y;
  constexpr int CHX = CIN / 8, CHY = COUT / 8;

  auto load_rows = [&](int r, int buf) {
    const int b = r / H, yy = r % H;
    const int ys = wrap_row(yy, (ky - 1) * dil, H);
    const bf16 *xs = x + ((size_t)b * H + ys) * kW * CIN;
    const bf16 *ds = dy + (size_t)r * kW * COUT;
    for (int i = tid; i < kW * CHX; i += kThreads)
      cp_async16(Xs + (buf * kW + i / CHX) * C::LDX + (i % CHX) * 8, xs + (size_t)i * 8);
    for (int i = tid; i < kW * CHY; i += kThreads)
      cp_async16(Ys + (buf * kW + i / CHY) * C::LDY + (i % CHY) * 8, ds + (size_t)i * 8);
  };

  // n8 tile t covers columns 8t..8t+7 of (kx, ci): kx = 8t / CIN, ci0 = 8t % CIN
  float acc[2][C::NT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < C::NT; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

  int r = blockIdx.x;
  if (r < rows) load_rows(r, 0);
  cp_async_commit();
  int buf = 0;
  const int mi = lane >> 3, rr = lane & 7;
  for (; r < rows; r += gridDim.x) {
    const int rn = r + gridDim.x;
    if (rn < rows) load_rows(rn, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const bf16 *Xb = Xs + buf * kW * C::LDX;
    const bf16 *Yb = Ys + buf * kW * C::LDY;
#pragma unroll 2
    for (int kc = 0; kc < kW / 16; ++kc) {
      const int p0 = kc * 16;
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int co = wm * 32 + mt * 16 + 8 * (mi & 1);
        const int p = p0 + rr + 8 * (mi >> 1);
        ldsm_x4_t(a[mt][0], a[mt][1], a[mt][2], a[mt][3], smem_addr(Yb + p * C::LDY + co));
      }
      uint32_t b[C::NT][2];
#pragma unroll
      for (int j = 0; j + 1 < C::NT; j += 2) {
        const int t = wn * C::NT + j + (mi >> 1);
        const int kx = (8 * t) / CIN, ci0 = (8 * t) % CIN;
        const int p = p0 + rr + 8 * (mi & 1);
        const int src = (p + (kx - 1) * dil) & (kW - 1);
        ldsm_x4_t(b[j][0], b[j][1], b[j + 1][0], b[j + 1][1], smem_addr(Xb + src * C::LDX + ci0));
      }
      if (C::NT & 1) {
        const int j = C::NT - 1;
        const int t = wn * C::NT + j;
        const int kx = (8 * t) / CIN, ci0 = (8 * t) % CIN;
        const int p = p0 + rr + 8 * (mi & 1);  // lanes 16-31 repeat valid addresses
        const int src = (p + (kx - 1) * dil) & (kW - 1);
        ldsm_x2_t(b[j][0], b[j][1], smem_addr(Xb + src * C::LDX + ci0));
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < C::NT; ++j) mma_bf16(acc[mt][j], a[mt], b[j][0], b[j][1]);
    }
    __syncthreads();
    buf ^= 1;
  }
  cp_async_wait<0>();

#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < C::NT; ++j) {
      const int t = wn * C::NT + j;
      const int n = 8 * t + (lane & 3) * 2;
      const int kx = n / CIN, ci = n % CIN;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int co = wm * 32 + mt * 16 + (lane >> 2) + hf * 8;
        float *dst = dw + ((size_t)co * 9 + ky * 3 + kx) * CIN + ci;
        atomicAdd(dst, acc[mt][j][2 * hf]);
        atomicAdd(dst + 1, acc[mt][j][2 * hf + 1]);
      }
    }
}

// ---------------------------------------------------------------------------
// Element-wise and reduction kernels
// ---------------------------------------------------------------------------
__global__ void flip_weights_kernel(const bf16 *__restrict__ w, int Cout, int Cin, bf16 *__restrict__ wt) {
  const int64_t n = (int64_t)Cout * 9 * Cin;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(i % Cout);
    const int tap = (int)((i / Cout) % 9);
    const int ci = (int)(i / ((int64_t)Cout * 9));
    wt[i] = w[((size_t)co * 9 + (8 - tap)) * Cin + ci];  // wt[ci][tap][co]
  }
}

// db[c] += sum_p dy[p][c]; blockDim 256, C divides 256
__global__ void bias_grad_kernel(const bf16 *__restrict__ dy, int64_t total, int C, float *__restrict__ db) {
  __shared__ float part[256];
  float s = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256)
    s += __bfloat162float(dy[i]);
  part[threadIdx.x] = s;
  __syncthreads();
  if ((int)threadIdx.x < C) {
    float t = 0.f;
    for (int k = threadIdx.x; k < 256; k += C) t += part[k];
    atomicAdd(db + threadIdx.x, t);
  }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  __syncthreads();
  return t;
}

__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ wch,
                           int64_t total, int C, float scale, double *loss, bf16 *__restrict__ dy) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float wc = wch[i % C];
    const float e = y[i] - t[i];
    s += (double)(wc * e) * (double)e;
    dy[i] = __float2bfloat16_rn(2.f * scale * wc * e);
  }
  if (loss) {
    const double tot = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(loss, tot * (double)scale);
  }
}

__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                            int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                            bf16 *__restrict__ p16) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    g[i] = 0.f;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void state_to_f32_kernel(const double *__restrict__ u, const double *__restrict__ v, int64_t n, int Nu,
                                    int Nv, double vscale, float *__restrict__ out, int ld) {
  const int C0 = Nu + Nv;
  const int64_t total = n * C0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / C0;
    const int c = (int)(i % C0);
    const double s = c < Nu ? u[node * Nu + c] : vscale * v[node * Nv + (c - Nu)];
    out[node * ld + c] = (float)s;
  }
}

// Network input: FP32 arithmetic with reciprocals staged once per block (the
// result is rounded to BF16); FP64 division is slow on this part.
__global__ void pack_state_kernel(const double *__restrict__ u, const double *__restrict__ v, int64_t n, int Nu,
                                  int Nv, double vscale, const double *__restrict__ shift,
                                  const double *__restrict__ scale, int C, bf16 *__restrict__ x) {
  __shared__ float sh_shift[64], sh_inv[64];
  if ((int)threadIdx.x < Nu + Nv) {
    sh_shift[threadIdx.x] = (float)shift[threadIdx.x];
    sh_inv[threadIdx.x] = (float)(1.0 / scale[threadIdx.x]);
  }
  __syncthreads();
  const float vs = (float)vscale;
  const int64_t total = n * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / C;
    const int c = (int)(i % C);
    float val = 0.f;
    if (c < Nu + Nv) {
      const float sv = c < Nu ? (float)u[node * Nu + c] : __fmul_rn((float)v[node * Nv + (c - Nu)], vs);
      val = __fmul_rn(__fsub_rn(sv, sh_shift[c]), sh_inv[c]);
    }
    x[i] = __float2bfloat16_rn(val);
  }
}

// Residual update: the change dscale * y in FP32, added to the FP64 state.
__global__ void unpack_state_kernel(const double *u, const double *v, const float *__restrict__ y, int64_t n, int Nu,
                                    int Nv, double inv_vscale, const double *__restrict__ dscale, int C, double *u_out,
                                    double *v_out) {
  __shared__ float sh_ds[64];
  if ((int)threadIdx.x < Nu + Nv) sh_ds[threadIdx.x] = (float)dscale[threadIdx.x];
  __syncthreads();
  const int C0 = Nu + Nv;
  const int64_t total = n * C0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / C0;
    const int c = (int)(i % C0);
    const double d = (double)__fmul_rn(sh_ds[c], y[node * C + c]);
    if (c < Nu)
      u_out[node * Nu + c] = u[node * Nu + c] + d;
    else
      v_out[node * Nv + (c - Nu)] = fma(d, inv_vscale, v[node * Nv + (c - Nu)]);
  }
}

__global__ void make_pairs_kernel(const float *__restrict__ levels, const int64_t *__restrict__ src,
                                  const int64_t *__restrict__ dst, int64_t n, int C0,
                                  const double *__restrict__ shift, const double *__restrict__ scale,
                                  const double *__restrict__ dscale, int C, bf16 *__restrict__ x,
                                  float *__restrict__ t) {
  __shared__ float sh_shift[64], sh_inv[64], sh_dinv[64];
  if ((int)threadIdx.x < C0) {
    sh_shift[threadIdx.x] = (float)shift[threadIdx.x];
    sh_inv[threadIdx.x] = (float)(1.0 / scale[threadIdx.x]);
    sh_dinv[threadIdx.x] = (float)(1.0 / dscale[threadIdx.x]);
  }
  __syncthreads();
  const int s = blockIdx.y;
  const float *a = levels + src[s];
  const float *b = levels + dst[s];
  const int64_t total = n * C;
  bf16 *xs = x + (int64_t)s * total;
  float *ts = t + (int64_t)s * total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = i / C;
    const int c = (int)(i % C);
    float xv = 0.f, tv = 0.f;
    if (c < C0) {
      const float av = a[node * C0 + c], bv = b[node * C0 + c];
      xv = __fmul_rn(__fsub_rn(av, sh_shift[c]), sh_inv[c]);
      tv = __fmul_rn(__fsub_rn(bv, av), sh_dinv[c]);
    }
    xs[i] = __float2bfloat16_rn(xv);
    ts[i] = tv;
  }
}

// out[c] += sum d, out[C + c] += sum d^2; blockDim 256, C <= 64
__global__ void moments_kernel(const float *__restrict__ a, const float *__restrict__ b, int64_t n, int C,
                               double *out) {
  __shared__ double s1[64], s2[64];
  if ((int)threadIdx.x < C) {
    s1[threadIdx.x] = 0.0;
    s2[threadIdx.x] = 0.0;
  }
  __syncthreads();
  const int64_t total = n * C;
  // each thread keeps one channel per pass when C divides the stride; use per-element atomics to shared
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const double d = b ? (double)a[i] - (double)b[i] : (double)a[i];
    atomicAdd(&s1[c], d);
    atomicAdd(&s2[c], d * d);
  }
  __syncthreads();
  if ((int)threadIdx.x < C) {
    atomicAdd(out + threadIdx.x, s1[threadIdx.x]);
    atomicAdd(out + C + threadIdx.x, s2[threadIdx.x]);
  }
}

__global__ void sqdiff_kernel(const double *__restrict__ au, const double *__restrict__ av,
                              const double *__restrict__ bu, const double *__restrict__ bv, int64_t n, int Nu, int Nv,
                              double vscale, double *out) {
  __shared__ double sh[32];
  double sd = 0.0, sb = 0.0;
  const int64_t nu = n * Nu, total = n * (Nu + Nv);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double x, y;
    if (i < nu) {
      x = au[i];
      y = bu[i];
    } else {
      x = vscale * av[i - nu];
      y = vscale * bv[i - nu];
    }
    sd += (x - y) * (x - y);
    sb += y * y;
  }
  const double td = block_sum(sd, sh);
  const double tb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    atomicAdd(out, td);
    atomicAdd(out + 1, tb);
  }
}

// per-sample distances: blockIdx.y = sample, states [nsamp][n][Nu] and [nsamp][n][Nv]
__global__ void sqdiff_batch_kernel(const double *__restrict__ au, const double *__restrict__ av,
                                    const double *__restrict__ bu, const double *__restrict__ bv, int64_t n, int Nu,
                                    int Nv, double vscale, double *out) {
  __shared__ double sh[32];
  const int s = blockIdx.y;
  const int64_t nu = n * Nu, nv = n * Nv, total = nu + nv;
  au += s * nu;
  bu += s * nu;
  if (av) av += s * nv;
  if (bv) bv += s * nv;
  double sd = 0.0, sb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double x, y;
    if (i < nu) {
      x = au[i];
      y = bu[i];
    } else {
      x = vscale * av[i - nu];
      y = vscale * bv[i - nu];
    }
    sd += (x - y) * (x - y);
    sb += y * y;
  }
  const double td = block_sum(sd, sh);
  const double tb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    atomicAdd(out + 2 * s, td);
    atomicAdd(out + 2 * s + 1, tb);
  }
}

__global__ void copy_blocks_kernel(const double *__restrict__ src, const int64_t *__restrict__ sidx,
                                   double *__restrict__ dst, const int64_t *__restrict__ didx, int64_t block) {
  const int i = blockIdx.y;
  const double *a = src + (sidx ? sidx[i] : i) * block;
  double *b = dst + (didx ? didx[i] : i) * block;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < block; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = a[e];
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
int g_num_sms = 0;
std::once_flag g_sm_once;

int num_sms() {
  std::call_once(g_sm_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  });
  return g_num_sms;
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int launched() { return cudaGetLastError() == cudaSuccess ? HERMITE_OK : HERMITE_ERR_CUDA; }

inline int elementwise_grid(int64_t total) {
  const int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

template <int CIN, int COUT>
int launch_fwd(const bf16 *x, const bf16 *w, const float *bias, const bf16 *mask, int rows, int H, int dil, int relu,
               bf16 *y16, float *y32, cudaStream_t s) {
  using C = FwdCfg<CIN, COUT>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(conv_fwd_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM);
  });
  if (attr != cudaSuccess) return HERMITE_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_fwd_kernel<CIN, COUT>, kThreads, C::SMEM) !=
          cudaSuccess ||
      per_sm < 1)
    return HERMITE_ERR_CUDA;
  const int grid = rows < num_sms() * per_sm ? rows : num_sms() * per_sm;
  conv_fwd_kernel<CIN, COUT><<<grid, kThreads, C::SMEM, s>>>(x, w, bias, mask, rows, H, dil, relu, y16, y32);
  return launched();
}

template <int CIN, int COUT>
int launch_wgrad(const bf16 *x, const bf16 *dy, int rows, int H, int dil, float *dw, cudaStream_t s) {
  using C = WgCfg<CIN, COUT>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(conv_wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM);
  });
  if (attr != cudaSuccess) return HERMITE_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_wgrad_kernel<CIN, COUT>, kThreads, C::SMEM) !=
          cudaSuccess ||
      per_sm < 1)
    return HERMITE_ERR_CUDA;
  // three kernel rows share the SMs; each CTA then sums many image rows before its atomics
  int gx = (num_sms() * per_sm + 2) / 3;
  if (gx > rows) gx = rows;
  conv_wgrad_kernel<CIN, COUT><<<dim3(gx, 3), kThreads, C::SMEM, s>>>(x, dy, rows, H, dil, dw);
  return launched();
}

inline bool chan_ok(int c) { return c == 32 || c == 64; }

}  // namespace
}  // namespace hermite_nn

using namespace hermite_nn;

extern "C" {

int hnn_conv3x3_fwd(const uint16_t *x, const uint16_t *w, const float *bias, const uint16_t *mask, int B, int H,
                    int W, int Cin, int Cout, int dil, int relu, uint16_t *y_bf16, float *y_f32, void *stream) {
  if (B < 0 || H < 0 || W != kW || !chan_ok(Cin) || !chan_ok(Cout) || dil < 1 || dil >= kW) return HERMITE_ERR_ARG;
  if (B == 0 || H == 0) return HERMITE_OK;
  if (!x || !w || (!y_bf16 && !y_f32)) return HERMITE_ERR_ARG;
  const int64_t rows64 = (int64_t)B * H;
  if (rows64 > INT32_MAX) return HERMITE_ERR_ARG;
  const int rows = (int)rows64;
  auto X = reinterpret_cast<const bf16 *>(x);
  auto Wt = reinterpret_cast<const bf16 *>(w);
  auto M = reinterpret_cast<const bf16 *>(mask);
  auto Y = reinterpret_cast<bf16 *>(y_bf16);
  cudaStream_t s = as_stream(stream);
  if (tc_conv_supported(Cin, Cout, dil)) return tc_conv_fwd(X, Wt, bias, M, rows, H, dil, relu, Y, y_f32, Cout, s);
  if (Cin == 32 && Cout == 64) return launch_fwd<32, 64>(X, Wt, bias, M, rows, H, dil, relu, Y, y_f32, s);
  if (Cin == 64 && Cout == 64) return launch_fwd<64, 64>(X, Wt, bias, M, rows, H, dil, relu, Y, y_f32, s);
  if (Cin == 64 && Cout == 32) return launch_fwd<64, 32>(X, Wt, bias, M, rows, H, dil, relu, Y, y_f32, s);
  return launch_fwd<32, 32>(X, Wt, bias, M, rows, H, dil, relu, Y, y_f32, s);
}

int hnn_flip_weights(const uint16_t *w, int Cout, int Cin, uint16_t *wt, void *stream) {
  if (!w || !wt || Cout <= 0 || Cin <= 0) return HERMITE_ERR_ARG;
  const int64_t n = (int64_t)Cout * 9 * Cin;
  flip_weights_kernel<<<elementwise_grid(n), 256, 0, as_stream(stream)>>>(reinterpret_cast<const bf16 *>(w), Cout,
                                                                          Cin, reinterpret_cast<bf16 *>(wt));
  return launched();
}

int hnn_conv3x3_wgrad(const uint16_t *x, const uint16_t *dy, int B, int H, int W, int Cin, int Cout, int dil,
                      float *dw, void *stream) {
  if (B < 0 || H < 0 || W != kW || !chan_ok(Cin) || !chan_ok(Cout) || dil < 1 || dil >= kW) return HERMITE_ERR_ARG;
  if (Cin == 32 && Cout == 32) return HERMITE_ERR_ARG;
  if (B == 0 || H == 0) return HERMITE_OK;
  if (!x || !dy || !dw) return HERMITE_ERR_ARG;
  const int64_t rows64 = (int64_t)B * H;
  if (rows64 > INT32_MAX) return HERMITE_ERR_ARG;
  const int rows = (int)rows64;
  auto X = reinterpret_cast<const bf16 *>(x);
  auto D = reinterpret_cast<const bf16 *>(dy);
  cudaStream_t s = as_stream(stream);
  if (Cin == 32) return launch_wgrad<32, 64>(X, D, rows, H, dil, dw, s);
  if (Cout == 64) return launch_wgrad<64, 64>(X, D, rows, H, dil, dw, s);
  return launch_wgrad<64, 32>(X, D, rows, H, dil, dw, s);
}

int hnn_bias_grad(const uint16_t *dy, int64_t npix, int C, float *db, void *stream) {
  if (npix < 0 || !chan_ok(C)) return HERMITE_ERR_ARG;
  if (npix == 0) return HERMITE_OK;
  if (!dy || !db) return HERMITE_ERR_ARG;
  const int64_t total = npix * C;
  bias_grad_kernel<<<elementwise_grid(total), 256, 0, as_stream(stream)>>>(reinterpret_cast<const bf16 *>(dy), total,
                                                                           C, db);
  return launched();
}

int hnn_mse(const float *y, const float *t, const float *wch, int64_t npix, int C, float scale, double *loss,
            uint16_t *dy, void *stream) {
  if (npix < 0 || C <= 0) return HERMITE_ERR_ARG;
  if (npix == 0) return HERMITE_OK;
  if (!y || !t || !wch || !dy) return HERMITE_ERR_ARG;
  const int64_t total = npix * C;
  mse_kernel<<<elementwise_grid(total), 256, 0, as_stream(stream)>>>(y, t, wch, total, C, scale, loss,
                                                                     reinterpret_cast<bf16 *>(dy));
  return launched();
}

int hnn_adam(float *p, float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2, float eps, int t,
             uint16_t *p_bf16, void *stream) {
  if (n < 0 || t < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f)) return HERMITE_ERR_ARG;
  if (n == 0) return HERMITE_OK;
  if (!p || !g || !m || !v) return HERMITE_ERR_ARG;
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  adam_kernel<<<elementwise_grid(n), 256, 0, as_stream(stream)>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2,
                                                                  reinterpret_cast<bf16 *>(p_bf16));
  return launched();
}

int hnn_state_to_f32(const double *u, const double *v, int64_t n, int Nu, int Nv, double vscale, float *out, int ld,
                     void *stream) {
  if (n < 0 || Nu < 1 || Nv < 0 || ld < Nu + Nv) return HERMITE_ERR_ARG;
  if (n == 0) return HERMITE_OK;
  if (!u || (Nv > 0 && !v) || !out) return HERMITE_ERR_ARG;
  state_to_f32_kernel<<<elementwise_grid(n * (Nu + Nv)), 256, 0, as_stream(stream)>>>(u, v, n, Nu, Nv, vscale, out,
                                                                                      ld);
  return launched();
}

int hnn_pack_state(const double *u, const double *v, int64_t n, int Nu, int Nv, double vscale, const double *shift,
                   const double *scale, int C, uint16_t *x, void *stream) {
  if (n < 0 || Nu < 1 || Nv < 0 || C < Nu + Nv || Nu + Nv > 64) return HERMITE_ERR_ARG;
  if (n == 0) return HERMITE_OK;
  if (!u || (Nv > 0 && !v) || !shift || !scale || !x) return HERMITE_ERR_ARG;
  pack_state_kernel<<<elementwise_grid(n * C), 256, 0, as_stream(stream)>>>(u, v, n, Nu, Nv, vscale, shift, scale, C,
                                                                            reinterpret_cast<bf16 *>(x));
  return launched();
}

int hnn_unpack_state(const double *u, const double *v, const float *y, int64_t n, int Nu, int Nv, double vscale,
                     const double *dscale, int C, double *u_out, double *v_out, void *stream) {
  if (n < 0 || Nu < 1 || Nv < 0 || C < Nu + Nv || Nu + Nv > 64 || (Nv > 0 && vscale == 0.0)) return HERMITE_ERR_ARG;
  if (n == 0) return HERMITE_OK;
  if (!u || !y || !dscale || !u_out || (Nv > 0 && (!v || !v_out))) return HERMITE_ERR_ARG;
  unpack_state_kernel<<<elementwise_grid(n * (Nu + Nv)), 256, 0, as_stream(stream)>>>(
      u, v, y, n, Nu, Nv, Nv > 0 ? 1.0 / vscale : 0.0, dscale, C, u_out, v_out);
  return launched();
}

int hnn_make_pairs(const float *levels, const int64_t *src, const int64_t *dst, int nsamp, int64_t n, int C0,
                   const double *shift, const double *scale, const double *dscale, int C, uint16_t *x, float *t,
                   void *stream) {
  if (nsamp < 0 || nsamp > 65535 || n < 0 || C0 < 1 || C0 > 64 || C < C0) return HERMITE_ERR_ARG;
  if (nsamp == 0 || n == 0) return HERMITE_OK;
  if (!levels || !src || !dst || !shift || !scale || !dscale || !x || !t) return HERMITE_ERR_ARG;
  int gx = elementwise_grid(n * C) / (nsamp < 8 ? 1 : 8);
  if (gx < 1) gx = 1;
  make_pairs_kernel<<<dim3(gx, nsamp), 256, 0, as_stream(stream)>>>(levels, src, dst, n, C0, shift, scale, dscale, C,
                                                                    reinterpret_cast<bf16 *>(x), t);
  return launched();
}

int hnn_moments(const float *a, const float *b, int64_t n, int C, double *out, void *stream) {
  if (n < 0 || C < 1 || C > 64) return HERMITE_ERR_ARG;
  if (n == 0) return HERMITE_OK;
  if (!a || !out) return HERMITE_ERR_ARG;
  moments_kernel<<<elementwise_grid(n * C), 256, 0, as_stream(stream)>>>(a, b, n, C, out);
  return launched();
}

int hnn_sqdiff(const double *a_u, const double *a_v, const double *b_u, const double *b_v, int64_t n, int Nu, int Nv,
               double vscale, double *out, void *stream) {
  if (n < 0 || Nu < 1 || Nv < 0) return HERMITE_ERR_ARG;
  if (n == 0) return HERMITE_OK;
  if (!a_u || !b_u || !out || (Nv > 0 && (!a_v || !b_v))) return HERMITE_ERR_ARG;
  sqdiff_kernel<<<elementwise_grid(n * (Nu + Nv)), 256, 0, as_stream(stream)>>>(a_u, a_v, b_u, b_v, n, Nu, Nv,
                                                                                vscale, out);
  return launched();
}

int hnn_sqdiff_batch(const double *a_u, const double *a_v, const double *b_u, const double *b_v, int nsamp, int64_t n,
                     int Nu, int Nv, double vscale, double *out, void *stream) {
  if (nsamp < 0 || nsamp > 65535 || n < 0 || Nu < 1 || Nv < 0) return HERMITE_ERR_ARG;
  if (nsamp == 0 || n == 0) return HERMITE_OK;
  if (!a_u || !b_u || !out || (Nv > 0 && (!a_v || !b_v))) return HERMITE_ERR_ARG;
  int gx = elementwise_grid(n * (Nu + Nv)) / 8;
  if (gx < 1) gx = 1;
  sqdiff_batch_kernel<<<dim3(gx, nsamp), 256, 0, as_stream(stream)>>>(a_u, a_v, b_u, b_v, n, Nu, Nv, vscale, out);
  return launched();
}

int hnn_copy_blocks(const double *src, const int64_t *sidx, double *dst, const int64_t *didx, int nblk, int64_t block,
                    void *stream) {
  if (nblk < 0 || nblk > 65535 || block < 0) return HERMITE_ERR_ARG;
  if (nblk == 0 || block == 0) return HERMITE_OK;
  if (!src || !dst) return HERMITE_ERR_ARG;
  int gx = elementwise_grid(block) / 8;
  if (gx < 1) gx = 1;
  copy_blocks_kernel<<<dim3(gx, nblk), 256, 0, as_stream(stream)>>>(src, sidx, dst, didx, block);
  return launched();
}

}  // extern "C"
