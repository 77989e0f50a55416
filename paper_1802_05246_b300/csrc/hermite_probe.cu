// Arithmetic-pipe probes: the FMA throughput a kernel of this library can
// reach on the device it runs on, measured rather than taken from a nominal
// lane count.  Each thread runs eight independent FMA chains x <- x*a + b
// (a just below 1, so the values settle at b / (1 - a): no overflow, no
// subnormals) and stores their sum so that nothing is optimised away.  An FMA
// counts as two floating-point operations.
#include <cuda_runtime.h>

#include "hermite_internal.h"

namespace hermite {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_f64_kernel(int iters, double *out) {
  double x[kProbeChains];
  const double a = 0.999999, b = 1e-7 * (1 + threadIdx.x % 7);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, b);
  double s = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_f32_kernel(int iters, double *out) {
  float x[kProbeChains];
  const float a = 0.99999f, b = 1e-6f * (1 + threadIdx.x % 7);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = (float)k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
  float s = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

// the packed FP32-pair form (two FMAs per instruction) the split kernels use
__global__ void __launch_bounds__(kProbeThreads) probe_f32x2_kernel(int iters, double *out) {
  float2 x[kProbeChains];
  const float2 a = make_float2(0.99999f, 0.99998f);
  const float2 b = make_float2(1e-6f * (1 + threadIdx.x % 7), 2e-6f);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = make_float2((float)k, (float)(k + 1));
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = __ffma2_rn(x[k], a, b);
  float s = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k].x + x[k].y;
  out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace hermite

extern "C" int hermite_peak_probe(int kind, double *flops_per_s) {
  using namespace hermite;
  if (!flops_per_s || kind < 0 || kind > 2) return HERMITE_ERR_ARG;
  *flops_per_s = 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HERMITE_ERR_CUDA;
  const int blocks = sms * 8;
  const int iters = kind == 0 ? 1 << 12 : 1 << 15;
  double *out = nullptr;
  if (device_alloc(&out, sizeof(double) * (size_t)blocks * kProbeThreads) != cudaSuccess) return HERMITE_ERR_ALLOC;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HERMITE_OK;
  float ms = 0;
  auto launch = [&] {
    if (kind == 0)
      probe_f64_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, out);
    else if (kind == 1)
      probe_f32_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, out);
    else
      probe_f32x2_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, out);
  };
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = HERMITE_ERR_CUDA;
  } else {
    launch();  // warm-up
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess || ms <= 0)
      rc = HERMITE_ERR_CUDA;
  }
  if (rc == HERMITE_OK) {
    const double fmas = (double)blocks * kProbeThreads * iters * kProbeChains * (kind == 2 ? 2 : 1);
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  return rc;
}
