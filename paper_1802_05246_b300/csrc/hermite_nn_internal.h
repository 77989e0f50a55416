// Internal interface between the network kernels (hermite_nn.cu) and the
// tensor-core forward convolution (hermite_nn_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace hermite_nn {

// true when the tensor-core path is selected and handles (Cin, Cout, dil)
bool tc_conv_supported(int Cin, int Cout, int dil);

// forward convolution with Cin = 64 on the tensor cores (tcgen05); arguments as
// hnn_conv3x3_fwd with rows = B * H; returns a HERMITE_* code
int tc_conv_fwd(const __nv_bfloat16 *x, const __nv_bfloat16 *w, const float *bias, const __nv_bfloat16 *mask,
                int rows, int H, int dil, int relu, __nv_bfloat16 *y16, float *y32, int Cout, cudaStream_t s);

}  // namespace hermite_nn
