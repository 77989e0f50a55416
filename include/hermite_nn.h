/*
 * hermite_nn.h -- C ABI of the learned super-stepper kernels (B300, sm_103a).
 *
 * A small convolutional network advances the primal nodal data of a periodic
 * 2-D dissipative Hermite problem by K full time steps at once; the Hermite
 * step itself (hermite.h) produces the training data, checks each answer and
 * is the fallback.  The paper has no counterpart: this is an extension built
 * beside the method (a learned surrogate of K applications of the half-step
 * pair of Sec. 3.1-3.4).
 *
 * Tensors are NHWC, x[b][y][x][c] (b = sample, y = node index along axis 0,
 * x = along axis 1, c = channel), periodic in y and x.  The image width W must
 * be 128 (one CTA row tile); H >= 1 is free.  Activations, gradients of
 * activations and the forward copies of the weights are BF16 (uint16_t bit
 * patterns, round-to-nearest-even); every product is accumulated in FP32 on
 * the tensor cores.  A 3x3 layer's weights are w[co][tap][ci], tap = 3*ky+kx,
 * reading the input at offset ((ky-1)*dil, (kx-1)*dil) from the output node.
 * Channel counts Cin, Cout must be 32 or 64 (inputs are zero-padded up to
 * 32); the supported (Cin, Cout) pairs are (32,64), (64,64), (64,32) and,
 * for the forward kernel only, (32,32).
 *
 * "Metric space" below is the solver's scaled nodal data with the v
 * coefficients multiplied by vscale = h/c, so that every entry is an
 * h^|k|/k!-scaled derivative of u or of (h/c) u_t.
 *
 * All pointers are device pointers; work is enqueued on the given
 * cudaStream_t (NULL = legacy default stream) and nothing synchronises.  No
 * call allocates device memory.  Every call returns 0 (HERMITE_OK), or
 * HERMITE_ERR_ARG (-1) for a NULL pointer or an unsupported size, or
 * HERMITE_ERR_CUDA (-3) if a launch fails.  Zero-sized inputs are a no-op.
 */
#ifndef HERMITE_NN_H
#define HERMITE_NN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y[p][co] = act(bias[co] + sum_{tap,ci} x[p + off(tap)][ci] w[co][tap][ci]),
 * x [B][H][128][Cin], w [Cout][9][Cin] (BF16), bias [Cout] FP32 or NULL.
 * relu = 1 applies max(0, .).  mask (BF16 [B][H][128][Cout] or NULL): the
 * result is set to 0 where mask <= 0 (the ReLU derivative, for the input
 * gradient).  Outputs: y_bf16 (BF16) and/or y_f32 (FP32), either may be NULL
 * but not both. */
int hnn_conv3x3_fwd(const uint16_t *x, const uint16_t *w, const float *bias, const uint16_t *mask, int B, int H,
                    int W, int Cin, int Cout, int dil, int relu, uint16_t *y_bf16, float *y_f32, void *stream);

/* Engine of hnn_conv3x3_fwd (process-wide): 0 (default) runs Cin = 64 layers
 * with dilation <= 8 on the fifth-generation tensor cores (tcgen05 MMAs with
 * tensor-memory accumulators, TMA-loaded input rows; other layers stay on
 * mma.sync),
 * 1 runs every layer on the mma.sync kernels.  Returns HERMITE_ERR_ARG for
 * another value. */
int hnn_set_conv_engine(int engine);

/* Synchronises the device, then returns HERMITE_ERR_TIMEOUT (and clears the
 * flag) if a tensor-core convolution gave up a bounded wait since the last
 * call (its output is then incomplete), else HERMITE_OK. */
int hnn_conv_status(void);

/* Self-test of the failure path: one block waits on an mbarrier that nothing
 * arrives at; its bounded wait (2^22 polls, well under a few seconds) gives up
 * and records the error that the next hnn_conv_status returns
 * (HERMITE_ERR_TIMEOUT).  The context stays usable. */
int hnn_wait_selftest(void *stream);

/* Self-test of the tensor-core path on one CTA: D[128][N] = A[128][64] B[N][64]^T,
 * A and B BF16 row-major, D FP32 row-major, N = 32 or 64; *status (device int,
 * caller-initialised to 0) is set to 1 if the MMA completion wait ran out. */
int hnn_tc_gemm_selftest(const uint16_t *A, const uint16_t *B, float *D, int N, int *status, void *stream);

/* Weights of the input-gradient convolution: wt[ci][tap][co] = w[co][8-tap][ci].
 * The gradient with respect to a layer's input is then
 * hnn_conv3x3_fwd(dy, wt, NULL, mask, ..., Cin = layer Cout, Cout = layer Cin). */
int hnn_flip_weights(const uint16_t *w, int Cout, int Cin, uint16_t *wt, void *stream);

/* Weight gradient, accumulated: dw[co][tap][ci] += sum_p dy[p][co] x[p + off(tap)][ci],
 * x [B][H][128][Cin], dy [B][H][128][Cout] (BF16), dw FP32. */
int hnn_conv3x3_wgrad(const uint16_t *x, const uint16_t *dy, int B, int H, int W, int Cin, int Cout, int dil,
                      float *dw, void *stream);

/* Bias gradient, accumulated: db[c] += sum_p dy[p][c], dy BF16 [npix][C]. */
int hnn_bias_grad(const uint16_t *dy, int64_t npix, int C, float *db, void *stream);

/* Weighted squared error of an FP32 prediction y against a target t, both
 * [npix][C]: loss[0] += scale * sum_{p,c} wch[c] (y - t)^2 (FP64 accumulation)
 * and dy = bf16(2 scale wch[c] (y - t)).  wch [C] FP32; loss may be NULL. */
int hnn_mse(const float *y, const float *t, const float *wch, int64_t npix, int C, float scale, double *loss,
            uint16_t *dy, void *stream);

/* One bias-corrected Adam step (step number t >= 1) on FP32 parameters p with
 * gradient g and moments m, v (all [n]); g is reset to 0 afterwards and
 * p_bf16 (may be NULL) receives the BF16 copy the forward kernels read. */
int hnn_adam(float *p, float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2, float eps,
             int t, uint16_t *p_bf16, void *stream);

/* Solver state of one problem (u [n][Nu], v [n][Nv], FP64, the layout of
 * hermite_get_grid_device) -> metric-space FP32 rows out[n][ld], channels
 * 0..Nu+Nv-1 written (ld >= Nu+Nv). */
int hnn_state_to_f32(const double *u, const double *v, int64_t n, int Nu, int Nv, double vscale, float *out, int ld,
                     void *stream);

/* Network input of n nodes (one problem, or several back to back):
 * x[i][c] = bf16((s_c - shift[c]) / scale[c]) for the metric-space value s_c of
 * node i, c < Nu+Nv <= 64, and 0 for Nu+Nv <= c < C.  Evaluated in FP32 as
 * (fl32(s_c) - fl32(shift[c])) * fl32(1 / scale[c]), with
 * fl32(s_c) = fl32(v) * fl32(vscale) for the v channels. */
int hnn_pack_state(const double *u, const double *v, int64_t n, int Nu, int Nv, double vscale, const double *shift,
                   const double *scale, int C, uint16_t *x, void *stream);

/* Residual update of n nodes: with the change d = fl32(fl32(dscale[c]) y[i][c])
 * (FP32), u_out = u + d and v_out = v + d / vscale (FP64; the outputs may
 * alias the inputs); y FP32 [n][C], Nu+Nv <= 64. */
int hnn_unpack_state(const double *u, const double *v, const float *y, int64_t n, int Nu, int Nv, double vscale,
                     const double *dscale, int C, double *u_out, double *v_out, void *stream);

/* Training pairs from stored metric-space levels (FP32 rows of C0 <= 64
 * channels): for sample s, a = levels + src[s], b = levels + dst[s] (element
 * offsets, n rows each): x[s][i][c] = bf16((a - shift[c]) / scale[c]) and
 * t[s][i][c] = (b - a) / dscale[c] for c < C0, zeros up to C (FP32 arithmetic
 * with the reciprocals rounded to FP32). */
int hnn_make_pairs(const float *levels, const int64_t *src, const int64_t *dst, int nsamp, int64_t n, int C0,
                   const double *shift, const double *scale, const double *dscale, int C, uint16_t *x, float *t,
                   void *stream);

/* Channel moments: out[c] += sum_i d[i][c], out[C + c] += sum_i d[i][c]^2 with
 * d = a - b (b may be NULL: d = a), rows of C FP32 values, FP64 sums. */
int hnn_moments(const float *a, const float *b, int64_t n, int C, double *out, void *stream);

/* Metric-space distance of two states of one problem: out[0] += sum (a - b)^2,
 * out[1] += sum b^2 (FP64, u and vscale * v entries together); a_v, b_v may
 * be NULL when Nv = 0. */
int hnn_sqdiff(const double *a_u, const double *a_v, const double *b_u, const double *b_v, int64_t n, int Nu, int Nv,
               double vscale, double *out, void *stream);

/* hnn_sqdiff for nsamp problems at once: a_u, b_u [nsamp][n][Nu], a_v, b_v
 * [nsamp][n][Nv] back to back; out[2 s], out[2 s + 1] += the sums of sample s. */
int hnn_sqdiff_batch(const double *a_u, const double *a_v, const double *b_u, const double *b_v, int nsamp, int64_t n,
                     int Nu, int Nv, double vscale, double *out, void *stream);

/* Block copy: dst[didx[i]] = src[sidx[i]] for i < nblk, blocks of `block`
 * doubles (sidx or didx NULL: the identity); index arrays are device int64. */
int hnn_copy_blocks(const double *src, const int64_t *sidx, double *dst, const int64_t *didx, int nblk, int64_t block,
                    void *stream);

#ifdef __cplusplus
}
#endif
#endif
