// Internal declarations of the Hermite CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hermite.h"

namespace hermite {

constexpr int kMaxDim = 3;
constexpr int kMaxCoef = 255;   // coefficients per node handled by the kernels
constexpr int kMaxBox = 512;    // (2m+2)^d polynomial box held in setup kernels
constexpr int kNumForms = 2;    // energy quadratic forms per context

// Geometry of one half-step or one energy pass: target nodes live on grid
// `dst`, the cell centred at each target takes its 2^d corners from grid
// 1-dst (with ghosts for non-periodic boundaries).
struct Geometry {
  int d;
  int bc;
  int dst;             // 0 primal, 1 dual
  int64_t n_dst;       // nodes per axis of the target grid
  int64_t n_src;       // nodes per axis of the source grid
  int64_t nodes_dst;   // n_dst^d
  int64_t ld_src;      // plane stride (elements) of the source SoA array
  int64_t ld_dst;      // plane stride of the target SoA array
};

}  // namespace hermite

struct hermite_ctx {
  int d = 0, m = 0, variant = 0, bc = 0;
  int64_t N = 0;
  double c = 0, h = 0, dt = 0, lam = 0;
  int Nu = 0, Nv = 0;      // u / v coefficients per node
  int ncoef = 0;           // coefficients stored per node (Nu+Nv or Nu)
  int nci = 0, nco = 0;    // operator inputs / outputs
  int64_t npts[2] = {0, 0}, nodes[2] = {0, 0}, ld[2] = {0, 0};
  double *grid[2] = {nullptr, nullptr};   // SoA [ncoef][ld] of the paper's scaled data
  double *M = nullptr;                     // half-step operator [nco][nci]
  double *Mstart = nullptr;                // conservative start-up [Nu][Nu+Nv]
  double *Q[hermite::kNumForms] = {nullptr, nullptr};  // energy forms [2^d][nq][nq]
  int nq[hermite::kNumForms] = {0, 0};
  // low-rank factors of the forms whose integrands span few monomials per
  // parity class: Q_c = L_c^T L_c, L stored [2^d][rmax][nq] (zero-padded rows)
  double *L[hermite::kNumForms] = {nullptr, nullptr};
  int rmax[hermite::kNumForms] = {0, 0};   // rows used per class
  int lrows[hermite::kNumForms] = {0, 0};  // rows allocated per class
  int ltri[hermite::kNumForms] = {0, 0};   // 1: pivoted Cholesky (triangular after permutation)
  int16_t *lperm[hermite::kNumForms] = {nullptr, nullptr};  // [2^d][nq] column order
  double formscale[hermite::kNumForms] = {0, 0};
  int8_t *par_in = nullptr;    // parity bits of each operator input coefficient
  int8_t *par_out = nullptr;   // parity bits of each operator output coefficient
  double *staging = nullptr;   // host-layout staging [max nodes][Nu+Nv]
  double *scratch_grid = nullptr;  // one grid of u (conservative energy)
  double *partials = nullptr;      // energy block partial sums
  double *result = nullptr;        // energy results (device)
  int64_t partials_len = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t half = 0;            // half-steps since the state was set
  // split precision (HERMITE_SPLIT32): state as FP32 hi + lo pairs; the FP64
  // grids above then serve as the staging copies for I/O and energies
  int precision = 0;
  bool has_energy = true;      // energy forms built (batch problems skip them)
  float2 *fgrid[2] = {nullptr, nullptr};  // SoA [ncoef][ld] of (hi, lo)
  float2 *Lf[hermite::kNumForms] = {nullptr, nullptr};  // energy factors split hi + lo
  float2 *fscratch = nullptr;  // one split grid (conservative energy)
  // slot layout of the split half-step kernels (single problem and batch):
  // warp w's slots [0, psplit) hold outputs of parity class pcls[2w], slots
  // [psplit, pslots) outputs of class pcls[2w+1]; the operator is laid out
  // per warp
  float2 *Mp = nullptr;        // [2^d warp][nci][pslots]
  int16_t *prow = nullptr;     // [2^d][pslots] output row of each slot (-1 unused)
  int8_t *pcls = nullptr;      // [2^d][2]
  int pslots = 0, psplit = 0;
  // tensor-core split half-step (d >= 2, every parity class of inputs and of
  // outputs at most 16 wide): the operator's BF16 digit image, the class
  // tables and row exponents; split_engine 1 runs it, 0 the CUDA-core kernel
  bool tc_ready = false;
  int split_engine = 0;
  int tc_vexp = 0;             // velocity inputs are scaled by 2^tc_vexp
  uint4 *tc_B = nullptr;       // [group][input class][class in group][96 x 16 BF16]
  int16_t *tc_inb = nullptr;   // [2^d][16]
  int16_t *tc_orow = nullptr;  // [2^d][16]
  int8_t *tc_er = nullptr;     // [nco]
  int *tc_status = nullptr;    // bounded-wait error word
  // 1-D matrices of the sum-factorised dissipative energies (two class bits)
  double *tpm = nullptr;
  float2 *tpmf = nullptr;
  std::string err;
};

namespace hermite {

// Setup kernels (FP64, hermite_setup.cu).
int build_operator(hermite_ctx *ctx, bool startup, double *out, int rows, int cols);
int build_energy_forms(hermite_ctx *ctx);
int build_parity_tables(hermite_ctx *ctx);

// Hot path (hermite_step.cu).
int launch_half_step(hermite_ctx *ctx, int dst, const double *M, int nci, int nco,
                     const double *src, double *dst_arr, bool subtract_old);
int launch_to_device_layout(hermite_ctx *ctx, const double *host_layout_u,
                            const double *host_layout_v, int grid, int64_t nodes,
                            double *soa, int64_t ld, int nu_count, bool has_v);
int launch_to_host_layout(hermite_ctx *ctx, const double *soa, int64_t ld, int64_t nodes,
                          double *out_u, double *out_v, bool want_v);

// Split precision (hermite_split.cu).
int build_split_operator(hermite_ctx *ctx);
int launch_half_step_split(hermite_ctx *ctx, int dst, bool subtract_old);
int split_from_fp64(hermite_ctx *ctx, int grid);
int split_to_fp64(hermite_ctx *ctx, int grid);
int build_split_forms(hermite_ctx *ctx);
int launch_energy_form_split(hermite_ctx *ctx, int form, int grid, const float2 *A, const float2 *B,
                             double *result_slot);
int launch_half_step_split_into(hermite_ctx *ctx, int dst, const float2 *src, float2 *out, bool subtract_old);

// Tensor-core split half-step (hermite_tc_step.cu).  build_tc_operator sets
// tc_ready (and split_engine = 1) where the shapes allow; the launch writes
// `out` from `src` like launch_half_step_split_into; tc_check_status returns
// HERMITE_ERR_TIMEOUT (once) if a bounded wait of the kernel ran out.
int build_tc_operator(hermite_ctx *ctx);
int launch_half_step_tc(hermite_ctx *ctx, int dst, const float2 *src, float2 *out, bool subtract_old);
int tc_check_status(hermite_ctx *ctx);

// Energy reduction (hermite_energy.cu).
int launch_energy_form(hermite_ctx *ctx, int form, int g, const double *A, const double *B,
                       double *result_slot);
// Sum-factorised energies (hermite_energy_tp.cu): both forms of the level
// held on `grid` into out[0..1] (dissipative: plain, invariant; conservative:
// seminorm, gradient); HERMITE_ERR_UNSUPPORTED when the context has no
// tensor-product matrices (m out of the compiled range).
bool energy_tp_supported(int d, int m, int variant);
int build_energy_tp(hermite_ctx *ctx);
int launch_energy_tp(hermite_ctx *ctx, int grid, double *out);
// conservative only: the forms of A + sigma * B (sigma in {0, 1, -1}), A and B
// levels on `grid` in the context's precision (double or float2 planes,
// stride ld[grid]); A = NULL means the context's own level
int launch_energy_tp_pair(hermite_ctx *ctx, int grid, const void *A, const void *B, float sigma, double *out);
// the same on a caller's FP64 coefficient-major level (plane stride ld) with
// the given partial-sum scratch (at least 2 x 1184 doubles)
int launch_energy_tp_level(hermite_ctx *ctx, int grid, const double *level, int64_t ld, double *partials,
                           int64_t partials_len, double *out);

// L2 error of the I_m interpolant of the FP64 u level on `grid` against
// exact values at tensor quadrature points (hermite_error.cu); cells and
// exact are device pointers, xq / wq host arrays; synchronises the stream.
int launch_l2_error(hermite_ctx *ctx, int grid, int64_t ncells, const int64_t *cells, int nq, const double *xq,
                    const double *wq, const double *exact, double out[2]);

Geometry make_geometry(const hermite_ctx *ctx, int dst);
int create_context(int d, int m, int64_t N, double c, double h, double dt, int variant, int bc, int precision,
                   bool with_energy, hermite_ctx **out);
bool cuda_ok(hermite_ctx *ctx, cudaError_t e, const char *what);

// Every device allocation of the library goes through here: cudaMalloc, unless
// hermite_debug_fail_alloc asked this call to fail (tests of the clean-up paths).
cudaError_t device_alloc(void **p, size_t bytes);
template <class T>
inline cudaError_t device_alloc(T **p, size_t bytes) {
  return device_alloc(reinterpret_cast<void **>(p), bytes);
}

}  // namespace hermite
