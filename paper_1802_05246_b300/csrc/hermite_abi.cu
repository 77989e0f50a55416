// C ABI of the Hermite library (declarations and contracts: include/hermite.h).
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "hermite_internal.h"

namespace hermite {

bool cuda_ok(hermite_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

namespace {
std::atomic<int> g_fail_alloc{0};  // > 0: the g_fail_alloc-th next allocation fails
}

cudaError_t device_alloc(void **p, size_t bytes) {
  int n = g_fail_alloc.load();
  while (n > 0) {
    if (g_fail_alloc.compare_exchange_weak(n, n - 1)) {
      if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

}  // namespace hermite

using namespace hermite;

namespace {

thread_local std::string g_create_error;

int fail(hermite_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int64_t ipow64(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

bool supported(int d, int m) {
  if (d == 1) return m <= 12;
  if (d == 2) return m <= 6;
  return m <= 3;
}

void release(hermite_ctx *ctx) {
  for (int g = 0; g < 2; ++g) cudaFree(ctx->grid[g]);
  cudaFree(ctx->M);
  cudaFree(ctx->Mstart);
  for (int f = 0; f < kNumForms; ++f) {
    cudaFree(ctx->Q[f]);
    cudaFree(ctx->L[f]);
    cudaFree(ctx->lperm[f]);
    cudaFree(ctx->Lf[f]);
  }
  cudaFree(ctx->par_in);
  cudaFree(ctx->staging);
  cudaFree(ctx->scratch_grid);
  cudaFree(ctx->partials);
  cudaFree(ctx->result);
  for (int g = 0; g < 2; ++g) cudaFree(ctx->fgrid[g]);
  cudaFree(ctx->fscratch);
  cudaFree(ctx->Mp);
  cudaFree(ctx->prow);
  cudaFree(ctx->pcls);
  cudaFree(ctx->tpm);
  cudaFree(ctx->tpmf);
  cudaFree(ctx->tc_B);
  cudaFree(ctx->tc_inb);
  cudaFree(ctx->tc_orow);
  cudaFree(ctx->tc_er);
  cudaFree(ctx->tc_status);
}

bool is_split(const hermite_ctx *ctx) { return ctx->precision == HERMITE_SPLIT32; }

// split precision: refresh the FP32 hi/lo state from the FP64 copies, or the
// FP64 copies from the state
int sync_split_from_fp64(hermite_ctx *ctx) {
  if (!is_split(ctx)) return HERMITE_OK;
  for (int g = 0; g < 2; ++g) {
    int rc = split_from_fp64(ctx, g);
    if (rc) return rc;
  }
  return HERMITE_OK;
}

int sync_fp64_from_split(hermite_ctx *ctx, int grid) {
  if (!is_split(ctx)) return HERMITE_OK;
  for (int g = 0; g < 2; ++g) {
    if (grid >= 0 && g != grid) continue;
    int rc = split_to_fp64(ctx, g);
    if (rc) return rc;
  }
  return HERMITE_OK;
}

bool is_cons(const hermite_ctx *ctx) { return ctx->variant == HERMITE_CONSERVATIVE; }

// grid holding the newest level
int newest_grid(const hermite_ctx *ctx) {
  if (is_cons(ctx)) return (ctx->half % 2 == 0) ? HERMITE_DUAL : HERMITE_PRIMAL;
  return (ctx->half % 2 == 0) ? HERMITE_PRIMAL : HERMITE_DUAL;
}

int one_half_step(hermite_ctx *ctx) {
  int rc;
  if (is_split(ctx)) {
    const int dst = is_cons(ctx) ? ((ctx->half % 2 == 0) ? HERMITE_PRIMAL : HERMITE_DUAL)
                                 : ((ctx->half % 2 == 0) ? HERMITE_DUAL : HERMITE_PRIMAL);
    rc = launch_half_step_split(ctx, dst, is_cons(ctx));
  } else if (is_cons(ctx)) {
    const int dst = (ctx->half % 2 == 0) ? HERMITE_PRIMAL : HERMITE_DUAL;
    rc = launch_half_step(ctx, dst, ctx->M, ctx->nci, ctx->nco, ctx->grid[1 - dst], ctx->grid[dst], true);
  } else {
    const int dst = (ctx->half % 2 == 0) ? HERMITE_DUAL : HERMITE_PRIMAL;
    rc = launch_half_step(ctx, dst, ctx->M, ctx->nci, ctx->nco, ctx->grid[1 - dst], ctx->grid[dst], false);
  }
  if (rc == HERMITE_OK) ctx->half += 1;
  return rc;
}

// host [node][coef] buffers -> device SoA grid (through the staging buffer)
int upload_grid(hermite_ctx *ctx, int grid, const double *u, const double *v, bool device_src) {
  const int64_t nodes = ctx->nodes[grid];
  const bool with_v = !is_cons(ctx) && ctx->Nv > 0;
  double *su = ctx->staging;
  double *sv = ctx->staging + nodes * ctx->Nu;
  const cudaMemcpyKind kind = device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (nodes * ctx->Nu > 0 &&
      !cuda_ok(ctx, cudaMemcpyAsync(su, u, sizeof(double) * nodes * ctx->Nu, kind, ctx->stream), "copy u"))
    return HERMITE_ERR_CUDA;
  const double *vsrc = nullptr;
  if (with_v && v) {
    if (!cuda_ok(ctx, cudaMemcpyAsync(sv, v, sizeof(double) * nodes * ctx->Nv, kind, ctx->stream), "copy v"))
      return HERMITE_ERR_CUDA;
    vsrc = sv;
  }
  int rc = launch_to_device_layout(ctx, su, vsrc, grid, nodes, ctx->grid[grid], ctx->ld[grid], ctx->Nu, with_v);
  if (rc) return rc;
  if (!device_src && !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "upload sync")) return HERMITE_ERR_CUDA;
  return HERMITE_OK;
}

int download_grid(hermite_ctx *ctx, int grid, double *u, double *v, bool device_dst) {
  if (int rc = sync_fp64_from_split(ctx, grid)) return rc;
  const int64_t nodes = ctx->nodes[grid];
  const bool want_v = !is_cons(ctx) && ctx->Nv > 0 && v != nullptr;
  double *su = ctx->staging;
  double *sv = ctx->staging + nodes * ctx->Nu;
  int rc = launch_to_host_layout(ctx, ctx->grid[grid], ctx->ld[grid], nodes, su, sv, want_v);
  if (rc) return rc;
  const cudaMemcpyKind kind = device_dst ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (u && nodes * ctx->Nu > 0 &&
      !cuda_ok(ctx, cudaMemcpyAsync(u, su, sizeof(double) * nodes * ctx->Nu, kind, ctx->stream), "copy u out"))
    return HERMITE_ERR_CUDA;
  if (want_v &&
      !cuda_ok(ctx, cudaMemcpyAsync(v, sv, sizeof(double) * nodes * ctx->Nv, kind, ctx->stream), "copy v out"))
    return HERMITE_ERR_CUDA;
  if (!cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "download sync")) return HERMITE_ERR_CUDA;
  return tc_check_status(ctx);
}

// conservative start-up: dual level at dt/2 from the primal (u, v) data held
// in the scratch grid as SoA planes (u then (h/c) v)
int cons_startup(hermite_ctx *ctx, const double *u, const double *v, bool device_src) {
  const int64_t nodes = ctx->nodes[0];
  double *su = ctx->staging;
  double *sv = ctx->staging + nodes * ctx->Nu;
  const cudaMemcpyKind kind = device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!cuda_ok(ctx, cudaMemcpyAsync(su, u, sizeof(double) * nodes * ctx->Nu, kind, ctx->stream), "copy u"))
    return HERMITE_ERR_CUDA;
  const bool with_v = ctx->Nv > 0;
  if (with_v) {
    if (v) {
      if (!cuda_ok(ctx, cudaMemcpyAsync(sv, v, sizeof(double) * nodes * ctx->Nv, kind, ctx->stream), "copy v"))
        return HERMITE_ERR_CUDA;
    } else if (!cuda_ok(ctx, cudaMemsetAsync(sv, 0, sizeof(double) * nodes * ctx->Nv, ctx->stream), "zero v")) {
      return HERMITE_ERR_CUDA;
    }
  }
  // primal u -> grid 0; (u, v) -> scratch SoA with Nu+Nv planes
  int rc = launch_to_device_layout(ctx, su, nullptr, 0, nodes, ctx->grid[0], ctx->ld[0], ctx->Nu, false);
  if (rc) return rc;
  rc = launch_to_device_layout(ctx, su, with_v ? sv : nullptr, 0, nodes, ctx->scratch_grid, ctx->ld[0], ctx->Nu,
                               with_v);
  if (rc) return rc;
  rc = launch_half_step(ctx, HERMITE_DUAL, ctx->Mstart, ctx->Nu + ctx->Nv, ctx->Nu, ctx->scratch_grid,
                        ctx->grid[1], false);
  if (rc) return rc;
  if (!device_src && !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "startup sync")) return HERMITE_ERR_CUDA;
  return HERMITE_OK;
}

}  // namespace

extern "C" {

int hermite_create(int d, int m, int64_t N, double c, double h, double dt, int variant, int bc,
                   hermite_ctx **out) {
  return hermite_create_ex(d, m, N, c, h, dt, variant, bc, HERMITE_FP64, out);
}

int hermite_create_ex(int d, int m, int64_t N, double c, double h, double dt, int variant, int bc,
                      int precision, hermite_ctx **out) {
  return hermite::create_context(d, m, N, c, h, dt, variant, bc, precision, true, out);
}

}  // extern "C"

namespace hermite {

int create_context(int d, int m, int64_t N, double c, double h, double dt, int variant, int bc, int precision,
                   bool with_energy, hermite_ctx **out) {
  if (precision != HERMITE_FP64 && precision != HERMITE_SPLIT32) {
    g_create_error = "unknown precision";
    if (out) *out = nullptr;
    return HERMITE_ERR_ARG;
  }
  if (!out) {
    g_create_error = "out is NULL";
    return HERMITE_ERR_ARG;
  }
  *out = nullptr;
  const bool cons = variant == HERMITE_CONSERVATIVE;
  if (d < 1 || d > 3 || N < 1 || !(c > 0) || !(h > 0) || !(dt > 0) || !std::isfinite(c) ||
      !std::isfinite(h) || !std::isfinite(dt) ||
      (variant != HERMITE_DISSIPATIVE && variant != HERMITE_CONSERVATIVE &&
       variant != HERMITE_DISSIPATIVE_SIMPLE) ||
      (bc != HERMITE_PERIODIC && bc != HERMITE_DIRICHLET && bc != HERMITE_NEUMANN) || (cons ? m < 0 : m < 1)) {
    g_create_error = "invalid argument to hermite_create";
    return HERMITE_ERR_ARG;
  }
  const double lam = c * dt / h;
  if (!(lam > 0) || lam > 1.0 + 1e-12) {
    g_create_error = "CFL number c*dt/h must lie in (0, 1]";
    return HERMITE_ERR_ARG;
  }
  if (!supported(d, m)) {
    g_create_error = "(d, m) outside the compiled range";
    return HERMITE_ERR_UNSUPPORTED;
  }
  hermite_ctx *ctx = new (std::nothrow) hermite_ctx;
  if (!ctx) {
    g_create_error = "host allocation failed";
    return HERMITE_ERR_ALLOC;
  }
  ctx->d = d;
  ctx->m = m;
  ctx->variant = variant;
  ctx->bc = bc;
  ctx->N = N;
  ctx->c = c;
  ctx->h = h;
  ctx->dt = dt;
  ctx->lam = lam;
  ctx->Nu = (int)ipow64(m + 1, d);
  ctx->Nv = (int)ipow64(m, d);
  ctx->ncoef = cons ? ctx->Nu : ctx->Nu + ctx->Nv;
  ctx->nci = ctx->ncoef;
  ctx->nco = ctx->ncoef;
  for (int g = 0; g < 2; ++g) {
    ctx->npts[g] = (bc == HERMITE_PERIODIC) ? N : (g == 0 ? N + 1 : N);
    ctx->nodes[g] = ipow64(ctx->npts[g], d);
    ctx->ld[g] = (ctx->nodes[g] + 31) / 32 * 32;
  }
  cudaGetDevice(&ctx->device);
  int rc = HERMITE_OK;
  const int64_t maxnodes = std::max(ctx->nodes[0], ctx->nodes[1]);
  const int64_t maxld = std::max(ctx->ld[0], ctx->ld[1]);
  auto alloc = [&](void **p, size_t bytes, const char *what) {
    if (rc) return;
    if (!cuda_ok(ctx, device_alloc(p, bytes ? bytes : 8), what)) rc = HERMITE_ERR_ALLOC;
  };
  for (int g = 0; g < 2; ++g) alloc((void **)&ctx->grid[g], sizeof(double) * ctx->ncoef * ctx->ld[g], "grid");
  alloc((void **)&ctx->M, sizeof(double) * ctx->nco * ctx->nci, "operator");
  alloc((void **)&ctx->staging, sizeof(double) * maxnodes * (ctx->Nu + ctx->Nv), "staging");
  if (cons) {
    alloc((void **)&ctx->Mstart, sizeof(double) * ctx->Nu * (ctx->Nu + ctx->Nv), "startup operator");
    alloc((void **)&ctx->scratch_grid, sizeof(double) * (ctx->Nu + ctx->Nv) * maxld, "scratch grid");
  }
  ctx->partials_len = 148 * 8 * (1 << d);
  alloc((void **)&ctx->partials, sizeof(double) * ctx->partials_len, "partials");
  alloc((void **)&ctx->result, sizeof(double) * 8, "result");
  for (int g = 0; g < 2 && rc == HERMITE_OK; ++g)
    if (!cuda_ok(ctx, cudaMemset(ctx->grid[g], 0, sizeof(double) * ctx->ncoef * ctx->ld[g]), "memset"))
      rc = HERMITE_ERR_CUDA;
  if (rc == HERMITE_OK) rc = build_parity_tables(ctx);
  if (rc == HERMITE_OK) rc = build_operator(ctx, false, ctx->M, ctx->nco, ctx->nci);
  if (rc == HERMITE_OK && cons) rc = build_operator(ctx, true, ctx->Mstart, ctx->Nu, ctx->Nu + ctx->Nv);
  ctx->has_energy = with_energy;
  if (rc == HERMITE_OK && with_energy) rc = build_energy_forms(ctx);
  ctx->precision = precision;
  if (rc == HERMITE_OK && precision == HERMITE_SPLIT32) {
    for (int g = 0; g < 2; ++g) alloc((void **)&ctx->fgrid[g], sizeof(float2) * ctx->ncoef * ctx->ld[g], "split grid");
    for (int g = 0; g < 2 && rc == HERMITE_OK; ++g)
      if (!cuda_ok(ctx, cudaMemset(ctx->fgrid[g], 0, sizeof(float2) * ctx->ncoef * ctx->ld[g]), "memset"))
        rc = HERMITE_ERR_CUDA;
    if (rc == HERMITE_OK) rc = build_split_operator(ctx);
    // batch problems (built without energy forms) run the batch kernels only
    if (rc == HERMITE_OK && with_energy) rc = build_tc_operator(ctx);
    if (rc == HERMITE_OK) rc = build_split_forms(ctx);
    if (cons) alloc((void **)&ctx->fscratch, sizeof(float2) * ctx->Nu * maxld, "split scratch");
  }
  if (rc == HERMITE_OK && with_energy) rc = build_energy_tp(ctx);
  if (rc == HERMITE_OK && !cuda_ok(ctx, cudaDeviceSynchronize(), "create sync")) rc = HERMITE_ERR_CUDA;
  if (rc != HERMITE_OK) {
    g_create_error = ctx->err.empty() ? "hermite_create failed" : ctx->err;
    release(ctx);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return HERMITE_OK;
}

}  // namespace hermite

extern "C" {

void hermite_destroy(hermite_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  release(ctx);
  delete ctx;
}

int hermite_set_stream(hermite_ctx *ctx, void *stream) {
  if (!ctx) return HERMITE_ERR_ARG;
  ctx->stream = (cudaStream_t)stream;
  return HERMITE_OK;
}

static int set_state_impl(hermite_ctx *ctx, const double *u, const double *v, bool device_src) {
  if (!ctx) return HERMITE_ERR_ARG;
  if (!u) return fail(ctx, HERMITE_ERR_ARG, "u is NULL");
  int rc;
  if (is_cons(ctx)) {
    rc = cons_startup(ctx, u, v, device_src);
  } else {
    rc = upload_grid(ctx, HERMITE_PRIMAL, u, v, device_src);
  }
  if (rc == HERMITE_OK) rc = sync_split_from_fp64(ctx);
  if (rc == HERMITE_OK) ctx->half = 0;
  return rc;
}

int hermite_set_state(hermite_ctx *ctx, const double *u, const double *v) {
  return set_state_impl(ctx, u, v, false);
}

int hermite_set_state_device(hermite_ctx *ctx, const double *u, const double *v) {
  return set_state_impl(ctx, u, v, true);
}

int hermite_set_state2(hermite_ctx *ctx, const double *u_primal, const double *u_dual) {
  if (!ctx) return HERMITE_ERR_ARG;
  if (!is_cons(ctx)) return fail(ctx, HERMITE_ERR_STATE, "hermite_set_state2 is for the conservative method");
  if (!u_primal || !u_dual) return fail(ctx, HERMITE_ERR_ARG, "NULL level");
  int rc = upload_grid(ctx, HERMITE_PRIMAL, u_primal, nullptr, false);
  if (rc == HERMITE_OK) rc = upload_grid(ctx, HERMITE_DUAL, u_dual, nullptr, false);
  if (rc == HERMITE_OK) rc = sync_split_from_fp64(ctx);
  if (rc == HERMITE_OK) ctx->half = 0;
  return rc;
}

int hermite_debug_fail_alloc(int n) {
  if (n < 0) return HERMITE_ERR_ARG;
  g_fail_alloc.store(n);
  return HERMITE_OK;
}

int hermite_step(hermite_ctx *ctx, int64_t nsteps) {
  if (!ctx) return HERMITE_ERR_ARG;
  if (nsteps < 0) return fail(ctx, HERMITE_ERR_ARG, "nsteps < 0");
  return hermite_advance_half(ctx, 2 * nsteps);
}

int hermite_advance_half(hermite_ctx *ctx, int64_t nhalf) {
  if (!ctx) return HERMITE_ERR_ARG;
  if (nhalf < 0) return fail(ctx, HERMITE_ERR_ARG, "nhalf < 0");
  for (int64_t i = 0; i < nhalf; ++i) {
    int rc = one_half_step(ctx);
    if (rc) return rc;
  }
  return HERMITE_OK;
}

int64_t hermite_half_steps(const hermite_ctx *ctx) { return ctx ? ctx->half : -1; }

double hermite_time(const hermite_ctx *ctx) {
  if (!ctx) return NAN;
  if (is_cons(ctx)) return (double)((ctx->half + 1) / 2) * ctx->dt;
  return (double)ctx->half * 0.5 * ctx->dt;
}

int hermite_l2_error(hermite_ctx *ctx, int grid, int64_t ncells, const int64_t *cells, int nq, const double *xq,
                     const double *wq, const double *exact, double out[2]) {
  if (!ctx) return HERMITE_ERR_ARG;
  if ((grid != 0 && grid != 1) || !xq || !wq || !exact || !out)
    return fail(ctx, HERMITE_ERR_ARG, "hermite_l2_error: bad grid or NULL pointer");
  if (int rc = sync_fp64_from_split(ctx, grid)) return rc;
  return launch_l2_error(ctx, grid, ncells, cells, nq, xq, wq, exact, out);
}

int hermite_get_state(hermite_ctx *ctx, double *u, double *v) {
  if (!ctx) return HERMITE_ERR_ARG;
  if (!u) return fail(ctx, HERMITE_ERR_ARG, "u is NULL");
  if (!is_cons(ctx) && ctx->half % 2 != 0)
    return fail(ctx, HERMITE_ERR_STATE, "the newest dissipative level is on the dual grid");
  return download_grid(ctx, HERMITE_PRIMAL, u, v, false);
}

int hermite_get_grid(hermite_ctx *ctx, int grid, double *u, double *v) {
  if (!ctx) return HERMITE_ERR_ARG;
  if ((grid != 0 && grid != 1) || !u) return fail(ctx, HERMITE_ERR_ARG, "bad grid or NULL u");
  return download_grid(ctx, grid, u, v, false);
}

int hermite_get_grid_device(hermite_ctx *ctx, int grid, double *u, double *v) {
  if (!ctx) return HERMITE_ERR_ARG;
  if ((grid != 0 && grid != 1) || !u) return fail(ctx, HERMITE_ERR_ARG, "bad grid or NULL u");
  return download_grid(ctx, grid, u, v, true);
}

int hermite_set_grid(hermite_ctx *ctx, int grid, const double *u, const double *v) {
  if (!ctx) return HERMITE_ERR_ARG;
  if ((grid != 0 && grid != 1) || !u) return fail(ctx, HERMITE_ERR_ARG, "bad grid or NULL u");
  if (int rc = sync_fp64_from_split(ctx, 1 - grid)) return rc;
  int rc = upload_grid(ctx, grid, u, v, false);
  if (rc == HERMITE_OK && is_split(ctx)) rc = split_from_fp64(ctx, grid);
  return rc;
}

// Conservative energies with the sum-factorised kernel: the forms of the
// newest level (slots 0, 1), of A + B and A - B for the tentative next level
// A and the older level B (slots 2, 4: polarisation of their inner product),
// and, when the newest level is the dual one, of the primal level (slot 7).
static int cons_energies_tp(hermite_ctx *ctx, int gnew, const void *A, const void *B) {
  const int gold = 1 - gnew;
  int rc = launch_energy_tp(ctx, gnew, ctx->result + 0);
  if (!rc) rc = launch_energy_tp_pair(ctx, gold, A, B, 1.0f, ctx->result + 2);
  if (!rc) rc = launch_energy_tp_pair(ctx, gold, A, B, -1.0f, ctx->result + 4);
  if (!rc && gnew != 0) rc = launch_energy_tp(ctx, 0, ctx->result + 6);
  return rc;
}

int hermite_energy(hermite_ctx *ctx, double out[3]) {
  if (!ctx || !out) return ctx ? fail(ctx, HERMITE_ERR_ARG, "out is NULL") : HERMITE_ERR_ARG;
  if (!ctx->has_energy) return fail(ctx, HERMITE_ERR_STATE, "this context was created without energy forms");
  int rc = HERMITE_OK;
  bool cons_tp = false;
  double host[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (is_split(ctx)) {
    // split contexts reduce their hi + lo levels in the same arithmetic
    if (!is_cons(ctx)) {
      const int g = newest_grid(ctx);
      rc = launch_energy_tp(ctx, g, ctx->result);
      if (rc == HERMITE_ERR_UNSUPPORTED) {
        rc = launch_energy_form_split(ctx, 0, g, ctx->fgrid[g], ctx->fgrid[g], ctx->result + 0);
        if (!rc) rc = launch_energy_form_split(ctx, 1, g, ctx->fgrid[g], ctx->fgrid[g], ctx->result + 1);
      }
    } else {
      const int gnew = newest_grid(ctx), gold = 1 - gnew;
      const size_t bytes = sizeof(float2) * ctx->Nu * ctx->ld[gold];
      if (!cuda_ok(ctx, cudaMemcpyAsync(ctx->fscratch, ctx->fgrid[gold], bytes, cudaMemcpyDeviceToDevice,
                                        ctx->stream),
                   "copy level"))
        return HERMITE_ERR_CUDA;
      rc = launch_half_step_split_into(ctx, gold, ctx->fgrid[gnew], ctx->fscratch, true);
      if (!rc && ctx->tpm) {
        rc = cons_energies_tp(ctx, gnew, ctx->fscratch, ctx->fgrid[gold]);
        cons_tp = true;
      } else {
        if (!rc) rc = launch_energy_form_split(ctx, 0, gnew, ctx->fgrid[gnew], ctx->fgrid[gnew], ctx->result + 0);
        if (!rc) rc = launch_energy_form_split(ctx, 0, gold, ctx->fscratch, ctx->fgrid[gold], ctx->result + 1);
        if (!rc) rc = launch_energy_form_split(ctx, 1, 0, ctx->fgrid[0], ctx->fgrid[0], ctx->result + 2);
      }
    }
  } else if (!is_cons(ctx)) {
    const int g = newest_grid(ctx);
    rc = launch_energy_tp(ctx, g, ctx->result);
    if (rc == HERMITE_ERR_UNSUPPORTED) {
      rc = launch_energy_form(ctx, 0, g, ctx->grid[g], ctx->grid[g], ctx->result + 0);
      if (!rc) rc = launch_energy_form(ctx, 1, g, ctx->grid[g], ctx->grid[g], ctx->result + 1);
    }
  } else {
    // G = |p_new|^2 - <p_next, p_old>: p_next is the tentative update of the
    // older level's grid, formed in the scratch grid
    const int gnew = newest_grid(ctx), gold = 1 - gnew;
    const size_t bytes = sizeof(double) * ctx->Nu * ctx->ld[gold];
    if (!cuda_ok(ctx, cudaMemcpyAsync(ctx->scratch_grid, ctx->grid[gold], bytes, cudaMemcpyDeviceToDevice,
                                      ctx->stream),
                 "copy level"))
      return HERMITE_ERR_CUDA;
    rc = launch_half_step(ctx, gold, ctx->M, ctx->nci, ctx->nco, ctx->grid[gnew], ctx->scratch_grid, true);
    if (!rc && ctx->tpm) {
      rc = cons_energies_tp(ctx, gnew, ctx->scratch_grid, ctx->grid[gold]);
      cons_tp = true;
    } else {
      if (!rc) rc = launch_energy_form(ctx, 0, gnew, ctx->grid[gnew], ctx->grid[gnew], ctx->result + 0);
      if (!rc) rc = launch_energy_form(ctx, 0, gold, ctx->scratch_grid, ctx->grid[gold], ctx->result + 1);
      if (!rc) rc = launch_energy_form(ctx, 1, 0, ctx->grid[0], ctx->grid[0], ctx->result + 2);
    }
  }
  if (rc) return rc;
  if (!cuda_ok(ctx, cudaMemcpyAsync(host, ctx->result, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx->stream),
               "energy copy") ||
      !cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "energy sync"))
    return HERMITE_ERR_CUDA;
  if (cons_tp) {
    // slots: [0,1] forms of the newest level, [2] |A+B|^2, [4] |A-B|^2 of the
    // tentative next level A and the older level B (their inner product is
    // the difference / 4), [1] or [7] the gradient form of the primal level
    out[0] = newest_grid(ctx) == 0 ? host[1] : host[7];
    out[1] = host[0] - 0.25 * (host[2] - host[4]);
  } else if (is_cons(ctx)) {
    out[0] = host[2];
    out[1] = host[0] - host[1];
  } else {
    out[0] = host[0];
    out[1] = host[1];
  }
  out[2] = 0.0;
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]))
    return fail(ctx, HERMITE_ERR_NONFINITE, "non-finite energy");
  return HERMITE_OK;
}

int64_t hermite_nodes(const hermite_ctx *ctx, int grid) {
  if (!ctx || (grid != 0 && grid != 1)) return -1;
  return ctx->nodes[grid];
}

int hermite_ncoef(const hermite_ctx *ctx, int *nu, int *nv) {
  if (!ctx) return HERMITE_ERR_ARG;
  if (nu) *nu = ctx->Nu;
  if (nv) *nv = ctx->Nv;
  return HERMITE_OK;
}

int hermite_operator(hermite_ctx *ctx, int which, double *out, int *rows, int *cols) {
  if (!ctx) return HERMITE_ERR_ARG;
  const double *src;
  int r, c;
  if (which == 0) {
    src = ctx->M;
    r = ctx->nco;
    c = ctx->nci;
  } else if (which == 1 && is_cons(ctx)) {
    src = ctx->Mstart;
    r = ctx->Nu;
    c = ctx->Nu + ctx->Nv;
  } else {
    return fail(ctx, HERMITE_ERR_ARG, "no such operator");
  }
  if (rows) *rows = r;
  if (cols) *cols = c;
  if (!out) return HERMITE_OK;
  if (!cuda_ok(ctx, cudaMemcpy(out, src, sizeof(double) * r * c, cudaMemcpyDeviceToHost), "operator copy"))
    return HERMITE_ERR_CUDA;
  return HERMITE_OK;
}

const char *hermite_last_error(const hermite_ctx *ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"
