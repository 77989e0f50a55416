// Device helpers shared by the split-precision half-step and the
// sum-factorised energy kernels: double-FP32 ("hi + lo") arithmetic and the
// corner gather of a cell with the ghost signs of Sec. 3.1.3.
#pragma once

#include "hermite_internal.h"

namespace hermite {
namespace dev {

// IEEE round-to-nearest intrinsics keep the compiler from contracting the
// error-free transformations into FMAs.
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float2 t = two_sum(a.x, b.x);
  t.y = __fadd_rn(t.y, __fadd_rn(a.y, b.y));
  return t;
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 df_norm(float2 a) {
  const float s = __fadd_rn(a.x, a.y);
  return make_float2(s, __fsub_rn(a.y, __fsub_rn(s, a.x)));
}

// acc += m * y with three split products and a compensated sum
__device__ __forceinline__ void df_fma(float2 &acc, const float2 m, const float2 y) {
  const float p = __fmul_rn(m.x, y.x);
  const float e = __fmaf_rn(m.x, y.x, -p);
  const float2 s = two_sum(acc.x, p);
  float c = __fadd_rn(acc.y, __fadd_rn(s.y, e));
  c = __fmaf_rn(m.x, y.y, c);
  c = __fmaf_rn(m.y, y.x, c);
  acc = make_float2(s.x, c);
}

// Two accumulators at once, (ahi, alo) holding slots (j, j+1) as hi and lo
// pairs: acc += m * y for both, with the operations of df_fma on packed FP32
// pairs (one instruction for the two slots; the same roundings, so the same
// results).  y is shared: yhi = (y.x, y.x), ylo = (y.y, y.y), nyhi = -yhi.
// A difference u - v is formed as fma(v, -1, u), which rounds like u - v.
__device__ __forceinline__ void df_fma_x2(float2 &ahi, float2 &alo, const float2 mhi, const float2 mlo,
                                          const float2 yhi, const float2 ylo, const float2 nyhi) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 pn = __fmul2_rn(mhi, nyhi);    // -p, p = fl(m.hi y.hi)
  const float2 e = __ffma2_rn(mhi, yhi, pn);  // m.hi y.hi - p, exact
  const float2 s = __ffma2_rn(pn, m1, ahi);   // fl(a + p)
  const float2 bb = __ffma2_rn(ahi, m1, s);   // fl(s - a)
  const float2 t1 = __ffma2_rn(bb, m1, s);    // fl(s - bb)
  const float2 t2 = __ffma2_rn(t1, m1, ahi);  // fl(a - (s - bb))
  const float2 t3 = __fadd2_rn(pn, bb);       // -fl(p - bb)
  const float2 err = __ffma2_rn(t3, m1, t2);  // rounding error of a + p
  float2 c = __fadd2_rn(alo, __fadd2_rn(err, e));
  c = __ffma2_rn(mhi, ylo, c);
  c = __ffma2_rn(mlo, yhi, c);
  ahi = s;
  alo = c;
}

// a * b with the same three split products, normalised
__device__ __forceinline__ float2 df_mul(const float2 a, const float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return df_norm(make_float2(p, e));
}

// Source-grid nodes of the 2^d corners of the cell centred at target node t
// (corner s: bit D-1-i of s selects the lower or upper node in axis i), and
// for non-periodic problems which of them are ghosts (mask bit per axis).
template <int D>
__device__ __forceinline__ void cell_corners(const Geometry &g, int64_t t, int64_t *idx, int *gmask) {
  int64_t ti[D];
  int64_t r = t;
#pragma unroll
  for (int i = D - 1; i >= 0; --i) {
    ti[i] = r % g.n_dst;
    r /= g.n_dst;
  }
  int64_t si[D][2];
  int gh[D][2];
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int64_t s = g.dst == 1 ? ti[i] + b : ti[i] - 1 + b;
      int ghost = 0;
      if (g.bc == HERMITE_PERIODIC) {
        if (s < 0) s += g.n_src;
        if (s >= g.n_src) s -= g.n_src;
      } else if (s < 0) {
        s = 0;
        ghost = 1;
      } else if (s >= g.n_src) {
        s = g.n_src - 1;
        ghost = 1;
      }
      si[i][b] = s;
      gh[i][b] = ghost;
    }
  }
#pragma unroll
  for (int s = 0; s < (1 << D); ++s) {
    int64_t id = 0;
    int mask = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const int bit = (s >> (D - 1 - i)) & 1;
      id = id * g.n_src + si[i][bit];
      if (gh[i][bit]) mask |= 1 << (D - 1 - i);
    }
    idx[s] = id;
    gmask[s] = mask;
  }
}

// Weight of the cell centred at target node t in an energy sum: a cell
// centred on a boundary primal node is cut in half by the boundary in that
// axis (its other half mirrors it), so it counts 1/2 per such axis.
template <int D>
__device__ __forceinline__ float cell_weight(const Geometry &g, int64_t t) {
  if (g.bc == HERMITE_PERIODIC || g.dst != 0) return 1.0f;
  float w = 1.0f;
#pragma unroll
  for (int i = D - 1; i >= 0; --i) {
    const int64_t ti = t % g.n_dst;
    t /= g.n_dst;
    if (ti == 0 || ti == g.n_dst - 1) w *= 0.5f;
  }
  return w;
}

// Does the ghost image of a coefficient with parity bits pb change sign?
// Odd extension (Dirichlet) gives (-1)^{k_i+1} per ghost axis, even
// extension (Neumann) (-1)^{k_i}.
__device__ __forceinline__ bool ghost_negates(int bc, int mask, int pb) {
  int neg = __popc(mask & pb) & 1;
  if (bc == HERMITE_DIRICHLET) neg ^= __popc(mask) & 1;
  return neg != 0;
}

}  // namespace dev
}  // namespace hermite
