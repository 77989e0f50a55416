"""Independent polynomial algebra for oracle pins (numpy only).

A d-variate polynomial is a coefficient array C with C[i0, .., i_{d-1}] the
coefficient of x0^i0 ... x_{d-1}^i_{d-1}.  Nothing here calls the oracle.
"""
from __future__ import annotations

import math

import numpy as np


def shift_scale(C, point, h):
    """Coefficients of xi -> P(point + h*xi); the coefficient of xi^k is the
    scaled derivative h^|k|/k! d^k P(point)."""
    C = np.asarray(C, dtype=np.float64)
    out = C.copy()
    for ax in range(C.ndim):
        n = C.shape[ax]
        T = np.zeros((n, n))
        a = float(point[ax])
        for j in range(n):
            for k in range(j + 1):
                T[k, j] = math.comb(j, k) * a ** (j - k) * h ** k
        out = np.moveaxis(np.tensordot(T, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def scaled_derivs(C, point, h, q):
    """[prod (q+1)] scaled derivatives k in [0,q]^d (C order) of P at point."""
    S = shift_scale(C, point, h)
    d = S.ndim
    pad = [(0, max(0, q + 1 - S.shape[i])) for i in range(d)]
    S = np.pad(S, pad)
    return S[tuple(slice(0, q + 1) for _ in range(d))].reshape(-1)


def deriv(C, ax, k=1):
    C = np.asarray(C, dtype=np.float64)
    out = np.zeros_like(C)
    n = C.shape[ax]
    for j in range(k, n):
        src = [slice(None)] * C.ndim
        dst = [slice(None)] * C.ndim
        src[ax] = j
        dst[ax] = j - k
        out[tuple(dst)] = C[tuple(src)] * math.perm(j, k)
    return out


def laplacian(C):
    return sum(deriv(C, ax, 2) for ax in range(np.ndim(C)))


def wave_taylor(U0, V0, t, c):
    """Exact solution of u_tt = c^2 Lap u for polynomial data (finite series)."""
    U0 = np.asarray(U0, dtype=np.float64)
    V0 = np.zeros_like(U0) if V0 is None else np.asarray(V0, dtype=np.float64)
    shape = tuple(max(a, b) for a, b in zip(U0.shape, V0.shape))
    U = np.zeros(shape)
    V = np.zeros(shape)
    U[tuple(slice(0, s) for s in U0.shape)] = U0
    V[tuple(slice(0, s) for s in V0.shape)] = V0
    u = np.zeros(shape)
    v = np.zeros(shape)
    r = 0
    a, b = U.copy(), V.copy()
    while np.any(a != 0) or np.any(b != 0):
        u += t ** (2 * r) * c ** (2 * r) / math.factorial(2 * r) * a
        u += t ** (2 * r + 1) * c ** (2 * r) / math.factorial(2 * r + 1) * b
        # v = u_t
        if r > 0:
            v += t ** (2 * r - 1) * c ** (2 * r) / math.factorial(2 * r - 1) * a
        v += t ** (2 * r) * c ** (2 * r) / math.factorial(2 * r) * b
        a, b = laplacian(a), laplacian(b)
        r += 1
    return u, v


def random_poly(rng, degs):
    return rng.standard_normal([d + 1 for d in degs])


def corner_points(d, h):
    """Corner offsets of a cell centred at 0, bit i of the corner index (axis 0
    most significant) = 1 meaning +h/2."""
    pts = []
    for s in range(1 << d):
        pts.append([(0.5 if (s >> (d - 1 - i)) & 1 else -0.5) * h for i in range(d)])
    return np.array(pts)


def corner_data(C, d, h, q):
    return np.stack([scaled_derivs(C, p, h, q) for p in corner_points(d, h)])
