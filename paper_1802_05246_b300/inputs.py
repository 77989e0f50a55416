"""Seeded synthetic inputs: exact scaled Taylor data of analytic functions.

This module is shared by the tests, the benchmark and the smoke check.  It
holds none of the Hermite method's arithmetic (no interpolation, no time
evolution): it only evaluates the nodal degrees of freedom the paper
initialises with (Sec. 3.1.1), i.e. the scaled derivatives

    h^|k| / k!  d^k f (x_node),   k in [0, q]^d,

of closed-form functions, returned in the host layout ``[node][coef]``
(nodes in C order with axis 0 slowest, coefficient multi-index in C order).

Functions provided
  * ``sine_data``: f = A sin(a . x + phi), any wave vector (plane and standing
    waves are sums of these);
  * ``gaussian_data``: sums of separable Gaussian pulses A exp(-|x-x0|^2/w^2),
    made periodic, odd (Dirichlet) or even (Neumann) by image sums;
  * pulse-parameter generators for the seeded workloads (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2


def npts(N: int, bc: int, grid: int) -> int:
    """Nodes per axis: periodic N on both grids; otherwise primal N+1, dual N."""
    if bc == PERIODIC:
        return N
    return N + 1 if grid == 0 else N


def axis_coords(N: int, h: float, bc: int, grid: int) -> np.ndarray:
    """Primal nodes at i*h, dual nodes at (j+1/2)*h (domain [0, N h])."""
    n = npts(N, bc, grid)
    return (np.arange(n, dtype=np.float64) + (0.5 if grid == 1 else 0.0)) * h


def _multi_indices(d: int, q: int) -> np.ndarray:
    if q < 0:
        return np.zeros((0, d), dtype=np.int64)
    g = np.meshgrid(*([np.arange(q + 1)] * d), indexing="ij")
    return np.stack([x.reshape(-1) for x in g], -1)


def tensor_data(per_axis: list[np.ndarray]) -> np.ndarray:
    """per_axis[i]: [n_i][q+1] scaled 1-D derivatives -> [prod n_i][(q+1)^d]."""
    out = per_axis[0]
    for a in per_axis[1:]:
        out = np.einsum("nk,ml->nmkl", out, a).reshape(out.shape[0] * a.shape[0], out.shape[1] * a.shape[1])
    return out


def sine_data(d, q, N, h, bc, grid, wavevec, phase=0.0, amp=1.0):
    """Scaled derivatives of amp*sin(wavevec . x + phase) at the nodes of grid."""
    wavevec = np.asarray(wavevec, dtype=np.float64).reshape(d)
    ax = axis_coords(N, h, bc, grid)
    g = np.meshgrid(*([ax] * d), indexing="ij")
    X = np.stack([x.reshape(-1) for x in g], -1)  # [nodes, d]
    K = _multi_indices(d, q)  # [ncoef, d]
    arg = X @ wavevec + phase
    kk = K.sum(1)
    fac = np.array([np.prod([(wavevec[i] * h) ** K[j, i] / math.factorial(K[j, i]) for i in range(d)])
                    for j in range(len(K))])
    return amp * np.sin(arg[:, None] + kk[None, :] * (np.pi / 2)) * fac[None, :]


def _hermite_phys(n: int, x: np.ndarray) -> np.ndarray:
    """Physicists' Hermite polynomials H_0..H_n at x: [n+1, ...]."""
    H = np.zeros((n + 1,) + x.shape)
    H[0] = 1.0
    if n >= 1:
        H[1] = 2 * x
    for k in range(1, n):
        H[k + 1] = 2 * x * H[k] - 2 * k * H[k - 1]
    return H


def gaussian_1d(x: np.ndarray, q: int, h: float, x0: float, w: float, L: float, bc: int) -> np.ndarray:
    """[n][q+1] scaled derivatives of the image sum of exp(-(x-x0)^2/w^2).

    Periodic: images at x0 + kL.  Dirichlet (odd about 0 and L): +images at
    x0 + 2kL, -images at -x0 + 2kL.  Neumann (even): both with +."""
    kmax = int(math.ceil(10.0 * w / L)) + 2
    out = np.zeros((x.size, q + 1))
    kf = np.array([h ** k / math.factorial(k) for k in range(q + 1)])

    def add(centre, sign):
        s = (x - centre) / w
        H = _hermite_phys(q, s)
        e = np.exp(-(s * s))
        for k in range(q + 1):
            out[:, k] += sign * (-1.0 / w) ** k * H[k] * e * kf[k]

    for k in range(-kmax, kmax + 1):
        if bc == PERIODIC:
            add(x0 + k * L, 1.0)
        else:
            add(x0 + 2 * k * L, 1.0)
            add(-x0 + 2 * k * L, -1.0 if bc == DIRICHLET else 1.0)
    return out


def gaussian_data(d, q, N, h, bc, grid, centres, widths, amps):
    """Sum over pulses p of amps[p] * prod_i gaussian_1d(axis i) (separable)."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, d)
    ax = axis_coords(N, h, bc, grid)
    L = N * h
    n = ax.size ** d
    if q < 0:
        return np.zeros((n, 0))
    out = np.zeros((n, (q + 1) ** d))
    for p in range(centres.shape[0]):
        per_axis = [gaussian_1d(ax, q, h, centres[p, i], float(widths[p]), L, bc) for i in range(d)]
        out += float(amps[p]) * tensor_data(per_axis)
    return out


def pulses_3d_config(seed: int = 0, n: int = 8):
    """3-D workload pulses: centres U[0,1)^3, widths U[0.05,0.1], amplitudes N(0,1),
    drawn in that order from numpy's PCG64 with the given seed."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n, 3))
    widths = rng.uniform(0.05, 0.1, size=n)
    amps = rng.normal(0.0, 1.0, size=n)
    return centres, widths, amps


def random_pulses(rng: np.random.Generator, d: int, nmin: int, nmax: int, wmin: float, wmax: float):
    """1..k pulses with centres U[0,1)^d, widths U[wmin,wmax], amplitudes N(0,1)."""
    n = int(rng.integers(nmin, nmax + 1))
    centres = rng.uniform(0.0, 1.0, size=(n, d))
    widths = rng.uniform(wmin, wmax, size=n)
    amps = rng.normal(0.0, 1.0, size=n)
    return centres, widths, amps


def gaussian_data_2d(q, N, h, bc, grid, centres, widths, amps):
    """Same values as ``gaussian_data`` for d = 2, with the sum over pulses
    taken as one matrix product (fast enough to generate thousands of
    initial conditions)."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 2)
    ax = axis_coords(N, h, bc, grid)
    L = N * h
    n = ax.size
    P = centres.shape[0]
    gx = np.stack([float(amps[p]) * gaussian_1d(ax, q, h, centres[p, 0], float(widths[p]), L, bc) for p in range(P)])
    gy = np.stack([gaussian_1d(ax, q, h, centres[p, 1], float(widths[p]), L, bc) for p in range(P)])
    k = q + 1
    U = gx.reshape(P, n * k).T @ gy.reshape(P, n * k)  # [(i, a), (j, b)]
    return np.ascontiguousarray(U.reshape(n, k, n, k).transpose(0, 2, 1, 3)).reshape(n * n, k * k)


def superstep_pulses(traj: int):
    """Initial pulses of learned-stepper trajectory number traj: 1-6 pulses,
    centres U[0,1)^2, widths U[0.05,0.15], amplitudes N(0,1), drawn from
    numpy's PCG64 seeded with traj."""
    return random_pulses(np.random.default_rng(traj), 2, 1, 6, 0.05, 0.15)


def pulse_wave_3d(points, t, centres, widths, amps, c=1.0, L=1.0, xp=np):
    """Exact solution u(x, t) of u_tt = c^2 Lap u on the periodic cube [0, L)^3
    with u(x, 0) = sum_p A_p sum_{n in Z^3} g_p(|x - x_p - n L|),
    g_p(r) = exp(-r^2 / w_p^2), and u_t(x, 0) = 0 (the 3-D pulse workload).

    Every periodic image is a radial pulse.  For radial data r*u solves the 1-D
    wave equation in r with an odd extension, so d'Alembert's formula gives
        u(r, t) = [(r - ct) g(r - ct) + (r + ct) g(r + ct)] / (2 r),
    whose limit at r = 0 is W'(ct) with W(s) = s g(s); for r below 1e-4 w the
    two-term Taylor series W'(ct) + W'''(ct) r^2 / 6 replaces the quotient.
    Images farther than 6.8 w from the sphere r = ct contribute below 1e-20
    and are skipped.

    points: [..., 3] array (numpy, or a torch tensor with xp=torch); returns
    an array of the leading shape."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    ct = c * float(t)
    out = xp.zeros_like(points[..., 0])
    for p in range(centres.shape[0]):
        w = float(widths[p])
        R = 6.8 * w
        K = int(math.ceil((ct + R) / L)) + 1
        d0 = points - xp.asarray(centres[p]) if xp is np else points - xp.tensor(centres[p], dtype=points.dtype,
                                                                                    device=points.device)
        # bounding box of the offsets: images whose distance range over the
        # box misses the shell |r - ct| <= R (and the ball r + ct <= R) are
        # skipped
        lo = [float(d0[..., i].min()) for i in range(3)]
        hi = [float(d0[..., i].max()) for i in range(3)]
        for n0 in range(-K, K + 1):
            for n1 in range(-K, K + 1):
                for n2 in range(-K, K + 1):
                    shift = (n0 * L, n1 * L, n2 * L)
                    near2 = far2 = 0.0
                    for i in range(3):
                        a0, a1 = lo[i] - shift[i], hi[i] - shift[i]
                        near2 += 0.0 if a0 <= 0.0 <= a1 else min(a0 * a0, a1 * a1)
                        far2 += max(a0 * a0, a1 * a1)
                    if math.sqrt(near2) > ct + R or (math.sqrt(far2) < ct - R and math.sqrt(far2) + ct > R):
                        continue
                    r2 = (d0[..., 0] - shift[0]) ** 2 + (d0[..., 1] - shift[1]) ** 2 + (d0[..., 2] - shift[2]) ** 2
                    r = xp.sqrt(r2)
                    a, b = r - ct, r + ct
                    far = (xp.abs(a) > R) & (b > R)
                    small = r < 1e-4 * w
                    rs = xp.where(small, xp.ones_like(r), r)
                    quo = (a * xp.exp(-(a * a) / (w * w)) + b * xp.exp(-(b * b) / (w * w))) / (2.0 * rs)
                    g = math.exp(-(ct * ct) / (w * w))
                    w1 = (1.0 - 2.0 * ct * ct / (w * w)) * g
                    w3 = (24.0 * ct * ct / w ** 4 - 6.0 / (w * w) - 8.0 * ct ** 4 / w ** 6) * g
                    ser = w1 + w3 * r2 / 6.0
                    val = xp.where(small, ser, quo)
                    out = out + float(amps[p]) * xp.where(far, xp.zeros_like(val), val)
    return out
