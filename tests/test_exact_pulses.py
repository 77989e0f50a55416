"""Pins of the exact 3-D pulse solution (inputs.pulse_wave_3d), the reference
that the L2 errors of the 3-D pulse workload are measured against.

The solution is built from d'Alembert's formula for r*u over periodic images;
it is checked here against things that do not share that construction:
  * t = 0: the separable 1-D image sums of inputs.gaussian_data;
  * t > 0: the Fourier series of the periodised Gaussian, each mode
    advancing as cos(2 pi c |k| t) (Gaussian Fourier transform
    (pi w^2)^{3/2} exp(-pi^2 w^2 |k|^2));
  * the wave equation itself, by central differences in x and t.
"""
import math

import numpy as np
import pytest

from paper_1802_05246_b300 import inputs as I


def fourier_pulse(points, t, centre, w, amp, c=1.0, kmax=20):
    k = np.arange(-kmax, kmax + 1)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    kn = np.sqrt((K * K).sum(1))
    coef = amp * (math.pi * w * w) ** 1.5 * np.exp(-(math.pi * w) ** 2 * kn * kn) * np.cos(2 * math.pi * c * kn * t)
    keep = np.abs(coef) > 1e-30
    K, coef = K[keep], coef[keep]
    ph = 2 * math.pi * (points - centre) @ K.T
    return np.cos(ph) @ coef


def test_initial_value_is_the_pulse_sum():
    cen, wid, amp = I.pulses_3d_config(0)
    N = 12
    h = 1.0 / N
    X = np.stack(np.meshgrid(*([np.arange(N) * h] * 3), indexing="ij"), -1).reshape(-1, 3)
    u = I.pulse_wave_3d(X, 0.0, cen, wid, amp)
    ref = I.gaussian_data(3, 0, N, h, I.PERIODIC, 0, cen, wid, amp)[:, 0]
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("w,t", [(0.1, 0.37), (0.1, 1.40625), (0.07, 0.9), (0.15, 2.3)])
def test_matches_the_fourier_series(w, t):
    rng = np.random.default_rng(7)
    centre = rng.uniform(0, 1, 3)
    pts = rng.uniform(0, 1, (40, 3))
    # points on and next to the pulse centre too (the r -> 0 limit)
    pts[0] = centre
    pts[1] = centre + 3e-6
    got = I.pulse_wave_3d(pts, t, centre[None, :], [w], [1.3], c=1.0)
    kmax = int(math.ceil(7.0 / (math.pi * w))) + 1
    ref = fourier_pulse(pts, t, centre, w, 1.3, kmax=kmax)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-13)


def test_solves_the_wave_equation():
    cen, wid, amp = I.pulses_3d_config(0)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (30, 3))
    c, t, d = 1.3, 0.41, 2e-3
    f = lambda x, tt: I.pulse_wave_3d(x, tt, cen, wid, amp, c=c)
    utt = (f(pts, t + d) - 2 * f(pts, t) + f(pts, t - d)) / d**2
    lap = sum((f(pts + d * e, t) - 2 * f(pts, t) + f(pts - d * e, t)) / d**2 for e in np.eye(3))
    scale = np.abs(utt).max()
    # second-order differences: error ~ d^2 u'''' / 12 with widths >= 0.05
    assert np.abs(utt - c * c * lap).max() <= 2e-3 * scale
    # and the velocity at t = 0 vanishes (even in t)
    np.testing.assert_allclose(f(pts, 1e-3), f(pts, -1e-3), rtol=0, atol=1e-14)


def test_oracle_converges_to_it_in_3d(orc):
    """The oracle's 3-D dissipative runs (m = 2, c dt/h <= 0.9, one pulse of
    width 0.2, T = 0.2) approach the exact solution at the order 2m - 1 = 3 of
    Sec. 3 as N = 8, 12, 16: the two pieces of code agree in the limit."""
    cen, wid, amp = np.array([[0.4, 0.55, 0.5]]), [0.2], [1.0]
    m, T = 2, 0.2
    errs = []
    for N in (8, 12, 16):
        h = 1.0 / N
        n = int(np.ceil(T / (0.9 * h)))
        P = orc.Problem(3, m, N, 1.0, h, T / n, orc.DISSIPATIVE, orc.PERIODIC)
        u0 = I.gaussian_data(3, m, N, h, I.PERIODIC, 0, cen, wid, amp)
        u, _ = P.run(u0, np.zeros((N**3, m**3)), nsteps=n)
        ex = lambda p: I.pulse_wave_3d(p.reshape(-1, 3), T, cen, wid, amp).reshape(p.shape[:-1])
        errs.append(P.l2_error(0, u, 2 * m + 2, ex))  # exact for the degree-(4m+2) square
    orders = [math.log(errs[0] / errs[1]) / math.log(1.5), math.log(errs[1] / errs[2]) / math.log(4 / 3)]
    assert errs[2] < 1e-4
    assert all(2.6 <= o <= 3.8 for o in orders), (errs, orders)
